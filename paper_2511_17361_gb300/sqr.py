"""Thin Python binding of libsqr (include/sqr.h) over ctypes.

Only argument marshalling lives here: every step of the renderer runs in the
CUDA library.  PyTorch provides device memory and the current stream.  The
library is loaded from the package's ``_lib/libsqr.so``; if it is missing the
import fails (there is no CPU fallback).

Names follow the C ABI: :func:`build_index`, :func:`render_fwd`,
:func:`render_bwd`, :func:`query_grid`, :func:`loss_ce_mse`, and
:class:`SQRender`, the ``torch.autograd.Function`` around forward/backward.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# SQR_CHECK=1 in the environment loads the debug build with bounds checks
# (libsqr_check.so, sq_check_query) instead of the library.
LIB_PATH = os.path.join(_PKG, "_lib", "libsqr_check.so" if os.environ.get("SQR_CHECK") == "1" else "libsqr.so")

SQ_OK, SQ_ERR_INVALID_ARG, SQ_ERR_CAPACITY, SQ_ERR_CUDA, SQ_ERR_TIMEOUT, SQ_ERR_NUMERIC = range(6)
SQ_INDEX_OBB, SQ_INDEX_CUBE, SQ_INDEX_OBB_OPACITY = 0, 1, 2
SQ_SEM_RAW, SQ_SEM_SOFTMAX = 0, 1
SQ_OP_INDEX, SQ_OP_FWD, SQ_OP_BWD, SQ_OP_QUERY = 0, 1, 2, 3
SQ_BWD_DEFAULT, SQ_BWD_RAY_MAJOR, SQ_BWD_PRIMITIVE_MAJOR = 0, 1, 2

_vp = ctypes.c_void_p


class SqGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("lo", ctypes.c_float * 3),
                ("vs", ctypes.c_float * 3)]


class SqPrims(ctypes.Structure):
    _fields_ = [("means", _vp), ("quats", _vp), ("scales", _vp), ("eps", _vp), ("opacity", _vp), ("logits", _vp),
                ("n", ctypes.c_int), ("n_classes", ctypes.c_int), ("sem_mode", ctypes.c_int)]


class SqIndexOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("tau_cut", ctypes.c_float), ("nv", ctypes.c_int)]


class SqIndex(ctypes.Structure):
    _fields_ = [("v_n", _vp), ("v_f", _vp), ("v_sq", _vp), ("ranges", _vp), ("capacity", ctypes.c_longlong),
                ("p_total", _vp), ("status", _vp), ("v_flags", _vp)]


class SqRays(ctypes.Structure):
    _fields_ = [("n_cam", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int), ("K", _vp), ("cam2world", _vp),
                ("t", _vp), ("L", ctypes.c_int), ("kappa", ctypes.c_float), ("alpha_max", ctypes.c_float)]


class SqScene(ctypes.Structure):
    _fields_ = [("prims", SqPrims), ("index", SqIndex), ("grid", SqGrid), ("rays", SqRays), ("depth", _vp),
                ("sem", _vp), ("t_final", _vp), ("saved", _vp), ("saved_bytes", ctypes.c_size_t), ("grad_depth", _vp),
                ("grad_sem", _vp), ("g_means", _vp), ("g_quats", _vp), ("g_scales", _vp), ("g_eps", _vp),
                ("g_opacity", _vp), ("g_logits", _vp), ("pair_visits", _vp)]


class SqTuning(ctypes.Structure):
    _fields_ = [("fwd_lanes_per_ray", ctypes.c_int), ("fwd_warps_per_cta", ctypes.c_int),
                ("bwd_warps_per_cta", ctypes.c_int), ("bwd_order", ctypes.c_int), ("fwd_ray_tile", ctypes.c_int)]


class SqrError(RuntimeError):
    pass


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_2511_17361_gb300._build")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    lib.sq_workspace_size.restype = ctypes.c_size_t
    lib.sq_workspace_size.argtypes = [ctypes.c_int, P(SqPrims), P(SqGrid), P(SqRays)]
    lib.sq_build_index.argtypes = [P(SqPrims), P(SqGrid), P(SqIndexOpts), P(SqIndex), _vp, ctypes.c_size_t, _vp]
    lib.sq_saved_size.restype = ctypes.c_size_t
    lib.sq_saved_size.argtypes = [P(SqRays), ctypes.c_int]
    lib.sq_saved_size_pages.restype = ctypes.c_size_t
    lib.sq_saved_size_pages.argtypes = [P(SqRays), ctypes.c_int, ctypes.c_longlong]
    lib.sq_render_fwd.argtypes = [P(SqPrims), P(SqIndex), P(SqGrid), P(SqRays), _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                  _vp, ctypes.c_size_t, _vp]
    lib.sq_render_bwd.argtypes = [P(SqPrims), P(SqIndex), P(SqGrid), P(SqRays), _vp, ctypes.c_size_t, _vp, _vp, _vp,
                                  _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
    lib.sq_query_grid.argtypes = [P(SqPrims), P(SqIndex), P(SqGrid), ctypes.c_float, _vp, _vp, _vp, _vp,
                                  ctypes.c_size_t, _vp]
    lib.sq_loss_ce_mse.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_float, _vp, _vp, _vp, _vp]
    lib.sq_loss_voxel.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                  _vp, _vp, _vp, _vp, _vp]
    lib.sq_count_pairs.argtypes = [P(SqIndex), P(SqGrid), P(SqRays), _vp, _vp]
    lib.sq_batched_workspace_size.restype = ctypes.c_size_t
    lib.sq_batched_workspace_size.argtypes = [P(SqScene), ctypes.c_int]
    lib.sq_render_batched.argtypes = [ctypes.c_int, P(SqScene), ctypes.c_int, P(SqTuning), _vp, ctypes.c_size_t, _vp]
    lib.sq_autotune.argtypes = [P(SqScene), ctypes.c_int, _vp, ctypes.c_size_t, _vp, ctypes.c_int, P(SqTuning),
                                _vp, _vp]
    for f in ("sq_build_index", "sq_render_fwd", "sq_render_bwd", "sq_query_grid", "sq_loss_ce_mse", "sq_loss_voxel",
              "sq_count_pairs", "sq_render_batched", "sq_autotune"):
        getattr(lib, f).restype = ctypes.c_int
    lib.sq_status_string.restype = ctypes.c_char_p
    lib.sq_status_string.argtypes = [ctypes.c_int]
    lib.sq_last_error.restype = ctypes.c_char_p
    lib.sq_query_grid_bwd.restype = ctypes.c_int
    lib.sq_query_grid_bwd.argtypes = [P(SqPrims), P(SqIndex), P(SqGrid), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                      _vp, ctypes.c_size_t, _vp]
    lib.sq_measure_sfu.restype = ctypes.c_int
    lib.sq_measure_sfu.argtypes = [ctypes.c_int, P(ctypes.c_double), _vp]
    lib.sq_check_query.restype = ctypes.c_int
    lib.sq_check_query.argtypes = [P(ctypes.c_int), P(ctypes.c_int)]
    lib.sq_profile_enable.restype = ctypes.c_int
    lib.sq_profile_enable.argtypes = [ctypes.c_int]
    lib.sq_profile_query.restype = ctypes.c_int
    lib.sq_profile_query.argtypes = [ctypes.c_char_p, P(ctypes.c_longlong), P(ctypes.c_double), P(ctypes.c_longlong)]
    return lib


lib = _load()


def _check(status: int, what: str):
    if status != SQ_OK:
        raise SqrError(f"{what}: {lib.sq_status_string(status).decode()} ({lib.sq_last_error().decode()})")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need_cuda_f32(t, name):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise SqrError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


PRIM_KEYS = ("means", "quats", "scales", "eps", "opacity", "logits")


def prims_struct(prims: dict) -> SqPrims:
    """The parameter tensors (PRIM_KEYS) and, optionally, prims["sem_mode"]
    (SQ_SEM_RAW by default, or SQ_SEM_SOFTMAX)."""
    for k in PRIM_KEYS:
        _need_cuda_f32(prims[k], k)
    n, C = prims["logits"].shape
    return SqPrims(*[_ptr(prims[k]) for k in PRIM_KEYS], n, C, int(prims.get("sem_mode", SQ_SEM_RAW)))


def grid_struct(grid: dict) -> SqGrid:
    nx, ny, nz = (int(v) for v in grid["n"])
    return SqGrid(nx, ny, nz, (ctypes.c_float * 3)(*[float(v) for v in grid["lo"]]),
                  (ctypes.c_float * 3)(*[float(v) for v in grid["vs"]]))


@dataclass
class Rays:
    """Camera rig and samples on the device: K [n_cam,4], cam2world [n_cam,3,4], t [L]."""
    K: torch.Tensor
    cam2world: torch.Tensor
    t: torch.Tensor
    H: int
    W: int
    kappa: float = 0.0
    alpha_max: float = 1.0

    @property
    def n_cam(self):
        return self.K.shape[0]

    @property
    def R(self):
        return self.n_cam * self.H * self.W

    def struct(self) -> SqRays:
        for name in ("K", "cam2world", "t"):
            _need_cuda_f32(getattr(self, name), name)
        return SqRays(self.n_cam, self.H, self.W, _ptr(self.K), _ptr(self.cam2world), _ptr(self.t), self.t.numel(),
                      self.kappa, self.alpha_max)

    @staticmethod
    def from_rig(rig: dict, t, device="cuda", kappa=0.0, alpha_max=1.0) -> "Rays":
        f = lambda a: torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        t_host = torch.as_tensor(t, dtype=torch.float32)
        if t_host.numel() > 1 and bool((t_host[1:] < t_host[:-1]).any()):
            raise SqrError("sample depths t must be non-decreasing")
        return Rays(f(rig["K"]), f(rig["cam2world"]), f(t), int(rig["H"]), int(rig["W"]), kappa, alpha_max)


class _Workspace:
    """Per-device scratch buffers, grown on demand and reused across calls."""

    def __init__(self):
        self.bufs = {}

    def get(self, key, nbytes, device):
        nbytes = max(int(nbytes), 256)
        b = self.bufs.get((key, device))
        if b is None or b.numel() < nbytes:
            b = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self.bufs[(key, device)] = b
        return b


_ws = _Workspace()


def workspace_size(op, prims=None, grid=None, rays=None) -> int:
    p = prims_struct(prims) if prims is not None else None
    g = grid_struct(grid) if grid is not None else None
    r = rays.struct() if rays is not None else None
    return int(lib.sq_workspace_size(op, ctypes.byref(p) if p else None, ctypes.byref(g) if g else None,
                                     ctypes.byref(r) if r else None))


# ------------------------------------------------------------------ index
class Index:
    """Device buffers of the voxel -> superquadric index (V_n, V_f, V_sq, ranges)
    and, with ``flags``, the per-entry range-boundary flags that the ray-major
    backward uses to find where a ray enters a range (the primitive-major default
    does not read them)."""

    def __init__(self, grid: dict, n: int, capacity: int, device, flags: bool = False):
        nvox = int(grid["n"][0]) * int(grid["n"][1]) * int(grid["n"][2])
        self.grid = grid
        self.v_n = torch.empty(nvox, dtype=torch.int32, device=device)
        self.v_f = torch.empty(nvox, dtype=torch.int32, device=device)
        self.v_sq = torch.empty(max(int(capacity), 1), dtype=torch.int32, device=device)
        self.v_flags = torch.empty(max(int(capacity), 1), dtype=torch.int16, device=device) if flags else None
        self.capacity = int(capacity)
        self.ranges = torch.empty((max(n, 1), 6), dtype=torch.int32, device=device)
        self.p_total = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)

    def struct(self) -> SqIndex:
        return SqIndex(_ptr(self.v_n), _ptr(self.v_f), _ptr(self.v_sq), _ptr(self.ranges), self.capacity,
                       _ptr(self.p_total), _ptr(self.status), _ptr(self.v_flags))

    def P(self) -> int:
        return int(self.p_total.item())

    def check(self):
        s = int(self.status.item())
        if s == SQ_ERR_CAPACITY:
            raise SqrError(f"index: {lib.sq_status_string(s).decode()} (needed {self.P()}, have {self.capacity})")
        if s != SQ_OK:
            raise SqrError(f"index: {lib.sq_status_string(s).decode()}")


def build_index(prims: dict, grid: dict, mode: int = SQ_INDEX_OBB, tau_cut: float = 0.01, nv: int = 5,
                capacity: int | None = None, index: Index | None = None, sync: bool = True,
                flags: bool = False) -> Index:
    """Builds the index on the current stream.  With ``sync`` the host reads P and
    re-runs once with a large enough V_sq when the capacity was too small.
    ``flags`` also writes the per-entry range-boundary flags (for the ray-major
    backward order)."""
    device = prims["means"].device
    n = prims["means"].shape[0]
    if index is None:
        if capacity is None:
            nvox = int(grid["n"][0]) * int(grid["n"][1]) * int(grid["n"][2])
            capacity = max(4 * nvox, 1024)
        index = Index(grid, n, capacity, device, flags)
    p, g = prims_struct(prims), grid_struct(grid)
    opts = SqIndexOpts(mode, tau_cut, nv)
    wsz = lib.sq_workspace_size(SQ_OP_INDEX, ctypes.byref(p), ctypes.byref(g), None)
    ws = _ws.get("index", wsz, device)
    idx_s = index.struct()
    _check(lib.sq_build_index(ctypes.byref(p), ctypes.byref(g), ctypes.byref(opts), ctypes.byref(idx_s),
                              _ptr(ws), ws.numel(), _stream()), "sq_build_index")
    if sync:
        P = index.P()
        if P > index.capacity:
            index = Index(grid, n, int(P * 1.25) + 1024, device, index.v_flags is not None)
            return build_index(prims, grid, mode, tau_cut, nv, index=index, sync=True)
        index.check()
    return index


# ------------------------------------------------------------------ render
SQ_SAVE_PAGE = 8


def saved_size(rays: Rays, n_classes: int, pages: int | None = None) -> int:
    """Bytes of the forward state the backward pass needs: T_j, alpha_j and s_j of
    the composited samples, in pages of SQ_SAVE_PAGE samples.  ``pages`` None: room
    for every sample of every ray (always enough); else room for that many pages."""
    r = rays.struct()
    if pages is None:
        n = int(lib.sq_saved_size(ctypes.byref(r), int(n_classes)))
    else:
        n = int(lib.sq_saved_size_pages(ctypes.byref(r), int(n_classes), max(int(pages), 1)))
    if n == 0 and rays.R > 0:
        raise ValueError(f"sq_saved_size: {lib.sq_last_error().decode()}")
    return n


def render_fwd(prims: dict, index: Index, grid: dict, rays: Rays, out=None, saved=None):
    """Returns depth [R], sem [R, C], t_final [R] (Eq. 4-6).  ``saved``: a uint8
    device tensor of saved_size(rays, C) bytes that receives the state for
    render_bwd, or None (inference)."""
    device = prims["means"].device
    C = prims["logits"].shape[1]
    R = rays.R
    if out is None:
        out = (torch.empty(R, device=device), torch.empty((R, C), device=device), torch.empty(R, device=device))
    depth, sem, tf = out
    p, g, r, ix = prims_struct(prims), grid_struct(grid), rays.struct(), index.struct()
    wsz = lib.sq_workspace_size(SQ_OP_FWD, ctypes.byref(p), ctypes.byref(g), ctypes.byref(r))
    ws = _ws.get("fwd", wsz, device)
    sv_n = 0 if saved is None else saved.numel() * saved.element_size()
    _check(lib.sq_render_fwd(ctypes.byref(p), ctypes.byref(ix), ctypes.byref(g), ctypes.byref(r), _ptr(depth),
                             _ptr(sem), _ptr(tf), _ptr(saved), sv_n, _ptr(ws), ws.numel(), _stream()),
           "sq_render_fwd")
    return depth, sem, tf


def new_saved(rays: Rays, n_classes: int, device="cuda", pages: int | None = None):
    """A saved-state buffer: room for every sample (pages None) or for ``pages``
    pages (after a forward, saved_header gives the pages it needed)."""
    return torch.empty(saved_size(rays, n_classes, pages), dtype=torch.uint8, device=device)


def saved_header(saved):
    """(pages the last forward needed, status SQ_OK or SQ_ERR_CAPACITY); waits
    for the stream."""
    h = saved[:16].cpu()
    return int(h[:8].view(torch.int64).item()), int(h[8:12].view(torch.int32).item())


def saved_counts(saved, rays: Rays, n_classes: int):
    """The per-ray composited sample counts [R] int32 of a saved forward state
    (its third block, layout as sq_saved_size documents)."""
    R, L = rays.R, rays.t.numel()
    npr = (L + SQ_SAVE_PAGE - 1) // SQ_SAVE_PAGE
    a256 = lambda b: (b + 255) // 256 * 256
    off = 256 + a256(R * npr * 4)
    return saved[off:off + R * 4].view(torch.int32)


def render_bwd(prims: dict, index: Index, grid: dict, rays: Rays, grad_depth, grad_sem, saved=None, out=None,
               order: int = SQ_BWD_DEFAULT, pair_visits=None) -> dict:
    """Gradients of sum(gD * depth) + sum(gS * sem) w.r.t. every parameter.  ``saved``
    comes from render_fwd on the same inputs; when None the forward is run here.
    ``order`` (SQ_BWD_*) other than the default goes through sq_render_batched
    with that backward order, and so does a ``pair_visits`` int64 tensor [n], which
    receives the pairs the primitive-major order evaluated per primitive."""
    device = prims["means"].device
    grad_depth = _need_cuda_f32(grad_depth.contiguous(), "grad_depth")
    grad_sem = _need_cuda_f32(grad_sem.contiguous(), "grad_sem")
    if saved is None:
        saved = new_saved(rays, prims["logits"].shape[1], device)
        render_fwd(prims, index, grid, rays, saved=saved)
    if out is None:
        out = {k: torch.empty_like(prims[k]) for k in PRIM_KEYS}
    p, g, r, ix = prims_struct(prims), grid_struct(grid), rays.struct(), index.struct()
    if order != SQ_BWD_DEFAULT or pair_visits is not None:
        sc = SqScene()
        sc.prims, sc.index, sc.grid, sc.rays = p, ix, g, r
        sc.saved, sc.saved_bytes = _ptr(saved), saved.numel() * saved.element_size()
        sc.grad_depth, sc.grad_sem = _ptr(grad_depth), _ptr(grad_sem)
        for k in PRIM_KEYS:
            setattr(sc, "g_" + k, _ptr(out[k]))
        if pair_visits is not None:
            if not (pair_visits.is_cuda and pair_visits.dtype == torch.int64 and pair_visits.is_contiguous()
                    and pair_visits.numel() == prims["means"].shape[0]):
                raise SqrError("pair_visits must be a contiguous int64 CUDA tensor with one entry per primitive")
            sc.pair_visits = _ptr(pair_visits)
        arr = (SqScene * 1)(sc)
        ws = _ws.get("bwd", lib.sq_batched_workspace_size(arr, 1), device)
        tn = SqTuning(4, 8, 0, order, 1)
        _check(lib.sq_render_batched(SQ_OP_BWD, arr, 1, ctypes.byref(tn), _ptr(ws), ws.numel(), _stream()),
               "sq_render_batched")
        return out
    wsz = lib.sq_workspace_size(SQ_OP_BWD, ctypes.byref(p), ctypes.byref(g), ctypes.byref(r))
    ws = _ws.get("bwd", wsz, device)
    _check(lib.sq_render_bwd(ctypes.byref(p), ctypes.byref(ix), ctypes.byref(g), ctypes.byref(r), _ptr(saved),
                             saved.numel() * saved.element_size(), _ptr(grad_depth), _ptr(grad_sem),
                             *[_ptr(out[k]) for k in PRIM_KEYS], _ptr(ws), ws.numel(), _stream()), "sq_render_bwd")
    return out


def query_grid(prims: dict, index: Index, grid: dict, tau: float = 0.05, with_label: bool = True, out=None):
    """Supp. A.4 voxelisation: density [V], sem [V, C], label [V] uint8 (C = free).
    ``out`` = (density, sem, label or None) to write into."""
    device = prims["means"].device
    C = prims["logits"].shape[1]
    nvox = index.v_n.numel()
    if out is not None:
        dens, sem, lab = out
    else:
        dens = torch.empty(nvox, device=device)
        sem = torch.empty((nvox, C), device=device)
        lab = torch.empty(nvox, dtype=torch.uint8, device=device) if with_label else None
    p, g, ix = prims_struct(prims), grid_struct(grid), index.struct()
    wsz = lib.sq_workspace_size(SQ_OP_QUERY, ctypes.byref(p), ctypes.byref(g), None)
    ws = _ws.get("query", wsz, device)
    _check(lib.sq_query_grid(ctypes.byref(p), ctypes.byref(ix), ctypes.byref(g), tau, _ptr(dens), _ptr(sem),
                             _ptr(lab), _ptr(ws), ws.numel(), _stream()), "sq_query_grid")
    return dens, sem, lab


def query_grid_bwd(prims: dict, index: Index, grid: dict, grad_density, grad_sem, out=None) -> dict:
    """Gradients of sum(gd * density) + sum(gs * sem) of the grid query w.r.t.
    every parameter (index held fixed)."""
    device = prims["means"].device
    grad_density = _need_cuda_f32(grad_density.contiguous(), "grad_density")
    grad_sem = _need_cuda_f32(grad_sem.contiguous(), "grad_sem")
    if out is None:
        out = {k: torch.empty_like(prims[k]) for k in PRIM_KEYS}
    p, g, ix = prims_struct(prims), grid_struct(grid), index.struct()
    wsz = lib.sq_workspace_size(SQ_OP_QUERY, ctypes.byref(p), ctypes.byref(g), None)
    ws = _ws.get("query", wsz, device)
    _check(lib.sq_query_grid_bwd(ctypes.byref(p), ctypes.byref(ix), ctypes.byref(g), _ptr(grad_density),
                                 _ptr(grad_sem), *[_ptr(out[k]) for k in PRIM_KEYS], _ptr(ws), ws.numel(),
                                 _stream()), "sq_query_grid_bwd")
    return out


def loss_ce_mse(depth, sem, target_depth, target_label, lambda_s=2.0, lambda_d=0.05, out=None):
    """Supp. A.5 loss (Eq. 8) and its gradients w.r.t. depth and sem."""
    R, C = sem.shape
    if out is None:
        out = (torch.empty(1, device=sem.device), torch.empty_like(depth), torch.empty_like(sem))
    loss, gd, gs = out
    _check(lib.sq_loss_ce_mse(_ptr(depth), _ptr(sem), _ptr(target_depth), _ptr(target_label), R, C, lambda_s,
                              lambda_d, _ptr(loss), _ptr(gd), _ptr(gs), _stream()), "sq_loss_ce_mse")
    return loss, gd, gs


def loss_voxel(density, sem, label, lambda_s=1.0, lambda_o=1.0, out=None):
    """Voxel losses of the grid query (CE on the semantic voxels, BCE on the
    occupancy 1 - exp(-density)); labels int32, C = free, -1 = ignored.  Returns
    (loss[3] = total, semantic, occupancy; counts[2]; grad_density; grad_sem)."""
    V, C = sem.shape
    if out is None:
        out = (torch.empty(3, device=sem.device), torch.empty(2, dtype=torch.int32, device=sem.device),
               torch.empty_like(density), torch.empty_like(sem))
    loss, counts, gd, gs = out
    _check(lib.sq_loss_voxel(_ptr(density), _ptr(sem), _ptr(label), V, C, lambda_s, lambda_o, _ptr(loss),
                             _ptr(counts), _ptr(gd), _ptr(gs), _stream()), "sq_loss_voxel")
    return loss, counts, gd, gs


def count_pairs(index: Index, grid: dict, rays: Rays):
    """(Q, in-grid samples): pairs the forward evaluates over all L samples."""
    out = torch.zeros(2, dtype=torch.int64, device=index.v_n.device)
    g, r, ix = grid_struct(grid), rays.struct(), index.struct()
    _check(lib.sq_count_pairs(ctypes.byref(ix), ctypes.byref(g), ctypes.byref(r), _ptr(out), _stream()),
           "sq_count_pairs")
    q, s = out.tolist()
    return int(q), int(s)


def measure_sfu(op: str) -> float:
    """Measured SFU instructions per second on the current device for op in
    ("ex2", "lg2", "rcp") (host-synchronous, a few milliseconds)."""
    v = ctypes.c_double()
    _check(lib.sq_measure_sfu({"ex2": 0, "lg2": 1, "rcp": 2}[op], ctypes.byref(v), _stream()), "sq_measure_sfu")
    return float(v.value)


def check_query():
    """(compiled, site) of the debug build's bounds checks (sq_check_query): whether
    the loaded library has them, and the site of a failed check since the last
    query (0: none), which it clears.  Host-synchronous."""
    c, site = ctypes.c_int(), ctypes.c_int()
    _check(lib.sq_check_query(ctypes.byref(c), ctypes.byref(site)), "sq_check_query")
    return bool(c.value), int(site.value)


def profile_enable(on: bool = True):
    """Start (clearing earlier records) or stop timing every kernel launch of the library."""
    _check(lib.sq_profile_enable(1 if on else 0), "sq_profile_enable")


def profile_query(name: str | None = None):
    """(launches, total ms, dropped) of the recorded launches of kernel ``name``
    (None = every kernel); waits for the recorded events."""
    n, ms, dropped = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_longlong()
    _check(lib.sq_profile_query(None if name is None else name.encode(), ctypes.byref(n), ctypes.byref(ms),
                                ctypes.byref(dropped)), "sq_profile_query")
    return int(n.value), float(ms.value), int(dropped.value)


# Pages of saved state to reserve per (rays, samples, classes): learnt from the
# forwards so far (the first forward of a shape reserves every sample).
_SAVED_PAGES: dict = {}


class SQRender(torch.autograd.Function):
    """(means, quats, scales, eps, opacity, logits) -> (depth [R], sem [R, C]).

    The index and rays are constants of the call; the backward runs
    sq_render_bwd with the incoming cotangents.  The saved state is sized from
    the pages earlier forwards of the same shape needed (plus 5%); the backward
    reads the page count (one wait for the stream), remembers it, and if the
    pages ran out re-runs the forward into a large enough buffer first."""

    @staticmethod
    def forward(ctx, means, quats, scales, eps, opacity, logits, index: Index, grid: dict, rays: Rays):
        prims = dict(zip(PRIM_KEYS, (t.contiguous() for t in (means, quats, scales, eps, opacity, logits))))
        key = (rays.R, rays.t.numel(), logits.shape[1])
        saved = new_saved(rays, logits.shape[1], means.device, _SAVED_PAGES.get(key))
        depth, sem, _ = render_fwd(prims, index, grid, rays, saved=saved)
        ctx.save_for_backward(*[prims[k] for k in PRIM_KEYS], saved)
        ctx.index, ctx.grid, ctx.rays, ctx.key = index, grid, rays, key
        return depth, sem

    @staticmethod
    def backward(ctx, g_depth, g_sem):
        prims = dict(zip(PRIM_KEYS, ctx.saved_tensors[:6]))
        saved = ctx.saved_tensors[6]
        C = prims["logits"].shape[1]
        if g_depth is None:
            g_depth = torch.zeros(ctx.rays.R, device=prims["means"].device)
        if g_sem is None:
            g_sem = torch.zeros((ctx.rays.R, C), device=prims["means"].device)
        needed, status = saved_header(saved)
        _SAVED_PAGES[ctx.key] = max(_SAVED_PAGES.get(ctx.key, 0), needed + needed // 20 + 16)
        if status != SQ_OK:  # the pages ran out: the forward again into a buffer that holds them
            saved = new_saved(ctx.rays, C, prims["means"].device, _SAVED_PAGES[ctx.key])
            render_fwd(prims, ctx.index, ctx.grid, ctx.rays, saved=saved)
        g = render_bwd(prims, ctx.index, ctx.grid, ctx.rays, g_depth, g_sem, saved=saved)
        return (g["means"], g["quats"], g["scales"], g["eps"], g["opacity"], g["logits"], None, None, None)


def render(prims: dict, index: Index, grid: dict, rays: Rays):
    """Differentiable render of ``prims`` (tensors may require grad)."""
    return SQRender.apply(*[prims[k] for k in PRIM_KEYS], index, grid, rays)


def to_device(prims_np: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(prims_np[k], dtype=torch.float32).contiguous().to(device) for k in PRIM_KEYS}


# ------------------------------------------------------------------ batched scenes
class Scene:
    """One scene of a batch: its parameters, index, grid and rays plus the device
    buffers the batched forward and backward read and write."""

    def __init__(self, prims: dict, index: Index, grid: dict, rays: Rays, training: bool = True):
        device = prims["means"].device
        C = prims["logits"].shape[1]
        R = rays.R
        self.prims, self.index, self.grid, self.rays = prims, index, grid, rays
        self.depth = torch.empty(R, device=device)
        self.sem = torch.empty((R, C), device=device)
        self.t_final = torch.empty(R, device=device)
        self.saved = new_saved(rays, C, device) if training else None
        self.C = C
        self.grad_depth = torch.zeros(R, device=device) if training else None
        self.grad_sem = torch.zeros((R, C), device=device) if training else None
        self.grads = {k: torch.empty_like(prims[k]) for k in PRIM_KEYS} if training else None

    def fit_saved(self, slack: float = 0.05):
        """Shrinks the saved-state buffer to the pages the last forward needed plus
        ``slack`` (waits for the stream); returns its bytes."""
        needed, _ = saved_header(self.saved)
        self.saved = new_saved(self.rays, self.C, self.saved.device, int(needed * (1 + slack)) + 16)
        return self.saved.numel()

    def struct(self) -> SqScene:
        sc = SqScene()
        sc.prims = prims_struct(self.prims)
        sc.index = self.index.struct()
        sc.grid = grid_struct(self.grid)
        sc.rays = self.rays.struct()
        sc.depth, sc.sem, sc.t_final = _ptr(self.depth), _ptr(self.sem), _ptr(self.t_final)
        if self.saved is not None:
            sc.saved, sc.saved_bytes = _ptr(self.saved), self.saved.numel()
            sc.grad_depth, sc.grad_sem = _ptr(self.grad_depth), _ptr(self.grad_sem)
            for k in PRIM_KEYS:
                setattr(sc, "g_" + k, _ptr(self.grads[k]))
        return sc


def _scene_array(scenes):
    arr = (SqScene * len(scenes))(*[s.struct() for s in scenes])
    return arr


def batched_workspace_size(scenes) -> int:
    arr = _scene_array(scenes)
    return int(lib.sq_batched_workspace_size(arr, len(scenes)))


def render_batched(op: int, scenes, tuning: dict | None = None):
    """One persistent launch over all scenes (op = SQ_OP_FWD or SQ_OP_BWD)."""
    arr = _scene_array(scenes)
    device = scenes[0].prims["means"].device
    ws = _ws.get("batched", lib.sq_batched_workspace_size(arr, len(scenes)), device)
    tn = None if tuning is None else SqTuning(tuning["fwd_lanes_per_ray"], tuning["fwd_warps_per_cta"],
                                              tuning["bwd_warps_per_cta"], tuning.get("bwd_order", SQ_BWD_DEFAULT),
                                              tuning.get("fwd_ray_tile", 1))
    _check(lib.sq_render_batched(op, arr, len(scenes), ctypes.byref(tn) if tn else None, _ptr(ws), ws.numel(),
                                 _stream()), "sq_render_batched")


TUNING_CACHE = os.path.join(_PKG, "_lib", "autotune.json")


def batch_signature(scenes) -> str:
    """Workload key for the tuning cache: scene sizes, rays, samples, classes."""
    parts = [f"{s.prims['means'].shape[0]}x{s.rays.R}x{s.rays.t.numel()}" for s in scenes]
    return f"C{scenes[0].prims['logits'].shape[1]}:" + ",".join(parts)


def autotune(scenes, reps: int = 3, use_cache: bool = True) -> dict:
    """Picks the fastest launch configuration for this batch with sq_autotune and
    caches it (JSON next to the library) under the batch signature."""
    import json
    key = batch_signature(scenes)
    cache = {}
    if use_cache and os.path.exists(TUNING_CACHE):
        try:
            cache = json.load(open(TUNING_CACHE))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return cache[key]
    arr = _scene_array(scenes)
    device = scenes[0].prims["means"].device
    ws = _ws.get("batched", lib.sq_batched_workspace_size(arr, len(scenes)), device)
    best = SqTuning()
    fms = (ctypes.c_float * 8)()
    bms = (ctypes.c_float * 4)()
    _check(lib.sq_autotune(arr, len(scenes), _ptr(ws), ws.numel(), _stream(), reps, ctypes.byref(best), fms, bms),
           "sq_autotune")
    out = {"fwd_lanes_per_ray": best.fwd_lanes_per_ray, "fwd_warps_per_cta": best.fwd_warps_per_cta,
           "bwd_warps_per_cta": best.bwd_warps_per_cta, "bwd_order": best.bwd_order,
           "fwd_ray_tile": best.fwd_ray_tile, "fwd_ms": list(fms),
           "bwd_ms": list(bms)}
    if use_cache:
        cache[key] = out
        try:
            os.makedirs(os.path.dirname(TUNING_CACHE), exist_ok=True)
            with open(TUNING_CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return out
