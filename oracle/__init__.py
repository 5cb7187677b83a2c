"""FP64 CPU oracle of the superquadric volume renderer -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  It wraps ``sqr_oracle.c`` (plain C, FP64,
OpenMP over rays), which shares nothing with the CUDA library.  See the header
of ``sqr_oracle.c`` for what each function computes and which equation of the
paper it restates.

All inputs are the same FP32 arrays the CUDA path receives (from
``paper_2511_17361_gb300.synth``); outputs are FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sqr_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so FP32 rules are exact)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", _SRC, "-lm"]
    tmp = _OUT + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_sq_f.restype = ctypes.c_double
            _lib.orc_sq_p.restype = ctypes.c_double
            _lib.orc_ranges.restype = ctypes.c_longlong
            _lib.orc_index.restype = ctypes.c_longlong
            _lib.orc_render_fwd.restype = ctypes.c_int
            _lib.orc_render_bwd.restype = ctypes.c_int
            _lib.orc_query_grid.restype = ctypes.c_int
            _lib.orc_trace_ray.restype = ctypes.c_int
            _lib.orc_max_threads.restype = ctypes.c_int
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _grid_args(grid):
    gn = np.asarray(grid["n"], np.int32)
    return gn, _f32(grid["lo"]), _f32(grid["vs"])


def max_threads() -> int:
    return _load().orc_max_threads()


# ----------------------------------------------------------------------- Eq. 1-2
def sq_f(xl, s, e1, e2) -> float:
    """Eq. 1 at a canonical-frame point."""
    xl = np.ascontiguousarray(xl, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    return _load().orc_sq_f(_p(xl), _p(s), ctypes.c_double(e1), ctypes.c_double(e2))


def sq_p(x, m, q, s, e1, e2) -> float:
    """Eq. 2 at a world point."""
    arr = [np.ascontiguousarray(a, np.float64) for a in (x, m, q, s)]
    return _load().orc_sq_p(*[_p(a) for a in arr], ctypes.c_double(e1), ctypes.c_double(e2))


# ----------------------------------------------------------------------- index
def ranges(prims, grid, mode=0, tau_cut=0.01, nv=5):
    """Per-primitive voxel box (i0,i1,j0,j1,k0,k1) and the near-tie count; mode 0
    OBB, 1 cube, 2 opacity-aware OBB."""
    n = prims["means"].shape[0]
    out = np.zeros((n, 6), np.int32)
    gn, glo, gvs = _grid_args(grid)
    P = prims
    ties = _load().orc_ranges(ctypes.c_int(n), _p(_f32(P["means"])), _p(_f32(P["quats"])), _p(_f32(P["scales"])),
                              _p(_f32(P["eps"])), _p(_f32(P["opacity"])), _p(gn), _p(glo), _p(gvs),
                              ctypes.c_int(mode), ctypes.c_float(tau_cut), ctypes.c_int(nv), _p(out))
    return out, int(ties)


def build_index(prims, grid, mode=0, tau_cut=0.01, nv=5) -> dict:
    """Voxel -> primitive lists (v_n, v_f, v_sq) walked in primitive-id order."""
    rg, ties = ranges(prims, grid, mode, tau_cut, nv)
    gn = np.asarray(grid["n"], np.int32)
    nvox = int(np.prod(grid["n"]))
    v_n = np.zeros(nvox, np.int32)
    v_f = np.zeros(nvox, np.int32)
    lib = _load()
    P = lib.orc_index(ctypes.c_int(rg.shape[0]), _p(rg), _p(gn), _p(v_n), _p(v_f), None, ctypes.c_longlong(0))
    v_sq = np.zeros(max(int(P), 1), np.int32)
    lib.orc_index(ctypes.c_int(rg.shape[0]), _p(rg), _p(gn), _p(v_n), _p(v_f), _p(v_sq), ctypes.c_longlong(P))
    return {"v_n": v_n, "v_f": v_f, "v_sq": v_sq[:P], "ranges": rg, "P": int(P), "ties": ties}


# ----------------------------------------------------------------------- render
def _softmax_rows(x):
    x = np.asarray(x, np.float32).astype(np.float64)  # the parameters are FP32
    e = np.exp(x - x.max(1, keepdims=True))
    return e / e.sum(1, keepdims=True)


def _semantic(prims, sem_mode):
    """The prims as the renderer sees them, class vectors in FP64: the FP32 logits
    (sem_mode 0, Eq. 4) or, with sem_mode 1 (per-primitive softmax), every
    primitive's softmax over the classes of those logits."""
    out = dict(prims)
    if sem_mode == 0:
        out["logits"] = np.asarray(prims["logits"], np.float32).astype(np.float64)
    else:
        assert sem_mode == 1, sem_mode
        out["logits"] = _softmax_rows(prims["logits"])
    return out


def _logit_grad(prims, sem_mode, g):
    """Logit gradient w.r.t. the raw logits: through s = softmax(c), s * (g - <g, s>)."""
    if sem_mode == 0:
        return g
    s = _softmax_rows(prims["logits"])
    return s * (g - (g * s).sum(1, keepdims=True))


def _scene_args(prims, grid, index, rig, t):
    P = prims
    n, C = P["logits"].shape
    gn, glo, gvs = _grid_args(grid)
    v_sq = index["v_sq"] if index["v_sq"].size else np.zeros(1, np.int32)
    keep = [_f32(P["means"]), _f32(P["quats"]), _f32(P["scales"]), _f32(P["eps"]), _f32(P["opacity"]),
            _f64(P["logits"]), gn, glo, gvs, _i32(index["v_n"]), _i32(index["v_f"]), _i32(v_sq),
            _f32(rig["K"]), _f32(rig["cam2world"]), _f32(t)]
    args = [ctypes.c_int(n), ctypes.c_int(C)] + [_p(a) for a in keep[:12]] + [
        ctypes.c_int(rig["n_cam"]), ctypes.c_int(rig["H"]), ctypes.c_int(rig["W"]), _p(keep[12]), _p(keep[13]),
        ctypes.c_int(len(t)), _p(keep[14])]
    return args, keep, C


def render_fwd(prims, grid, index, rig, t, kappa=0.0, alpha_max=1.0, ray_ids=None, threads=0, sem_mode=0):
    """Eq. 4-6 per ray: returns depth [R], sem [R, C], t_final [R], n_used [R]."""
    args, keep, C = _scene_args(_semantic(prims, sem_mode), grid, index, rig, t)
    R = rig["n_cam"] * rig["H"] * rig["W"] if ray_ids is None else len(ray_ids)
    ids = None if ray_ids is None else np.ascontiguousarray(ray_ids, np.int64)
    depth = np.zeros(R); sem = np.zeros((R, C)); tf = np.zeros(R); nu = np.zeros(R, np.int32)
    _load().orc_render_fwd(*args, ctypes.c_double(kappa), ctypes.c_double(alpha_max), _p(ids), ctypes.c_longlong(R),
                           _p(depth), _p(sem), _p(tf), _p(nu), ctypes.c_int(threads))
    return depth, sem, tf, nu


def render_bwd(prims, grid, index, rig, t, grad_depth, grad_sem, kappa=0.0, alpha_max=1.0, ray_ids=None, threads=0,
               sem_mode=0):
    """Gradient of sum(gD*D) + sum(gS*S) over the listed rays w.r.t. every parameter."""
    raw = prims
    prims = _semantic(prims, sem_mode)
    args, keep, C = _scene_args(prims, grid, index, rig, t)
    n = prims["means"].shape[0]
    R = rig["n_cam"] * rig["H"] * rig["W"] if ray_ids is None else len(ray_ids)
    ids = None if ray_ids is None else np.ascontiguousarray(ray_ids, np.int64)
    gd = np.ascontiguousarray(grad_depth, np.float64).reshape(R)
    gs = np.ascontiguousarray(grad_sem, np.float64).reshape(R, C)
    out = {"means": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "scales": np.zeros((n, 3)), "eps": np.zeros((n, 2)),
           "opacity": np.zeros(n), "logits": np.zeros((n, C))}
    _load().orc_render_bwd(*args, ctypes.c_double(kappa), ctypes.c_double(alpha_max), _p(ids), ctypes.c_longlong(R),
                           _p(gd), _p(gs), _p(out["means"]), _p(out["quats"]), _p(out["scales"]), _p(out["eps"]),
                           _p(out["opacity"]), _p(out["logits"]), ctypes.c_int(threads))
    out["logits"] = _logit_grad(raw, sem_mode, out["logits"])
    return out


def trace_ray(prims, grid, index, rig, t, ray, kappa=0.0, alpha_max=1.0, sem_mode=0):
    """Per-sample alpha, raw sum, T (length L+1), voxel ids and FP32 positions of one ray."""
    args, keep, C = _scene_args(_semantic(prims, sem_mode), grid, index, rig, t)
    L = len(t)
    alpha = np.zeros(L); ssum = np.zeros(L); T = np.zeros(L + 1); vox = np.zeros(L, np.int64)
    xyz = np.zeros((L, 3), np.float32)
    used = _load().orc_trace_ray(*args, ctypes.c_double(kappa), ctypes.c_double(alpha_max), ctypes.c_longlong(ray),
                                 _p(alpha), _p(ssum), _p(T), _p(vox), _p(xyz))
    return {"alpha": alpha, "ssum": ssum, "T": T, "vox": vox, "xyz": xyz, "used": used}


def query_grid_bwd(prims, grid, index, grad_density, grad_sem, voxel_ids=None, sem_mode=0):
    """Gradient of sum(gd * density) + sum(gs * sem) of the grid query over the
    listed voxels (None: all, gd/gs in voxel order) w.r.t. every parameter."""
    raw = prims
    P = prims = _semantic(prims, sem_mode)
    n, C = P["logits"].shape
    gn, glo, gvs = _grid_args(grid)
    nvox = int(np.prod(grid["n"]))
    V = nvox if voxel_ids is None else len(voxel_ids)
    ids = None if voxel_ids is None else np.ascontiguousarray(voxel_ids, np.int64)
    v_sq = index["v_sq"] if index["v_sq"].size else np.zeros(1, np.int32)
    keep = [_f32(P["means"]), _f32(P["quats"]), _f32(P["scales"]), _f32(P["eps"]), _f32(P["opacity"]),
            _f64(P["logits"]), gn, glo, gvs, _i32(index["v_n"]), _i32(index["v_f"]), _i32(v_sq)]
    gd = np.ascontiguousarray(grad_density, np.float64).reshape(V)
    gs = np.ascontiguousarray(grad_sem, np.float64).reshape(V, C)
    out = {"means": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "scales": np.zeros((n, 3)), "eps": np.zeros((n, 2)),
           "opacity": np.zeros(n), "logits": np.zeros((n, C))}
    _load().orc_query_grid_bwd(ctypes.c_int(n), ctypes.c_int(C), *[_p(a) for a in keep], _p(ids),
                               ctypes.c_longlong(V), _p(gd), _p(gs), _p(out["means"]), _p(out["quats"]),
                               _p(out["scales"]), _p(out["eps"]), _p(out["opacity"]), _p(out["logits"]))
    out["logits"] = _logit_grad(raw, sem_mode, out["logits"])
    return out


def ray_samples(K, c2w, u, v, t, grid):
    """FP32 sample positions and voxel ids (-1 outside) of pixel (u, v)."""
    gn, glo, gvs = _grid_args(grid)
    t = _f32(t)
    L = len(t)
    xyz = np.zeros((L, 3), np.float32)
    vox = np.zeros(L, np.int64)
    _load().orc_ray_samples(_p(_f32(K)), _p(_f32(c2w)), ctypes.c_int(u), ctypes.c_int(v), ctypes.c_int(L), _p(t),
                            _p(gn), _p(glo), _p(gvs), _p(xyz), _p(vox))
    return xyz, vox


def sample_voxels(rig, t, grid, threads=0):
    """Voxel id (-1 outside) of every sample of every ray: int32 [R, L]."""
    gn, glo, gvs = _grid_args(grid)
    t = _f32(t)
    R = rig["n_cam"] * rig["H"] * rig["W"]
    vox = np.zeros((R, len(t)), np.int32)
    _load().orc_sample_voxels(ctypes.c_int(rig["n_cam"]), ctypes.c_int(rig["H"]), ctypes.c_int(rig["W"]),
                              _p(_f32(rig["K"])), _p(_f32(rig["cam2world"])), ctypes.c_int(len(t)), _p(t), _p(gn),
                              _p(glo), _p(gvs), _p(vox), ctypes.c_int(threads))
    return vox


def query_grid(prims, grid, index, tau=0.05, voxel_ids=None, threads=0, sem_mode=0):
    """Supp. A.4 voxelisation: density [V], sem [V, C], label [V] (C = free)."""
    P = _semantic(prims, sem_mode)
    n, C = P["logits"].shape
    gn, glo, gvs = _grid_args(grid)
    nvox = int(np.prod(grid["n"]))
    V = nvox if voxel_ids is None else len(voxel_ids)
    ids = None if voxel_ids is None else np.ascontiguousarray(voxel_ids, np.int64)
    v_sq = index["v_sq"] if index["v_sq"].size else np.zeros(1, np.int32)
    keep = [_f32(P["means"]), _f32(P["quats"]), _f32(P["scales"]), _f32(P["eps"]), _f32(P["opacity"]),
            _f64(P["logits"]), gn, glo, gvs, _i32(index["v_n"]), _i32(index["v_f"]), _i32(v_sq)]
    dens = np.zeros(V); sem = np.zeros((V, C)); lab = np.zeros(V, np.int32)
    _load().orc_query_grid(ctypes.c_int(n), ctypes.c_int(C), *[_p(a) for a in keep], ctypes.c_double(tau), _p(ids),
                           ctypes.c_longlong(V), _p(dens), _p(sem), _p(lab), ctypes.c_int(threads))
    return dens, sem, lab


def voxel_loss(density, sem, label, lambda_s=1.0, lambda_o=1.0, d_min=1e-6):
    """Voxel losses of the grid query (Supp. A.4 / A.5: cross-entropy on the
    semantic voxels, binary cross-entropy on the density voxels), in FP64.

    Labels: 0..C-1 occupied voxel of that class, C free, -1 ignored.  The density
    d = max(v_d, 0) enters the BCE through the occupancy probability
    p = 1 - exp(-d); free voxels cost -log(1 - p) = d, occupied ones
    -log(p) with d clamped below at d_min (zero gradient under the clamp).  The
    CE is averaged over occupied voxels, the BCE over labelled ones.

    Returns (total, semantic term, occupancy term, grad_density, grad_sem)."""
    d_raw = np.asarray(density, np.float64)
    s = np.asarray(sem, np.float64)
    y = np.asarray(label, np.int64)
    V, C = s.shape
    occ = (y >= 0) & (y < C)
    free = y == C
    n_occ, n_lab = int(occ.sum()), int((occ | free).sum())
    ws = lambda_s / n_occ if n_occ else 0.0
    wo = lambda_o / n_lab if n_lab else 0.0
    gs = np.zeros_like(s)
    ce = 0.0
    if n_occ:
        so = s[occ]
        mx = so.max(1, keepdims=True)
        e = np.exp(so - mx)
        z = e.sum(1, keepdims=True)
        yo = y[occ]
        ce = float(np.sum(mx[:, 0] + np.log(z[:, 0]) - so[np.arange(len(yo)), yo]))
        g = e / z
        g[np.arange(len(yo)), yo] -= 1.0
        gs[occ] = ws * g
    d = np.maximum(d_raw, 0.0)
    gd = np.zeros_like(d)
    bce = float(np.sum(d[free]))
    gd[free] = np.where(d_raw[free] > 0.0, wo, 0.0)
    dc = np.maximum(d[occ], d_min)
    bce += float(np.sum(-np.log(-np.expm1(-dc))))
    gd[occ] = np.where(d[occ] > d_min, -wo / np.expm1(np.maximum(d[occ], d_min)), 0.0)
    return ws * ce + wo * bce, ws * ce, wo * bce, gd, gs
