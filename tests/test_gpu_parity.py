"""CUDA path vs the FP64 oracle on the same seeded inputs (needs a GPU).

Index contents are compared bit for bit; renders, grid queries and gradients
element by element at the tolerances in tests/gpu_common.py.  Small workloads
are compared in full; the 540,000-ray frames on sampled rays (sparse
cotangents for the backward), which the oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_17361_gb300 import synth
from tests.gpu_common import (assert_index_equal, check_depth, check_grad, check_sem, dev_grid, lib, np_index,
                              oracle_index, scene_to_gpu)
from tests.helpers import prims_from, small_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    return lib()


def _index_pair(sqr, cfg, mode=0, tau=0.01, nv=5):
    prims_d = sqr.to_device(cfg["prims"])
    ix = sqr.build_index(prims_d, dev_grid(cfg["grid"]), mode=mode, tau_cut=tau, nv=nv, flags=True)
    ref = oracle.build_index(cfg["prims"], cfg["grid"], mode, tau, nv)
    return prims_d, ix, ref


def _assert_index_equal(ix, ref):
    assert_index_equal(ix, ref)


# ----------------------------------------------------------------------- index
@pytest.mark.parametrize("ci", [0, 1, 2, 4])
def test_index_bit_exact(sqr, ci):
    cfg = synth.make_config(ci)
    _, ix, ref = _index_pair(sqr, cfg)
    _assert_index_equal(ix, ref)


def test_index_bit_exact_batch_and_horizon_scenes(sqr):
    """The 12 scenes of the uneven batch and the 13 frames of the temporal horizon."""
    for c in synth.make_batch_config(3) + synth.make_temporal_config():
        _, ix, ref = _index_pair(sqr, c)
        _assert_index_equal(ix, ref)


@pytest.mark.parametrize("ci", [0, 1])
def test_index_opacity_mode_bit_exact(sqr, ci):
    """Opacity-aware OBB index (the paper's future-work refinement): identical to
    the oracle's, and smaller than the plain OBB index."""
    cfg = synth.make_config(ci)
    _, ix, ref = _index_pair(sqr, cfg, mode=2)
    _assert_index_equal(ix, ref)
    assert ref["P"] < oracle.build_index(cfg["prims"], cfg["grid"])["P"]


def test_index_cube_mode_bit_exact(sqr):
    cfg = synth.make_config(0)
    _, ix, ref = _index_pair(sqr, cfg, mode=1, nv=5)
    _assert_index_equal(ix, ref)


def test_index_long_lists_sorted(sqr):
    """Lists longer than a warp (33..2000 entries) take the shared- and global-memory
    sort paths; still identical to the oracle."""
    rng = np.random.default_rng(5)
    for n in (40, 300, 2000):
        pr = prims_from(rng.uniform(0, 4, (n, 3)), rng.standard_normal((n, 4)), rng.uniform(0.5, 3.0, (n, 3)),
                        rng.uniform(0.3, 1.8, (n, 2)), rng.uniform(0, 1, n), rng.standard_normal((n, 3)))
        grid = synth.grid_spec(4, 3, 2, lo=(0, 0, 0), hi=(4, 3, 2))
        _, ix, ref = _index_pair(sqr, {"prims": pr, "grid": grid})
        _assert_index_equal(ix, ref)
        assert ref["v_n"].max() > 32


def test_index_empty_and_outside(sqr):
    """N = 0, and primitives entirely outside the grid, give empty lists."""
    grid = synth.grid_spec(5, 5, 5, lo=(0, 0, 0), hi=(5, 5, 5))
    pr = prims_from([[50, 50, 50], [-30, 2, 2]], [[1, 0, 0, 0]] * 2, [[1, 1, 1]] * 2, [[1, 1]] * 2, [0.5] * 2,
                    np.zeros((2, 3)))
    _, ix, ref = _index_pair(sqr, {"prims": pr, "grid": grid})
    _assert_index_equal(ix, ref)
    assert ref["P"] == 0
    pr0 = prims_from(np.zeros((0, 3)), np.zeros((0, 4)), np.zeros((0, 3)), np.zeros((0, 2)), np.zeros(0),
                     np.zeros((0, 3)))
    _, ix0, ref0 = _index_pair(sqr, {"prims": pr0, "grid": grid})
    assert ix0.P() == 0 and np.all(ix0.v_n.cpu().numpy() == 0)


def _expected_flags(ix):
    """Range-boundary flags of every index entry, from their definition: per axis
    a, bit 4a: lo == v, 4a+1: lo == v - 1, 4a+2: hi == v, 4a+3: hi == v + 1, for
    the entry's voxel v and its primitive's voxel range."""
    ny, nz = int(ix.grid["n"][1]), int(ix.grid["n"][2])
    got = np_index(ix)
    vox = np.repeat(np.arange(len(got["v_n"]), dtype=np.int64), got["v_n"])
    coords = (vox // (ny * nz), (vox // nz) % ny, vox % nz)
    r = got["ranges"][got["v_sq"]]
    f = np.zeros(got["P"], np.int64)
    for a, c in enumerate(coords):
        lo, hi = r[:, 2 * a].astype(np.int64), r[:, 2 * a + 1].astype(np.int64)
        f |= ((lo == c) * 1 | (lo == c - 1) * 2 | (hi == c) * 4 | (hi == c + 1) * 8) << (4 * a)
    return f


@pytest.mark.parametrize("ci", [0, 2])
def test_index_boundary_flags(sqr, ci):
    """The optional per-entry flags equal their definition, bit for bit."""
    cfg = synth.make_config(ci)
    _, ix, _ = _index_pair(sqr, cfg)
    P = ix.P()
    got = ix.v_flags[:P].cpu().numpy().astype(np.int64) & 0xFFFF
    assert np.array_equal(got, _expected_flags(ix))
    assert np.count_nonzero(got) > 0


def test_index_boundary_flags_long_lists(sqr):
    rng = np.random.default_rng(7)
    n = 1500
    pr = prims_from(rng.uniform(0, 4, (n, 3)), rng.standard_normal((n, 4)), rng.uniform(0.2, 1.5, (n, 3)),
                    rng.uniform(0.3, 1.8, (n, 2)), rng.uniform(0, 1, n), rng.standard_normal((n, 3)))
    grid = synth.grid_spec(8, 6, 4, lo=(0, 0, 0), hi=(4, 3, 2))
    _, ix, _ = _index_pair(sqr, {"prims": pr, "grid": grid})
    got = ix.v_flags[:ix.P()].cpu().numpy().astype(np.int64) & 0xFFFF
    assert np.array_equal(got, _expected_flags(ix))
    assert np_index(ix)["v_n"].max() > 32


def test_index_capacity_overflow_reported(sqr):
    """Too small a V_sq: status = SQ_ERR_CAPACITY and p_total = the needed size."""
    cfg = synth.make_config(0)
    prims_d = sqr.to_device(cfg["prims"])
    ix = sqr.build_index(prims_d, dev_grid(cfg["grid"]), capacity=1000, sync=False)
    torch.cuda.synchronize()
    assert int(ix.status.item()) == sqr.SQ_ERR_CAPACITY
    ref = oracle.build_index(cfg["prims"], cfg["grid"])
    assert ix.P() == ref["P"]
    with pytest.raises(sqr.SqrError):
        ix.check()
    # render on an overflowed index does no work (outputs left as given)
    rays = sqr.Rays.from_rig(cfg["rig"], cfg["t"])
    depth = torch.full((rays.R,), -7.0, device="cuda")
    sem = torch.zeros((rays.R, 18), device="cuda")
    tf = torch.zeros(rays.R, device="cuda")
    sqr.render_fwd(prims_d, ix, dev_grid(cfg["grid"]), rays, out=(depth, sem, tf))
    assert torch.all(depth == -7.0)
    # the auto-growing path recovers
    ix2 = sqr.build_index(prims_d, dev_grid(cfg["grid"]), capacity=1000)
    _assert_index_equal(ix2, ref)


@pytest.mark.parametrize("field,index,value", [("scales", (7, 1), float("nan")), ("scales", (3, 0), 0.0),
                                               ("eps", (5, 0), 2.5), ("eps", (9, 1), -0.1),
                                               ("quats", (2, slice(None)), 0.0), ("means", (4, 2), float("inf")),
                                               ("opacity", (11,), float("nan")), ("logits", (6, 17), float("-inf"))])
def test_index_numeric_status(sqr, field, index, value):
    """A parameter outside its domain (set on the host): the index build reports
    SQ_ERR_NUMERIC (over a capacity overflow too), the forward leaves its outputs
    untouched, the backward and the query backward return zero gradients, and the
    grid query writes nothing."""
    cfg = synth.make_config(0)
    pr = {k: v.copy() for k, v in cfg["prims"].items()}
    pr[field][index] = value
    prims_d = sqr.to_device(pr)
    g = dev_grid(cfg["grid"])
    for cap in (None, 1000):
        ix = sqr.build_index(prims_d, g, capacity=cap, sync=False)
        torch.cuda.synchronize()
        assert int(ix.status.item()) == sqr.SQ_ERR_NUMERIC
    with pytest.raises(sqr.SqrError, match="NUMERIC"):
        sqr.build_index(prims_d, g)
    rays = sqr.Rays.from_rig(cfg["rig"], cfg["t"])
    depth = torch.full((rays.R,), -7.0, device="cuda")
    sem = torch.full((rays.R, 18), 3.0, device="cuda")
    tf = torch.full((rays.R,), 5.0, device="cuda")
    saved = sqr.new_saved(rays, 18)
    sqr.render_fwd(prims_d, ix, g, rays, out=(depth, sem, tf), saved=saved)
    torch.cuda.synchronize()
    assert torch.all(depth == -7.0) and torch.all(sem == 3.0) and torch.all(tf == 5.0)
    gd, gs = torch.ones(rays.R, device="cuda"), torch.ones((rays.R, 18), device="cuda")
    for order in (sqr.SQ_BWD_DEFAULT, sqr.SQ_BWD_RAY_MAJOR):
        grads = {k: torch.full_like(prims_d[k], 9.0) for k in sqr.PRIM_KEYS}
        sqr.render_bwd(prims_d, ix, g, rays, gd, gs, saved=saved, out=grads, order=order)
        torch.cuda.synchronize()
        assert all(torch.all(v == 0.0) for v in grads.values())
    nvox = ix.v_n.numel()
    dens = torch.full((nvox,), -1.0, device="cuda")
    qs = torch.full((nvox, 18), -1.0, device="cuda")
    sqr.query_grid(prims_d, ix, g, out=(dens, qs, None))
    qg = sqr.query_grid_bwd(prims_d, ix, g, torch.ones(nvox, device="cuda"), torch.ones((nvox, 18), device="cuda"))
    torch.cuda.synchronize()
    assert torch.all(dens == -1.0) and torch.all(qs == -1.0)
    assert all(torch.all(v == 0.0) for v in qg.values())


# ----------------------------------------------------------------------- forward
def _fwd_pair(sqr, prims, grid, rig, t, kappa=0.0, alpha_max=1.0, ray_ids=None, mode=0, tau=0.01, nv=5):
    prims_d, rays = scene_to_gpu(sqr, prims, rig, t, kappa, alpha_max)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g, mode=mode, tau_cut=tau, nv=nv)
    depth, sem, tf = sqr.render_fwd(prims_d, ix, g, rays)
    torch.cuda.synchronize()
    ref_ix = oracle_index(ix, prims, grid, mode, tau, nv)
    D, S, T, NU = oracle.render_fwd(prims, grid, ref_ix, rig, t, kappa, alpha_max, ray_ids=ray_ids)
    sel = slice(None) if ray_ids is None else np.asarray(ray_ids)
    return depth.cpu().numpy()[sel], sem.cpu().numpy()[sel], tf.cpu().numpy()[sel], D, S, T, NU


def test_forward_small_workload_full(sqr):
    cfg = synth.make_config(0)
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"])
    check_depth(d, D, 0.5)
    check_sem(s, S)
    assert np.max(np.abs(tf - T)) < 1e-5
    # transmittance identity on the GPU side: sum w + T = 1 is implied by D, T
    assert np.all((tf >= 0) & (tf <= 1))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forward_ragged_small_scenes(sqr, seed):
    """Odd image sizes (ragged warps and tiles), several class counts."""
    C = [5, 3, 18][seed]
    pr, grid, rig, t = small_scene(seed, n=9, H=7, W=13, L=[24, 33, 48][seed], C=C, sigma_max=0.9)
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, pr, grid, rig, t)
    check_depth(d, D, 0.5)
    check_sem(s, S)
    assert np.max(np.abs(tf - T)) < 1e-5


def test_forward_clamp_active(sqr):
    """Dense overlapping primitives: alpha = min(sum, 1) saturates."""
    pr, grid, rig, t = small_scene(4, n=12, sigma_max=3.0, s_range=(1.0, 2.5))
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, pr, grid, rig, t)
    check_depth(d, D, 0.5)
    check_sem(s, S)
    assert np.any(T == 0.0)


def test_forward_heavy_voxels(sqr):
    """Voxel lists longer than a chunk's pair buffer (> 256 primitives)."""
    rng = np.random.default_rng(9)
    n = 400
    pr = prims_from(np.c_[rng.uniform(2, 6, n), rng.uniform(-1, 1, n), rng.uniform(0, 2, n)],
                    rng.standard_normal((n, 4)), rng.uniform(0.5, 2.0, (n, 3)), rng.uniform(0.3, 1.8, (n, 2)),
                    rng.uniform(0.0, 0.02, n), rng.standard_normal((n, 4)))
    grid = synth.grid_spec(4, 4, 2, lo=(-8, -8, -1), hi=(8, 8, 3))
    rig = synth.rig_single(H=5, W=9, f=6.0, centre=(-1.0, 0.0, 1.0))
    t = synth.sample_depths(30, 0.5, 9.5)
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, pr, grid, rig, t)
    check_depth(d, D, 0.5)
    check_sem(s, S)


def test_forward_early_termination(sqr):
    """kappa > 0: rays stop after T < kappa; compared on rays whose T is not within
    1e-4 (relative) of kappa at any sample."""
    cfg = synth.make_config(0)
    kappa = 1e-2
    d, s, tf, D, S, T, NU = _fwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], kappa=kappa)
    assert (NU < 48).any()
    ok = np.ones(len(D), bool)
    ix_ref = oracle.build_index(cfg["prims"], cfg["grid"])
    for r in np.flatnonzero(NU < 48):
        tr = oracle.trace_ray(cfg["prims"], cfg["grid"], ix_ref, cfg["rig"], cfg["t"], r, kappa=kappa)
        if np.any(np.abs(tr["T"][:tr["used"] + 1] - kappa) < 1e-4 * kappa):
            ok[r] = False
    check_depth(d[ok], D[ok], 0.5)
    check_sem(s[ok], S[ok])


@pytest.mark.parametrize("ci", [1, 2])
def test_forward_full_frame_sampled_rays(sqr, ci):
    """Six-camera 225x400 frames (540,000 rays), 3000 sampled rays vs the oracle."""
    cfg = synth.make_config(ci)
    R = synth.n_rays(cfg["rig"])
    rng = np.random.default_rng(ci)
    rays = np.unique(np.r_[rng.integers(0, R, 2990), [0, R - 1, 399, 400, 90000, 89999]])
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], ray_ids=rays)
    check_depth(d, D, 0.5)
    check_sem(s, S)
    assert np.max(np.abs(tf - T)) < 2e-5


def test_forward_cube_index(sqr):
    cfg = synth.make_config(0)
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], mode=1, nv=3)
    check_depth(d, D, 0.5)
    check_sem(s, S)


# ----------------------------------------------------------------------- backward
@pytest.fixture(params=["ray_major", "primitive_major"])
def bwd_order(request, sqr):
    """Both backward orders (Sec. 3.3.3): ray-major run walk, primitive-major tiles."""
    return {"ray_major": sqr.SQ_BWD_RAY_MAJOR, "primitive_major": sqr.SQ_BWD_PRIMITIVE_MAJOR}[request.param]


def _bwd_pair(sqr, prims, grid, rig, t, gd, gs, ray_ids=None, alpha_max=1.0, kappa=0.0, flags=True, mode=0,
              order=0):
    prims_d, rays = scene_to_gpu(sqr, prims, rig, t, kappa, alpha_max)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g, mode=mode, flags=flags)
    R = rays.R
    gd_full = np.zeros(R, np.float32)
    gs_full = np.zeros((R, prims["logits"].shape[1]), np.float32)
    sel = np.arange(R) if ray_ids is None else np.asarray(ray_ids)
    gd_full[sel] = gd
    gs_full[sel] = gs
    out = sqr.render_bwd(prims_d, ix, g, rays, torch.from_numpy(gd_full).cuda(), torch.from_numpy(gs_full).cuda(),
                         order=order)
    torch.cuda.synchronize()
    ref = oracle.render_bwd(prims, grid, oracle_index(ix, prims, grid, mode), rig, t, gd_full[sel].astype(np.float64),
                            gs_full[sel].astype(np.float64), alpha_max=alpha_max, kappa=kappa,
                            ray_ids=None if ray_ids is None else sel)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_small_scene_full(sqr, seed, bwd_order):
    """Every gradient of a small scene, for 5, 18 and 32 classes (the logit
    gradients of 32 classes span two 32-lane blocks of the accumulator)."""
    pr, grid, rig, t = small_scene(seed, n=8, H=9, W=11, L=32, C=[5, 18, 32][seed], sigma_max=0.6)
    R = 9 * 11
    rng = np.random.default_rng(seed)
    gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, pr["logits"].shape[1])).astype(
        np.float32)
    got, ref = _bwd_pair(sqr, pr, grid, rig, t, gd, gs, order=bwd_order)
    for k in ref:
        check_grad(got[k], ref[k], k)


@pytest.mark.parametrize("flags", [True, False])
def test_backward_long_sample_steps(sqr, flags, bwd_order):
    """Samples several voxels apart (run starts then come from a test of each list
    entry's range, not from the boundary flags), with and without the index's
    flags; and the default spacing without flags."""
    pr, grid, rig, t = small_scene(9, n=10, H=8, W=10, L=10, gn=(64, 64, 16))
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(9)
    gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, 5)).astype(np.float32)
    got, ref = _bwd_pair(sqr, pr, grid, rig, t, gd, gs, flags=flags, order=bwd_order)
    assert np.count_nonzero(ref["opacity"]) > 3
    for k in ref:
        check_grad(got[k], ref[k], k)
    if not flags:
        pr, grid, rig, t = small_scene(10, n=8, H=9, W=11, L=32)
        R = rig["H"] * rig["W"]
        gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, 5)).astype(np.float32)
        got, ref = _bwd_pair(sqr, pr, grid, rig, t, gd, gs, flags=False, order=bwd_order)
        for k in ref:
            check_grad(got[k], ref[k], k)


def test_render_with_opacity_index(sqr, bwd_order):
    """Forward and backward over the opacity-aware index, against the oracle
    rendering the same index."""
    cfg = synth.make_config(0)
    d, s, tf, D, S, T, _ = _fwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], mode=2)
    check_depth(d, D, 0.5)
    check_sem(s, S)
    pr, grid, rig, t = small_scene(13, n=10, H=9, W=11, L=32, sigma_max=0.6)
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(13)
    gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, 5)).astype(np.float32)
    got, ref = _bwd_pair(sqr, pr, grid, rig, t, gd, gs, mode=2, order=bwd_order)
    for k in ref:
        check_grad(got[k], ref[k], k)


def test_backward_clamp_active(sqr, bwd_order):
    pr, grid, rig, t = small_scene(6, n=12, sigma_max=2.5, s_range=(1.0, 2.5))
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(6)
    gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, 5)).astype(np.float32)
    got, ref = _bwd_pair(sqr, pr, grid, rig, t, gd, gs, order=bwd_order)
    for k in ref:
        check_grad(got[k], ref[k], k)


def test_backward_early_termination(sqr, bwd_order):
    """kappa > 0: gradients flow only through the composited samples; cotangents on
    rays whose T stays clear of kappa (1e-4 relative) at every sample."""
    cfg = synth.make_config(0)
    kappa = 1e-2
    ix_ref = oracle.build_index(cfg["prims"], cfg["grid"])
    D, S, T, NU = oracle.render_fwd(cfg["prims"], cfg["grid"], ix_ref, cfg["rig"], cfg["t"], kappa=kappa)
    safe = []
    for r in range(0, len(D), 7):
        tr = oracle.trace_ray(cfg["prims"], cfg["grid"], ix_ref, cfg["rig"], cfg["t"], r, kappa=kappa)
        if not np.any(np.abs(tr["T"][:tr["used"] + 1] - kappa) < 1e-4 * kappa):
            safe.append(r)
    safe = np.array(safe)
    assert (NU[safe] < 48).sum() > 20
    rng = np.random.default_rng(8)
    gd = rng.standard_normal(len(safe)).astype(np.float32)
    gs = rng.standard_normal((len(safe), 18)).astype(np.float32)
    got, ref = _bwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], gd, gs, ray_ids=safe, kappa=kappa,
                         order=bwd_order)
    for k in ref:
        check_grad(got[k], ref[k], k)


def test_backward_stress_crop(sqr, bwd_order):
    """16,384 clustered superquadrics, 32x32-ray crop of camera 0 (cotangents zero
    elsewhere): every parameter's gradient vs the FP64 oracle."""
    cfg = synth.make_config(2)
    H, W = cfg["rig"]["H"], cfg["rig"]["W"]
    v0, u0 = 96, 184
    rays = np.array([(v0 + i) * W + (u0 + j) for i in range(32) for j in range(32)])
    rng = np.random.default_rng(2)
    gd = rng.standard_normal(len(rays)).astype(np.float32)
    gs = rng.standard_normal((len(rays), 18)).astype(np.float32)
    got, ref = _bwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], gd, gs, ray_ids=rays,
                         order=bwd_order)
    touched = np.abs(ref["opacity"]) > 0
    assert touched.sum() > 100
    for k in ref:
        check_grad(got[k], ref[k], k)


def test_backward_full_frame_sparse_cotangents(sqr, bwd_order):
    """540,000-ray frame, cotangents on 400 sampled rays only."""
    cfg = synth.make_config(1)
    R = synth.n_rays(cfg["rig"])
    rng = np.random.default_rng(11)
    rays = np.unique(rng.integers(0, R, 400))
    gd = rng.standard_normal(len(rays)).astype(np.float32)
    gs = rng.standard_normal((len(rays), 18)).astype(np.float32)
    got, ref = _bwd_pair(sqr, cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], gd, gs, ray_ids=rays,
                         order=bwd_order)
    for k in ref:
        check_grad(got[k], ref[k], k)


def test_autograd_function_matches_entry_point(sqr):
    """SQRender (torch.autograd.Function) routes the cotangents of a loss into
    sq_render_bwd: its .grad equals the direct call."""
    pr, grid, rig, t = small_scene(3, n=7, C=4)
    prims_d, rays = scene_to_gpu(sqr, pr, rig, t)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g)
    leaves = {k: v.clone().requires_grad_(True) for k, v in prims_d.items()}
    depth, sem = sqr.render(leaves, ix, g, rays)
    tgt = torch.linspace(1, 5, rays.R, device="cuda")
    loss = ((depth - tgt) ** 2).sum() + (sem[:, 1] * 0.3).sum()
    loss.backward()
    gd = 2 * (depth.detach() - tgt)
    gs = torch.zeros_like(sem)
    gs[:, 1] = 0.3
    direct = sqr.render_bwd(prims_d, ix, g, rays, gd, gs)
    for k in direct:
        torch.testing.assert_close(leaves[k].grad, direct[k], rtol=1e-5, atol=1e-6)


# ----------------------------------------------------------------------- grid query
def test_query_grid_full(sqr):
    """Supp. A.4 voxelisation of 8192 superquadrics at all 640,000 voxel centres."""
    cfg = synth.make_config(4)
    prims_d = sqr.to_device(cfg["prims"])
    g = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims_d, g)
    dens, sem, lab = sqr.query_grid(prims_d, ix, g, tau=0.05)
    torch.cuda.synchronize()
    rd, rs, rl = oracle.query_grid(cfg["prims"], cfg["grid"], oracle_index(ix, cfg["prims"], cfg["grid"]), tau=0.05)
    dens, sem, lab = dens.cpu().numpy(), sem.cpu().numpy(), lab.cpu().numpy()
    assert np.max(np.abs(dens - rd) / np.maximum(1.0, rd)) < 5e-5
    assert np.max(np.abs(sem - rs) / np.maximum(1.0, np.abs(rs))) < 5e-5
    # labels: the GPU's own FP32 decision must be self-consistent everywhere ...
    own = np.where(dens >= 0.05, np.argmax(sem, 1), 18)
    assert np.array_equal(own, lab)
    # ... and equal the FP64 label wherever the decision has a clear margin
    srt = np.sort(rs, 1)
    clear = (np.abs(rd - 0.05) > 1e-4) & (srt[:, -1] - srt[:, -2] > 1e-4)
    assert clear.mean() > 0.99
    assert np.array_equal(lab[clear], rl[clear])


def _query_scene(seed, n, gn, lo, hi, C=7):
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    means = rng.uniform(lo, hi, (n, 3))
    pr = prims_from(means, rng.standard_normal((n, 4)), rng.uniform(0.1, 1.2, (n, 3)), rng.uniform(0.2, 1.8, (n, 2)),
                    rng.uniform(0.05, 0.9, n), rng.standard_normal((n, C)))
    return pr, synth.grid_spec(*gn, lo=lo, hi=hi)


@pytest.mark.parametrize("gn", [(13, 11, 7), (9, 17, 5), (1, 1, 1)])
def test_query_grid_partial_tiles(sqr, gn):
    """Grids whose sides are not multiples of the 8 x 8 x 4 voxel tiles, with more
    primitives than one scan round (1,024 ids): density, semantics and labels
    against the oracle at every voxel centre."""
    pr, grid = _query_scene(31, 2500, gn, (-6.0, -6.0, -2.0), (6.0, 6.0, 2.0))
    prims_d = sqr.to_device(pr)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g)
    dens, sem, lab = sqr.query_grid(prims_d, ix, g, tau=0.05)
    torch.cuda.synchronize()
    rd, rs, rl = oracle.query_grid(pr, grid, oracle_index(ix, pr, grid), tau=0.05)
    dens, sem, lab = dens.cpu().numpy(), sem.cpu().numpy(), lab.cpu().numpy()
    assert np.max(np.abs(dens - rd) / np.maximum(1.0, rd)) < 5e-5
    assert np.max(np.abs(sem - rs) / np.maximum(1.0, np.abs(rs))) < 5e-5
    assert np.array_equal(np.where(dens >= 0.05, np.argmax(sem, 1), 7), lab)


def test_query_grid_long_axis(sqr):
    """A grid with more than 65,535 voxels along x: the query runs without voxel
    tiles (one lane per voxel, lane groups merging their lists) and still matches
    the oracle."""
    pr, grid = _query_scene(32, 300, (66000, 2, 2), (0.0, -1.0, -1.0), (6600.0, 1.0, 1.0))
    prims_d = sqr.to_device(pr)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g)
    sqr.profile_enable(True)
    dens, sem, lab = sqr.query_grid(prims_d, ix, g, tau=0.05)
    torch.cuda.synchronize()
    sqr.profile_enable(False)
    assert sqr.profile_query("k_query")[0] == 1 and sqr.profile_query("k_query_tiles")[0] == 0
    rd, rs, rl = oracle.query_grid(pr, grid, oracle_index(ix, pr, grid), tau=0.05)
    dens, sem = dens.cpu().numpy(), sem.cpu().numpy()
    assert rd.max() > 0.05
    assert np.max(np.abs(dens - rd) / np.maximum(1.0, rd)) < 5e-5
    assert np.max(np.abs(sem - rs) / np.maximum(1.0, np.abs(rs))) < 5e-5


def test_query_backward_full(sqr):
    """Backward of the grid query (dense cotangents on all 20,000 voxels of the
    256-superquadric scene) against the FP64 oracle."""
    cfg = synth.make_config(0)
    prims_d = sqr.to_device(cfg["prims"])
    g = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims_d, g)
    nvox = int(np.prod(cfg["grid"]["n"]))
    rng = np.random.default_rng(31)
    gd = rng.standard_normal(nvox).astype(np.float32)
    gs = rng.standard_normal((nvox, 18)).astype(np.float32)
    got = sqr.query_grid_bwd(prims_d, ix, g, torch.from_numpy(gd).cuda(), torch.from_numpy(gs).cuda())
    torch.cuda.synchronize()
    ref = oracle.query_grid_bwd(cfg["prims"], cfg["grid"], oracle_index(ix, cfg["prims"], cfg["grid"]),
                                gd.astype(np.float64),
                                gs.astype(np.float64))
    assert np.count_nonzero(ref["opacity"]) > 100
    for k in ref:
        check_grad(got[k].cpu().numpy(), ref[k], k)


def test_query_backward_sparse_large(sqr):
    """8192 superquadrics on the 200x200x16 grid, cotangents on 600 voxels only:
    every primitive's gradient (most are exactly zero) against the oracle."""
    cfg = synth.make_config(4)
    prims_d = sqr.to_device(cfg["prims"])
    g = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims_d, g)
    nvox = int(np.prod(cfg["grid"]["n"]))
    rng = np.random.default_rng(32)
    sel = np.sort(rng.choice(nvox, 600, replace=False))
    gd, gs = rng.standard_normal(600).astype(np.float32), rng.standard_normal((600, 18)).astype(np.float32)
    gd_full, gs_full = np.zeros(nvox, np.float32), np.zeros((nvox, 18), np.float32)
    gd_full[sel], gs_full[sel] = gd, gs
    got = sqr.query_grid_bwd(prims_d, ix, g, torch.from_numpy(gd_full).cuda(), torch.from_numpy(gs_full).cuda())
    torch.cuda.synchronize()
    ref = oracle.query_grid_bwd(cfg["prims"], cfg["grid"], oracle_index(ix, cfg["prims"], cfg["grid"]),
                                gd.astype(np.float64),
                                gs.astype(np.float64), voxel_ids=sel)
    assert np.count_nonzero(ref["opacity"]) > 50
    for k in ref:
        check_grad(got[k].cpu().numpy(), ref[k], k)


def test_softmax_sem_mode(sqr):
    """Per-primitive softmax of the logits (sem_mode 1): render forward and
    backward and the grid query and its backward against the oracle in the same
    mode."""
    pr, grid, rig, t = small_scene(40, n=8, H=9, W=11, L=32, C=6, sigma_max=0.6)
    prims_d, rays = scene_to_gpu(sqr, pr, rig, t)
    prims_d["sem_mode"] = sqr.SQ_SEM_SOFTMAX
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g)
    idx = oracle_index(ix, pr, grid)
    d, s, _ = sqr.render_fwd(prims_d, ix, g, rays)
    D, S, _, _ = oracle.render_fwd(pr, grid, idx, rig, t, sem_mode=1)
    check_depth(d.cpu().numpy(), D, 0.5)
    check_sem(s.cpu().numpy(), S)
    R = rays.R
    rng = np.random.default_rng(40)
    gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, 6)).astype(np.float32)
    got = sqr.render_bwd(prims_d, ix, g, rays, torch.from_numpy(gd).cuda(), torch.from_numpy(gs).cuda())
    ref = oracle.render_bwd(pr, grid, idx, rig, t, gd.astype(np.float64), gs.astype(np.float64), sem_mode=1)
    for k in ref:
        check_grad(got[k].cpu().numpy(), ref[k], k)
    assert np.allclose(got["logits"].cpu().numpy().sum(1), 0.0, atol=1e-5 * np.abs(ref["logits"]).max())
    dens, sem, _ = sqr.query_grid(prims_d, ix, g, tau=0.05)
    rd, rs, _ = oracle.query_grid(pr, grid, idx, tau=0.05, sem_mode=1)
    assert np.max(np.abs(sem.cpu().numpy() - rs) / np.maximum(1.0, np.abs(rs))) < 5e-5
    nvox = int(np.prod(grid["n"]))
    qd, qs = rng.standard_normal(nvox).astype(np.float32), rng.standard_normal((nvox, 6)).astype(np.float32)
    gq = sqr.query_grid_bwd(prims_d, ix, g, torch.from_numpy(qd).cuda(), torch.from_numpy(qs).cuda())
    rq = oracle.query_grid_bwd(pr, grid, idx, qd.astype(np.float64), qs.astype(np.float64), sem_mode=1)
    for k in rq:
        check_grad(gq[k].cpu().numpy(), rq[k], k)


def test_kernel_timing_records_every_launch(sqr):
    """sq_profile_*: while enabled, every launch of the library is recorded with a
    positive duration on its stream; disabled, nothing is recorded."""
    cfg = synth.make_config(0)
    prims_d, rays = scene_to_gpu(sqr, cfg["prims"], cfg["rig"], cfg["t"])
    g = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims_d, g)
    sqr.profile_enable(True)
    sqr.build_index(prims_d, g, index=ix, sync=False)  # 9 kernels
    sqr.render_fwd(prims_d, ix, g, rays)  # pack, descriptors, forward
    torch.cuda.synchronize()
    sqr.profile_enable(False)
    n_all, ms_all, dropped = sqr.profile_query(None)
    n_fwd, ms_fwd, _ = sqr.profile_query("k_forward")
    assert (n_all, dropped) == (12, 0) and n_fwd == 1
    assert 0.0 < ms_fwd < ms_all
    sqr.render_fwd(prims_d, ix, g, rays)
    torch.cuda.synchronize()
    assert sqr.profile_query(None)[0] == 12  # disabled: unchanged
    sqr.profile_enable(True)
    assert sqr.profile_query(None)[0] == 0  # enabling clears
    sqr.profile_enable(False)


# ----------------------------------------------------------------------- loss
@pytest.mark.parametrize("R,C", [(1000, 18), (77, 5), (4097, 32), (64, 1)])
def test_loss_kernel_matches_torch(sqr, R, C):
    """Ray counts that leave a partial 32-ray chunk, odd and even class counts up to
    the maximum, a single class."""
    rng = np.random.default_rng(R + C)
    d = torch.from_numpy(rng.uniform(0, 40, R).astype(np.float32)).cuda()
    s = torch.from_numpy(rng.standard_normal((R, C)).astype(np.float32)).cuda()
    td = torch.from_numpy(rng.uniform(0.5, 45, R).astype(np.float32)).cuda()
    tl = torch.from_numpy(rng.integers(0, C, R).astype(np.int32)).cuda()
    loss, gd, gs = sqr.loss_ce_mse(d, s, td, tl)
    dc, sc = d.cpu().double().requires_grad_(), s.cpu().double().requires_grad_()
    ref = 2.0 * torch.nn.functional.cross_entropy(sc, tl.cpu().long()) + 0.05 * ((dc - td.cpu().double()) ** 2).mean()
    ref.backward()
    assert abs(loss.item() - ref.item()) < 1e-4 * abs(ref.item())
    torch.testing.assert_close(gd.cpu().double(), dc.grad, rtol=1e-5, atol=1e-9)
    torch.testing.assert_close(gs.cpu().double(), sc.grad, rtol=1e-4, atol=1e-9)


def test_loss_label_outside_classes_gives_nan(sqr):
    """A label outside [0, C) makes the loss NaN; the other rays' gradient rows are
    those of a valid batch, and that ray's row is its softmax without a one-hot term."""
    rng = np.random.default_rng(5)
    R, C = 100, 18
    d = torch.from_numpy(rng.uniform(0, 40, R).astype(np.float32)).cuda()
    s = torch.from_numpy(rng.standard_normal((R, C)).astype(np.float32)).cuda()
    td = torch.from_numpy(rng.uniform(0.5, 45, R).astype(np.float32)).cuda()
    good = rng.integers(0, C, R).astype(np.int32)
    bad = good.copy()
    bad[37] = C + 3
    loss_b, _, gs_b = sqr.loss_ce_mse(d, s, td, torch.from_numpy(bad).cuda())
    _, _, gs_g = sqr.loss_ce_mse(d, s, td, torch.from_numpy(good).cuda())
    assert np.isnan(loss_b.item())
    keep = np.arange(R) != 37
    assert torch.equal(gs_b[keep], gs_g[keep])
    row = gs_g[37].clone()
    row[int(good[37])] += 2.0 / R  # lambda_s / R times the one-hot term
    torch.testing.assert_close(gs_b[37], row, rtol=1e-6, atol=1e-8)
    with pytest.raises(sqr.SqrError):
        sqr.loss_ce_mse(d, torch.zeros((R, 33), device="cuda"), td, torch.from_numpy(good).cuda())


@pytest.mark.parametrize("V,C", [(20000, 18), (1001, 7), (77, 32)])
def test_voxel_loss_kernel_matches_oracle(sqr, V, C):
    """sq_loss_voxel (CE on semantic voxels, BCE on 1 - exp(-density)) against the
    FP64 oracle: counts exact, loss terms 1e-5 relative, gradients 1e-5 of each
    tensor's largest entry (FP32 exp/log/expm1 of single terms); voxel counts with a
    partial 32-voxel chunk, odd and maximal class counts."""
    rng = np.random.default_rng(7 + V + C)
    dens = rng.uniform(-0.2, 4.0, V).astype(np.float32)
    dens[::17] = 0.0
    sem = (rng.standard_normal((V, C)) * 3).astype(np.float32)
    lab = rng.integers(-1, C + 1, V).astype(np.int32)
    loss, counts, gd, gs = sqr.loss_voxel(torch.from_numpy(dens).cuda(), torch.from_numpy(sem).cuda(),
                                          torch.from_numpy(lab).cuda(), lambda_s=2.0, lambda_o=0.5)
    torch.cuda.synchronize()
    tot, ce, bce, rgd, rgs = oracle.voxel_loss(dens, sem, lab, lambda_s=2.0, lambda_o=0.5)
    occ = int(((lab >= 0) & (lab < C)).sum())
    assert counts.cpu().tolist() == [occ, int(((lab >= 0) & (lab <= C)).sum())]
    got = loss.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, [tot, ce, bce], rtol=1e-5)
    np.testing.assert_allclose(gd.cpu().numpy(), rgd, rtol=0, atol=1e-5 * np.abs(rgd).max())
    np.testing.assert_allclose(gs.cpu().numpy(), rgs, rtol=0, atol=1e-5 * np.abs(rgs).max())


# ----------------------------------------------------------------------- argument errors
def test_invalid_arguments_rejected_on_host(sqr):
    cfg = synth.make_config(0)
    prims_d = sqr.to_device(cfg["prims"])
    g = dev_grid(cfg["grid"])
    with pytest.raises(sqr.SqrError):
        sqr.build_index(prims_d, g, tau_cut=1.5)
    with pytest.raises(sqr.SqrError):
        sqr.build_index(prims_d, {"n": (0, 5, 5), "lo": [0, 0, 0], "vs": [1, 1, 1]})
    ix = sqr.build_index(prims_d, g)
    rays = sqr.Rays.from_rig(cfg["rig"], np.linspace(0.5, 45, 2000))
    with pytest.raises(sqr.SqrError):
        sqr.render_fwd(prims_d, ix, g, rays)  # L > SQ_MAX_SAMPLES
