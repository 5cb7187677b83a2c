"""The saved forward state in pages of composited samples (needs a GPU).

The forward saves T_j, alpha_j and s_j only for the samples a ray composites,
in pages of SQ_SAVE_PAGE samples handed out as rays advance; the header reports
the pages it needed and whether they fitted.  These tests check the count, the
overflow path (outputs unchanged, backward refused with zero gradients, a rerun
into a buffer of the reported size giving the same gradients bit for bit), and
the autograd wrapper's re-sizing."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_17361_gb300 import synth
from tests.gpu_common import check_grad, dev_grid, lib, oracle_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    return lib()


def _scene(sqr, ci):
    cfg = synth.make_config(ci)
    prims = sqr.to_device(cfg["prims"])
    rays = sqr.Rays.from_rig(cfg["rig"], cfg["t"])
    grid = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims, grid)
    return cfg, prims, rays, grid, ix


@pytest.mark.parametrize("ci", [0, 1])
def test_pages_needed_and_overflow(sqr, ci):
    cfg, prims, rays, grid, ix = _scene(sqr, ci)
    C = cfg["prims"]["logits"].shape[1]
    full = sqr.new_saved(rays, C)
    d0, s0, t0 = (x.clone() for x in sqr.render_fwd(prims, ix, grid, rays, saved=full))
    needed, status = sqr.saved_header(full)
    assert status == sqr.SQ_OK
    le = sqr.saved_counts(full, rays, C).cpu().numpy().astype(np.int64)
    # pages of SQ_SAVE_PAGE samples up to each ray's stop (4-sample chunks never straddle a page)
    ps = sqr.SQ_SAVE_PAGE
    assert needed == int(((le + ps - 1) // ps).sum())
    assert needed * 4 < rays.R * len(cfg["t"])  # fewer than every sample
    rng = np.random.default_rng(ci)
    gd = torch.from_numpy(rng.standard_normal(rays.R).astype(np.float32)).cuda()
    gs = torch.from_numpy(rng.standard_normal((rays.R, C)).astype(np.float32)).cuda()
    g_full = {k: v.clone() for k, v in sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=full).items()}

    small = sqr.new_saved(rays, C, pages=max(needed // 3, 1))
    d1, s1, t1 = sqr.render_fwd(prims, ix, grid, rays, saved=small)
    n_small, st_small = sqr.saved_header(small)
    assert st_small == sqr.SQ_ERR_CAPACITY and n_small == needed
    assert torch.equal(d1, d0) and torch.equal(s1, s0) and torch.equal(t1, t0)
    g_small = sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=small)
    assert all(torch.all(v == 0) for v in g_small.values())

    exact = sqr.new_saved(rays, C, pages=needed)
    assert exact.numel() < full.numel()
    sqr.render_fwd(prims, ix, grid, rays, saved=exact)
    assert sqr.saved_header(exact) == (needed, sqr.SQ_OK)
    g_exact = sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=exact)
    for k in g_full:
        assert torch.equal(g_exact[k], g_full[k]), k


def test_bench_frame_saved_state_size(sqr):
    """The six-camera frame of the benchmark: the pages of its composited samples
    take less than half the memory of the state for every sample."""
    cfg, prims, rays, grid, ix = _scene(sqr, 1)
    C = cfg["prims"]["logits"].shape[1]
    full = sqr.new_saved(rays, C)
    sqr.render_fwd(prims, ix, grid, rays, saved=full)
    needed, status = sqr.saved_header(full)
    assert status == sqr.SQ_OK
    fitted = sqr.saved_size(rays, C, pages=needed)
    assert fitted < 2.0e9 and fitted < 0.45 * full.numel(), (fitted, full.numel())


def test_autograd_resizes_after_an_overflow(sqr):
    """SQRender reserves the pages earlier forwards of the shape needed; when they
    run out it reruns the forward into a large enough buffer, and the gradients
    match the FP64 oracle."""
    cfg, prims, rays, grid, ix = _scene(sqr, 0)
    C = cfg["prims"]["logits"].shape[1]
    key = (rays.R, rays.t.numel(), C)
    sqr._SAVED_PAGES[key] = 10  # far too few
    leaves = {k: v.clone().requires_grad_(True) for k, v in prims.items()}
    depth, sem = sqr.render(leaves, ix, grid, rays)
    rng = np.random.default_rng(3)
    gd = rng.standard_normal(rays.R).astype(np.float32)
    gs = rng.standard_normal((rays.R, C)).astype(np.float32)
    (depth * torch.from_numpy(gd).cuda()).sum().add((sem * torch.from_numpy(gs).cuda()).sum()).backward()
    assert sqr._SAVED_PAGES[key] > 10
    ref_ix = oracle_index(ix, cfg["prims"], cfg["grid"])
    ref = oracle.render_bwd(cfg["prims"], cfg["grid"], ref_ix, cfg["rig"], cfg["t"], gd.astype(np.float64),
                            gs.astype(np.float64))
    for k in ref:
        check_grad(leaves[k].grad.cpu().numpy(), ref[k], k)
    del sqr._SAVED_PAGES[key]
