"""Whole six-camera frames against the FP64 oracle (needs a GPU).

* Every (composited sample, primitive) pair is visited exactly once by the
  primitive-major backward (Sec. 3.3.3 sums the gradient over exactly these
  pairs): per primitive, the pairs its tiles evaluated equal the count derived
  from the oracle's index and the forward's composited sample counts.
* The forward and the dense-cotangent backward of the full 540,000-ray frame,
  every ray and every gradient element, against the oracle at the tolerances of
  tests/gpu_common.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_17361_gb300 import synth
from tests.gpu_common import check_depth, check_grad, check_sem, dev_grid, lib, oracle_index
from tests.helpers import box_sums

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    return lib()


def _frame(sqr, cfg):
    prims = sqr.to_device(cfg["prims"])
    rays = sqr.Rays.from_rig(cfg["rig"], cfg["t"])
    grid = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims, grid)
    ref_ix = oracle_index(ix, cfg["prims"], cfg["grid"])
    C = cfg["prims"]["logits"].shape[1]
    saved = sqr.new_saved(rays, C)
    depth, sem, tf = sqr.render_fwd(prims, ix, grid, rays, saved=saved)
    return prims, rays, grid, ix, ref_ix, saved, (depth, sem, tf)


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_pair_visits_equal_index_count(sqr, ci):
    """Workloads 0, 1 (the bench frame) and 2 (16,384 clustered primitives): the
    primitive-major backward's per-primitive pair counts equal, integer for integer,
    sum over the voxels v of the primitive's range of #{(r, j): j < composited(r),
    voxel(r, j) = v}, the voxels of the samples taken by the oracle's FP32 rule."""
    cfg = synth.make_config(ci)
    prims, rays, grid, ix, ref_ix, saved, _ = _frame(sqr, cfg)
    R, L, C = rays.R, len(cfg["t"]), cfg["prims"]["logits"].shape[1]
    n = cfg["prims"]["means"].shape[0]
    rng = np.random.default_rng(50 + ci)
    gd = torch.from_numpy(rng.standard_normal(R).astype(np.float32)).cuda()
    gs = torch.from_numpy(rng.standard_normal((R, C)).astype(np.float32)).cuda()
    visits = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=saved, pair_visits=visits)
    torch.cuda.synchronize()
    got = visits.cpu().numpy()
    le = sqr.saved_counts(saved, rays, C).cpu().numpy().astype(np.int64)
    assert np.all((le >= 0) & (le <= L))
    vox = oracle.sample_voxels(cfg["rig"], cfg["t"], cfg["grid"])
    keep = (np.arange(L)[None, :] < le[:, None]) & (vox >= 0)
    nvox = int(np.prod(cfg["grid"]["n"]))
    per_voxel = np.bincount(vox[keep], minlength=nvox).reshape(tuple(int(v) for v in cfg["grid"]["n"]))
    want = box_sums(per_voxel, ref_ix["ranges"])
    assert want.sum() > 0
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (f"{bad.size} primitives differ, e.g. {bad[:5]}: got {got[bad[:5]]}, "
                           f"want {want[bad[:5]]}")


def test_full_frame_dense_backward_against_oracle(sqr):
    """The bench frame (six 225x400 cameras, 4096 superquadrics, L = 100): depth and
    semantics of all 540,000 rays, then the gradients of seeded dense cotangents on
    every ray, element by element against the FP64 oracle on the host cores."""
    cfg = synth.make_config(1)
    prims, rays, grid, ix, ref_ix, saved, (depth, sem, tf) = _frame(sqr, cfg)
    R, C = rays.R, cfg["prims"]["logits"].shape[1]
    rng = np.random.default_rng(77)
    gd = (rng.standard_normal(R) / R).astype(np.float32)
    gs = (rng.standard_normal((R, C)) / R).astype(np.float32)
    got = sqr.render_bwd(prims, ix, grid, rays, torch.from_numpy(gd).cuda(), torch.from_numpy(gs).cuda(),
                         saved=saved)
    torch.cuda.synchronize()
    D, S, T, _ = oracle.render_fwd(cfg["prims"], cfg["grid"], ref_ix, cfg["rig"], cfg["t"])
    check_depth(depth.cpu().numpy(), D, float(cfg["t"][0]))
    check_sem(sem.cpu().numpy(), S)
    assert np.max(np.abs(tf.cpu().numpy() - T)) < 2e-5
    ref = oracle.render_bwd(cfg["prims"], cfg["grid"], ref_ix, cfg["rig"], cfg["t"], gd.astype(np.float64),
                            gs.astype(np.float64))
    for k in ref:
        check_grad(got[k].cpu().numpy(), ref[k], k)
