"""The two backward orders of Sec. 3.3.3 (needs a GPU): the primitive-major
backward (each primitive's interactions generated from its projected box and
reduced in fixed order) against the FP64 oracle on rigs that exercise its
camera geometry, bitwise reproducibility, agreement with the ray-major backward
on a full frame, and the batched path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_17361_gb300 import synth
from tests.gpu_common import check_grad, dev_grid, lib, oracle_index, per_ray_magnitude, scene_to_gpu
from tests.helpers import axis_camera, small_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    return lib()


def _grads(sqr, prims_d, ix, g, rays, gd, gs, order):
    out = sqr.render_bwd(prims_d, ix, g, rays, gd, gs, order=order)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle_case(sqr, pr, grid, rig, t, seed):
    prims_d, rays = scene_to_gpu(sqr, pr, rig, t)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g)
    R = rays.R
    rng = np.random.default_rng(seed)
    C = pr["logits"].shape[1]
    gd, gs = rng.standard_normal(R).astype(np.float32), rng.standard_normal((R, C)).astype(np.float32)
    got = _grads(sqr, prims_d, ix, g, rays, torch.from_numpy(gd).cuda(), torch.from_numpy(gs).cuda(),
                 sqr.SQ_BWD_PRIMITIVE_MAJOR)
    idx = oracle_index(ix, pr, grid)
    ref = oracle.render_bwd(pr, grid, idx, rig, t, gd.astype(np.float64), gs.astype(np.float64))
    mag = per_ray_magnitude(pr, grid, idx, rig, t, gd, gs)
    return got, ref, mag


def test_rays_from_the_camera_centre(sqr):
    """t_0 = 0: samples at the camera centre and boxes reaching behind the camera
    (their rectangle is the whole image)."""
    pr, grid, rig, t = small_scene(21, n=9, H=9, W=11, L=30)
    t = synth.sample_depths(30, 0.0, 9.5)
    got, ref, mag = _oracle_case(sqr, pr, grid, rig, t, 21)
    assert np.count_nonzero(ref["opacity"]) >= 5
    for k in ref:
        check_grad(got[k], ref[k], k, mag=mag[k])


def test_camera_inside_boxes(sqr):
    """Primitives around the camera: boxes that hold the camera centre or straddle
    its image plane are clipped at the nearest sample depth."""
    rng = np.random.default_rng(22)
    pr, grid, rig, t = small_scene(22, n=10, H=10, W=12, L=36)
    means = pr["means"].copy()
    means[:4] = np.stack([rng.uniform(-2.0, 0.0, 4), rng.uniform(-1.0, 1.0, 4), rng.uniform(0.5, 1.5, 4)], 1)
    pr["means"] = means.astype(np.float32)
    got, ref, mag = _oracle_case(sqr, pr, grid, rig, t, 22)
    for k in ref:
        check_grad(got[k], ref[k], k, mag=mag[k])


def test_uneven_sample_spacing(sqr):
    """Geometrically spaced samples: the interval ends' estimate (from even spacing)
    is off by several samples, so the exact search takes over."""
    pr, grid, rig, _ = small_scene(26, n=9, H=9, W=11, L=36)
    t = (0.5 * 1.085 ** np.arange(36)).astype(np.float32)
    got, ref, mag = _oracle_case(sqr, pr, grid, rig, t, 26)
    assert np.count_nonzero(ref["opacity"]) >= 5
    for k in ref:
        check_grad(got[k], ref[k], k, mag=mag[k])


def test_axis_aligned_ray(sqr):
    """A ray along a grid axis (two direction components exactly zero): the
    per-axis interval searches see constant coordinates."""
    pr, grid, _, t = small_scene(23, n=6, L=40)
    rig = axis_camera(centre=(-1.0, 0.25, 1.0))
    got, ref, mag = _oracle_case(sqr, pr, grid, rig, t, 23)
    assert np.count_nonzero(ref["opacity"]) >= 1
    for k in ref:
        check_grad(got[k], ref[k], k, mag=mag[k])


def test_multi_camera_ring(sqr):
    """Six cameras of a small ring, primitives all around (rectangles in several
    cameras, boxes behind some of them)."""
    pr = synth.prims_driving(300, 24)
    grid = synth.grid_spec(50, 50, 8)
    rig = synth.rig_ring(n_cam=6, H=12, W=20, f=9.0)
    t = synth.sample_depths(40)
    got, ref, mag = _oracle_case(sqr, pr, grid, rig, t, 24)
    for k in ref:
        check_grad(got[k], ref[k], k, mag=mag[k])


def test_many_cameras(sqr):
    """18 cameras (more than a tile stages in shared memory: the rectangles are then
    read from global memory), small images, primitives all around."""
    pr = synth.prims_driving(200, 25)
    grid = synth.grid_spec(50, 50, 8)
    n_cam, H, W, f = 18, 5, 7, 3.0
    K = np.ascontiguousarray([[f, f, W / 2.0, H / 2.0]] * n_cam, np.float32)
    poses = [synth.camera_pose(np.deg2rad(20.0 * i), np.array([np.cos(np.deg2rad(20.0 * i)),
                                                               np.sin(np.deg2rad(20.0 * i)), 1.6]))
             for i in range(n_cam)]
    rig = {"n_cam": n_cam, "H": H, "W": W, "K": K, "cam2world": np.ascontiguousarray(poses, np.float32)}
    t = synth.sample_depths(40)
    got, ref, mag = _oracle_case(sqr, pr, grid, rig, t, 25)
    assert np.count_nonzero(ref["opacity"]) > 20
    for k in ref:
        check_grad(got[k], ref[k], k, mag=mag[k])


def test_full_frame_reproducible_and_matches_ray_major(sqr):
    """540,000-ray frame with dense cotangents: two primitive-major runs agree bit
    for bit; against the ray-major backward (itself checked against the oracle)
    the sums differ only in FP32 summation order."""
    cfg = synth.make_config(1)
    prims_d, rays = scene_to_gpu(sqr, cfg["prims"], cfg["rig"], cfg["t"])
    g = dev_grid(cfg["grid"])
    ix = sqr.build_index(prims_d, g)
    gd_np, gs_np = synth.cotangents(rays.R, 5)
    gd, gs = torch.from_numpy(gd_np).cuda(), torch.from_numpy(gs_np).cuda()
    a = _grads(sqr, prims_d, ix, g, rays, gd, gs, sqr.SQ_BWD_PRIMITIVE_MAJOR)
    b = _grads(sqr, prims_d, ix, g, rays, gd, gs, sqr.SQ_BWD_PRIMITIVE_MAJOR)
    rm = _grads(sqr, prims_d, ix, g, rays, gd, gs, sqr.SQ_BWD_RAY_MAJOR)
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
        check_grad(a[k], rm[k].astype(np.float64), k, rtol=2e-3)


def test_batched_primitive_major(sqr):
    """Three scenes of uneven size in one batched backward in primitive-major order
    against each scene's ray-major backward."""
    cfgs = [small_scene(31, n=20, H=13, W=17, L=40, C=18, sigma_max=0.8),
            (synth.prims_driving(600, 32), synth.grid_spec(100, 100, 8), synth.rig_ring(n_cam=2, H=30, W=52, f=35.0),
             synth.sample_depths(33)),
            (synth.prims_uniform(400, 33), synth.grid_spec(50, 50, 8), synth.rig_ring(n_cam=3, H=17, W=23, f=14.0),
             synth.sample_depths(61))]
    scenes = []
    for i, (pr, grid, rig, t) in enumerate(cfgs):
        prims_d, rays = scene_to_gpu(sqr, pr, rig, t)
        g = dev_grid(grid)
        ix = sqr.build_index(prims_d, g)
        sc = sqr.Scene(prims_d, ix, g, rays)
        gd, gs = synth.cotangents(rays.R, 40 + i)
        sc.grad_depth.copy_(torch.from_numpy(gd))
        sc.grad_sem.copy_(torch.from_numpy(gs))
        scenes.append(sc)
    sqr.render_batched(sqr.SQ_OP_FWD, scenes)
    sqr.render_batched(sqr.SQ_OP_BWD, scenes, tuning={"fwd_lanes_per_ray": 4, "fwd_warps_per_cta": 8,
                                                      "bwd_warps_per_cta": 0,
                                                      "bwd_order": sqr.SQ_BWD_PRIMITIVE_MAJOR})
    torch.cuda.synchronize()
    for sc in scenes:
        ref = _grads(sqr, sc.prims, sc.index, sc.grid, sc.rays, sc.grad_depth, sc.grad_sem, sqr.SQ_BWD_RAY_MAJOR)
        for k in ref:
            check_grad(sc.grads[k].cpu().numpy(), ref[k].astype(np.float64), k, rtol=2e-3)


def test_unknown_order_rejected(sqr):
    pr, grid, rig, t = small_scene(34, n=4)
    prims_d, rays = scene_to_gpu(sqr, pr, rig, t)
    g = dev_grid(grid)
    ix = sqr.build_index(prims_d, g)
    gd = torch.zeros(rays.R, device="cuda")
    gs = torch.zeros((rays.R, 5), device="cuda")
    with pytest.raises(sqr.SqrError):
        sqr.render_bwd(prims_d, ix, g, rays, gd, gs, order=7)
