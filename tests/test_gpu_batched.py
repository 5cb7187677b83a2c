"""Batched persistent launches (many scenes of uneven size in one launch), the
launch-configuration autotuner and CUDA-graph capture (needs a GPU).  The batched
path is checked against per-scene calls (themselves checked against the FP64
oracle in test_gpu_parity.py) and against the oracle directly on every scene.
Gradients of two GPU runs differ by the order of FP32 atomic additions; each is
within the gradient tolerance of the FP64 result, so two runs are compared at
twice that tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_17361_gb300 import synth
from tests.gpu_common import check_depth, check_grad, check_sem, dev_grid, lib, oracle_index, per_ray_magnitude
from tests.helpers import small_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    return lib()


def _scenes(sqr, seed=0):
    """Four scenes of uneven size sharing 18 classes: different N, cameras, image
    sizes and sample counts."""
    rng = np.random.default_rng(seed)
    cfgs = []
    c0 = synth.make_config(0)
    cfgs.append((c0["prims"], c0["grid"], c0["rig"], c0["t"]))
    pr, g, rig, t = small_scene(seed + 1, n=30, H=21, W=35, L=40, C=18, sigma_max=0.8)
    cfgs.append((pr, g, rig, t))
    pr = synth.prims_driving(900, seed + 2)
    cfgs.append((pr, synth.grid_spec(100, 100, 8), synth.rig_ring(n_cam=2, H=30, W=52, f=35.0), synth.sample_depths(33)))
    pr = synth.prims_uniform(500, seed + 3)
    cfgs.append((pr, synth.grid_spec(50, 50, 8), synth.rig_ring(n_cam=3, H=17, W=23, f=14.0), synth.sample_depths(61)))
    scenes, host = [], []
    for pr, g, rig, t in cfgs:
        prims_d = sqr.to_device(pr)
        rays = sqr.Rays.from_rig(rig, t)
        gd = dev_grid(g)
        ix = sqr.build_index(prims_d, gd)
        sc = sqr.Scene(prims_d, ix, gd, rays, training=True)
        R = rays.R
        sc.grad_depth.copy_(torch.from_numpy(rng.standard_normal(R).astype(np.float32)))
        sc.grad_sem.copy_(torch.from_numpy(rng.standard_normal((R, 18)).astype(np.float32)))
        scenes.append(sc)
        host.append((pr, g, rig, t))
    return scenes, host


def _per_scene(sqr, sc):
    saved = sqr.new_saved(sc.rays, sc.prims["logits"].shape[1])
    d, s, tf = sqr.render_fwd(sc.prims, sc.index, sc.grid, sc.rays, saved=saved)
    g = sqr.render_bwd(sc.prims, sc.index, sc.grid, sc.rays, sc.grad_depth, sc.grad_sem, saved=saved)
    return d.clone(), s.clone(), tf.clone(), {k: v.clone() for k, v in g.items()}


def test_batched_equals_per_scene(sqr):
    scenes, _ = _scenes(sqr)
    refs = [_per_scene(sqr, sc) for sc in scenes]
    sqr.render_batched(sqr.SQ_OP_FWD, scenes)
    sqr.render_batched(sqr.SQ_OP_BWD, scenes)
    torch.cuda.synchronize()
    for sc, (d, s, tf, g) in zip(scenes, refs):
        assert torch.equal(sc.depth, d) and torch.equal(sc.sem, s) and torch.equal(sc.t_final, tf)
        for k in g:
            check_grad(sc.grads[k].cpu().numpy(), g[k].cpu().numpy(), k, rtol=2e-3)


def test_batched_scene_against_oracle(sqr):
    scenes, host = _scenes(sqr, seed=5)
    sqr.render_batched(sqr.SQ_OP_FWD, scenes)
    sqr.render_batched(sqr.SQ_OP_BWD, scenes)
    torch.cuda.synchronize()
    for sc, (pr, g, rig, t) in zip(scenes, host):
        idx = oracle_index(sc.index, pr, g)
        D, S, T, _ = oracle.render_fwd(pr, g, idx, rig, t)
        check_depth(sc.depth.cpu().numpy(), D, 0.5)
        check_sem(sc.sem.cpu().numpy(), S)
        ref = oracle.render_bwd(pr, g, idx, rig, t, sc.grad_depth.cpu().numpy().astype(np.float64),
                                sc.grad_sem.cpu().numpy().astype(np.float64))
        for k in ref:
            check_grad(sc.grads[k].cpu().numpy(), ref[k], k)


@pytest.mark.parametrize("lanes,fw,bw,tile", [(4, 4, 4, 1), (8, 8, 8, 16), (16, 4, 2, 3), (4, 8, 0, 64)])
def test_every_tuning_gives_the_same_render(sqr, lanes, fw, bw, tile):
    scenes, _ = _scenes(sqr, seed=2)
    sqr.render_batched(sqr.SQ_OP_FWD, scenes)
    sqr.render_batched(sqr.SQ_OP_BWD, scenes)
    base = [(sc.depth.clone(), sc.sem.clone(), {k: v.clone() for k, v in sc.grads.items()}) for sc in scenes]
    tn = {"fwd_lanes_per_ray": lanes, "fwd_warps_per_cta": fw, "bwd_warps_per_cta": bw, "fwd_ray_tile": tile}
    sqr.render_batched(sqr.SQ_OP_FWD, scenes, tn)
    sqr.render_batched(sqr.SQ_OP_BWD, scenes, tn)
    torch.cuda.synchronize()
    for sc, (d, s, g) in zip(scenes, base):
        torch.testing.assert_close(sc.depth, d, rtol=1e-5, atol=1e-5)
        torch.testing.assert_close(sc.sem, s, rtol=1e-5, atol=1e-5)
        for k in g:
            check_grad(sc.grads[k].cpu().numpy(), g[k].cpu().numpy(), k, rtol=2e-3)


def test_autotuner_picks_a_measured_candidate(sqr):
    scenes, _ = _scenes(sqr, seed=3)
    best = sqr.autotune(scenes, reps=2, use_cache=False)
    assert best["fwd_lanes_per_ray"] in (4, 8) and best["fwd_warps_per_cta"] in (4, 8)
    assert best["bwd_warps_per_cta"] in (0, 4, 8)
    assert all(ms > 0 for ms in best["fwd_ms"]) and all(ms > 0 for ms in best["bwd_ms"])
    cands = [(lanes, warps, tile) for tile in (1, 16) for lanes, warps in ((4, 4), (4, 8), (8, 4), (8, 8))]
    assert len(best["fwd_ms"]) == 8
    i = cands.index((best["fwd_lanes_per_ray"], best["fwd_warps_per_cta"], best["fwd_ray_tile"]))
    assert best["fwd_ms"][i] == min(best["fwd_ms"])
    assert len(best["bwd_ms"]) == 4 and best["bwd_order"] in (sqr.SQ_BWD_RAY_MAJOR, sqr.SQ_BWD_PRIMITIVE_MAJOR)
    bc = [(sqr.SQ_BWD_RAY_MAJOR, 0), (sqr.SQ_BWD_RAY_MAJOR, 4), (sqr.SQ_BWD_RAY_MAJOR, 8),
          (sqr.SQ_BWD_PRIMITIVE_MAJOR, 0)]
    j = bc.index((best["bwd_order"], best["bwd_warps_per_cta"]))
    assert best["bwd_ms"][j] == min(best["bwd_ms"])


def test_ray_tile_outside_range_is_refused(sqr):
    scenes, _ = _scenes(sqr, seed=2)
    with pytest.raises(sqr.SqrError, match="ray tile"):
        sqr.render_batched(sqr.SQ_OP_FWD, scenes, {"fwd_lanes_per_ray": 4, "fwd_warps_per_cta": 8,
                                                   "bwd_warps_per_cta": 0, "fwd_ray_tile": 65})


def test_cuda_graph_replay_matches_eager(sqr):
    """The whole training step of a batch (index rebuilds, batched forward, loss
    gradient, batched backward) captured once and replayed."""
    scenes, _ = _scenes(sqr, seed=4)
    targets = []
    for sc in scenes:
        R = sc.rays.R
        rng = np.random.default_rng(R)
        targets.append((torch.from_numpy(rng.uniform(0.5, 40, R).astype(np.float32)).cuda(),
                        torch.from_numpy(rng.integers(0, 18, R).astype(np.int32)).cuda(),
                        (torch.empty(1, device="cuda"), torch.empty(R, device="cuda"),
                         torch.empty((R, 18), device="cuda"))))

    def step():
        for sc in scenes:
            sqr.build_index(sc.prims, sc.grid, index=sc.index, sync=False)
        sqr.render_batched(sqr.SQ_OP_FWD, scenes)
        for sc, (td, tl, out) in zip(scenes, targets):
            sqr.loss_ce_mse(sc.depth, sc.sem, td, tl, out=out)
            sc.grad_depth.copy_(out[1])
            sc.grad_sem.copy_(out[2])
        sqr.render_batched(sqr.SQ_OP_BWD, scenes)

    step()
    torch.cuda.synchronize()
    eager = [(sc.depth.clone(), sc.sem.clone(), {k: v.clone() for k, v in sc.grads.items()}) for sc in scenes]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()  # warm-up on the capture stream (workspaces already sized)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for sc in scenes:
        sc.depth.zero_()
        for v in sc.grads.values():
            v.zero_()
    g.replay()
    torch.cuda.synchronize()
    for sc, (d, s, gr) in zip(scenes, eager):
        assert torch.equal(sc.depth, d) and torch.equal(sc.sem, s)
        for k in gr:
            check_grad(sc.grads[k].cpu().numpy(), gr[k].cpu().numpy(), k, rtol=2e-3)


def test_temporal_horizon_batch(sqr):
    """The 2T+1 frames of a temporal horizon (Sec. 3.2; T = 2 here, small images):
    the batched launch equals per-frame calls, and the first and last frames
    match the FP64 oracle."""
    frames = synth.make_temporal_config(T=2, n=300, H=18, W=30, f=20.0, L=40)
    assert len(frames) == 5
    rng = np.random.default_rng(12)
    scenes = []
    for fr in frames:
        prims_d = sqr.to_device(fr["prims"])
        rays = sqr.Rays.from_rig(fr["rig"], fr["t"])
        gd = dev_grid(fr["grid"])
        sc = sqr.Scene(prims_d, sqr.build_index(prims_d, gd), gd, rays, training=True)
        sc.grad_depth.copy_(torch.from_numpy(rng.standard_normal(rays.R).astype(np.float32)))
        sc.grad_sem.copy_(torch.from_numpy(rng.standard_normal((rays.R, 18)).astype(np.float32)))
        scenes.append(sc)
    refs = [_per_scene(sqr, sc) for sc in scenes]
    sqr.render_batched(sqr.SQ_OP_FWD, scenes)
    sqr.render_batched(sqr.SQ_OP_BWD, scenes)
    torch.cuda.synchronize()
    for sc, (d, s, tf, g) in zip(scenes, refs):
        assert torch.equal(sc.depth, d) and torch.equal(sc.sem, s)
        for k in g:
            check_grad(sc.grads[k].cpu().numpy(), g[k].cpu().numpy(), k, rtol=2e-3)
    for i in (0, len(frames) - 1):
        fr, sc = frames[i], scenes[i]
        idx = oracle_index(sc.index, fr["prims"], fr["grid"])
        D, S, T, _ = oracle.render_fwd(fr["prims"], fr["grid"], idx, fr["rig"], fr["t"])
        check_depth(sc.depth.cpu().numpy(), D, 0.5)
        check_sem(sc.sem.cpu().numpy(), S)
        ref = oracle.render_bwd(fr["prims"], fr["grid"], idx, fr["rig"], fr["t"],
                                sc.grad_depth.cpu().numpy().astype(np.float64),
                                sc.grad_sem.cpu().numpy().astype(np.float64))
        for k in ref:
            check_grad(sc.grads[k].cpu().numpy(), ref[k], k)


def _batch_sampled_parity(sqr, cfgs, n_rays=24, seed=0):
    """All scenes in one batched forward and backward (default tuning); each scene
    checked against the oracle on sampled rays (cotangents on those rays only).  With
    few rays their contributions can cancel, so the gradient check carries the FP32
    summation term of per_ray_magnitude.  (This test found the primitive records'
    FP32 construction too coarse near the planes u_j = 0 of a primitive's frame;
    they are now computed in FP64 and rounded once.)"""
    scenes = []
    for i, c in enumerate(cfgs):
        prims_d = sqr.to_device(c["prims"])
        rays = sqr.Rays.from_rig(c["rig"], c["t"])
        g = dev_grid(c["grid"])
        sc = sqr.Scene(prims_d, sqr.build_index(prims_d, g), g, rays)
        rng = np.random.default_rng(seed + i)
        ids = np.unique(rng.integers(0, rays.R, n_rays))
        C = c["prims"]["logits"].shape[1]
        gd = np.zeros(rays.R, np.float32)
        gs = np.zeros((rays.R, C), np.float32)
        gd[ids] = rng.standard_normal(len(ids))
        gs[ids] = rng.standard_normal((len(ids), C))
        sc.grad_depth.copy_(torch.from_numpy(gd))
        sc.grad_sem.copy_(torch.from_numpy(gs))
        scenes.append((sc, c, ids, gd, gs))
    batch = [s[0] for s in scenes]
    sqr.render_batched(sqr.SQ_OP_FWD, batch)
    sqr.render_batched(sqr.SQ_OP_BWD, batch)
    torch.cuda.synchronize()
    for sc, c, ids, gd, gs in scenes:
        idx = oracle_index(sc.index, c["prims"], c["grid"])
        D, S, _, _ = oracle.render_fwd(c["prims"], c["grid"], idx, c["rig"], c["t"], ray_ids=ids)
        check_depth(sc.depth.cpu().numpy()[ids], D, float(c["t"][0]))
        check_sem(sc.sem.cpu().numpy()[ids], S)
        ref = oracle.render_bwd(c["prims"], c["grid"], idx, c["rig"], c["t"], gd[ids].astype(np.float64),
                                gs[ids].astype(np.float64), ray_ids=ids)
        mag = per_ray_magnitude(c["prims"], c["grid"], idx, c["rig"], c["t"], gd, gs)
        for k in ref:
            check_grad(sc.grads[k].cpu().numpy(), ref[k], k, mag=mag[k])


def test_uneven_batch_of_12_full_size(sqr):
    """The bench's uneven batch at full size (12 scenes, 1-6 cameras, 225x400 or
    450x800 pixels, L 64-128, N 1000-12000): sampled rays of every scene."""
    _batch_sampled_parity(sqr, synth.make_batch_config(3), seed=30)


def test_eight_frames_of_8192(sqr):
    """Eight six-camera frames of 8,192 superquadrics each (the grid-query scene's
    distribution, 8 seeds) in one batched forward and backward."""
    _batch_sampled_parity(sqr, [synth.make_config(4, seed=40 + i) for i in range(8)], seed=40)
