"""The two conservative tests the primitive-major backward relies on, restated in
numpy FP32 with the kernels' formulas and checked against every ray of small
scenes (CPU): a primitive's projected pixel rectangle (k_pm_rects) holds every
pixel whose ray has a sample in the primitive's voxel box, and the slab test of a
candidate ray (k_pm_tiles) never rejects such a ray.  The GPU tests check the
kernels themselves against the oracle; these check that the geometry they use
cannot miss a run on inputs of the workloads' kinds."""
import numpy as np
import pytest

import oracle
from paper_2511_17361_gb300 import synth
from tests.helpers import box_sums, small_scene

f32 = np.float32


def _rays(rig):
    """FP32 ray directions and origins of every pixel, in the pinhole rule's op order."""
    dirs, origins = [], []
    H, W = rig["H"], rig["W"]
    for cam in range(rig["n_cam"]):
        fx, fy, cx, cy = rig["K"][cam]
        vv, uu = np.meshgrid(np.arange(H, dtype=f32), np.arange(W, dtype=f32), indexing="ij")
        dx = ((uu + f32(0.5)) - cx) / fx
        dy = ((vv + f32(0.5)) - cy) / fy
        nrm = np.sqrt((dx * dx + dy * dy) + f32(1.0))
        cd = np.stack([dx / nrm, dy / nrm, f32(1.0) / nrm], -1).reshape(-1, 3)
        R = rig["cam2world"][cam][:, :3]
        dirs.append(np.stack([(R[i, 0] * cd[:, 0] + R[i, 1] * cd[:, 1]) + R[i, 2] * cd[:, 2] for i in range(3)],
                             -1).astype(f32))
        origins.append(np.repeat(rig["cam2world"][cam][:, 3][None], H * W, 0))
    return np.concatenate(dirs).astype(f32), np.concatenate(origins).astype(f32)


def _rect(K, c2w, H, W, bl, bh, t0):
    """The box's pixel rectangle as k_pm_rects forms it (FP32), or None."""
    fx, fy, cx, cy = [f32(v) for v in K]
    R = c2w[:, :3].astype(f32)
    o = c2w[:, 3].astype(f32)
    A = np.zeros((3, 3), f32)
    A[0, 0] = R[1, 1] * R[2, 2] - R[1, 2] * R[2, 1]
    A[0, 1] = R[0, 2] * R[2, 1] - R[0, 1] * R[2, 2]
    A[0, 2] = R[0, 1] * R[1, 2] - R[0, 2] * R[1, 1]
    A[1, 0] = R[1, 2] * R[2, 0] - R[1, 0] * R[2, 2]
    A[1, 1] = R[0, 0] * R[2, 2] - R[0, 2] * R[2, 0]
    A[1, 2] = R[0, 2] * R[1, 0] - R[0, 0] * R[1, 2]
    A[2, 0] = R[1, 0] * R[2, 1] - R[1, 1] * R[2, 0]
    A[2, 1] = R[0, 1] * R[2, 0] - R[0, 0] * R[2, 1]
    A[2, 2] = R[0, 0] * R[1, 1] - R[0, 1] * R[1, 0]
    idet = f32(1) / f32(R[0, 0] * A[0, 0] + R[0, 1] * A[1, 0] + R[0, 2] * A[2, 0])
    P = []
    for c in range(8):
        w = np.array([bh[0] if c & 1 else bl[0], bh[1] if c & 2 else bl[1], bh[2] if c & 4 else bl[2]], f32)
        dw = (w - o).astype(f32)
        P.append(np.array([(A[i, 0] * dw[0] + A[i, 1] * dw[1] + A[i, 2] * dw[2]) * idet for i in range(3)], f32))
    P = np.array(P, f32)
    if t0 > 0:
        mx = f32(max(abs(f32(0.5) - cx), abs(f32(W) - f32(0.5) - cx)) / abs(fx))
        my = f32(max(abs(f32(0.5) - cy), abs(f32(H) - f32(0.5) - cy)) / abs(fy))
        zc = f32(f32(0.5) * f32(t0) / np.sqrt(f32(1) + mx * mx + my * my))
    else:
        if np.any(P[:, 2] <= 0):
            return 0, 0, W - 1, H - 1
        zc = f32(0)
    pts = [p for p in P if p[2] >= zc and p[2] > 0]
    if zc > 0:
        for c in range(8):
            for b in (1, 2, 4):
                if c & b:
                    continue
                za, zb = P[c][2], P[c | b][2]
                if (za < zc) == (zb < zc):
                    continue
                s = f32((zc - za) / (zb - za))
                q = (P[c] + s * (P[c | b] - P[c])).astype(f32)
                q[2] = zc
                pts.append(q)
    if not pts:
        return None
    pts = np.array(pts, f32)
    iz = (f32(1) / pts[:, 2]).astype(f32)
    u = (fx * pts[:, 0] * iz + cx - f32(0.5)).astype(f32)
    v = (fy * pts[:, 1] * iz + cy - f32(0.5)).astype(f32)
    u0, u1 = max(np.floor(u.min()) - 2, 0), min(np.ceil(u.max()) + 2, W - 1)
    v0, v1 = max(np.floor(v.min()) - 2, 0), min(np.ceil(v.max()) + 2, H - 1)
    if u0 > u1 or v0 > v1:
        return None
    return int(u0), int(v0), int(u1), int(v1)


def _slab_passes(o, d, bwl, bwh, glo, t0, tlast):
    """k_pm_tiles' slab test of rays (o, d) against the box grown by its FP32 margin."""
    tm = max(abs(t0), abs(tlast))
    dl = (f32(1e-5) * (np.abs(o) + np.abs(glo) + np.abs(bwl) + np.abs(bwh) + tm * np.abs(d)) + f32(1e-6)).astype(f32)
    flat = np.abs(d) < 1e-20
    with np.errstate(divide="ignore", invalid="ignore"):
        idd = np.where(flat, f32(0), f32(1) / np.where(flat, f32(1), d)).astype(f32)
        t1 = ((bwl - dl - o) * idd).astype(f32)
        t2 = ((bwh + dl - o) * idd).astype(f32)
    lo_t = np.where(flat, -np.inf, np.minimum(t1, t2) - (f32(1e-5) * np.abs(np.minimum(t1, t2)) + f32(1e-6)))
    hi_t = np.where(flat, np.inf, np.maximum(t1, t2) + (f32(1e-5) * np.abs(np.maximum(t1, t2)) + f32(1e-6)))
    flat_miss = np.any(flat & ((o < bwl - dl) | (o > bwh + dl)), 1)
    return (np.maximum(t0, lo_t.max(1)) <= np.minimum(tlast, hi_t.min(1))) & ~flat_miss


def _check(pr, grid, rig, t, kmax=None):
    ix = oracle.build_index(pr, grid)
    ranges = ix["ranges"]
    d_all, o_all = _rays(rig)
    t = t.astype(f32)
    lo = np.asarray(grid["lo"], f32)
    inv = (f32(1.0) / np.asarray(grid["vs"], f32)).astype(f32)
    nf = np.asarray(grid["n"]).astype(f32)
    H, W = rig["H"], rig["W"]
    prims = [k for k in range(len(pr["means"]) if kmax is None else kmax)
             if ranges[k][1] >= ranges[k][0] and ranges[k][3] >= ranges[k][2] and ranges[k][5] >= ranges[k][4]]
    boxes = {}
    for k in prims:
        r6 = ranges[k]
        boxes[k] = (np.array([f32(grid["lo"][a]) + f32(r6[2 * a]) * f32(grid["vs"][a]) for a in range(3)], f32),
                    np.array([f32(grid["lo"][a]) + f32(r6[2 * a + 1] + 1) * f32(grid["vs"][a]) for a in range(3)], f32))
    runs = 0
    for c in range(rig["n_cam"]):  # one camera's rays at a time
        d, o = d_all[c * H * W:(c + 1) * H * W], o_all[c * H * W:(c + 1) * H * W]
        x = (o[:, None, :] + (t[None, :, None] * d[:, None, :]).astype(f32)).astype(f32)
        u = ((x - lo).astype(f32) * inv).astype(f32)
        inside = np.all((u >= 0) & (u < nf), -1)
        idx = np.floor(np.where(inside[..., None], u, 0)).astype(np.int16)
        for k in prims:
            r6 = ranges[k]
            hit = (inside & np.all((idx >= r6[[0, 2, 4]]) & (idx <= r6[[1, 3, 5]]), -1)).any(1)
            runs += hit.sum()
            bl, bh = boxes[k]
            rc = _rect(rig["K"][c], rig["cam2world"][c], H, W, bl, bh, float(t[0]))
            m = np.zeros((H, W), bool)
            if rc is not None:
                m[rc[1]:rc[3] + 1, rc[0]:rc[2] + 1] = True
            assert not (hit.reshape(H, W) & ~m).any(), f"primitive {k}, camera {c}: a run lies outside the rectangle"
            passes = _slab_passes(o, d, bl, bh, lo, t[0], t[-1])
            assert not (hit & ~passes).any(), f"primitive {k}, camera {c}: the slab test misses a run"
    return runs


@pytest.mark.parametrize("case", ["near_plane_from_zero", "camera_among_boxes", "ring"])
def test_rectangles_and_slab_test_never_miss_a_run(case):
    if case == "near_plane_from_zero":
        pr, grid, rig, _ = small_scene(21, n=9, H=9, W=11, L=30)
        t = synth.sample_depths(30, 0.0, 9.5)
    elif case == "camera_among_boxes":
        rng = np.random.default_rng(22)
        pr, grid, rig, t = small_scene(22, n=10, H=10, W=12, L=36)
        means = pr["means"].copy()
        means[:4] = np.stack([rng.uniform(-2.0, 0.0, 4), rng.uniform(-1.0, 1.0, 4), rng.uniform(0.5, 1.5, 4)], 1)
        pr["means"] = means.astype(np.float32)
    else:
        pr, grid = synth.prims_driving(300, 24), synth.grid_spec(50, 50, 8)
        rig, t = synth.rig_ring(n_cam=6, H=12, W=20, f=9.0), synth.sample_depths(40)
    assert _check(pr, grid, rig, t) > 500


def test_full_frame_primitives_never_miss_a_run():
    """Every ray of the six-camera frame for its first 12 primitives."""
    cfg = synth.make_config(1)
    assert _check(cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], kmax=12) > 10000


def _runs_from_estimates(pr, grid, rig, t, kmax=None):
    """For every (ray, primitive) of the scene: the samples whose FP32 voxel lies in
    the primitive's box form one interval, and whenever k_pm_tiles' four voxel-rule
    tests accept the interval the six plane-crossing estimates give (its end samples
    inside the box, the samples just outside it outside), that interval is the exact
    one.  Returns (runs, runs accepted by the tests)."""
    ix = oracle.build_index(pr, grid)
    ranges = ix["ranges"]
    d_all, o_all = _rays(rig)
    t = t.astype(f32)
    L = len(t)
    lo = np.asarray(grid["lo"], f32)
    vs = np.asarray(grid["vs"], f32)
    inv = (f32(1.0) / vs).astype(f32)
    nf = np.asarray(grid["n"]).astype(f32)
    inv_dt = f32((L - 1) / (t[-1] - t[0])) if L > 1 and t[-1] > t[0] else f32(0)
    H, W = rig["H"], rig["W"]
    prims = [k for k in range(len(pr["means"]) if kmax is None else kmax)
             if ranges[k][1] >= ranges[k][0] and ranges[k][3] >= ranges[k][2] and ranges[k][5] >= ranges[k][4]]
    runs = accepted = 0
    for c in range(rig["n_cam"]):
        d, o = d_all[c * H * W:(c + 1) * H * W], o_all[c * H * W:(c + 1) * H * W]
        x = (o[:, None, :] + (t[None, :, None] * d[:, None, :]).astype(f32)).astype(f32)
        u = ((x - lo).astype(f32) * inv).astype(f32)
        inside = np.all((u >= 0) & (u < nf), -1)
        idx = np.floor(np.where(inside[..., None], u, 0)).astype(np.int32)
        rows = np.arange(H * W)
        for k in prims:
            r6 = ranges[k]
            hit = inside & np.all((idx >= r6[[0, 2, 4]]) & (idx <= r6[[1, 3, 5]]), -1)
            n_in = hit.sum(1)
            has = n_in > 0
            first = np.argmax(hit, 1)
            last = L - 1 - np.argmax(hit[:, ::-1], 1)
            assert np.all(n_in[has] == last[has] - first[has] + 1), f"primitive {k}: a run is not one interval"
            runs += int(has.sum())
            # the estimates, as k_pm_tiles forms them (an exact quotient stands in for the approximate 1 / d)
            blo = np.asarray(r6[[0, 2, 4]], f32)
            bhi = (np.asarray(r6[[1, 3, 5]]) + 1).astype(f32)
            neg = d < 0
            ok = np.all(d != 0, 1)
            with np.errstate(divide="ignore", invalid="ignore"):
                def est(thr):
                    ts = ((thr * vs + lo - o) / np.where(d != 0, d, f32(1))).astype(f32)
                    return np.clip(np.ceil((ts - t[0]) * inv_dt), 0, L).astype(np.int64)
                j0e = est(np.where(neg, bhi, blo)).max(1)
                j1e = est(np.where(neg, blo, bhi)).min(1)
            cand = ok & (j0e < j1e)
            j0c, j1c = np.clip(j0e, 0, L - 1), np.clip(j1e - 1, 0, L - 1)
            before = np.where(j0e > 0, hit[rows, np.clip(j0e - 1, 0, L - 1)], False)
            after = np.where(j1e < L, hit[rows, np.clip(j1e, 0, L - 1)], False)
            acc = cand & hit[rows, j0c] & hit[rows, j1c] & ~before & ~after
            assert np.all(first[acc] == j0e[acc]) and np.all(last[acc] + 1 == j1e[acc]), \
                f"primitive {k}, camera {c}: an accepted interval is not the run"
            accepted += int(acc.sum())
    return runs, accepted


def test_confirmed_estimates_give_the_exact_run():
    """The run ends k_pm_tiles takes without a search: on the ring scene and on the
    six-camera frame's first 12 primitives (every ray, every sample), each run is one
    interval, every interval the four tests accept is the run, and they accept nearly
    all runs (the rest go to the per-axis searches)."""
    pr, grid = synth.prims_driving(300, 24), synth.grid_spec(50, 50, 8)
    rig, t = synth.rig_ring(n_cam=6, H=12, W=20, f=9.0), synth.sample_depths(40)
    runs, accepted = _runs_from_estimates(pr, grid, rig, t)
    assert runs > 500 and accepted >= 0.95 * runs
    cfg = synth.make_config(1)
    runs, accepted = _runs_from_estimates(cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"], kmax=12)
    assert runs > 10000 and accepted >= 0.95 * runs


def test_box_sums_equal_brute_force():
    """The summed-volume box sums used by the pair-visit check equal direct sums
    over every inclusive range, empty ranges giving 0."""
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 50, (7, 5, 4))
    ranges = []
    for _ in range(200):
        r = []
        for n in counts.shape:
            a, b = sorted(rng.integers(0, n, 2))
            r += [a, b]
        ranges.append(r)
    ranges += [[0, -1, 0, -1, 0, -1], [3, 2, 0, 4, 0, 3], [0, 6, 0, 4, 0, 3]]
    ranges = np.array(ranges, np.int32)
    got = box_sums(counts, ranges)
    for r, g in zip(ranges, got):
        want = counts[r[0]:r[1] + 1, r[2]:r[3] + 1, r[4]:r[5] + 1].sum() if r[1] >= r[0] and r[3] >= r[2] and \
            r[5] >= r[4] else 0
        assert g == want
