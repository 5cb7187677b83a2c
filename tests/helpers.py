"""Shared helpers for the tests: tiny hand-made scenes and an independent
brute-force renderer for small inputs (numpy + scipy's rotation, no index)."""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

from paper_2511_17361_gb300 import synth


def prims_from(means, quats, scales, eps, opacity, logits) -> dict:
    f = lambda a: np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    return {"means": f(means).reshape(-1, 3), "quats": f(quats).reshape(-1, 4), "scales": f(scales).reshape(-1, 3),
            "eps": f(eps).reshape(-1, 2), "opacity": f(opacity).reshape(-1), "logits": f(logits)}


def axis_camera(centre=(0.0, 0.0, 0.0), yaw=0.0) -> dict:
    """A 1x1 camera whose single ray is exactly the camera's forward axis."""
    c2w = synth.camera_pose(yaw, np.asarray(centre, np.float64))[None]
    return {"n_cam": 1, "H": 1, "W": 1, "K": np.array([[1.0, 1.0, 0.5, 0.5]], np.float32),
            "cam2world": np.ascontiguousarray(c2w, np.float32)}


def small_scene(seed, n=6, H=6, W=8, L=24, gn=(8, 8, 4), s_range=(0.6, 1.6), eps_range=(0.3, 1.7),
                sigma_max=0.35, C=5):
    """A small random scene in a 16x16x4 m box seen by one camera; opacities are
    kept low so that the alpha clamp stays far from active."""
    rng = np.random.default_rng(seed)
    lo, hi = (-8.0, -8.0, -1.0), (8.0, 8.0, 3.0)
    grid = synth.grid_spec(*gn, lo=lo, hi=hi)
    means = np.stack([rng.uniform(1.0, 7.0, n), rng.uniform(-3, 3, n), rng.uniform(-0.5, 2.5, n)], 1)
    q = rng.standard_normal((n, 4))
    q *= rng.uniform(0.5, 2.0, (n, 1))  # deliberately not unit length
    prims = prims_from(means, q, rng.uniform(*s_range, (n, 3)), rng.uniform(*eps_range, (n, 2)),
                       rng.uniform(0.05, sigma_max, n), rng.standard_normal((n, C)))
    rig = synth.rig_single(H=H, W=W, f=6.0, centre=(-1.0, 0.0, 1.0))
    t = synth.sample_depths(L, 0.5, 9.5)
    return prims, grid, rig, t


# ---------------------------------------------------------------- brute force
def _fp32_samples(rig, t):
    """FP32 sample positions [R, L, 3] with the documented op order."""
    K, c2w = rig["K"], rig["cam2world"]
    out = []
    for cam in range(rig["n_cam"]):
        fx, fy, cx, cy = K[cam]
        vv, uu = np.meshgrid(np.arange(rig["H"], dtype=np.float32), np.arange(rig["W"], dtype=np.float32),
                             indexing="ij")
        dx = ((uu + np.float32(0.5)) - cx) / fx
        dy = ((vv + np.float32(0.5)) - cy) / fy
        n2 = (dx * dx + dy * dy) + np.float32(1.0)
        nrm = np.sqrt(n2)
        cam_d = np.stack([dx / nrm, dy / nrm, np.float32(1.0) / nrm], -1).reshape(-1, 3)
        R = c2w[cam, :, :3]
        d = np.stack([(R[i, 0] * cam_d[:, 0] + R[i, 1] * cam_d[:, 1]) + R[i, 2] * cam_d[:, 2] for i in range(3)], -1)
        o = c2w[cam, :, 3]
        x = o[None, None, :] + (t.astype(np.float32)[None, :, None] * d[:, None, :])
        out.append(x.astype(np.float32))
    return np.concatenate(out, 0)


def _inside(grid, x):
    lo, vs = grid["lo"], grid["vs"]
    inv = (np.float32(1.0) / vs).astype(np.float32)
    u = ((x - lo) * inv).astype(np.float32)
    n = np.asarray(grid["n"], np.float32)
    return np.all((u >= 0) & (u < n), axis=-1)


def brute_p(prims, x):
    """p_o of every primitive at points x [..., 3] -> [..., N] (FP64, scipy rotation)."""
    q = prims["quats"].astype(np.float64)
    Rm = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # local -> world
    d = x[..., None, :].astype(np.float64) - prims["means"].astype(np.float64)
    xl = np.einsum("nij,...ni->...nj", Rm, d)
    s = prims["scales"].astype(np.float64)
    e1 = prims["eps"][:, 0].astype(np.float64)
    e2 = prims["eps"][:, 1].astype(np.float64)
    a = np.abs(xl) / s
    A = a[..., 0] ** (2 / e2) + a[..., 1] ** (2 / e2)
    f = A ** (e2 / e1) + a[..., 2] ** (2 / e1)
    return np.exp(-f)


def brute_render(prims, grid, rig, t, alpha_max=1.0):
    """Eq. 4-6 summing over ALL primitives at every in-grid sample."""
    x = _fp32_samples(rig, t)
    inside = _inside(grid, x)
    p = brute_p(prims, x) * inside[..., None]
    sig = prims["opacity"].astype(np.float64)
    c = prims["logits"].astype(np.float64)
    ssum = p @ sig
    alpha = np.minimum(ssum, alpha_max)
    sem_s = p @ c
    R, L = alpha.shape
    T = np.ones(R)
    D = np.zeros(R)
    S = np.zeros((R, c.shape[1]))
    for j in range(L):
        w = T * alpha[:, j]
        D += w * t[j]
        S += w[:, None] * sem_s[:, j]
        T = T * (1 - alpha[:, j])
    return D, S, T


def richardson_fd(loss, prims, name, i, h):
    """Central difference of loss(prims) in prims[name].flat[i], Richardson-extrapolated
    from steps h and h/2 (removes the O(h^2) term).  Steps are exact in FP32."""
    flat = prims[name].reshape(-1)
    x = flat[i]

    def cd(hh):
        hf = np.float32(hh)
        xp, xm = x + hf, x - hf
        assert float(xp) - float(x) == hh and float(x) - float(xm) == hh
        vals = []
        for xv in (xp, xm):
            f2 = flat.copy()
            f2[i] = xv
            p2 = dict(prims)
            p2[name] = f2.reshape(prims[name].shape)
            vals.append(loss(p2))
        return (vals[0] - vals[1]) / (2 * hh)

    return (4 * cd(h / 2) - cd(h)) / 3


def box_sums(counts, ranges):
    """Per primitive, the sum of counts [nx, ny, nz] over its inclusive voxel range
    (i0, i1, j0, j1, k0, k1); 0 for an empty range.  A summed-volume table in int64."""
    sat = np.zeros(tuple(n + 1 for n in counts.shape), np.int64)
    sat[1:, 1:, 1:] = counts.astype(np.int64).cumsum(0).cumsum(1).cumsum(2)
    r = ranges.astype(np.int64)
    i0, i1, j0, j1, k0, k1 = (r[:, c] for c in range(6))
    empty = (i1 < i0) | (j1 < j0) | (k1 < k0)
    i0, j0, k0 = [np.where(empty, 0, a) for a in (i0, j0, k0)]
    i1, j1, k1 = [np.where(empty, -1, a) + 1 for a in (i1, j1, k1)]
    tot = (sat[i1, j1, k1] - sat[i0, j1, k1] - sat[i1, j0, k1] - sat[i1, j1, k0] + sat[i0, j0, k1] + sat[i0, j1, k0]
           + sat[i1, j0, k0] - sat[i0, j0, k0])
    return np.where(empty, 0, tot)
