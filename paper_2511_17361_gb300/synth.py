"""Seeded synthetic scenes, camera rigs and sample depths.

This module only draws inputs.  It holds none of the renderer's arithmetic
(no inside-outside function, no index, no compositing), so both the CUDA path
and the FP64 oracle can be fed from it without sharing any of the method.

The recipes follow the paper's driving workloads:

* scene box [-40, 40] x [-40, 40] x [-1, 5.4] m at 0.4 m voxels (Sec. 4.1),
* a surround rig of six pinhole cameras (Sec. 4.2, six-camera renders of Tab. 3a),
* N = 1.6k-16k superquadrics (Tab. 4c), L = 48-128 uniform samples (Tab. 4d),
* parameter ranges of Supp. A.9 (eps in [0.1, 2.0], opacity in [0, 1]) with the
  trained-parameter shapes of the supplementary parameter-distribution study
  (flat ground primitives with small eps1, objects with rounder shapes).

Every array is float32 (int32 for labels) and C-contiguous.  Quaternions are
(w, x, y, z).  Cameras use OpenCV axes (x right, y down, z forward) mapped to
the ego frame (x forward, y left, z up); ``cam2world`` is [R | centre] with the
columns of R the camera axes in world coordinates.
"""
from __future__ import annotations

import numpy as np

N_CLASSES = 18
SCENE_LO = (-40.0, -40.0, -1.0)
SCENE_HI = (40.0, 40.0, 5.4)


# --------------------------------------------------------------------------- grids
def grid_spec(nx: int, ny: int, nz: int, lo=SCENE_LO, hi=SCENE_HI) -> dict:
    """Axis-aligned voxel grid over [lo, hi] with nx*ny*nz cells (voxel size per axis)."""
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    n = np.array([nx, ny, nz], np.float64)
    vs = ((hi.astype(np.float64) - lo.astype(np.float64)) / n).astype(np.float32)
    return {"n": (int(nx), int(ny), int(nz)), "lo": lo, "vs": vs}


# --------------------------------------------------------------------------- primitives
def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _yaw_quats(rng, n):
    yaw = rng.uniform(-np.pi, np.pi, n)
    q = np.zeros((n, 4))
    q[:, 0] = np.cos(0.5 * yaw)
    q[:, 3] = np.sin(0.5 * yaw)
    return q


def _sigmoid_normal(rng, n):
    return 1.0 / (1.0 + np.exp(-rng.standard_normal(n)))


def _pack(means, quats, scales, eps, opacity, logits) -> dict:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"means": f(means), "quats": f(quats), "scales": f(scales), "eps": f(eps),
            "opacity": f(opacity), "logits": f(logits)}


def prims_uniform(n, seed, s_range=(0.2, 3.0), eps_range=(0.2, 1.8), n_classes=N_CLASSES,
                  lo=SCENE_LO, hi=SCENE_HI) -> dict:
    """Objects: centres uniform in the scene box, scales U(s_range)^3, random unit
    quaternions, eps1, eps2 ~ U(eps_range), opacity = sigmoid(N(0,1)), logits N(0,1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, (n, 3))
    scales = rng.uniform(*s_range, (n, 3))
    quats = _unit_quats(rng, n)
    eps = rng.uniform(*eps_range, (n, 2))
    opacity = _sigmoid_normal(rng, n)
    logits = rng.standard_normal((n, n_classes))
    return _pack(means, quats, scales, eps, opacity, logits)


def prims_driving(n, seed, ground_frac=0.7, n_classes=N_CLASSES) -> dict:
    """Driving-scene mix: ``ground_frac`` flat ground primitives (centres over the
    xy box with z in U(-1, 0.5), yaw-only rotation, s_xy ~ U(0.2, 3), s_z ~ U(0.2, 0.5),
    eps1 ~ U(0.1, 0.3), eps2 ~ U(0.2, 1.8)) and the rest objects drawn as in
    :func:`prims_uniform`.  The ground rows come first, then the objects, then
    the whole set is shuffled with the same seed."""
    rng = np.random.default_rng(seed)
    ng = int(round(ground_frac * n))
    no = n - ng
    gm = np.stack([rng.uniform(-40, 40, ng), rng.uniform(-40, 40, ng), rng.uniform(-1.0, 0.5, ng)], 1)
    gs = np.stack([rng.uniform(0.2, 3.0, ng), rng.uniform(0.2, 3.0, ng), rng.uniform(0.2, 0.5, ng)], 1)
    gq = _yaw_quats(rng, ng)
    ge = np.stack([rng.uniform(0.1, 0.3, ng), rng.uniform(0.2, 1.8, ng)], 1)
    om = rng.uniform(SCENE_LO, SCENE_HI, (no, 3))
    os_ = rng.uniform(0.2, 3.0, (no, 3))
    oq = _unit_quats(rng, no)
    oe = rng.uniform(0.2, 1.8, (no, 2))
    means = np.concatenate([gm, om])
    scales = np.concatenate([gs, os_])
    quats = np.concatenate([gq, oq])
    eps = np.concatenate([ge, oe])
    opacity = _sigmoid_normal(rng, n)
    logits = rng.standard_normal((n, n_classes))
    perm = rng.permutation(n)
    return _pack(means[perm], quats[perm], scales[perm], eps[perm], opacity[perm], logits[perm])


def prims_clustered(n, seed, n_clusters=512, spread=1.5, s_range=(0.15, 0.6), eps_range=(0.1, 1.9),
                    n_classes=N_CLASSES) -> dict:
    """Heavy-overlap stress set: ``n_clusters`` cluster centres uniform in the scene
    box (z in [-1, 3]), members offset by N(0, spread) m, scales U(s_range)^3, random
    rotations, eps1, eps2 ~ U(eps_range)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform((-38, -38, -1.0), (38, 38, 3.0), (n_clusters, 3))
    which = rng.integers(0, n_clusters, n)
    means = centres[which] + rng.normal(0.0, spread, (n, 3))
    scales = rng.uniform(*s_range, (n, 3))
    quats = _unit_quats(rng, n)
    eps = rng.uniform(*eps_range, (n, 2))
    opacity = _sigmoid_normal(rng, n)
    logits = rng.standard_normal((n, n_classes))
    return _pack(means, quats, scales, eps, opacity, logits)


# --------------------------------------------------------------------------- cameras
def camera_pose(yaw, centre):
    """cam2world [3, 4] of a level camera looking along world yaw ``yaw`` (rad)."""
    c, s = np.cos(yaw), np.sin(yaw)
    fwd = np.array([c, s, 0.0])
    right = np.array([s, -c, 0.0])
    down = np.array([0.0, 0.0, -1.0])
    m = np.zeros((3, 4))
    m[:, 0], m[:, 1], m[:, 2], m[:, 3] = right, down, fwd, centre
    return m


def rig_single(H=64, W=112, f=80.0, centre=(0.0, 0.0, 1.6)) -> dict:
    K = np.array([[f, f, W / 2.0, H / 2.0]], np.float32)
    c2w = camera_pose(0.0, np.asarray(centre, np.float64))[None]
    return {"n_cam": 1, "H": int(H), "W": int(W), "K": K, "cam2world": np.ascontiguousarray(c2w, np.float32)}


def rig_ring(n_cam=6, H=225, W=400, f=250.0, radius=1.0, height=1.6, cams=None) -> dict:
    """Surround ring at 60 degree yaw spacing; ``cams`` selects a subset of the six."""
    idx = list(range(6)) if cams is None else list(cams)
    idx = idx[:n_cam]
    Ks, poses = [], []
    for i in idx:
        yaw = np.deg2rad(60.0 * i)
        centre = np.array([radius * np.cos(yaw), radius * np.sin(yaw), height])
        Ks.append([f, f, W / 2.0, H / 2.0])
        poses.append(camera_pose(yaw, centre))
    return {"n_cam": len(idx), "H": int(H), "W": int(W),
            "K": np.ascontiguousarray(Ks, np.float32), "cam2world": np.ascontiguousarray(poses, np.float32)}


def sample_depths(L, t_near=0.5, t_far=45.0) -> np.ndarray:
    """L uniformly spaced depths including both ends (float32, ascending)."""
    return np.linspace(t_near, t_far, L).astype(np.float32)


def loss_targets(R, seed, n_classes=N_CLASSES, t_near=0.5, t_far=45.0):
    """Random per-pixel depth targets U(t_near, t_far) and labels U{0..C-1}."""
    rng = np.random.default_rng(seed + 1000)
    depth = rng.uniform(t_near, t_far, R).astype(np.float32)
    labels = rng.integers(0, n_classes, R).astype(np.int32)
    return depth, labels


def cotangents(R, seed, n_classes=N_CLASSES, scale_d=1.0, scale_s=1.0):
    """Random output cotangents (dL/dD, dL/dS) for linear-loss gradient checks."""
    rng = np.random.default_rng(seed + 2000)
    gd = (scale_d * rng.standard_normal(R)).astype(np.float32)
    gs = (scale_s * rng.standard_normal((R, n_classes))).astype(np.float32)
    return gd, gs


# --------------------------------------------------------------------------- configs
def make_config(idx: int, seed: int | None = None) -> dict:
    """The five workloads: 0 small single camera, 1 six-camera training frame,
    2 backward stress, 4 grid-query scene.  (Workload 3, the batch, is
    :func:`make_batch_config`.)"""
    s = idx if seed is None else seed
    if idx == 0:
        return {"name": "cam1_64x112_L48_N256", "prims": prims_uniform(256, s), "grid": grid_spec(50, 50, 8),
                "rig": rig_single(), "t": sample_depths(48), "kappa": 0.0, "alpha_max": 1.0}
    if idx == 1:
        return {"name": "ring6_225x400_L100_N4096", "prims": prims_driving(4096, s), "grid": grid_spec(200, 200, 16),
                "rig": rig_ring(), "t": sample_depths(100), "kappa": 0.0, "alpha_max": 1.0}
    if idx == 2:
        return {"name": "ring6_225x400_L100_N16384_clustered", "prims": prims_clustered(16384, s),
                "grid": grid_spec(200, 200, 16), "rig": rig_ring(), "t": sample_depths(100),
                "kappa": 0.0, "alpha_max": 1.0}
    if idx == 4:
        return {"name": "grid200x200x16_N8192", "prims": prims_driving(8192, s), "grid": grid_spec(200, 200, 16),
                "rig": rig_ring(), "t": sample_depths(100), "kappa": 0.0, "alpha_max": 1.0}
    raise ValueError(f"unknown workload {idx}")


def make_temporal_config(T: int = 6, n: int = 1600, seed: int = 6, H: int = 225, W: int = 400, f: float = 250.0,
                         L: int = 100, ego_step: float = 0.5, speed: float = 0.4) -> list[dict]:
    """Temporal horizon of Sec. 3.2: the 2T+1 frames t = -T..T of one superquadric
    set (N = 1600, T = 6 as in the paper's training, Sec. 4.2) whose properties
    are shared and whose means move by a per-frame offset v(t) = t * u_i (u_i per
    primitive: 0 for the ground, N(0, speed^2) m per frame in x and y for objects),
    each frame rendered by the six-camera rig moved by the ego motion t * ego_step m
    along +x.  The grid stays centred on the current frame's ego pose."""
    base = prims_driving(n, seed)
    rng = np.random.default_rng(seed + 17)
    ground = base["scales"][:, 2] <= 0.5
    ground &= (base["eps"][:, 0] <= 0.3)
    u = np.zeros((n, 3))
    u[~ground, :2] = rng.normal(0.0, speed, (int((~ground).sum()), 2))
    frames = []
    for t in range(-T, T + 1):
        pr = {k: v.copy() for k, v in base.items()}
        pr["means"] = (base["means"].astype(np.float64) + t * u).astype(np.float32)
        rig = rig_ring(H=H, W=W, f=f)
        rig["cam2world"] = rig["cam2world"].copy()
        rig["cam2world"][:, 0, 3] += np.float32(t * ego_step)
        frames.append({"name": f"frame{t:+d}", "t_index": t, "prims": pr, "grid": grid_spec(200, 200, 16),
                       "rig": rig, "t": sample_depths(L), "kappa": 0.0, "alpha_max": 1.0})
    return frames


def make_batch_config(seed: int = 3, n_scenes: int = 12) -> list[dict]:
    """Uneven batch: per scene N ~ U{1000..12000}, 1-6 ring cameras, 225x400 (f=250)
    or 450x800 (f=500) rays, L ~ U{64..128}, each with its own 200x200x16 grid."""
    rng = np.random.default_rng(seed)
    scenes = []
    for i in range(n_scenes):
        n = int(rng.integers(1000, 12001))
        n_cam = int(rng.integers(1, 7))
        hi_res = bool(rng.integers(0, 2))
        L = int(rng.integers(64, 129))
        H, W, f = (450, 800, 500.0) if hi_res else (225, 400, 250.0)
        scenes.append({"name": f"scene{i}", "prims": prims_driving(n, 100 * seed + i), "grid": grid_spec(200, 200, 16),
                       "rig": rig_ring(n_cam=n_cam, H=H, W=W, f=f), "t": sample_depths(L),
                       "kappa": 0.0, "alpha_max": 1.0})
    return scenes


def n_rays(rig: dict) -> int:
    return rig["n_cam"] * rig["H"] * rig["W"]
