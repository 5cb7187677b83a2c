"""Pins of the FP64 oracle against things other than itself: closed forms of
Eq. 1-2, the rotation convention, hand-computed voxel boxes, brute force over
all primitives, a 1-D compositing recurrence along an axis ray, the
transmittance identity, and central finite differences of the backward.
CPU only."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2511_17361_gb300 import synth
from tests.helpers import _fp32_samples, axis_camera, brute_p, brute_render, prims_from, richardson_fd, small_scene


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


# --------------------------------------------------------------------- Eq. 1, 2
def test_sphere_is_isotropic_gaussian():
    """eps1 = eps2 = 1 and equal scales r: p_o = exp(-|x - m|^2 / r^2) for any rotation."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        m = rng.uniform(-5, 5, 3)
        q = rng.standard_normal(4)
        r = rng.uniform(0.3, 3)
        x = m + rng.normal(0, r, 3)
        want = math.exp(-np.sum((x - m) ** 2) / r ** 2)
        assert oracle.sq_p(x, m, q, [r, r, r], 1.0, 1.0) == pytest.approx(want, rel=1e-13, abs=1e-300)


def test_ellipsoid_axis_aligned():
    """eps = 1, identity rotation: p_o = exp(-sum((x_i - m_i)/s_i)^2)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        m, s = rng.uniform(-5, 5, 3), rng.uniform(0.2, 3, 3)
        x = m + rng.normal(0, 1.5, 3)
        want = math.exp(-np.sum(((x - m) / s) ** 2))
        assert oracle.sq_p(x, m, [1, 0, 0, 0], s, 1.0, 1.0) == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_along_a_local_axis_exponent_is_two_over_eps1(axis):
    """On a local axis only one coordinate is non-zero and f = (|x_i|/s_i)^(2/eps1):
    the eps2 exponents cancel on the x and y axes (Eq. 1)."""
    rng = np.random.default_rng(2 + axis)
    for _ in range(30):
        s = rng.uniform(0.2, 3, 3)
        e1, e2 = rng.uniform(0.1, 2.0, 2)
        xl = np.zeros(3)
        xl[axis] = rng.uniform(-2, 2) * s[axis]
        want = (abs(xl[axis]) / s[axis]) ** (2 / e1)
        assert oracle.sq_f(xl, s, e1, e2) == pytest.approx(want, rel=1e-12)


def test_equator_plane_uses_eps2_roundness():
    """In the z = 0 plane with |x|/sx = |y|/sy = a: f = (2 a^(2/e2))^(e2/e1)."""
    for a, e1, e2 in [(0.7, 0.5, 1.5), (1.3, 1.2, 0.3), (0.4, 2.0, 0.1)]:
        s = np.array([1.5, 0.5, 2.0])
        xl = np.array([a * s[0], -a * s[1], 0.0])
        assert oracle.sq_f(xl, s, e1, e2) == pytest.approx((2 * a ** (2 / e2)) ** (e2 / e1), rel=1e-12)


def test_rotation_convention_local_x_to_world_y():
    """q = (cos 45, 0, 0, sin 45) turns local +x onto world +y (Hamilton, local->world),
    so a primitive long along local x is long along world y."""
    q = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]
    m = np.array([1.0, 2.0, 3.0])
    s = [3.0, 0.5, 0.5]
    assert oracle.sq_p(m + [0, 2.0, 0], m, q, s, 1.0, 1.0) == pytest.approx(math.exp(-(2 / 3) ** 2), rel=1e-13)
    assert oracle.sq_p(m + [2.0, 0, 0], m, q, s, 1.0, 1.0) == pytest.approx(math.exp(-(2 / 0.5) ** 2), rel=1e-12)


def test_quaternion_sign_and_scale_invariance():
    rng = np.random.default_rng(5)
    for _ in range(30):
        m, s = rng.uniform(-2, 2, 3), rng.uniform(0.3, 2, 3)
        q = rng.standard_normal(4)
        e1, e2 = rng.uniform(0.1, 2, 2)
        x = m + rng.normal(0, 1, 3)
        p = oracle.sq_p(x, m, q, s, e1, e2)
        assert oracle.sq_p(x, m, -q, s, e1, e2) == pytest.approx(p, rel=1e-12, abs=1e-300)
        assert oracle.sq_p(x, m, 3.7 * q, s, e1, e2) == pytest.approx(p, rel=1e-12, abs=1e-300)


def test_swap_x_y_with_scales():
    """f is symmetric under swapping (x, sx) with (y, sy)."""
    rng = np.random.default_rng(6)
    for _ in range(30):
        xl, s = rng.normal(0, 1, 3), rng.uniform(0.3, 2, 3)
        e1, e2 = rng.uniform(0.1, 2, 2)
        f1 = oracle.sq_f(xl, s, e1, e2)
        f2 = oracle.sq_f(xl[[1, 0, 2]], s[[1, 0, 2]], e1, e2)
        assert f2 == pytest.approx(f1, rel=1e-13)


def test_matches_scipy_rotation_at_random_points():
    """Eq. 2 against an independent evaluation using scipy's quaternion rotation."""
    pr, grid, rig, t = small_scene(7, n=10)
    rng = np.random.default_rng(7)
    x = rng.uniform(-3, 8, (40, 3))
    bp = brute_p(pr, x)
    for k in range(10):
        for i in range(40):
            got = oracle.sq_p(x[i], pr["means"][k], pr["quats"][k], pr["scales"][k], float(pr["eps"][k, 0]),
                              float(pr["eps"][k, 1]))
            assert got == pytest.approx(bp[i, k], rel=1e-11, abs=1e-300)


# --------------------------------------------------------------------- index
def test_obb_box_axis_aligned_by_hand():
    """Identity rotation: half-extent h = s * ln(1/tau)^(eps1/2); the box is
    floor((m -+ h - lo)/vs), clipped.  At m + h e_i the occupancy equals tau."""
    grid = synth.grid_spec(20, 20, 10, lo=(-10, -10, -5), hi=(10, 10, 5))
    means = [[0.3, -2.2, 1.1], [9.5, 9.5, 4.5], [-30, 0, 0]]
    scales = [[1.0, 2.0, 0.5], [2.0, 2.0, 2.0], [1.0, 1.0, 1.0]]
    eps = [[1.0, 0.5], [0.25, 1.0], [1.0, 1.0]]
    pr = prims_from(means, [[1, 0, 0, 0]] * 3, scales, eps, [0.5] * 3, np.zeros((3, 2)))
    tau = 0.01
    rg, ties = oracle.ranges(pr, grid, 0, tau, 5)
    assert ties == 0
    K = math.log(1 / np.float32(tau))
    for k in range(2):
        h = np.array(scales[k]) * K ** (eps[k][0] / 2)
        for j in range(3):
            lo = math.floor((means[k][j] - h[j] - grid["lo"][j]) / grid["vs"][j])
            hi = math.floor((means[k][j] + h[j] - grid["lo"][j]) / grid["vs"][j])
            assert rg[k, 2 * j] == max(lo, 0)
            assert rg[k, 2 * j + 1] == min(hi, grid["n"][j] - 1)
            e = np.zeros(3)
            e[j] = h[j]
            p_edge = oracle.sq_p(np.array(means[k]) + e, means[k], [1, 0, 0, 0], scales[k], *eps[k])
            assert p_edge == pytest.approx(np.float32(tau), rel=1e-9)
    assert list(rg[2]) == [0, -1, 0, -1, 0, -1]  # entirely outside: empty box


def test_obb_box_contains_level_set():
    """Every point with p_o >= tau_cut (found by bisection along random directions)
    lies inside the primitive's voxel box (unless outside the grid)."""
    pr, grid, rig, t = small_scene(11, n=12, gn=(16, 16, 8))
    tau = 0.01
    rg, _ = oracle.ranges(pr, grid, 0, tau, 5)
    rng = np.random.default_rng(11)
    lo, vs, n = grid["lo"].astype(float), grid["vs"].astype(float), np.array(grid["n"])
    for k in range(12):
        m, q, s, (e1, e2) = pr["means"][k], pr["quats"][k], pr["scales"][k], pr["eps"][k]
        for _ in range(40):
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            a, b = 0.0, 50.0
            for _ in range(80):
                c = 0.5 * (a + b)
                if oracle.sq_p(m + c * u, m, q, s, float(e1), float(e2)) >= tau:
                    a = c
                else:
                    b = c
            x = m + a * u
            iv = np.floor((x - lo) / vs).astype(int)
            if np.any(iv < 0) or np.any(iv >= n):
                continue
            for j in range(3):
                assert rg[k, 2 * j] <= iv[j] <= rg[k, 2 * j + 1]


def test_cube_mode_box():
    grid = synth.grid_spec(20, 20, 10, lo=(-10, -10, -5), hi=(10, 10, 5))
    pr = prims_from([[0.3, -2.2, 1.1], [9.9, -9.9, 0.0]], [[1, 0, 0, 0]] * 2, [[1, 1, 1]] * 2, [[1, 1]] * 2,
                    [0.5] * 2, np.zeros((2, 2)))
    rg, _ = oracle.ranges(pr, grid, 1, 0.01, 3)
    # centre voxels (10, 7, 6) and (19, 0, 5)
    assert list(rg[0]) == [7, 13, 4, 10, 3, 9]
    assert list(rg[1]) == [16, 19, 0, 3, 2, 8]


def _brute_lists(rg, gn):
    lists = {}
    for ix in range(gn[0]):
        for iy in range(gn[1]):
            for iz in range(gn[2]):
                v = (ix * gn[1] + iy) * gn[2] + iz
                lists[v] = [k for k in range(len(rg)) if rg[k, 0] <= ix <= rg[k, 1] and rg[k, 2] <= iy <= rg[k, 3]
                            and rg[k, 4] <= iz <= rg[k, 5]]
    return lists


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_index_equals_brute_force_tiny(seed):
    """Per voxel of a 4x3x2 grid: the list is exactly the ids whose box holds it, ascending."""
    rng = np.random.default_rng(seed)
    gn = (4, 3, 2)
    grid = synth.grid_spec(*gn, lo=(0, 0, 0), hi=(4, 3, 2))
    n = 8
    pr = prims_from(rng.uniform(0, [4, 3, 2], (n, 3)), rng.standard_normal((n, 4)), rng.uniform(0.2, 1.2, (n, 3)),
                    rng.uniform(0.2, 1.8, (n, 2)), rng.uniform(0, 1, n), rng.standard_normal((n, 3)))
    idx = oracle.build_index(pr, grid, 0, 0.01, 5)
    lists = _brute_lists(idx["ranges"], gn)
    assert np.array_equal(idx["v_f"], np.concatenate([[0], np.cumsum(idx["v_n"])[:-1]]))
    for v, want in lists.items():
        got = idx["v_sq"][idx["v_f"][v]:idx["v_f"][v] + idx["v_n"][v]]
        assert list(got) == want


def test_index_counts_equal_box_coverage_small_config():
    """On the 50x50x8 workload: v_n equals the number of boxes covering each voxel
    (vectorised count), and the total P equals the sum of box volumes."""
    cfg = synth.make_config(0)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    rg = idx["ranges"].astype(np.int64)
    gn = cfg["grid"]["n"]
    ix, iy, iz = np.meshgrid(*[np.arange(g) for g in gn], indexing="ij")
    cov = np.zeros(gn, np.int64)
    for r in rg:
        cov += (ix >= r[0]) & (ix <= r[1]) & (iy >= r[2]) & (iy <= r[3]) & (iz >= r[4]) & (iz <= r[5])
    assert np.array_equal(cov.reshape(-1), idx["v_n"])
    vol = np.prod(np.maximum(rg[:, 1::2] - rg[:, 0::2] + 1, 0), axis=1).sum()
    assert idx["P"] == vol
    assert idx["ties"] == 0


# --------------------------------------------------------------------- samples
def test_axis_ray_samples_closed_form():
    """A ray on the camera's optical axis: x_j = o + t_j (1, 0, 0) exactly, and the
    voxel is floor((x - lo)/vs) with outside samples marked -1."""
    grid = synth.grid_spec(50, 50, 8)
    t = synth.sample_depths(48)
    K = np.array([80, 80, 56.5, 32.5], np.float32)  # pixel (56, 32) centre on the axis
    c2w = synth.camera_pose(0.0, np.array([0.0, 0.0, 1.6]))
    xyz, vox = oracle.ray_samples(K, c2w, 56, 32, t, grid)
    assert np.array_equal(xyz[:, 0], t)
    assert np.all(xyz[:, 1] == 0) and np.all(xyz[:, 2] == np.float32(1.6))
    for j in range(48):
        if t[j] >= 40.0:
            assert vox[j] == -1
        else:
            ix = int(np.floor((t[j] + 40.0) / 1.6))
            assert vox[j] == (ix * 50 + 25) * 8 + int(np.floor((np.float32(1.6) + 1.0) / 0.8))


def test_sample_voxels_of_every_ray_match_numpy_fp32():
    """The oracle's voxel of every sample of every ray of workload 0 equals a numpy
    FP32 restatement of the rule (pixel-centre ray, x = o + t d, floor((x - lo) * (1/vs)),
    -1 outside), element by element."""
    cfg = synth.make_config(0)
    grid, rig, t = cfg["grid"], cfg["rig"], cfg["t"]
    vox = oracle.sample_voxels(rig, t, grid)
    x = _fp32_samples(rig, t)
    inv = (np.float32(1.0) / np.asarray(grid["vs"], np.float32)).astype(np.float32)
    u = ((x - np.asarray(grid["lo"], np.float32)) * inv).astype(np.float32)
    n = np.asarray(grid["n"])
    inside = np.all((u >= 0) & (u < n.astype(np.float32)), axis=-1)
    i = np.floor(u).astype(np.int64)
    ref = np.where(inside, (i[..., 0] * n[1] + i[..., 1]) * n[2] + i[..., 2], -1)
    assert vox.shape == ref.shape
    assert np.array_equal(vox, ref)
    assert 0 < inside.sum() < inside.size


# --------------------------------------------------------------------- forward
def _recurrence(alpha, t, c):
    T, D, S = 1.0, 0.0, np.zeros_like(c[0])
    for j in range(len(t)):
        w = T * alpha[j]
        D += w * t[j]
        S = S + w * c[j]
        T *= 1 - alpha[j]
    return D, S, T


@pytest.mark.parametrize("b,sigma,n_sph", [(0.0, 0.7, 1), (0.8, 0.4, 1), (0.3, 0.9, 2)])
def test_sphere_ray_closed_form(b, sigma, n_sph):
    """Ray along +x past spheres at impact parameter b: p_j = exp(-((t_j-t0)^2 + b^2)/r^2);
    the 1-D recurrence T, D, S (clamp active when two spheres overlap) matches to 1e-12."""
    r = 1.5
    centres = [(8.0, b, 0.0), (8.5, -b, 0.2)][:n_sph]
    logits = np.array([[0.3, -1.2, 2.0], [1.0, 0.5, -0.5]])[:n_sph]
    pr = prims_from(centres, [[1, 0, 0, 0], [0.6, 0.0, 0.8, 0.0]][:n_sph], [[r, r, r]] * n_sph, [[1, 1]] * n_sph,
                    [sigma] * n_sph, logits)
    grid = synth.grid_spec(21, 10, 10, lo=(-1, -5, -5), hi=(20, 5, 5))
    rig = axis_camera()
    t = synth.sample_depths(40, 0.5, 15.0)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    D, S, T, nu = oracle.render_fwd(pr, grid, idx, rig, t)
    tt = t.astype(np.float64)
    p = np.stack([np.exp(-(((tt - c[0]) ** 2) + c[1] ** 2 + c[2] ** 2) / r ** 2) for c in np.asarray(pr["means"],
                                                                                                     np.float64)], 1)
    alpha = np.minimum(p @ pr["opacity"].astype(np.float64), 1.0)
    sem = p @ pr["logits"].astype(np.float64)
    D0, S0, T0 = _recurrence(alpha, tt, sem)
    assert D[0] == pytest.approx(D0, rel=1e-12)
    np.testing.assert_allclose(S[0], S0, rtol=1e-12, atol=1e-14)
    assert T[0] == pytest.approx(T0, rel=1e-12, abs=1e-300)
    if n_sph == 2:
        assert np.any(p @ pr["opacity"] > 1.0)  # the clamp was exercised


def _recurrence_kappa(alpha, t, c, kappa):
    """The 1-D recurrence cut after the first sample j whose T_{j+1} < kappa."""
    T, D, S = 1.0, 0.0, np.zeros_like(c[0])
    for j in range(len(t)):
        w = T * alpha[j]
        D += w * t[j]
        S = S + w * c[j]
        T *= 1 - alpha[j]
        if T < kappa:
            return D, S, T, j + 1
    return D, S, T, len(t)


@pytest.mark.parametrize("kappa", [1e-2, 0.3])
@pytest.mark.parametrize("b,sigma,n_sph", [(0.0, 0.7, 1), (0.3, 0.9, 2)])
def test_sphere_ray_closed_form_early_termination(kappa, b, sigma, n_sph):
    """Early termination (Tab. 4b): the sphere ray of the closed form above with
    kappa > 0 stops after the first sample whose following transmittance is below
    kappa.  D, S, T_final and the composited count match the truncated 1-D
    recurrence to 1e-12, and stopping one sample earlier or later (testing T_j, or
    testing before compositing j) would move D by that sample's w_j t_j."""
    r = 1.5
    centres = [(8.0, b, 0.0), (8.5, -b, 0.2)][:n_sph]
    logits = np.array([[0.3, -1.2, 2.0], [1.0, 0.5, -0.5]])[:n_sph]
    pr = prims_from(centres, [[1, 0, 0, 0], [0.6, 0.0, 0.8, 0.0]][:n_sph], [[r, r, r]] * n_sph, [[1, 1]] * n_sph,
                    [sigma] * n_sph, logits)
    grid = synth.grid_spec(21, 10, 10, lo=(-1, -5, -5), hi=(20, 5, 5))
    t = synth.sample_depths(40, 0.5, 15.0)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    D, S, T, nu = oracle.render_fwd(pr, grid, idx, axis_camera(), t, kappa=kappa)
    tt = t.astype(np.float64)
    p = np.stack([np.exp(-(((tt - c[0]) ** 2) + c[1] ** 2 + c[2] ** 2) / r ** 2) for c in np.asarray(pr["means"],
                                                                                                     np.float64)], 1)
    alpha = np.minimum(p @ pr["opacity"].astype(np.float64), 1.0)
    sem = p @ pr["logits"].astype(np.float64)
    D0, S0, T0, n0 = _recurrence_kappa(alpha, tt, sem, kappa)
    assert 1 < n0 < len(t)  # the ray really stops early, after at least one weighted sample
    assert nu[0] == n0
    assert D[0] == pytest.approx(D0, rel=1e-12)
    np.testing.assert_allclose(S[0], S0, rtol=1e-12, atol=1e-14)
    assert T[0] == pytest.approx(T0, rel=1e-12, abs=1e-300)
    # the neighbouring stop rules give visibly different depths
    w = np.cumprod(np.concatenate([[1.0], 1 - alpha]))[:-1] * alpha
    assert abs(w[n0 - 1] * tt[n0 - 1]) > 1e-6 * abs(D0)


def test_box_like_superquadric_entry_depth():
    """eps1 = 0.1 (eps2 = 1): along local x, p = exp(-(|t - t0|/s)^20), a near-hard wall.
    With sigma = 1 the rendered depth sits at the entry face t0 - s (the weight
    of every sample lies within 0.25 m of it), and T_final ~ 0."""
    s = 2.0
    pr = prims_from([(10.0, 0, 0)], [[1, 0, 0, 0]], [[s, 1.0, 1.0]], [[0.1, 1.0]], [1.0], [[1.0]])
    grid = synth.grid_spec(22, 10, 10, lo=(-1, -5, -5), hi=(21, 5, 5))
    t = synth.sample_depths(301, 0.5, 15.5)  # 0.05 m spacing
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    D, S, T, _ = oracle.render_fwd(pr, grid, idx, axis_camera(), t)
    assert T[0] < 1e-6
    assert abs(D[0] / (1 - T[0]) - (10.0 - s)) < 0.25
    # a Gaussian profile (wrong exponent) would start absorbing much earlier
    tr = oracle.trace_ray(pr, grid, idx, axis_camera(), t, 0)
    w = tr["T"][:-1] * tr["alpha"]
    assert w[t < 10 - s - 0.3].sum() < 1e-3


def test_transmittance_identity():
    """sum_j w_j + T_final = 1 on every ray (Eq. 5)."""
    cfg = synth.make_config(0)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    for ray in range(0, 64 * 112, 397):
        tr = oracle.trace_ray(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], ray)
        w = tr["T"][:-1] * tr["alpha"]
        assert w.sum() + tr["T"][tr["used"]] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_full_coverage_index_equals_brute_force(seed):
    """With every primitive's box covering the whole grid, the indexed render is the
    plain sum over all primitives (numpy, scipy rotations) at every in-grid sample."""
    pr, grid, rig, t = small_scene(seed, n=7, sigma_max=0.9)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    assert np.all(idx["v_n"] == 7)
    D, S, T, _ = oracle.render_fwd(pr, grid, idx, rig, t)
    D0, S0, T0 = brute_render(pr, grid, rig, t)
    np.testing.assert_allclose(D, D0, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(S, S0, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(T, T0, rtol=1e-11, atol=1e-14)


def test_truncated_index_drops_only_weak_terms():
    """With tau_cut = 1e-4 the indexed render differs from the all-primitive sum by
    no more than the dropped occupancies allow."""
    pr, grid, rig, t = small_scene(3, n=9, gn=(16, 16, 8))
    idx = oracle.build_index(pr, grid, 0, 1e-4, 5)
    D, S, T, _ = oracle.render_fwd(pr, grid, idx, rig, t)
    D0, S0, T0 = brute_render(pr, grid, rig, t)
    assert np.max(np.abs(T - T0)) < 24 * 9 * 1e-4
    assert np.max(np.abs(T - T0)) > 0  # truncation is real


def test_out_of_grid_samples_contribute_nothing():
    """A sphere straddling the grid's far face: samples past the face add nothing."""
    r = 1.0
    pr = prims_from([(9.8, 0, 0)], [[1, 0, 0, 0]], [[r, r, r]], [[1, 1]], [0.8], [[1.0, 2.0]])
    grid = synth.grid_spec(10, 10, 10, lo=(0, -5, -5), hi=(10, 5, 5))
    t = synth.sample_depths(60, 0.5, 12.3)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    D, S, T, _ = oracle.render_fwd(pr, grid, idx, axis_camera(), t)
    tt = t.astype(np.float64)
    m = float(np.float32(9.8))
    po = np.where(tt < 10.0, np.exp(-((tt - m) ** 2) / r ** 2), 0.0)
    alpha = np.minimum(float(np.float32(0.8)) * po, 1)
    D0, S0, T0 = _recurrence(alpha, tt, po[:, None] * [1.0, 2.0])
    np.testing.assert_allclose(S[0], S0, rtol=1e-12)
    assert D[0] == pytest.approx(D0, rel=1e-12)
    assert T[0] == pytest.approx(T0, rel=1e-12)


def test_early_termination_stops_after_threshold():
    """kappa > 0: compositing stops after the first sample whose T drops below kappa."""
    cfg = synth.make_config(0)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    D, S, T, nu = oracle.render_fwd(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], kappa=1e-2)
    D0, S0, T0, nu0 = oracle.render_fwd(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"])
    stopped = nu < 48
    assert stopped.any()
    assert np.all(T[stopped] < 1e-2)
    for ray in np.flatnonzero(stopped)[:20]:
        tr = oracle.trace_ray(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], ray)
        k = nu[ray]
        assert tr["T"][k - 1] >= 1e-2 > tr["T"][k]
        w = tr["T"][:k] * tr["alpha"][:k]
        assert D[ray] == pytest.approx(np.dot(w, cfg["t"][:k].astype(float)), rel=1e-12)
    assert np.all(nu0 == 48)


# --------------------------------------------------------------------- backward
def _linear_loss(pr, grid, idx, rig, t, gd, gs, alpha_max=1.0):
    D, S, _, _ = oracle.render_fwd(pr, grid, idx, rig, t, alpha_max=alpha_max)
    return float(np.dot(gd, D) + np.sum(gs * S))


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_central_differences(seed):
    """Analytic FP64 gradient vs central finite differences (index frozen) for every
    parameter of every primitive of a small scene."""
    pr, grid, rig, t = small_scene(seed, n=5, H=5, W=6, L=20)
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(100 + seed)
    gd, gs = rng.standard_normal(R), rng.standard_normal((R, pr["logits"].shape[1]))
    g = oracle.render_bwd(pr, grid, idx, rig, t, gd, gs)
    # clamp far from active
    for ray in range(R):
        tr = oracle.trace_ray(pr, grid, idx, rig, t, ray)
        assert np.all(np.abs(tr["ssum"] - 1.0) > 1e-2)
    h = 2.0 ** -13  # ~1e-4; x +- h and x +- h/2 are exact in FP32 for |x| < 512
    checked = 0
    for name in ["means", "quats", "scales", "eps", "opacity", "logits"]:
        for i in range(pr[name].size):
            fd = richardson_fd(lambda p2: _linear_loss(p2, grid, idx, rig, t, gd, gs), pr, name, i, h)
            an = g[name].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, np.abs(g[name]).max())), (name, i, an, fd)
            checked += 1
    assert checked == 5 * (3 + 4 + 3 + 2 + 1 + 5)


def test_backward_matches_central_differences_on_stress_crop():
    """The same check on the clustered 16,384-primitive scene (sharp and flat
    shapes, eps down to 0.1), cotangents on every 8th ray of a 32x32 crop of camera
    0 whose samples all stay clear of the alpha clamp: every parameter of the six
    primitives with the largest opacity gradient."""
    cfg = synth.make_config(2)
    pr, grid, rig, t = cfg["prims"], cfg["grid"], cfg["rig"], cfg["t"]
    idx = oracle.build_index(pr, grid)
    W = rig["W"]
    crop = np.array([(96 + i) * W + (184 + j) for i in range(32) for j in range(32)])[::8]
    safe = np.array([r for r in crop
                     if np.all(np.abs(oracle.trace_ray(pr, grid, idx, rig, t, r)["ssum"] - 1.0) > 1e-2)])
    assert len(safe) > 100
    rng = np.random.default_rng(7)
    gd, gs = rng.standard_normal(len(safe)), rng.standard_normal((len(safe), pr["logits"].shape[1]))
    g = oracle.render_bwd(pr, grid, idx, rig, t, gd, gs, ray_ids=safe)

    def loss(p2):
        D, S, _, _ = oracle.render_fwd(p2, grid, idx, rig, t, ray_ids=safe)
        return float(np.dot(gd, D) + np.sum(gs * S))

    prims = np.argsort(-np.abs(g["opacity"]))[:6]
    assert np.abs(g["opacity"][prims]).min() > 0
    # a smaller step than on the tiny scenes: the sharper primitives' higher
    # derivatives leave 4e-4 of truncation error at 2^-13 (one quaternion component
    # of primitive 16208 goes -1.02938, -1.02353, -1.023938, -1.0239386 for steps
    # 2^-11 .. 2^-17, the analytic value -1.0239386); x +- 2^-17 stays exact in FP32
    # for |x| < 128, which holds for every parameter of this scene
    h = 2.0 ** -17
    sizes = {"means": 3, "quats": 4, "scales": 3, "eps": 2, "opacity": 1, "logits": pr["logits"].shape[1]}
    for name, m in sizes.items():
        scale = np.abs(g[name]).max()
        for k in prims:
            for c in range(m):
                i = int(k) * m + c
                fd = richardson_fd(loss, pr, name, i, h)
                an = g[name].reshape(-1)[i]
                assert an == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, scale)), (name, int(k), c, an, fd)


def test_backward_with_early_termination_matches_central_differences():
    """kappa > 0: the analytic gradient through the truncated composite (Tab. 4b)
    against central differences, on rays whose transmittance stays clear of kappa
    (at least 2% relative at every sample), so that a step of 2^-13 moves no ray's
    stopping sample."""
    kappa = 0.4
    pr, grid, rig, t = small_scene(4, n=6, H=5, W=6, L=20, sigma_max=0.6)
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    R = rig["H"] * rig["W"]
    _, _, _, nu = oracle.render_fwd(pr, grid, idx, rig, t, kappa=kappa)
    safe = []
    for ray in range(R):
        tr = oracle.trace_ray(pr, grid, idx, rig, t, ray, kappa=kappa)
        Tn = tr["T"][1:tr["used"] + 1]
        if np.all(np.abs(Tn - kappa) > 0.02 * kappa) and np.all(np.abs(tr["ssum"] - 1.0) > 1e-2):
            safe.append(ray)
    safe = np.array(safe)
    assert np.any(nu[safe] < len(t)), "no checked ray stops early"
    assert len(safe) > R // 3
    rng = np.random.default_rng(11)
    gd, gs = rng.standard_normal(len(safe)), rng.standard_normal((len(safe), pr["logits"].shape[1]))
    g = oracle.render_bwd(pr, grid, idx, rig, t, gd, gs, kappa=kappa, ray_ids=safe)

    def loss(p2):
        D, S, _, _ = oracle.render_fwd(p2, grid, idx, rig, t, kappa=kappa, ray_ids=safe)
        return float(np.dot(gd, D) + np.sum(gs * S))

    h = 2.0 ** -13
    for name in ["means", "quats", "scales", "eps", "opacity", "logits"]:
        scale = np.abs(g[name]).max()
        for i in range(pr[name].size):
            fd = richardson_fd(loss, pr, name, i, h)
            an = g[name].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, scale)), (name, i, an, fd)


def test_quaternion_gradient_is_orthogonal_to_q():
    """p_o depends on q only through q/|q|, so q . dL/dq = 0."""
    pr, grid, rig, t = small_scene(4, n=6)
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(4)
    g = oracle.render_bwd(pr, grid, idx, rig, t, rng.standard_normal(R), rng.standard_normal((R, 5)))
    dots = np.sum(g["quats"] * pr["quats"].astype(np.float64), 1)
    assert np.all(np.abs(dots) <= 1e-10 * np.abs(g["quats"]).max())


def test_logit_gradient_closed_form_single_primitive():
    """One primitive: dL/dc = gS_r * sum_j w_j p_j and p_j = alpha_j / sigma (unclamped)."""
    pr = prims_from([(8.0, 0.3, 0)], [[0.9, 0.1, 0.3, -0.2]], [[1.5, 1.0, 2.0]], [[0.7, 1.3]], [0.6],
                    [[0.2, -0.4, 1.0]])
    grid = synth.grid_spec(21, 10, 10, lo=(-1, -5, -5), hi=(20, 5, 5))
    t = synth.sample_depths(50, 0.5, 15.0)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    gs = np.array([[0.5, -1.5, 2.0]])
    g = oracle.render_bwd(pr, grid, idx, axis_camera(), t, np.array([0.0]), gs)
    tr = oracle.trace_ray(pr, grid, idx, axis_camera(), t, 0)
    w = tr["T"][:-1] * tr["alpha"]
    Wp = np.sum(w * tr["alpha"] / float(np.float32(0.6)))
    np.testing.assert_allclose(g["logits"][0], gs[0] * Wp, rtol=1e-12)


def test_opacity_gradient_closed_form_single_primitive():
    """One primitive, L = depth: with alpha_j = p_j sigma (unclamped) and
    T_j = prod_{l<j} (1 - alpha_l), dD/dsigma = sum_j t_j (p_j T_j + alpha_j dT_j/dsigma)
    with dT_j/dsigma = -T_j sum_{l<j} p_l / (1 - alpha_l) (forward-mode, written
    from Eq. 5-6, not the reverse sweep the oracle uses)."""
    pr = prims_from([(8.0, 0.3, 0)], [[0.9, 0.1, 0.3, -0.2]], [[1.5, 1.0, 2.0]], [[0.7, 1.3]], [0.6],
                    [[0.2, -0.4, 1.0]])
    grid = synth.grid_spec(21, 10, 10, lo=(-1, -5, -5), hi=(20, 5, 5))
    t = synth.sample_depths(50, 0.5, 15.0)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    g = oracle.render_bwd(pr, grid, idx, axis_camera(), t, np.array([1.0]), np.zeros((1, 3)))
    tr = oracle.trace_ray(pr, grid, idx, axis_camera(), t, 0)
    sigma = float(np.float32(0.6))
    alpha, T = tr["alpha"], tr["T"][:-1]
    assert alpha.max() < 1.0 and np.count_nonzero(alpha) > 5
    p = alpha / sigma
    dT = -T * np.concatenate([[0.0], np.cumsum(p / (1.0 - alpha))[:-1]])
    dD = np.sum(t.astype(np.float64) * (p * T + alpha * dT))
    assert g["opacity"][0] == pytest.approx(dD, rel=1e-10)


def test_clamped_samples_pass_no_alpha_gradient():
    """Where sum p sigma > alpha_max the alpha gradient is zero: a sigma change that
    keeps every sample clamped leaves the loss unchanged."""
    pr = prims_from([(8.0, 0, 0)], [[1, 0, 0, 0]], [[3.0, 3.0, 3.0]], [[1, 1]], [5.0], [[1.0]])
    grid = synth.grid_spec(21, 10, 10, lo=(-1, -5, -5), hi=(20, 5, 5))
    t = synth.sample_depths(10, 7.0, 9.0)  # all samples deep inside: p sigma > 4
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    g = oracle.render_bwd(pr, grid, idx, axis_camera(), t, np.array([1.0]), np.array([[0.0]]))
    assert g["opacity"][0] == 0.0


# --------------------------------------------------------------------- voxelisation
def test_grid_query_single_sphere():
    """Supp. A.4 with one sphere: density = sigma exp(-|p - m|^2/r^2) at FP32 voxel
    centres, sem = c * that occupancy, label = argmax c where density >= tau else C."""
    r, sigma = 1.7, 0.8
    c = np.array([0.1, 2.0, -1.0, 0.5])
    pr = prims_from([(0.3, -0.4, 0.2)], [[0.8, 0.2, -0.3, 0.4]], [[r, r, r]], [[1, 1]], [sigma], c[None])
    grid = synth.grid_spec(10, 10, 5, lo=(-4, -4, -2), hi=(4, 4, 2))
    idx = oracle.build_index(pr, grid, 1, 0.01, 20)
    dens, sem, lab = oracle.query_grid(pr, grid, idx, tau=0.05)
    gn = grid["n"]
    ii = np.stack(np.meshgrid(*[np.arange(g, dtype=np.float32) for g in gn], indexing="ij"), -1).reshape(-1, 3)
    pc = (grid["lo"] + ((ii + np.float32(0.5)) * grid["vs"]).astype(np.float32)).astype(np.float32)
    r32 = float(np.float32(r))
    po = np.exp(-np.sum((pc.astype(np.float64) - pr["means"][0].astype(np.float64)) ** 2, 1) / r32 ** 2)
    np.testing.assert_allclose(dens, np.float32(sigma) * po, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(sem, po[:, None] * c.astype(np.float32), rtol=1e-12, atol=1e-300)
    want = np.where(dens >= 0.05, 1, 4)
    assert np.array_equal(lab, want)
    assert (want == 1).any() and (want == 4).any()


def test_grid_query_full_coverage_equals_brute_force():
    pr, grid, rig, t = small_scene(9, n=8)
    idx = oracle.build_index(pr, grid, 1, 0.01, 100)
    dens, sem, lab = oracle.query_grid(pr, grid, idx, tau=0.05)
    gn = grid["n"]
    ii = np.stack(np.meshgrid(*[np.arange(g, dtype=np.float32) for g in gn], indexing="ij"), -1).reshape(-1, 3)
    pc = (grid["lo"] + ((ii + np.float32(0.5)) * grid["vs"]).astype(np.float32)).astype(np.float32)
    p = brute_p(pr, pc)
    np.testing.assert_allclose(dens, p @ pr["opacity"].astype(np.float64), rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(sem, p @ pr["logits"].astype(np.float64), rtol=1e-11, atol=1e-14)


# ------------------------------------------------- opacity-aware index (mode 2)
def test_opacity_mode_axis_aligned_box():
    """Axis-aligned primitive: the box holds the level set sigma p_o >= tau, whose
    local half-extents are s_i (ln(sigma/tau))^(eps1/2) (along a local axis
    f = (|x_i|/s_i)^(2/eps1))."""
    grid = synth.grid_spec(20, 20, 10, lo=(-10, -10, -5), hi=(10, 10, 5))
    m, s, e1, sig, tau = np.array([0.3, -2.2, 1.1]), np.array([1.0, 2.0, 0.5]), 1.0, 0.5, 0.01
    pr = prims_from([m], [[1, 0, 0, 0]], [s], [[e1, 1.0]], [sig], np.zeros((1, 2)))
    rg, ties = oracle.ranges(pr, grid, 2, tau, 0)
    h = s * np.log(sig / tau) ** (e1 / 2)
    lo = np.floor((m - h - np.array([-10, -10, -5])) / 1.0).astype(int)
    hi = np.floor((m + h - np.array([-10, -10, -5])) / 1.0).astype(int)
    assert ties == 0
    assert list(rg[0]) == [lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]] == [8, 12, 3, 11, 5, 7]


def test_opacity_mode_drops_faint_and_matches_obb_at_full_opacity():
    rng = np.random.default_rng(4)
    n = 200
    grid = synth.grid_spec(40, 40, 10, lo=(-20, -20, -2), hi=(20, 20, 8))
    base = prims_from(rng.uniform(-15, 15, (n, 3)), rng.standard_normal((n, 4)), rng.uniform(0.2, 2.5, (n, 3)),
                      rng.uniform(0.2, 1.8, (n, 2)), rng.uniform(0, 1, n), rng.standard_normal((n, 3)))
    obb, _ = oracle.ranges(base, grid, 0, 0.01, 0)
    opa, _ = oracle.ranges(base, grid, 2, 0.01, 0)
    empty = (opa[:, 1] < opa[:, 0]) | (opa[:, 3] < opa[:, 2]) | (opa[:, 5] < opa[:, 4])
    # sigma <= tau: listed nowhere
    assert np.all(empty[base["opacity"] <= 0.01])
    # otherwise contained in the OBB-mode box (sigma <= 1 shrinks the level set)
    ok = ~empty
    assert np.all(opa[ok, 0::2] >= obb[ok, 0::2]) and np.all(opa[ok, 1::2] <= obb[ok, 1::2])
    assert np.any(opa[ok] != obb[ok])
    # sigma = 1: ln(1) - ln(tau) = ln(1/tau) exactly, the same boxes as mode 0
    full = dict(base)
    full["opacity"] = np.ones(n, np.float32)
    opa1, _ = oracle.ranges(full, grid, 2, 0.01, 0)
    assert np.array_equal(opa1, obb)


def test_opacity_mode_box_holds_level_set():
    """Points of a rotated primitive with sigma p_o >= tau (brute force over a
    lattice around it) all fall in its opacity-aware voxel box."""
    grid = synth.grid_spec(40, 40, 40, lo=(-4, -4, -4), hi=(4, 4, 4))
    rng = np.random.default_rng(9)
    for _ in range(4):
        m = rng.uniform(-0.5, 0.5, 3)
        q = rng.standard_normal(4)
        s = rng.uniform(0.3, 1.0, 3)
        e = rng.uniform(0.3, 1.7, 2)
        sig = rng.uniform(0.05, 1.0)
        pr = prims_from([m], [q], [s], [e], [sig], np.zeros((1, 2)))
        rg, _ = oracle.ranges(pr, grid, 2, 0.01, 0)
        pts = m + rng.uniform(-3.9, 3.9, (4000, 3))
        pts = pts[np.all(np.abs(pts) < 3.99, 1)]
        inside = np.array([sig * oracle.sq_p(x, m, q, s, e[0], e[1]) >= 0.01 for x in pts])
        vox = np.floor((pts + 4.0) / 0.2).astype(int)
        in_box = ((vox[:, 0] >= rg[0, 0]) & (vox[:, 0] <= rg[0, 1]) & (vox[:, 1] >= rg[0, 2]) & (vox[:, 1] <= rg[0, 3])
                  & (vox[:, 2] >= rg[0, 4]) & (vox[:, 2] <= rg[0, 5]))
        assert inside.sum() > 0
        assert np.all(in_box[inside])


# ------------------------------------------------------ grid query backward
def _query_loss(pr, grid, idx, gd, gs):
    dens, sem, _ = oracle.query_grid(pr, grid, idx, 0.05)
    return float(np.dot(gd, dens) + np.sum(gs * sem))


@pytest.mark.parametrize("seed", [0, 1])
def test_query_backward_matches_central_differences(seed):
    """The grid query's analytic FP64 gradient (index frozen) vs central finite
    differences of the FP64 query, for every parameter of every primitive."""
    pr, grid, _, _ = small_scene(20 + seed, n=4, gn=(8, 8, 4))
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    nvox = int(np.prod(grid["n"]))
    rng = np.random.default_rng(200 + seed)
    gd, gs = rng.standard_normal(nvox), rng.standard_normal((nvox, pr["logits"].shape[1]))
    g = oracle.query_grid_bwd(pr, grid, idx, gd, gs)
    h = 2.0 ** -13
    for name in ["means", "quats", "scales", "eps", "opacity", "logits"]:
        for i in range(pr[name].size):
            fd = richardson_fd(lambda p2: _query_loss(p2, grid, idx, gd, gs), pr, name, i, h)
            an = g[name].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, np.abs(g[name]).max())), (name, i, an, fd)


def test_query_backward_voxel_subset_is_the_restriction():
    """Cotangents on a voxel subset give the same gradient as the full grid with
    the other voxels' cotangents zero."""
    pr, grid, _, _ = small_scene(23, n=6, gn=(8, 8, 4))
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    nvox = int(np.prod(grid["n"]))
    rng = np.random.default_rng(5)
    sel = np.sort(rng.choice(nvox, 50, replace=False))
    gd, gs = rng.standard_normal(50), rng.standard_normal((50, pr["logits"].shape[1]))
    gd_full, gs_full = np.zeros(nvox), np.zeros((nvox, gs.shape[1]))
    gd_full[sel], gs_full[sel] = gd, gs
    a = oracle.query_grid_bwd(pr, grid, idx, gd, gs, voxel_ids=sel)
    b = oracle.query_grid_bwd(pr, grid, idx, gd_full, gs_full)
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------ per-primitive softmax
def test_softmax_mode_backward_matches_central_differences():
    """sem_mode 1 (c_k -> softmax(c_k)): the logit gradient through the softmax,
    and the other parameters, against central differences of the FP64 render."""
    pr, grid, rig, t = small_scene(30, n=4, H=5, W=6, L=20)
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(30)
    gd, gs = rng.standard_normal(R), rng.standard_normal((R, pr["logits"].shape[1]))
    g = oracle.render_bwd(pr, grid, idx, rig, t, gd, gs, sem_mode=1)

    def loss(p2):
        D, S, _, _ = oracle.render_fwd(p2, grid, idx, rig, t, sem_mode=1)
        return float(np.dot(gd, D) + np.sum(gs * S))

    h = 2.0 ** -13
    for name in ["logits", "opacity", "means"]:
        for i in range(pr[name].size):
            fd = richardson_fd(loss, pr, name, i, h)
            an = g[name].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=2e-5, abs=1e-6 * max(1.0, np.abs(g[name]).max())), (name, i, an, fd)


def test_softmax_mode_invariances():
    """A constant added to a primitive's logits changes nothing in softmax mode, so
    every primitive's logit gradient sums to zero; with one class the semantic sum
    is the plain occupancy sum (softmax of one logit is 1)."""
    pr, grid, rig, t = small_scene(31, n=5)
    idx = oracle.build_index(pr, grid, 0, 1e-3, 5)
    R = rig["H"] * rig["W"]
    rng = np.random.default_rng(31)
    D0, S0, _, _ = oracle.render_fwd(pr, grid, idx, rig, t, sem_mode=1)
    shifted = dict(pr)
    shifted["logits"] = (pr["logits"] + rng.uniform(-3, 3, (pr["logits"].shape[0], 1))).astype(np.float32)
    D1, S1, _, _ = oracle.render_fwd(shifted, grid, idx, rig, t, sem_mode=1)
    np.testing.assert_allclose(S1, S0, rtol=1e-6, atol=1e-9)
    np.testing.assert_array_equal(D1, D0)
    g = oracle.render_bwd(pr, grid, idx, rig, t, rng.standard_normal(R), rng.standard_normal((R, 5)), sem_mode=1)
    np.testing.assert_allclose(g["logits"].sum(1), 0.0, atol=1e-12 * max(1.0, np.abs(g["logits"]).max()))
    one = dict(pr)
    one["logits"] = rng.standard_normal((pr["logits"].shape[0], 1)).astype(np.float32)
    _, S_soft, _, _ = oracle.render_fwd(one, grid, idx, rig, t, sem_mode=1)
    ones = dict(pr)
    ones["logits"] = np.ones((pr["logits"].shape[0], 1), np.float32)
    _, S_ones, _, _ = oracle.render_fwd(ones, grid, idx, rig, t)
    np.testing.assert_allclose(S_soft, S_ones, rtol=1e-12, atol=1e-15)


# ----------------------------------------------------------------------- voxel losses
def test_voxel_loss_closed_forms():
    """Uniform logits cost log C per occupied voxel; an occupied voxel of density
    ln 2 (p = 1/2) costs ln 2; a free voxel costs its density; ignored voxels and
    empty sets cost nothing."""
    C = 6
    s = np.zeros((4, C))
    d = np.array([np.log(2.0), 0.7, 5.0, 0.3])
    y = np.array([2, C, -1, -1])
    tot, ce, bce, gd, gs = oracle.voxel_loss(d, s, y, lambda_s=1.0, lambda_o=1.0)
    assert np.isclose(ce, np.log(C), rtol=1e-14)
    assert np.isclose(bce, (np.log(2.0) + 0.7) / 2, rtol=1e-14)
    assert np.isclose(tot, ce + bce, rtol=1e-14)
    assert gd[2] == 0.0 and gd[3] == 0.0 and np.all(gs[1:] == 0.0)
    assert np.isclose(gd[1], 0.5) and np.isclose(gd[0], -0.5 / (2.0 - 1.0))  # -w/(e^d - 1) at d = ln 2
    tot, ce, bce, gd, gs = oracle.voxel_loss(d, s, np.full(4, -1))
    assert tot == 0.0 and not gd.any() and not gs.any()


def test_voxel_loss_matches_torch_library():
    """Against torch's cross_entropy and binary_cross_entropy (FP64) on p = 1 -
    exp(-d), gradients by autograd, densities away from the clamp."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(5)
    V, C = 300, 7
    d = rng.uniform(0.01, 4.0, V)
    s = rng.standard_normal((V, C)) * 2
    y = rng.integers(-1, C + 1, V)
    tot, ce, bce, gd, gs = oracle.voxel_loss(d, s, y, lambda_s=2.0, lambda_o=0.5)
    dt = torch.tensor(d, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    yt = torch.tensor(y)
    occ, lab = (yt >= 0) & (yt < C), (yt >= 0) & (yt <= C)
    p = 1.0 - torch.exp(-dt)
    ref = 2.0 * F.cross_entropy(st[occ], yt[occ]) + 0.5 * F.binary_cross_entropy(p[lab], (yt[lab] < C).double())
    ref.backward()
    assert np.isclose(tot, ref.item(), rtol=1e-12)
    np.testing.assert_allclose(gd, dt.grad.numpy(), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(gs, st.grad.numpy(), rtol=1e-10, atol=1e-14)
