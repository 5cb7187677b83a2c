"""Helpers for the GPU parity tests: build/load the CUDA library, move seeded
inputs to the device, and the tolerance checks (each stated where it is used)."""
from __future__ import annotations

import json
import os

import numpy as np
import torch

import oracle
from paper_2511_17361_gb300 import synth


def lib():
    from paper_2511_17361_gb300 import _build
    _build.build()
    from paper_2511_17361_gb300 import sqr
    return sqr


def dev_grid(grid):
    return {"n": tuple(int(v) for v in grid["n"]), "lo": [float(v) for v in grid["lo"]],
            "vs": [float(v) for v in grid["vs"]]}


def scene_to_gpu(sqr, prims, rig, t, kappa=0.0, alpha_max=1.0):
    return sqr.to_device(prims), sqr.Rays.from_rig(rig, t, kappa=kappa, alpha_max=alpha_max)


def np_index(ix):
    P = ix.P()
    return {"v_n": ix.v_n.cpu().numpy(), "v_f": ix.v_f.cpu().numpy(), "v_sq": ix.v_sq[:P].cpu().numpy(),
            "ranges": ix.ranges.cpu().numpy(), "P": P}


def assert_index_equal(ix, ref, no_ties=True):
    """The GPU index equals the oracle's bit for bit (P, ranges, V_n, V_f, V_sq);
    with no_ties the seeded scene also has no voxel-boundary near-tie."""
    got = np_index(ix)
    if no_ties:
        assert ref["ties"] == 0, "seeded workload has a voxel-boundary near-tie"
    assert got["P"] == ref["P"]
    assert np.array_equal(got["ranges"][:len(ref["ranges"])], ref["ranges"])
    assert np.array_equal(got["v_n"], ref["v_n"])
    assert np.array_equal(got["v_f"], ref["v_f"])
    assert np.array_equal(got["v_sq"], ref["v_sq"])


def oracle_index(ix, prims, grid, mode=0, tau=0.01, nv=5):
    """The oracle's own index of the scene, after checking that the GPU's index ix
    (built with the same options) equals it bit for bit: the oracle then renders
    over lists it built itself, never over the GPU's."""
    ref = oracle.build_index(prims, grid, mode, tau, nv)
    assert_index_equal(ix, ref, no_ties=False)
    return ref


def _log_error(kind, **vals):
    """Append the observed worst error of one check to the JSON-lines file named
    by SQR_TOL_LOG (when set), with the test that made it: the record the
    tolerances are set from."""
    path = os.environ.get("SQR_TOL_LOG")
    if not path:
        return
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "check": kind}
    rec.update({k: float(v) for k, v in vals.items()})
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def softmax(x):
    x = np.asarray(x, np.float64)
    e = np.exp(x - x.max(-1, keepdims=True))
    return e / e.sum(-1, keepdims=True)


def check_depth(d_gpu, d_ref, t_near):
    """Depth within 1e-4 relative: |dD| <= 1e-4 * max(D_ref, t_near)."""
    d_gpu = np.asarray(d_gpu, np.float64)
    tol = 1e-4 * np.maximum(np.abs(d_ref), t_near)
    if d_gpu.size:
        _log_error("depth", rel_to_tol=np.max(np.abs(d_gpu - d_ref) / tol))
    bad = np.abs(d_gpu - d_ref) > tol
    assert not bad.any(), f"{bad.sum()} depths off; worst {np.max(np.abs(d_gpu - d_ref) / tol):.3g} x tol"


def check_sem(s_gpu, s_ref, raw_tol=1e-5):
    """Class probabilities softmax(S) within 1e-5 absolute; raw S within
    raw_tol * max(1, |S_ref|) (FP32 accumulation of ~10^3 SFU-evaluated terms)."""
    s_gpu = np.asarray(s_gpu, np.float64)
    dp = np.abs(softmax(s_gpu) - softmax(s_ref))
    rel = np.abs(s_gpu - s_ref) / np.maximum(1.0, np.abs(s_ref))
    if s_gpu.size:
        _log_error("sem", prob_abs=dp.max(), raw_rel=rel.max(), raw_rel_p999=np.quantile(rel, 0.999),
                   max_abs_ref=np.abs(s_ref).max())
    assert dp.max() <= 1e-5, f"class probabilities off by {dp.max():.3g}"
    assert rel.max() <= raw_tol, f"raw semantics off by {rel.max():.3g} (rel)"


def check_grad(g_gpu, g_ref, name, rtol=1e-3, mag=None):
    """Per element |g - g_ref| <= rtol * max(|g_ref|, 1e-3 * max|g_ref| over the tensor).
    ``mag`` (optional, same shape): sum over rays of |per-ray gradient| from the
    oracle.  An FP32 sum of terms whose magnitudes add up to mag carries a rounding
    error of order 2^-24 * mag whatever the order of summation, so 16 * 2^-24 * mag
    is added to the tolerance: this matters only where the rays' contributions
    cancel (|g_ref| far below mag)."""
    g_gpu = np.asarray(g_gpu, np.float64)
    g_ref = np.asarray(g_ref, np.float64)
    scale = np.max(np.abs(g_ref)) if g_ref.size else 0.0
    tol = rtol * np.maximum(np.abs(g_ref), 1e-3 * scale)
    if mag is not None:
        tol = tol + 16.0 * 2.0 ** -24 * np.asarray(mag, np.float64)
    err = np.abs(g_gpu - g_ref)
    if g_gpu.size:
        _log_error(f"grad:{name}", ratio=np.max(err / (tol + 1e-30)))
    bad = err > tol + 1e-30
    assert not bad.any(), (f"{name}: {bad.sum()}/{bad.size} elements off; worst ratio "
                           f"{np.max(err / (tol + 1e-30)):.3g}; norm ratio "
                           f"{np.linalg.norm(g_gpu) / max(np.linalg.norm(g_ref), 1e-300):.6f}")


def per_ray_magnitude(prims, grid, idx, rig, t, gd, gs, **kw):
    """Sum over rays of |the oracle's gradient from that ray alone| per parameter
    (the magnitude an FP32 sum over the rays' contributions rounds against)."""
    out = None
    for r in np.nonzero((np.asarray(gd) != 0) | np.any(np.asarray(gs) != 0, axis=1))[0]:
        g = oracle.render_bwd(prims, grid, idx, rig, t, np.asarray(gd, np.float64)[[r]],
                              np.asarray(gs, np.float64)[[r]], ray_ids=np.array([r]), **kw)
        if out is None:
            out = {k: np.abs(v) for k, v in g.items()}
        else:
            for k in out:
                out[k] += np.abs(g[k])
    return out
