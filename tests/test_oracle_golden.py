"""The oracle, rebuilt on this machine, reproduces the stored outputs written by
tests/golden/make_golden.py (same index bytes, same FP64 renders to 1e-12)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_17361_gb300 import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_small.json")


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_oracle_reproduces_golden():
    g = json.load(open(GOLD))
    cfg = synth.make_config(0)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    assert idx["P"] == g["P"]
    assert _digest(idx["v_n"].astype(np.int32)) == g["sha256_v_n"]
    assert _digest(idx["v_sq"].astype(np.int32)) == g["sha256_v_sq"]
    assert _digest(idx["ranges"].astype(np.int32)) == g["sha256_ranges"]
    D, S, T, _ = oracle.render_fwd(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], ray_ids=g["rays"])
    np.testing.assert_allclose(D, g["depth"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(T, g["t_final"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(S, g["sem"], rtol=1e-12, atol=1e-13)
    dens, sem, lab = oracle.query_grid(cfg["prims"], cfg["grid"], idx, voxel_ids=g["voxels"])
    np.testing.assert_allclose(dens, g["density"], rtol=1e-12, atol=1e-14)
    assert lab.tolist() == g["label"]
