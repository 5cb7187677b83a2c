"""Writes tests/golden/oracle_small.json from the FP64 oracle alone.

The paper prints no worked numeric example of its renderer, so these values
are not the paper's: they are the oracle's own outputs on the seeded 50x50x8,
256-superquadric, 64x112-ray workload, kept so that a rebuild of the oracle on
another machine (for instance an aarch64 host) can be checked to reproduce the
same discrete decisions (index contents, sample voxels) and the same FP64
renders.  Run:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_17361_gb300 import synth  # noqa: E402

RAYS = [0, 111, 2000, 3571, 4480, 5000, 7167]
VOXELS = [0, 777, 10000, 19999]


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main():
    cfg = synth.make_config(0)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    D, S, T, _ = oracle.render_fwd(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], ray_ids=RAYS)
    dens, sem, lab = oracle.query_grid(cfg["prims"], cfg["grid"], idx, voxel_ids=VOXELS)
    out = {
        "workload": cfg["name"],
        "P": idx["P"],
        "sha256_v_n": digest(idx["v_n"].astype(np.int32)),
        "sha256_v_sq": digest(idx["v_sq"].astype(np.int32)),
        "sha256_ranges": digest(idx["ranges"].astype(np.int32)),
        "rays": RAYS,
        "depth": D.tolist(),
        "t_final": T.tolist(),
        "sem": S.tolist(),
        "voxels": VOXELS,
        "density": dens.tolist(),
        "label": lab.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
