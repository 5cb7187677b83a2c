"""Cases run in a subprocess on the debug build with bounds checks (SQR_CHECK=1 loads
libsqr_check.so): ``python -m tests.checked_cases <case>`` prints one JSON object.

valid     a small scene through the index, forward, both backward orders and the
          grid query: no check fails, and the forward agrees with the oracle.
bad_id    one V_sq entry replaced by an id past the last primitive: the forward
          reports site 2 (a listed id that is not a primitive) and skips it.
bad_list  the V_f offsets of the listed voxels moved past V_sq's capacity: site 1.
bad_page  one entry of the saved state's page table moved past the saved buffer:
          the backward's sweep reports site 3.
The planted values are only ever given to this build, whose kernels check them.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from tests.helpers import small_scene  # noqa: E402


def _scene(sqr):
    pr, grid, rig, t = small_scene(7, n=9, C=5)
    prims = sqr.to_device(pr)
    g = {"n": grid["n"], "lo": [float(v) for v in grid["lo"]], "vs": [float(v) for v in grid["vs"]]}
    rays = sqr.Rays.from_rig(rig, t)
    ix = sqr.build_index(prims, g)
    return pr, grid, rig, t, prims, g, rays, ix


def run(case: str) -> dict:
    os.environ["SQR_CHECK"] = "1"
    from paper_2511_17361_gb300 import sqr
    compiled, site = sqr.check_query()
    out = {"compiled": compiled, "lib": os.path.basename(sqr.LIB_PATH), "before": site}
    pr, grid, rig, t, prims, g, rays, ix = _scene(sqr)
    P = ix.P()
    if case == "valid":
        import oracle
        from tests.gpu_common import check_depth, check_sem, oracle_index
        depth, sem, tf = sqr.render_fwd(prims, ix, g, rays)
        gd = torch.ones(rays.R, device="cuda")
        gs = torch.ones((rays.R, 5), device="cuda")
        for order in (sqr.SQ_BWD_DEFAULT, sqr.SQ_BWD_RAY_MAJOR):
            sqr.render_bwd(prims, ix, g, rays, gd, gs, order=order)
        sqr.query_grid(prims, ix, g, tau=0.05)
        torch.cuda.synchronize()
        out["site"] = sqr.check_query()[1]
        D, S, _, _ = oracle.render_fwd(pr, grid, oracle_index(ix, pr, grid), rig, t)
        check_depth(depth.cpu().numpy(), D, 0.5)
        check_sem(sem.cpu().numpy(), S)
        out["parity"] = True
    elif case == "bad_id":
        assert P > 4
        ix.v_sq[P // 2] = prims["means"].shape[0] + 7
        sqr.render_fwd(prims, ix, g, rays)
        torch.cuda.synchronize()
        out["site"] = sqr.check_query()[1]
    elif case == "bad_list":
        ix.v_f[ix.v_n > 0] = ix.capacity + 100  # every listed voxel, so that samples reach one
        sqr.render_fwd(prims, ix, g, rays)
        torch.cuda.synchronize()
        out["site"] = sqr.check_query()[1]
    elif case == "bad_page":
        saved = sqr.new_saved(rays, 5)
        sqr.render_fwd(prims, ix, g, rays, saved=saved)
        torch.cuda.synchronize()
        pages, status = sqr.saved_header(saved)
        assert status == sqr.SQ_OK and pages > 0
        npr = (rays.t.numel() + sqr.SQ_SAVE_PAGE - 1) // sqr.SQ_SAVE_PAGE
        table = saved[256:256 + rays.R * npr * 4].view(torch.int32)
        first = int(torch.nonzero(table >= 0)[0].item())
        table[first] = int(saved.numel())  # far past the buffer's pages
        sqr.render_bwd(prims, ix, g, rays, torch.ones(rays.R, device="cuda"),
                       torch.ones((rays.R, 5), device="cuda"), saved=saved)
        torch.cuda.synchronize()
        out["site"] = sqr.check_query()[1]
    else:
        raise SystemExit(f"unknown case {case}")
    return out


if __name__ == "__main__":
    print(json.dumps(run(sys.argv[1])))
