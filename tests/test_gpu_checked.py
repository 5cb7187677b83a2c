"""The debug build with bounds checks (libsqr_check.so, include/sqr.h sq_check_query):
each case runs in its own process with SQR_CHECK=1 (tests/checked_cases.py), so
that the planted bad indices only ever reach kernels that check them."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _case(name: str) -> dict:
    env = dict(os.environ, SQR_CHECK="1")
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases", name], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.gpu
def test_checked_build_valid_scene():
    """Valid inputs: no check fails through index, forward, both backward orders and
    the query, and the checked forward still agrees with the oracle."""
    out = _case("valid")
    assert out["compiled"] and out["lib"] == "libsqr_check.so"
    assert out["before"] == 0 and out["site"] == 0 and out["parity"]


@pytest.mark.gpu
@pytest.mark.parametrize("case,site", [("bad_id", 2), ("bad_list", 1), ("bad_page", 3)])
def test_checked_build_reports_planted_index(case, site):
    """A planted out-of-range id, list offset or saved-state page is reported with its
    site (and the access skipped) instead of being dereferenced."""
    out = _case(case)
    assert out["compiled"] and out["site"] == site
