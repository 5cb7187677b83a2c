import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


import pytest  # noqa: E402


@pytest.fixture(autouse=True)
def _no_failed_bounds_check(request):
    """With SQR_CHECK=1 the binding loads the debug build with bounds checks
    (libsqr_check.so): then every GPU test must also end with no failed check."""
    yield
    if os.environ.get("SQR_CHECK") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2511_17361_gb300 import sqr
    compiled, site = sqr.check_query()
    assert compiled, "SQR_CHECK=1 but the loaded library has no bounds checks"
    assert site == 0, f"a bounds check failed during the test (site {site})"
