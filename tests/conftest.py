import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CHECKED = os.environ.get("IVHD_CHECKED", "") not in ("", "0")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libivhd")
    config.addinivalue_line("markers", "plants_violations: corrupts a layout on purpose "
                                       "(checked builds only)")


@pytest.fixture(autouse=True)
def _no_bounds_violations(request):
    """With the checked library (IVHD_CHECKED=1), every GPU test must end
    without an out-of-range index or row met by the step kernels."""
    yield
    if CHECKED and "gpu" in request.keywords and "plants_violations" not in request.keywords:
        from paper_2303_05455_gb300 import ivhd
        assert ivhd.check_violations(reset=True) == 0
