import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU-side oracle runs")


def pytest_sessionfinish(session, exitstatus):
    """With MATEX_TEST_REPORT set, write the adaptive-m records of the GPU
    parity comparisons there (JSON)."""
    path = os.environ.get("MATEX_TEST_REPORT")
    if not path:
        return
    import json
    from tests import parity_util
    with open(path, "w") as f:
        json.dump(parity_util.REPORT, f, indent=1)
