import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


def pytest_sessionfinish(session, exitstatus):
    """Write the parity gate's per-result figures (tests/parity.py) to the file named by
    BFGP_PARITY_REPORT, if set."""
    path = os.environ.get("BFGP_PARITY_REPORT")
    if not path:
        return
    import parity
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as fh:
        json.dump(parity.REPORT, fh, indent=1)
