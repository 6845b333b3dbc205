import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbm.so")
    config.addinivalue_line("markers", "slow: long-running CPU check (minutes)")
    config.addinivalue_line("markers", "gpu_long: GPU run of several minutes, only with -m gpu_long (not part of -m gpu)")


# Relative L2 errors against the FP64 oracle measured by the GPU tests; written as JSON to the path
# in LBM_ACCURACY_OUT (if set) when the session ends.
_ACCURACY = []


@pytest.fixture(scope="session")
def accuracy():
    return _ACCURACY


def _with_target(case):
    """The entry with its accuracy target (the stated bound, or the target a bounded-only run
    misses) and whether every recorded error meets it."""
    c = dict(case)
    target = c.get("target", c.get("bound"))
    errs = [v for k, v in c.items() if k.startswith(("rel_", "max_rel_")) and isinstance(v, float)]
    if target is not None and errs:
        c["target"] = target
        c["meets_target"] = bool(max(errs) <= target)
    return c


def pytest_sessionfinish(session, exitstatus):
    out = os.environ.get("LBM_ACCURACY_OUT")
    if out and _ACCURACY:
        with open(out, "w") as fh:
            json.dump({"source": "python -m pytest tests -m gpu (FP64 oracle vs liblbm.so on the same seeded inputs)",
                       "cases": [_with_target(c) for c in _ACCURACY]}, fh, indent=1)
