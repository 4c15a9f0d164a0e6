import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


# The 4096-cell 14-moment Sod tube's oracle trajectories take minutes: when
# its test is collected, start them in a spawn-started process pool right
# away (no GPU work is done in the workers), so that they run while the rest
# of the suite does.
_SOD4096 = {}


def pytest_collection_finish(session):
    if any("test_gpu_zsod14_4096" in it.nodeid for it in session.items):
        from tests._sod14_4096 import Runs
        _SOD4096["runs"] = Runs()


def pytest_sessionfinish(session, exitstatus):
    runs = _SOD4096.pop("runs", None)
    if runs is not None:
        runs.close()


@pytest.fixture(scope="session")
def sod14_4096_runs():
    if "runs" not in _SOD4096:
        from tests._sod14_4096 import Runs
        _SOD4096["runs"] = Runs()
    return _SOD4096["runs"]
