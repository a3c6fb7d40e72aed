import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_sessionfinish(session, exitstatus):
    # the GPU parity tests' largest float errors per workload, when SEG_PARITY_REPORT is set
    helpers = sys.modules.get("gpu_helpers")
    if helpers is not None:
        helpers.write_report()


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
