import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


@pytest.fixture(scope="session", autouse=True)
def _built_host_libs():
    """Compile the gcc-built helpers (workload generators, oracle) once."""
    import oracle
    import paper_2205_14503_gb300.workloads as wl
    wl.build()
    oracle.build()
    yield
