import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built amgc library")
    config.addinivalue_line("markers", "slow: larger CPU case (still part of the default CPU suite)")


@pytest.fixture(scope="session")
def cfg0():
    from paper_1912_09056_gb300.problem import workload
    return workload(0, keep_full=True)


@pytest.fixture(scope="session")
def large_problem():
    """The large workload (110x110x55 + 97x97x49 hex8, 3.47 M rows), generated once per session."""
    from paper_1912_09056_gb300.problem import workload
    return workload(2)
