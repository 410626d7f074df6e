import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def c2_full():
    """The benchmark's full-size 2D workload (512 x 512 cells, 64 per species
    per cell on average, seed 2), generated once per test session."""
    from paper_2206_02937_gb300 import workloads as wl
    return wl.c2(512, 512, 64, seed=2)
