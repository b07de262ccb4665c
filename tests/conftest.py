import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session", autouse=True)
def _build_oracle():
    """Builds the oracle and lets it use every host core (its results do not
    depend on the thread count: every sum keeps its order)."""
    import oracle
    oracle.build()
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    for kind in ("f64", "ld"):
        oracle.set_threads(n, kind)
