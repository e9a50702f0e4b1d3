import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def cpu_pool():
    """Process pool for the slow brute-force pins of the oracle: spawned
    workers (safe whether or not CUDA was initialised in this process), one
    per available core, at most 8."""
    import concurrent.futures as cf
    import multiprocessing as mp
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=max(1, min(8, n)), mp_context=mp.get_context("spawn")) as ex:
        yield ex
