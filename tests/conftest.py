import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built sipf library")
    config.addinivalue_line("markers", "slow: longer CPU pins (still part of the CPU suite)")
    config.addinivalue_line("markers", "oracle_job(name): the test reads a long oracle run "
                                       "that a background process computes meanwhile")


@pytest.hookimpl(trylast=True)
def pytest_collection_modifyitems(session, config, items):
    """After -m/-k deselection: start the background oracle runs the selected
    tests need, in a process of their own ('spawn': nothing is inherited from
    this process, which may hold a CUDA context later)."""
    names = sorted({m.args[0] for it in items for m in it.iter_markers("oracle_job")})
    if not names:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return          # the GPU tests skip; no oracle run is needed
    except ImportError:
        return
    import multiprocessing as mp

    import oracle_jobs
    pool = mp.get_context("spawn").Pool(processes=len(names))
    config._oracle_pool = pool
    config._oracle_jobs = {n: pool.apply_async(oracle_jobs.JOBS[n][0], oracle_jobs.JOBS[n][1])
                           for n in names}


def pytest_unconfigure(config):
    pool = getattr(config, "_oracle_pool", None)
    if pool is not None:
        pool.terminate()
        pool.join()


@pytest.fixture
def oracle_job(request):
    """Result of the background oracle run named by the test's oracle_job mark."""
    name = request.node.get_closest_marker("oracle_job").args[0]
    jobs = getattr(request.config, "_oracle_jobs", {})
    if name not in jobs:
        import oracle_jobs
        fn, args = oracle_jobs.JOBS[name]
        return fn(*args)
    return jobs[name].get(timeout=3600)
