"""Serving with continuous batching through the C ABI: requests submitted at
different times, admitted while their device memory fits the budget,
advanced together and collected as they finish.  Every request's fields are
bit for bit those of the same run alone, and the device memory in use never
exceeds the budget."""

import os

import numpy as np
import pytest

from paper_2605_20140_gb300 import sipf
from sipf_inputs import Params, ensemble_workloads, workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(sipf.LIB_PATH):
        from paper_2605_20140_gb300 import build
        build.build()
    sipf.load()


@pytest.mark.parametrize("H,N,H0", [(32, 5000, 0.0), (48, 70000, 0.0), (64, 3000, 10.0),
                                    (192, 20000, 0.0)])
def test_device_bytes_match_the_estimate(H, N, H0):
    p = sipf.make_params(Params(H0=H0))
    g = sipf.make_grid(H, 1.0)
    ctx = sipf.sipf_create(g, N, p)
    try:
        assert sipf.load().sipf_device_bytes(ctx) == sipf.sipf_context_bytes(g, N, p)
    finally:
        sipf.sipf_destroy(ctx)


def test_served_results_equal_solo_runs():
    runs = ensemble_workloads(6, seed=5, max_log2_N=15)
    steps = [5, 9, 4, 12, 7, 3]
    need = [sipf.sipf_context_bytes(sipf.make_grid(w.H, w.L), w.N, sipf.make_params(w.params))
            for w in runs]
    budget = int(2.2 * max(need))
    results = {}
    with sipf.Server(budget) as srv:
        ids = {}
        for i in range(3):
            w = runs[i]
            ids[srv.submit(w.H, w.L, w.origin, w.N, w.params, w.x, w.mass, w.v, w.m, w.w,
                           w.dt, steps[i])] = i
        srv.advance(2)
        srv.advance(2)
        for i in range(3, 6):
            w = runs[i]
            ids[srv.submit(w.H, w.L, w.origin, w.N, w.params, w.x, w.mass, w.v, w.m, w.w,
                           w.dt, steps[i])] = i
        rounds = 0
        while len(results) < len(runs):
            srv.advance(2)
            for rid in srv.poll():
                results[ids[rid]] = srv.collect(rid)
            rounds += 1
            assert rounds < 10000
        st = srv.stats()
        assert st["peak"] <= budget and st["in_use"] == 0 and st["live"] == 0
    for i, w in enumerate(runs):
        with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
            solo.set_state(w.x, w.mass, None, w.v, w.m, w.w)
            solo.step(w.dt, steps[i])
            ref = solo.fields()
        for k in ref:
            np.testing.assert_array_equal(results[i][k], ref[k], err_msg=f"request {i} {k}")


def test_collect_rejects_unknown_and_unfinished_requests():
    wl = workload("small", H=32, N=4096)
    with sipf.Server(1 << 34) as srv:
        rid = srv.submit(wl.H, wl.L, wl.origin, wl.N, wl.params, wl.x, wl.mass, wl.v, wl.m, wl.w,
                         wl.dt, 40)
        srv.H[rid + 100] = wl.H
        with pytest.raises(sipf.SipfError):
            srv.collect(rid + 100)
        srv.advance(1)                      # admitted, one step enqueued
        if rid not in srv.poll():
            with pytest.raises(sipf.SipfError):
                srv.collect(rid)            # not finished
            srv.H[rid] = wl.H
        while srv.advance(8):
            pass
        srv.poll()
        f = srv.collect(rid, sipf.FIELD_M)
        assert f["m"].shape == (32, 32, 32)
