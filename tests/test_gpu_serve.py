"""Serving with continuous batching through the C ABI: requests submitted at
different times, admitted while their device memory fits the budget,
advanced together and collected as they finish.  Every request's fields are
bit for bit those of the same run alone, and the device memory in use never
exceeds the budget."""

import os

import numpy as np
import pytest

from oracle import sipf_oracle as O
from paper_2605_20140_gb300 import sipf
from parity_helpers import compare_fields, oracle_state
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


def _submit(srv, w, steps):
    return srv.submit(w.H, w.L, w.origin, w.N, w.params, w.x, w.mass, w.v, w.m, w.w, w.dt, steps)


def _drain(srv, want):
    out, rounds = {}, 0
    while len(out) < want:
        srv.advance(2)
        for rid in srv.poll():
            try:
                out[rid] = srv.collect(rid)
            except sipf.SipfError as e:
                out[rid] = e
        rounds += 1
        assert rounds < 20000
    return out


def test_served_request_matches_oracle():
    """A request on a radix-3 grid with drawn chi, alpha, Du and seed, served
    in a mix with other requests, against the FP64 oracle run of it alone."""
    runs = ensemble_workloads(8, seed=21, max_log2_N=15)
    pick = [i for i, w in enumerate(runs) if w.H in (48, 96)]
    assert pick, [w.H for w in runs]
    i = pick[0]
    steps = 30
    with sipf.Server(1 << 36) as srv:
        rids = {_submit(srv, w, steps if j == i else 10 + j): j for j, w in enumerate(runs)}
        got = _drain(srv, len(runs))
    f = next(got[r] for r, j in rids.items() if j == i)
    w = runs[i]
    st = O.run(oracle_state(w), w.dt, steps)
    errs = compare_fields(f, st, w)
    print(f"served request (H={w.H}, N={w.N}) rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_a_failed_admission_does_not_block_the_queue():
    """Fault injected on the host: the first admission fails as if device
    memory were short.  That request is reported failed, with its code, and
    the requests behind it run to completion with the results of solo runs;
    no device memory stays accounted to it."""
    runs = ensemble_workloads(3, seed=7, max_log2_N=14)
    with sipf.Server(1 << 36) as srv:
        srv.fail_next_admission(sipf.SIPF_ENOMEM)
        rids = [_submit(srv, w, 6) for w in runs]
        got = _drain(srv, 3)
        st = srv.stats()
    assert isinstance(got[rids[0]], sipf.SipfError) and got[rids[0]].code == sipf.SIPF_ENOMEM
    assert st["in_use"] == 0 and st["live"] == 0 and st["queued"] == 0
    for rid, w in zip(rids[1:], runs[1:]):
        with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
            solo.set_state(w.x, w.mass, None, w.v, w.m, w.w)
            solo.step(w.dt, 6)
            ref = solo.fields()
        for k in ref:
            np.testing.assert_array_equal(got[rid][k], ref[k], err_msg=k)


def test_submit_rejects_a_non_finite_mass():
    """A request with a NaN mass is refused at submission (what set_state
    would refuse at admission); the requests around it are served."""
    runs = ensemble_workloads(2, seed=8, max_log2_N=14)
    bad = runs[0]
    mass = bad.mass.copy()
    mass[5] = np.nan
    with sipf.Server(1 << 36) as srv:
        a = _submit(srv, runs[0], 4)
        with pytest.raises(sipf.SipfError) as e:
            srv.submit(bad.H, bad.L, bad.origin, bad.N, bad.params, bad.x, mass, bad.v, bad.m,
                       bad.w, bad.dt, 4)
        assert e.value.code == sipf.SIPF_EINVAL
        b = _submit(srv, runs[1], 4)
        got = _drain(srv, 2)
    assert set(got) == {a, b} and all(isinstance(v, dict) for v in got.values())


def test_one_at_a_time_limit():
    """With max_live = 1 the server admits one request at a time (the
    one-at-a-time arm of the serving benchmark); results are unchanged."""
    runs = ensemble_workloads(4, seed=9, max_log2_N=14)
    with sipf.Server(1 << 36, max_live=1) as srv:
        rids = [_submit(srv, w, 5) for w in runs]
        out, rounds = {}, 0
        while len(out) < len(runs):
            srv.advance(2)
            assert srv.stats()["live"] <= 1
            for rid in srv.poll():
                out[rid] = srv.collect(rid)
            rounds += 1
            assert rounds < 20000
    w = runs[2]
    with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
        solo.set_state(w.x, w.mass, None, w.v, w.m, w.w)
        solo.step(w.dt, 5)
        ref = solo.fields()
    for k in ref:
        np.testing.assert_array_equal(out[rids[2]][k], ref[k], err_msg=k)
