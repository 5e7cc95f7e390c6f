"""Ensembles of independent runs through the C ABI: every member, advanced
together with the others on its own stream, ends bit for bit where the same
run advanced alone ends (same kernels, deterministic integer deposit)."""

import os

import numpy as np
import pytest

from oracle import sipf_oracle as O
from paper_2605_20140_gb300 import sipf
from parity_helpers import compare, oracle_state
from sipf_inputs import ensemble_workloads

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


def snapshot(sim):
    f = sim.fields()
    s, loga, ids = sim.particle_state()
    o = np.argsort(ids, kind="stable")
    return f, s[o], loga[o]


@pytest.mark.parametrize("mode,steps", [(sipf.SIPF_ENSEMBLE_BATCHED, 12),
                                        (sipf.SIPF_ENSEMBLE_BATCHED, 13),
                                        (sipf.SIPF_ENSEMBLE_STREAMS, 12)])
def test_members_equal_their_solo_runs(mode, steps):
    """Batched launches across members (one particle-step launch for all
    runs, one launch per spectral pass and grid size, replayed as a graph;
    an odd step count ends with one step enqueued launch by launch) or one
    stream per member: every member ends bit for bit where its solo run ends."""
    runs = ensemble_workloads(6, seed=3, max_log2_N=16)
    assert len({w.H for w in runs}) > 1          # uneven grids
    dts = np.array([w.dt * (1.0 + 0.1 * i) for i, w in enumerate(runs)])
    with sipf.Ensemble([(w.H, w.L, w.origin, w.N, w.params) for w in runs], mode=mode) as ens:
        for sim, w in zip(ens.members, runs):
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        ens.step(dts, steps)
        ens.sync()
        assert ens.last_path() == mode
        got = [snapshot(sim) for sim in ens.members]
        assert all(sim.diagnostics()["step"] == steps for sim in ens.members)
    for w, dt, (f, s, l) in zip(runs, dts, got):
        with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
            solo.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
            solo.step(dt, steps)
            f0, s0, l0 = snapshot(solo)
        for k in f0:
            np.testing.assert_array_equal(f[k], f0[k], err_msg=f"{w.name} {k}")
        np.testing.assert_array_equal(s, s0)
        np.testing.assert_array_equal(l, l0)


def test_step_checks_every_member():
    runs = ensemble_workloads(2, seed=1, max_log2_N=14)
    with sipf.Ensemble([(w.H, w.L, w.origin, w.N, w.params) for w in runs]) as ens:
        ens.members[0].set_state(runs[0].x, runs[0].mass, runs[0].ids, runs[0].v, runs[0].m,
                                 runs[0].w)
        with pytest.raises(sipf.SipfError) as e:
            ens.step([1e-3, 1e-3], 1)      # member 1 has no state
        assert e.value.code == sipf.SIPF_EINVAL
        ens.members[1].set_state(runs[1].x, runs[1].mass, runs[1].ids, runs[1].v, runs[1].m,
                                 runs[1].w)
        with pytest.raises(sipf.SipfError):
            ens.step([1e-3, 0.0], 1)
        ens.step([1e-3, 1e-3], 2)
        ens.sync()


def test_member_with_drawn_parameters_matches_oracle():
    """A member on a radix-3 grid (H = 48) with its own drawn chi, alpha, Du and
    Philox key, advanced inside an uneven ensemble, against the FP64 oracle
    run of the same member alone: fields, positions and log-masses within the
    parity tolerances."""
    runs = ensemble_workloads(8, seed=21, max_log2_N=15)
    pick = [i for i, w in enumerate(runs) if w.H == 48]
    assert pick, [w.H for w in runs]
    i = pick[0]
    steps = 40
    with sipf.Ensemble([(w.H, w.L, w.origin, w.N, w.params) for w in runs]) as ens:
        for sim, w in zip(ens.members, runs):
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        ens.step(np.array([w.dt for w in runs]), steps)
        ens.sync()
        w = runs[i]
        st = O.run(oracle_state(w), w.dt, steps)
        errs = compare(ens.members[i], st, w)
    print(f"member {i} (H={w.H}, N={w.N}, chi={w.params.chi:.4f}, alpha={w.params.alpha:.2f}, "
          f"Du={w.params.Du:.2e}) rel-L2:", {k: f"{v:.1e}" for k, v in errs.items()})


def test_batched_launches_split_above_the_batch_size():
    """70 members of one grid size: the spectral passes take them in two
    launches (64 + 6); every member still equals its solo run."""
    from sipf_inputs import Params, workload
    specs, states = [], []
    for i in range(70):
        w = workload("small", H=16, N=300 + 7 * i, seed=i)
        w.params = Params(seed=1000 + i, chi=0.01 + 1e-4 * i)
        specs.append((w.H, w.L, w.origin, w.N, w.params))
        states.append(w)
    with sipf.Ensemble(specs) as ens:
        for sim, w in zip(ens.members, states):
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        ens.step([w.dt for w in states], 4)
        ens.sync()
        assert ens.last_path() == sipf.SIPF_ENSEMBLE_BATCHED
        got = {i: snapshot(ens.members[i]) for i in (0, 63, 64, 69)}
    for i, (f, s, l) in got.items():
        w = states[i]
        with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
            solo.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
            solo.step(w.dt, 4)
            f0, s0, l0 = snapshot(solo)
        for k in f0:
            np.testing.assert_array_equal(f[k], f0[k], err_msg=f"member {i} {k}")
        np.testing.assert_array_equal(s, s0)
        np.testing.assert_array_equal(l, l0)


def test_a_member_outside_the_batched_form_falls_back_to_streams():
    """A member with the low-pass filter on cannot join the batched launches:
    the ensemble steps one stream per member, with the same results."""
    import dataclasses
    runs = ensemble_workloads(3, seed=4, max_log2_N=14)
    runs[1].params = dataclasses.replace(runs[1].params, H0=runs[1].H ** (8 / 13))
    with sipf.Ensemble([(w.H, w.L, w.origin, w.N, w.params) for w in runs]) as ens:
        for sim, w in zip(ens.members, runs):
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        ens.step([w.dt for w in runs], 3)
        ens.sync()
        assert ens.last_path() == sipf.SIPF_ENSEMBLE_STREAMS
        f, s, l = snapshot(ens.members[1])
    w = runs[1]
    with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
        solo.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        solo.step(w.dt, 3)
        f0, s0, l0 = snapshot(solo)
    for k in f0:
        np.testing.assert_array_equal(f[k], f0[k], err_msg=k)


def test_members_on_the_lane_group_pipeline_equal_their_solo_runs():
    """Members whose tuning selects radix plan 2 (the lane-group spectral
    pipeline) run its passes member by member inside the batched step, and
    members of one grid size on different plans are batched apart: here three
    of the four H = 64 members take plan 2, the fourth keeps its table plan,
    and every member ends bit for bit where its solo run with the same plan
    ends."""
    runs = ensemble_workloads(12, seed=3, max_log2_N=15)
    h64 = [i for i, w in enumerate(runs) if w.H == 64]
    assert len(h64) >= 4 and len({w.H for w in runs}) > 2
    on_plan2 = set(h64[:3])

    def tune(sim, i):
        if i in on_plan2:
            t = sipf.sipf_get_tuning(sim.ctx)
            t["radix_plan"] = 2
            sipf.sipf_set_tuning(sim.ctx, **t)
            assert sipf.sipf_get_tuning(sim.ctx)["radix_plan"] == 2

    steps = 12
    dts = np.array([w.dt for w in runs])
    with sipf.Ensemble([(w.H, w.L, w.origin, w.N, w.params) for w in runs],
                       mode=sipf.SIPF_ENSEMBLE_BATCHED) as ens:
        for i, (sim, w) in enumerate(zip(ens.members, runs)):
            tune(sim, i)
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        assert sipf.sipf_get_tuning(ens.members[h64[3]].ctx)["radix_plan"] != 2
        ens.step(dts, steps)
        ens.sync()
        assert ens.last_path() == sipf.SIPF_ENSEMBLE_BATCHED
        got = [snapshot(sim) for sim in ens.members]
    for i, (w, dt, (f, s, l)) in enumerate(zip(runs, dts, got)):
        with sipf.Simulation(w.H, w.L, w.origin, w.N, w.params) as solo:
            tune(solo, i)
            solo.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
            solo.step(dt, steps)
            f0, s0, l0 = snapshot(solo)
        for k in f0:
            np.testing.assert_array_equal(f[k], f0[k], err_msg=f"{w.name} {k}")
        np.testing.assert_array_equal(s, s0)
        np.testing.assert_array_equal(l, l0)
