"""Residual resampling (paper Alg. 4) through the C ABI against the oracle.

The integer work -- which parent each new particle copies, the new ids -- is
compared bit for bit (both sides take the decisions on the same fixed-point
weights of the exported masses and the same Philox draws), positions are
copies and must be bit-identical, and the common new mass a_0 agrees to
float64 rounding of its log-mass (the GPU stores log a_0 - logref)."""

import os

import numpy as np
import pytest

from oracle import resample_oracle as RO
from paper_2605_20140_gb300 import sipf
from sipf_inputs import workload

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


def make_sim(name, H, N, steps, sigma=1.0, ids=None):
    wl = workload(name, H=H, N=N)
    rng = np.random.default_rng(17)
    mass = rng.lognormal(0.0, sigma, N)
    mass *= wl.mass.sum() / mass.sum()
    sim = sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params)
    sim.set_state(wl.x, mass, ids, wl.v, wl.m, wl.w)
    if steps:
        sim.step(wl.dt, steps)
    return wl, sim


def state(sim):
    s, _, ids = sim.particle_state()
    _, mass, ids2 = sim.particles()
    assert np.array_equal(ids, ids2)
    return s, mass, ids


@pytest.mark.parametrize("name,H,N,steps", [("small", 32, 1 << 15, 3), ("small", 48, 20000, 2),
                                            ("headline", 128, 1 << 22, 1)])
def test_resampling_matches_oracle(name, H, N, steps):
    wl, sim = make_sim(name, H, N, steps)
    s0, m0, i0 = state(sim)
    assert sim.resample(0.0)
    s1, m1, i1 = state(sim)
    d = sim.diagnostics()
    sim.step(wl.dt, 2)            # the resampled store steps normally
    sim.close()
    s_exp, a_exp, ids_exp, parent = RO.resample_state(s0, m0, i0, n=steps, seed=wl.params.seed)
    o = np.argsort(i1, kind="stable")
    np.testing.assert_array_equal(i1[o], ids_exp)
    np.testing.assert_array_equal(s1[o], s_exp.astype(np.float32))
    # a_0 is stored as log a_0 - logref: log, the two additions and exp each round
    # to float64 on values of magnitude |log a_0| (about 10 here), so the mass
    # carries a few ulp of that magnitude in relative terms
    rtol = 4.0 * 2.0 ** -52 * (abs(np.log(a_exp[0])) + 1.0)
    np.testing.assert_allclose(m1, a_exp[0], rtol=rtol, atol=0)
    assert abs(d["mass_particles"] - m0.sum()) <= 1e-14 * m0.sum()
    # the deterministic copies: particle p appears at least floor(a_p / a_0) times
    k = np.floor(np.sort(m0)[::-1][:8] / a_exp[0])
    counts = np.sort(np.bincount(parent, minlength=N))[::-1][:8]
    assert np.all(counts >= k)


def test_ratio_threshold_leaves_the_state_unchanged():
    wl, sim = make_sim("small", 32, 4096, 1, sigma=0.1)
    s0, m0, i0 = state(sim)
    ratio = float(m0.max() / m0.min()) * 1.01
    assert not sim.resample(ratio)
    s1, m1, i1 = state(sim)
    o0, o1 = np.argsort(i0), np.argsort(i1)
    np.testing.assert_array_equal(s0[o0], s1[o1])
    np.testing.assert_array_equal(m0[o0], m1[o1])
    assert sim.resample(ratio * 0.5)
    sim.close()


def test_ids_must_be_a_permutation():
    wl = workload("small", H=32, N=4096)
    with sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params) as sim:
        sim.set_state(wl.x, wl.mass, (2 * np.arange(4096)).astype(np.uint32), wl.v, wl.m, wl.w)
        with pytest.raises(sipf.SipfError) as e:
            sim.resample(0.0)
        assert e.value.code == sipf.SIPF_EINVAL
        sim.step(wl.dt, 1)        # the context stays usable
