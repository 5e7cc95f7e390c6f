"""Pins of the residual-resampling oracle (paper Alg. 4) against what the
algorithm and the mathematics fix: a worked example, exact rational
arithmetic of k_p = floor(a_p / a_0) and r_p = a_p - k_p a_0, the unbiasedness
E[copies of p] = a_p / a_0, the equal-weight and single-heavy-particle special
cases, mass conservation and independence of the storage order."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import resample_oracle as R


def test_worked_example():
    # a = (1, 2, 3, 2): a_0 = 2, k = (0, 1, 1, 1), r = (1, 0, 1, 0), one draw
    # between particles 0 and 2 with equal probability
    a = np.array([1.0, 2.0, 3.0, 2.0])
    seen = set()
    for n in range(64):
        parent, a0 = R.residual_resample(a, n, seed=5)
        assert a0 == 2.0
        assert list(parent[:3]) == [1, 2, 3]
        assert parent[3] in (0, 2)
        seen.add(int(parent[3]))
    assert seen == {0, 2}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_integer_parts_and_residuals_match_exact_rationals(seed):
    rng = np.random.default_rng(seed)
    P = 257
    m = rng.integers(1, 1 << 20, size=P)
    m[rng.integers(0, P, 8)] = rng.integers(1 << 18, 1 << 20, 8)
    a = m.astype(np.float64) * 2.0 ** -10          # dyadic: Q is exact
    E, Q = R.fixed_point_weights(a)
    S, k, Rr = R.split_counts(Q)
    a0 = Fraction(int(m.sum()), P) * Fraction(1, 1 << 10)
    scale = Fraction(1 << (31 - E))                  # Q = a * scale exactly
    for p in range(P):
        ap = Fraction(int(m[p]), 1 << 10)
        kp = math.floor(ap / a0)
        assert k[p] == kp
        assert Fraction(int(Rr[p]), P) / scale == ap - kp * a0
    assert int(k.sum()) + (int(Rr.sum()) // S) == P


def test_copies_are_unbiased():
    rng = np.random.default_rng(7)
    P = 48
    a = rng.uniform(0.05, 3.0, size=P)
    a[3] = 9.0
    trials = 600
    counts = np.zeros((trials, P))
    for t in range(trials):
        parent, a0 = R.residual_resample(a, n=t + 1, seed=11)
        assert len(parent) == P
        counts[t] = np.bincount(parent, minlength=P)
    expect = a / a.mean()
    mean = counts.mean(axis=0)
    sd = counts.std(axis=0, ddof=1) / math.sqrt(trials)
    # deterministic parts are exact; residual parts within 5 standard errors
    ok = np.abs(mean - expect) <= 5.0 * np.maximum(sd, 1e-12) + 1e-12
    assert ok.all(), (mean[~ok], expect[~ok])
    np.testing.assert_array_less(np.floor(expect) - 1e-12, counts.min(axis=0) + 1e-12)


def test_equal_masses_are_an_identity():
    parent, a0 = R.residual_resample(np.full(100, 0.25), n=3, seed=1)
    np.testing.assert_array_equal(parent, np.arange(100))
    assert a0 == 0.25


def test_single_heavy_particle_takes_the_deterministic_copies():
    a = np.full(64, 1e-9)
    a[17] = 1.0
    parent, a0 = R.residual_resample(a, n=1, seed=2)
    k17 = math.floor(1.0 / a0)
    assert np.count_nonzero(parent[:k17] == 17) == k17


def test_mass_is_conserved_and_storage_order_does_not_matter():
    rng = np.random.default_rng(3)
    P = 1000
    a = rng.lognormal(0.0, 1.0, P) / P
    s = rng.uniform(0, 32, (P, 3))
    ids = rng.permutation(P)
    s1, a1, i1, par1 = R.resample_state(s, a, ids, n=9, seed=4)
    perm = rng.permutation(P)
    s2, a2, i2, par2 = R.resample_state(s[perm], a[perm], ids[perm], n=9, seed=4)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(par1, par2)
    assert abs(a1.sum() - a.sum()) <= 1e-14 * a.sum()
    np.testing.assert_array_equal(i1, np.arange(P))
    with pytest.raises(ValueError):
        R.resample_state(s, a, np.zeros(P, np.int64), n=1, seed=0)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_fixed_point_decisions_against_real_masses(seed):
    """Ordinary (non-dyadic) float64 masses: Alg. 4 on the exact rational
    masses gives k_p = floor(a_p / a_bar) with a_bar = sum(a) / P and the
    residual r_p / a_bar = a_p / a_bar - k_p.  The oracle decides on 31-bit
    fixed-point weights Q_p = floor(a_p 2^(31-E)), so x_p = a_p / a_bar is
    replaced by Q_p P / S.  With s = 2^(31-E), Q_p = a_p s - d_p and
    S = (sum a) s - D (0 <= d_p < 1, 0 <= D < P), which moves x_p by at most
    eps_p = (1 + x_p) P / ((sum a) s - P) (first order, plus a 1% margin).  So
    k_p may differ from the real-mass decision only where x_p lies within
    eps_p of an integer, and the residual probabilities agree to eps_p / P."""
    rng = np.random.default_rng(100 + seed)
    P = 2000
    a = rng.lognormal(0.0, 1.2, P) / P
    a[rng.integers(0, P, 5)] *= 40.0                     # a few heavy particles
    E, Q = R.fixed_point_weights(a)
    S, k, Rr = R.split_counts(Q)
    fa = [Fraction(float(v)) for v in a]                 # exact values of the float64 masses
    A = sum(fa)
    s = Fraction(2) ** (31 - E)
    margin = Fraction(101, 100) * P / (A * s - P)
    mismatches = 0
    for p in range(P):
        x = fa[p] * P / A                                # a_p / a_bar, exact
        kp = math.floor(x)
        eps = (1 + x) * margin
        if k[p] != kp:
            mismatches += 1
            near = min(x - math.floor(x), math.ceil(x) - x)
            assert near <= eps, (p, float(x), int(k[p]), kp)
            assert abs(int(k[p]) - kp) == 1
        else:
            # residual probability r_p / sum(r) with sum(r) = P - sum(k) in units of a_bar
            got = Fraction(int(Rr[p]), S)                # = Q_p P / S - k_p
            assert abs(got - (x - kp)) <= eps, (p, float(got), float(x - kp))
    # the bound is tight enough that decisions essentially never flip
    assert mismatches <= 2
    assert float(margin) < 1e-5
