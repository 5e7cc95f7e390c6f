"""Convergence-rate pins of the oracle: first order in the time step
(Lemma temporal, Sec. 4) and the Monte-Carlo rate P^-1/2 in the particle
count (Theorem overall), measured with the metric E of Sec. 5.1."""

import math

import numpy as np
import pytest

from oracle import sipf_oracle as O
from sipf_inputs import Params, node_coordinates, periodic_sq_distance


def _cloud_state(H, N, p, seed, L=1.0):
    rng = np.random.default_rng(seed)
    c = (0.5, 0.5, 0.5)
    x = (np.asarray(c) + 0.08 * rng.standard_normal((N, 3))) % L
    X, Y, Z = node_coordinates(H, L, (0, 0, 0))
    g = np.exp(-periodic_sq_distance(X, Y, Z, c, L) / 0.02)
    v = 1.0 - 0.6 * g
    m = 0.5 * g
    w = np.full((H, H, H), 0.5)
    return O.make_state(H, L, (0, 0, 0), p, x.astype(np.float32), np.full(N, 1.0 / N),
                        np.arange(N, dtype=np.uint32), v, m, w)


def _slope(xs, ys):
    return np.polyfit(np.log2(xs), np.log2(ys), 1)[0]


def test_first_order_in_the_time_step():
    """Runs with tau = 8, 4, 2 x tau_ref on shared Brownian paths (the coarse
    increment is the sum of the fine ones) converge to the tau_ref run at
    first order in tau, in the fields and in the particle positions."""
    H, N, T = 16, 2048, 0.032
    p = Params(chi=0.5, Du=1e-3, Dm=5e-3, Dw=1e-2, alpha=10.0, beta=0.1, gamma=0.5, seed=3)
    nref = 256
    tau_ref = T / nref
    st0 = _cloud_state(H, N, p, 1)
    z_ref = [O.brownian_normals(st0.ids, n, p.seed) for n in range(1, nref + 1)]
    ref = st0
    for n in range(nref):
        ref = O.step(ref, tau_ref, z_ref[n])
    taus, em, es = [], [], []
    for r in (32, 16, 8):
        st = st0
        for j in range(nref // r):
            z = sum(z_ref[j * r:(j + 1) * r]) / math.sqrt(r)
            st = O.step(st, r * tau_ref, z)
        taus.append(r * tau_ref)
        em.append(np.linalg.norm(st.m - ref.m) / np.linalg.norm(ref.m))
        ds = st.s - ref.s
        ds -= H * np.round(ds / H)
        es.append(np.sqrt(np.mean(ds ** 2)))
    assert 0.7 <= _slope(taus, em) <= 1.3, em
    assert 0.7 <= _slope(taus, es) <= 1.3, es


def test_particle_count_rate_half():
    """E between independent runs (different samples and noise) falls like
    P^-1/2 (Theorem overall's Monte-Carlo term)."""
    H, tau, steps = 16, 2e-3, 5
    p = Params(chi=0.2, Du=1e-3, seed=0)
    Ns = [2 ** 10, 2 ** 12, 2 ** 14]
    errs = []
    for N in Ns:
        e = []
        for pair in range(4):
            sts = []
            for k in range(2):
                pk = Params(**{**p.__dict__, "seed": 100 * pair + k})
                st = O.run(_cloud_state(H, N, pk, 1000 * N + 10 * pair + k), tau, steps)
                sts.append(O.density(st))
            e.append(O.error_E(sts[0], sts[1], K=8))
        errs.append(np.mean(e))
    assert -0.65 <= _slope(Ns, errs) <= -0.35, errs


def test_error_metric_truncation_properties():
    """Truncation keeps low modes exactly and removes high ones; E is 0 for
    equal fields and symmetric."""
    H = 16
    q = np.arange(H) / H
    Z, Y, X = np.meshgrid(q, q, q, indexing="ij")
    low = np.cos(2 * np.pi * (X + 2 * Y)) + 0.5
    high = np.cos(2 * np.pi * 6 * Z)
    t = O.fourier_truncate(low + high, 8)
    q8 = np.arange(8) / 8
    Z8, Y8, X8 = np.meshgrid(q8, q8, q8, indexing="ij")
    np.testing.assert_allclose(t, np.cos(2 * np.pi * (X8 + 2 * Y8)) + 0.5, atol=1e-12)
    assert O.error_E(low, low) == 0.0
    assert O.error_E(low, low + high, 8) < 1e-14
    assert math.isclose(O.error_E(low, 2 * low), O.error_E(2 * low, low))
