"""CPU oracle of residual resampling (paper Alg. 4) -- TEST INFRASTRUCTURE ONLY.

Same rules as ``sipf_oracle``: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; it shares no code with
the CUDA path.  Exact integer arithmetic (NumPy int64 and Python integers)
plus the oracle's own Philox4x32-10.

Alg. 4 in the paper's order.  Readings where the paper leaves a choice open:

* The loop over p = 1..P runs in the order of the particle ids 0..P-1 (the
  ids must be a permutation of 0..P-1).
* The integer decisions use fixed-point weights: with E the binary exponent of
  the largest mass (a_max < 2^E, from frexp), Q_p = floor(a_p 2^(31-E)) and
  S = sum_p Q_p.  Then the threshold weight a_0 = S / P, the integer part
  k_p = floor(Q_p / a_0) = floor(Q_p P / S) and the residual, scaled by P,
  R_p = Q_p P - k_p S are exact integers; a particle's decision therefore does
  not depend on rounding order.
* N_stoch = P - sum_p k_p indices are drawn independently with probabilities
  R_p / C, C = sum_p R_p (= S N_stoch).  Draw j uses the 64-bit integer
  U_j = b0 + 2^32 b1 of the Philox4x32-10 block with key (seed mod 2^32,
  seed >> 32) and counter (n, 1, j, 0) (the Brownian increments use word 1 = 0),
  the target t_j = floor(U_j C / 2^64), and the first p whose inclusive prefix
  sum of R exceeds t_j.
* The new list holds the k_p copies of each p in order of p, then the drawn
  particles in draw order; the new ids are 0..P-1 in list order, and every new
  particle has the mass a_0 = T 2^(E-62) / P with T = sum_p round(a_p 2^(62-E))
  (an exact fixed-point total rounded once to float64).
"""

from __future__ import annotations

import bisect
import itertools
import math

import numpy as np

from oracle.sipf_oracle import philox4x32_10


def fixed_point_weights(a: np.ndarray):
    """(E, Q): a_max < 2^E and Q_p = floor(a_p 2^(31-E)) (int64, < 2^31)."""
    a = np.asarray(a, dtype=np.float64)
    amax = float(a.max())
    if not amax > 0.0:
        raise ValueError("resampling needs a positive total mass")
    _, E = math.frexp(amax)
    Q = np.floor(np.ldexp(a, 31 - E)).astype(np.int64)
    return E, Q


def split_counts(Q: np.ndarray):
    """Deterministic part of Alg. 4 on fixed-point weights:
    (S, k_p, R_p) with k_p = floor(Q_p P / S), R_p = Q_p P - k_p S."""
    P = len(Q)
    S = int(Q.sum())
    k = (Q * P) // S
    R = Q * P - k * S
    return S, k, R


def draw_targets(n: int, seed: int, n_stoch: int, C: int) -> list:
    """t_j = floor(U_j C / 2^64), U_j from Philox counter (n, 1, j, 0)."""
    if n_stoch == 0:
        return []
    j = np.arange(n_stoch, dtype=np.uint32)
    ones = np.ones(n_stoch, dtype=np.uint32)
    zero = np.zeros(n_stoch, dtype=np.uint32)
    step = np.full(n_stoch, n & 0xFFFFFFFF, dtype=np.uint32)
    b = philox4x32_10(step, ones, j, zero, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return [((int(b0) | (int(b1) << 32)) * C) >> 64 for b0, b1 in zip(b[0], b[1])]


def residual_resample(a: np.ndarray, n: int, seed: int):
    """Alg. 4 for masses a (indexed by particle id).  Returns (parent, a0):
    parent[j] is the id whose position the new particle j copies, a0 the
    common new mass."""
    a = np.asarray(a, dtype=np.float64)
    P = len(a)
    E, Q = fixed_point_weights(a)
    S, k, R = split_counts(Q)
    # deterministic splitting: k_p copies of particle p, in order of p
    parent_det = np.repeat(np.arange(P, dtype=np.int64), k)
    n_stoch = P - int(k.sum())
    # stochastic part: n_stoch draws with probabilities proportional to R_p
    prefix = list(itertools.accumulate(int(r) for r in R))
    C = prefix[-1]
    assert C == S * n_stoch
    picks = [bisect.bisect_right(prefix, t) for t in draw_targets(n, seed, n_stoch, C)]
    parent = np.concatenate([parent_det, np.asarray(picks, dtype=np.int64)])
    T = sum(int(round(x)) for x in np.ldexp(a, 62 - E))
    a0 = math.ldexp(float(T), -(62 - E)) / P
    return parent, a0


def resample_state(s: np.ndarray, a: np.ndarray, ids: np.ndarray, n: int, seed: int):
    """Resample particles given in any storage order: (s_new, a_new, ids_new)
    with positions s (P, 3) copied from the parents, ids 0..P-1."""
    ids = np.asarray(ids, dtype=np.int64)
    P = len(ids)
    if not np.array_equal(np.sort(ids), np.arange(P)):
        raise ValueError("ids must be a permutation of 0..P-1")
    order = np.argsort(ids)
    s_by_id = np.asarray(s)[order]
    a_by_id = np.asarray(a, dtype=np.float64)[order]
    parent, a0 = residual_resample(a_by_id, n, seed)
    return s_by_id[parent], np.full(P, a0), np.arange(P, dtype=np.int64), parent
