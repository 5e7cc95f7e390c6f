"""The seeded input generators: the uneven ensemble follows its stated
distribution and is reproducible."""

import numpy as np

from sipf_inputs import ensemble_workloads


def test_ensemble_workloads_follow_their_ranges():
    runs = ensemble_workloads(24, seed=2, max_log2_N=15)
    assert {w.H for w in runs} <= {32, 48, 64, 96} and len({w.H for w in runs}) > 1
    for w in runs:
        assert 2 ** 14 - 1 <= w.N <= 2 ** 15 + 1 and w.x.shape == (w.N, 3)
        assert 0.005 <= w.params.chi <= 0.03 and 5.0 <= w.params.alpha <= 20.0
        assert 5e-4 <= w.params.Du <= 2e-3
        assert w.v.shape == (w.H, w.H, w.H) and abs(w.mass.sum() - 1.0) < 1e-12
    assert len({w.params.seed for w in runs}) == len(runs)
    again = ensemble_workloads(24, seed=2, max_log2_N=15)
    for a, b in zip(runs, again):
        np.testing.assert_array_equal(a.x, b.x)
