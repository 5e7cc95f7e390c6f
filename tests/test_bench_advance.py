"""The timed loop of bench.py on CPU: sipf_step calls cover exactly the
requested steps, with the diagnostics read every DIAG_EVERY steps and a
non-finite count stopping the run (a stand-in object replaces the GPU
simulation)."""

import pytest

import bench


class _Sim:
    def __init__(self, nonfinite_at=None):
        self.steps = 0
        self.calls = []
        self.diag_at = []
        self.nonfinite_at = nonfinite_at

    def step(self, dt, k):
        assert k >= 1
        self.calls.append(k)
        self.steps += k

    def diagnostics(self):
        self.diag_at.append(self.steps)
        bad = self.nonfinite_at is not None and self.steps >= self.nonfinite_at
        return {"nonfinite": 1 if bad else 0, "step": self.steps}


@pytest.mark.parametrize("steps", [0, 1, 99, 100, 101, 250, 1000])
def test_steps_and_diagnostics_schedule(steps):
    sim = _Sim()
    n = bench._advance(sim, 1e-3, steps)
    every = bench.DIAG_EVERY
    assert sim.steps == steps
    assert n == steps // every
    assert sim.diag_at == [every * (i + 1) for i in range(steps // every)]
    assert all(k <= every for k in sim.calls)


def test_non_finite_values_stop_the_run():
    sim = _Sim(nonfinite_at=200)
    with pytest.raises(SystemExit):
        bench._advance(sim, 1e-3, 1000)
    assert sim.steps == 200
