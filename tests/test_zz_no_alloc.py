"""The allocation-free deposit against the context path.

sipf_deposit_noalloc is for callers that must not allocate device memory
when they need a density (code under another framework's memory budget,
real-time loops, plug-ins given only pre-allocated buffers).  Its result
must match the deposit of the regular context path (sipf_fields with
SIPF_FIELD_U) within the deposit tolerance of the parity tests, on two
calls in a row (the second call must not see the first call's sums)."""

import numpy as np
import pytest

from paper_2605_20140_gb300 import sipf
from sipf_inputs import workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _context_deposit(wl):
    with sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params) as sim:
        sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
        return sim.fields(sipf.FIELD_U)["u"].astype(np.float64)


def _noalloc_deposit(wl):
    x = torch.from_numpy(np.ascontiguousarray(wl.x.T)).cuda()
    mass = torch.from_numpy(np.ascontiguousarray(wl.mass)).cuda()
    u = torch.full((wl.H ** 3,), -1.0, dtype=torch.float32, device="cuda")
    sipf.sipf_deposit_noalloc(sipf.make_grid(wl.H, wl.L, wl.origin), x, mass, wl.N, u)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64).reshape(wl.H, wl.H, wl.H)


def test_noalloc_deposit_matches_context_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    if not os.path.exists(sipf.LIB_PATH):
        from paper_2605_20140_gb300 import build
        build.build()
    first = workload("small", H=32, N=1 << 15)
    second = workload("headline", H=64, N=1 << 17, seed=3)
    second.mass = second.mass * (0.5 + np.random.default_rng(1).random(second.N))
    for wl in (first, second):
        ref = _context_deposit(wl)
        got = _noalloc_deposit(wl)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-6, rel
        assert np.max(np.abs(got - ref)) <= 2e-6 * ref.max()
        h3 = (wl.L / wl.H) ** 3
        assert abs(got.sum() * h3 - wl.mass.sum()) <= 1e-6 * wl.mass.sum()


def test_noalloc_skips_non_finite_masses():
    """An infinite or NaN mass contributes nothing (it must not set the scale
    of every node): the result equals the context path's deposit of the same
    particles with those masses set to zero (massless tracers)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = workload("small", H=32, N=1 << 14, seed=5)
    bad = wl.mass.copy()
    bad[[3, 77]] = [np.inf, np.nan]
    clean = wl.mass.copy()
    clean[[3, 77]] = 0.0
    wl.mass = clean
    ref = _context_deposit(wl)
    wl.mass = bad
    got = _noalloc_deposit(wl)
    assert np.isfinite(got).all()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-6, rel


def test_noalloc_rejects_grids_beyond_its_scratch():
    """H = 128 needs more nodes than the fixed scratch holds: refused up front."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = torch.zeros(30, dtype=torch.float32, device="cuda")
    mass = torch.ones(10, dtype=torch.float64, device="cuda")
    u = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(sipf.SipfError) as e:
        sipf.sipf_deposit_noalloc(sipf.make_grid(128, 1.0), x, mass, 10, u)
    assert e.value.code == sipf.SIPF_EINVAL
