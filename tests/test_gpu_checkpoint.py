"""Checkpoint / resume through the C ABI (sipf_save, sipf_load, sipf_describe).

The state after step n of Alg. 3 (particles, log-masses, ids, v, m, w, the
gather array, step, time and the deposit's fixed-point reference) is written
to a file; a context loaded from it must hold bit for bit the same state and,
advanced with the same dt sequence, reach bit for bit the same later states
as the context that was saved (the deposit is an exact integer sum, so the
re-binned particle order does not change any value).
"""

import os

import numpy as np
import pytest

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


def snapshot(sim):
    f = sim.fields()
    s, loga, ids = sim.particle_state()
    o = np.argsort(ids, kind="stable")
    return f, s[o], loga[o], ids[o], sim.diagnostics()


def assert_same(a, b):
    fa, sa, la, ia, da = a
    fb, sb, lb, ib, db = b
    for k in fa:
        np.testing.assert_array_equal(fa[k], fb[k], err_msg=k)
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(ia, ib)
    for k in ("step", "time", "mass_particles", "mass_grid", "min_u", "min_v", "min_m", "min_w"):
        assert da[k] == db[k], k


@pytest.mark.parametrize("H,N", [(32, 1 << 15), (64, 1 << 17)])
def test_resume_is_bit_exact(tmp_path, H, N):
    wl = workload("small", H=H, N=N)
    path = str(tmp_path / "state.sipf")
    sim = sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params)
    sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    sim.step(wl.dt, 5)
    sim.save(path)
    at_save = snapshot(sim)
    sim.step(wl.dt, 4)
    sim.step(0.5 * wl.dt, 3)
    later = snapshot(sim)
    sim.close()

    res = sipf.Simulation.load(path)
    d = sipf.sipf_describe(res.ctx)
    assert (d["H"], d["N"], d["step"]) == (wl.H, wl.N, 5)
    assert d["params"]["seed"] == wl.params.seed
    assert_same(snapshot(res), at_save)
    res.step(wl.dt, 4)
    res.step(0.5 * wl.dt, 3)
    assert_same(snapshot(res), later)
    res.close()


def test_damaged_files_are_rejected(tmp_path):
    wl = workload("small", H=32, N=4096)
    path = str(tmp_path / "state.sipf")
    with sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params) as sim:
        sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
        sim.step(wl.dt, 2)
        sim.save(path)
    raw = bytearray(open(path, "rb").read())
    flipped = raw.copy()
    flipped[-5] ^= 0x40                      # one payload byte
    cut = raw[:-16]                          # truncated payload
    for name, data in (("flipped", flipped), ("cut", cut)):
        bad = str(tmp_path / name)
        open(bad, "wb").write(bytes(data))
        with pytest.raises(sipf.SipfError) as e:
            sipf.sipf_load(bad)
        assert e.value.code == sipf.SIPF_EINVAL
    # the intact file still loads
    ctx = sipf.sipf_load(path)
    sipf.sipf_destroy(ctx)
