"""CPU checks of the C ABI: the library builds, loads, exports every function
declared in include/sipf.h, its structs have the layout gcc gives the header,
and argument validation rejects bad input before any CUDA work."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2605_20140_gb300 import sipf
from sipf_inputs import Params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sipf.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sipf.LIB_PATH):
        from paper_2605_20140_gb300 import build
        build.build()
    return sipf.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sipf_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(sipf.EXPORTED) == sorted(n for n in names if n in sipf.EXPORTED)


def test_struct_layout_matches_the_header():
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "sipf.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(sipf_grid), sizeof(sipf_params), sizeof(sipf_diag));
  printf("%zu %zu %zu\n", offsetof(sipf_grid, origin), offsetof(sipf_params, diffusion),
         offsetof(sipf_params, H0));
  printf("%zu %zu %zu %zu\n", offsetof(sipf_params, seed), offsetof(sipf_diag, nonfinite),
         offsetof(sipf_params, p2g_order), offsetof(sipf_params, sigma));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(sipf.sipf_grid), ctypes.sizeof(sipf.sipf_params),
            ctypes.sizeof(sipf.sipf_diag), sipf.sipf_grid.origin.offset,
            sipf.sipf_params.diffusion.offset, sipf.sipf_params.H0.offset,
            sipf.sipf_params.seed.offset, sipf.sipf_diag.nonfinite.offset,
            sipf.sipf_params.p2g_order.offset, sipf.sipf_params.sigma.offset]
    assert got == want


def _create(lib, H=32, L=1.0, N=100, **kw):
    g = sipf.make_grid(H, L)
    p = sipf.sipf_params()
    p.chi, p.Du, p.Dm, p.Dw, p.alpha, p.beta, p.gamma = 0.01, 1e-3, 1e-3, 1e-2, 10, 0.1, 0.5
    for k, v in kw.items():
        setattr(p, k, v)
    out = ctypes.c_void_p()
    return lib.sipf_create(ctypes.byref(g), N, ctypes.byref(p), None, ctypes.byref(out)), out


@pytest.mark.parametrize("kw,code", [
    (dict(N=0), sipf.SIPF_EINVAL),
    (dict(N=1 << 31), sipf.SIPF_EINVAL),
    (dict(H=40), sipf.SIPF_EINVAL),
    (dict(H=36), sipf.SIPF_EINVAL),
    (dict(H=12), sipf.SIPF_EINVAL),
    (dict(H=1024), sipf.SIPF_EINVAL),
    (dict(H=40 * 8), sipf.SIPF_EINVAL),
    (dict(L=0.0), sipf.SIPF_EINVAL),
    (dict(L=float("nan")), sipf.SIPF_EINVAL),
    (dict(chi=-1.0), sipf.SIPF_EINVAL),
    (dict(Du=float("inf")), sipf.SIPF_EINVAL),
    (dict(diffusion=7), sipf.SIPF_EINVAL),
    (dict(v_update=2), sipf.SIPF_EINVAL),
    (dict(p2g_order=3), sipf.SIPF_EINVAL),
    (dict(sigma=-1e-3), sipf.SIPF_EINVAL),
    (dict(reserved=1), sipf.SIPF_EINVAL),
])
def test_create_rejects_bad_arguments_without_touching_the_gpu(lib, kw, code):
    r, out = _create(lib, **kw)
    assert r == code and out.value is None


def test_null_arguments_and_strerror(lib):
    assert lib.sipf_create(None, 10, None, None, None) == sipf.SIPF_EINVAL
    assert lib.sipf_step(None, 1e-3, 1) == sipf.SIPF_EINVAL
    assert lib.sipf_sync(None) == sipf.SIPF_EINVAL
    lib.sipf_destroy(None)
    for code in (0, -1, -2, -3, -4, -6, -7):
        assert lib.sipf_strerror(code)
    assert lib.sipf_last_error(None) == b""


def test_load_rejects_missing_and_foreign_files_without_touching_the_gpu(lib, tmp_path):
    out = ctypes.c_void_p()
    assert lib.sipf_load(b"/nonexistent/dir/state.sipf", None, ctypes.byref(out)) == sipf.SIPF_EINVAL
    junk = tmp_path / "junk.sipf"
    junk.write_bytes(b"not a checkpoint" * 64)
    assert lib.sipf_load(os.fsencode(str(junk)), None, ctypes.byref(out)) == sipf.SIPF_EINVAL
    assert out.value is None
    assert lib.sipf_load(None, None, ctypes.byref(out)) == sipf.SIPF_EINVAL
    assert lib.sipf_save(None, b"x") == sipf.SIPF_EINVAL
    assert lib.sipf_describe(None, None, None, None, None, None) == sipf.SIPF_EINVAL


def test_ensemble_calls_reject_bad_arguments_without_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    g = sipf.make_grid(32, 1.0)
    p = sipf.sipf_params()
    n = ctypes.c_int64(100)
    assert lib.sipf_ensemble_create(0, ctypes.byref(g), ctypes.byref(n), ctypes.byref(p),
                                    ctypes.byref(out)) == sipf.SIPF_EINVAL
    assert lib.sipf_ensemble_create(1, None, None, None, ctypes.byref(out)) == sipf.SIPF_EINVAL
    assert out.value is None
    assert lib.sipf_ensemble_step(None, None, 1) == sipf.SIPF_EINVAL
    assert lib.sipf_ensemble_sync(None) == sipf.SIPF_EINVAL
    assert lib.sipf_ensemble_member(None, 0) is None
    assert lib.sipf_ensemble_last_error(None) == b""
    lib.sipf_ensemble_destroy(None)


def test_context_bytes_without_touching_the_gpu(lib):
    p = sipf.sipf_params()
    p.chi, p.Du, p.Dm, p.Dw, p.alpha, p.beta, p.gamma = 0.01, 1e-3, 1e-3, 1e-2, 10, 0.1, 0.5
    b = lambda H, N: sipf.sipf_context_bytes(sipf.make_grid(H, 1.0), N, p)
    assert b(32, 1000) > 0 and b(32, 2000) > b(32, 1000) and b(64, 1000) > b(32, 1000)
    spec = 64 * 64 * (64 // 2 + 2) * 8
    p.H0 = 10.0                                   # the filtered v spectrum adds one spectrum
    assert b(64, 1000) == sipf.sipf_context_bytes(sipf.make_grid(64, 1.0), 1000, p)
    filt = b(64, 1000)
    p.H0 = 0.0
    assert filt - b(64, 1000) == spec
    assert b(40, 1000) == sipf.SIPF_EINVAL and b(32, 0) == sipf.SIPF_EINVAL
    assert lib.sipf_device_bytes(None) == sipf.SIPF_EINVAL


def test_server_queues_and_validates_without_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.sipf_server_create(0, ctypes.byref(out)) == sipf.SIPF_EINVAL
    assert lib.sipf_server_advance(None, 1, None) == sipf.SIPF_EINVAL
    assert lib.sipf_server_last_error(None) == b""
    lib.sipf_server_destroy(None)
    from sipf_inputs import workload
    wl = workload("small", H=32, N=2048)
    need = sipf.sipf_context_bytes(sipf.make_grid(32, 1.0), 2048, sipf.make_params(wl.params))
    srv = sipf.Server(10 * need)
    try:
        rid = srv.submit(wl.H, wl.L, wl.origin, wl.N, wl.params, wl.x, wl.mass, wl.v, wl.m, wl.w,
                         wl.dt, 4)
        assert rid == 1 and srv.stats() == {"in_use": 0, "peak": 0, "queued": 1, "live": 0}
        with pytest.raises(sipf.SipfError):
            srv.submit(wl.H, wl.L, wl.origin, wl.N, wl.params, wl.x, wl.mass, wl.v, wl.m, wl.w,
                       0.0, 4)
    finally:
        srv.close()
    small = sipf.Server(need - 1)                 # larger than the whole budget
    try:
        with pytest.raises(sipf.SipfError) as e:
            small.submit(wl.H, wl.L, wl.origin, wl.N, wl.params, wl.x, wl.mass, wl.v, wl.m,
                         wl.w, wl.dt, 4)
        assert e.value.code == sipf.SIPF_EINVAL
    finally:
        small.close()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every entry point raises."""
    monkeypatch.setattr(sipf, "LIB_PATH", str(tmp_path / "libsipf.so"))
    monkeypatch.setattr(sipf, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        sipf.load()
    with pytest.raises(RuntimeError, match="missing"):
        sipf.Simulation(16, 1.0, (0.0, 0.0, 0.0), 64, Params())


def _restore_shipped_table():
    """Put back the table that ships next to the library (later tests in the
    same process create contexts with it, as bench.py does)."""
    shipped = os.path.join(os.path.dirname(sipf.LIB_PATH), "sipf_tuning.txt")
    sipf.sipf_tuning_load(shipped if os.path.exists(shipped) else None)


def test_tuning_table_is_parsed_and_looked_up(lib, tmp_path):
    """The autotuner's table (host only): the first line matching (H, N)
    applies; malformed or out-of-range lines are refused; NULL empties it."""
    good = tmp_path / "t.txt"
    good.write_text("# comment\n128 1000 5000000 1 4 16 16   # ms\n\n96 1 999 0 0 32 8\n"
                    "128 1 999 0 3 8 32\n")
    sipf.sipf_tuning_load(good)
    assert sipf.sipf_tuning_lookup(128, 4194304) == {
        "radix_plan": 1, "step_blocks_per_sm": 4, "bucket_slack_div": 16, "bucket_slack_add": 16}
    assert sipf.sipf_tuning_lookup(128, 500)["step_blocks_per_sm"] == 3
    assert sipf.sipf_tuning_lookup(96, 1000) is None
    assert sipf.sipf_tuning_lookup(64, 10) is None
    for text in ("128 1 10 3 0 8 32\n", "128 1 10 0 0 4 32\n", "128 1 10 0 0 8 64\n",
                 "128 10 1 0 0 8 32\n", "128 1 10 0\n"):
        bad = tmp_path / "bad.txt"
        bad.write_text(text)
        with pytest.raises(sipf.SipfError):
            sipf.sipf_tuning_load(bad)
    with pytest.raises(sipf.SipfError):
        sipf.sipf_tuning_load(tmp_path / "missing.txt")
    sipf.sipf_tuning_load(None)
    assert sipf.sipf_tuning_lookup(128, 4194304) is None
    _restore_shipped_table()


def test_autotuner_candidates_are_valid():
    from paper_2605_20140_gb300 import autotune
    cands = autotune.candidates()
    assert len(cands) == len({tuple(sorted(c.items())) for c in cands}) >= 12
    for c in cands:
        assert c["radix_plan"] in (0, 1, 2) and 0 <= c["step_blocks_per_sm"] <= 32
        assert 8 <= c["bucket_slack_div"] <= 1024 and 0 <= c["bucket_slack_add"] <= 32
    for H, lo, hi, rep, recipe in autotune.TARGETS:
        assert lo <= rep <= hi and recipe in ("headline", "large")


def test_autotuner_partial_table_keeps_the_other_sizes(tmp_path):
    """A re-tune of some grid sizes (--only) rewrites their lines and keeps
    the others; the result parses."""
    from paper_2605_20140_gb300 import autotune
    path = tmp_path / "t.txt"
    path.write_text("# old table\n128 1 10 0 0 8 32   # 0.2 (0.2)\n256 1 10 1 0 16 16   # 2.0\n"
                    "96 1 10 1 3 16 16   # 0.05\n")
    best = dict(radix_plan=2, step_blocks_per_sm=0, bucket_slack_div=16, bucket_slack_add=16)
    autotune.write_table(str(path), [(256, 1, 10, best, 1.5, 1.9)], keep={128, 96})
    lines = [ln.split("#")[0].split() for ln in path.read_text().splitlines()]
    rows = [ln for ln in lines if ln]
    assert sorted(int(r[0]) for r in rows) == [96, 128, 256]
    assert [r for r in rows if r[0] == "256"] == [["256", "1", "10", "2", "0", "16", "16"]]
    assert [r for r in rows if r[0] == "128"] == [["128", "1", "10", "0", "0", "8", "32"]]
    sipf.sipf_tuning_load(path)
    try:
        assert sipf.sipf_tuning_lookup(256, 5)["radix_plan"] == 2
        assert sipf.sipf_tuning_lookup(96, 5)["step_blocks_per_sm"] == 3
    finally:
        _restore_shipped_table()
