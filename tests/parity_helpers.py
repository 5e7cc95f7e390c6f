"""Comparison helpers shared by the GPU parity tests: the CUDA path's fields
and particles against the FP64 oracle's, with the tolerances derived in the
module docstring of test_gpu_parity.py (relative L2 1e-5 on u_bar, v, m, w;
grad v from the float32 rounding of v^n; positions 1e-4 grid units;
log-masses 1e-6)."""

import numpy as np

from oracle import sipf_oracle as O

FIELD_TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def oracle_state(wl, x=None, mass=None, v=None, m=None, w=None, p=None):
    return O.make_state(wl.H, wl.L, wl.origin, p or wl.params,
                        wl.x if x is None else x, wl.mass if mass is None else mass, wl.ids,
                        wl.v if v is None else v, wl.m if m is None else m,
                        wl.w if w is None else w)


def oracle_fields(st):
    return {"u": O.density(st), "v": st.v, "m": st.m, "w": st.w,
            "gx": st.grad_v[0], "gy": st.grad_v[1], "gz": st.grad_v[2]}


def by_id(s, loga, ids):
    order = np.argsort(ids, kind="stable")
    return s[order], loga[order], ids[order]


def periodic_diff(a, b, H):
    d = np.asarray(a, np.float64) - b
    return d - H * np.round(d / H)


def grad_tolerance(st, axis, L):
    """Expected relative L2 effect on d_axis v of float32 rounding of v^n over
    st.n steps (4x margin), floored at FIELD_TOL."""
    H = st.H
    n = max(st.n, 1)
    k_rms = 2 * np.pi / L * H / np.sqrt(12.0)
    dv_rms = 2.0 ** -24 * np.sqrt(2.0 * n / 3.0) * np.sqrt(np.mean(st.v ** 2))
    g_rms = np.sqrt(np.mean(st.grad_v[axis] ** 2))
    return max(FIELD_TOL, 4.0 * k_rms * dv_rms / g_rms)


def u_tolerance(st, N):
    """Relative L2 bound on u_bar: FIELD_TOL, or on sparse grids (N < H^3) the
    effect of float32 position rounding on one particle's weights."""
    if N >= st.H ** 3:
        return FIELD_TOL
    return max(FIELD_TOL, 4.0 * np.sqrt(3.0) * st.H * 2.0 ** -24 * np.sqrt(max(st.n, 1)))


def position_tolerance(H, N, n):
    """Bound on the periodic position difference (grid units) after n steps:
    1e-4, or the largest of 3N float32 rounding walks of two roundings per
    step, ulp = 2^(ceil(log2 H) - 24) for positions below H."""
    ulp = 2.0 ** (np.ceil(np.log2(H)) - 24)
    walk = ulp * np.sqrt(2.0 * max(n, 1) / 12.0)
    return max(1e-4, (np.sqrt(2.0 * np.log(3.0 * N)) + 1.5) * walk)


def compare(sim, st, wl, field_tol=FIELD_TOL, pos_tol=1e-4, loga_tol=1e-6):
    f = sim.fields()
    ref = oracle_fields(st)
    errs = {k: rel_l2(f[k], ref[k]) for k in ref}
    tols = {k: field_tol for k in ("u", "v", "m", "w")}
    tols["u"] = max(field_tol, u_tolerance(st, wl.N))
    for axis, k in enumerate(("gx", "gy", "gz")):
        tols[k] = grad_tolerance(st, axis, wl.L)
    s, loga, ids = sim.particle_state()
    s_id, l_id, i_id = by_id(s, loga, ids)
    np.testing.assert_array_equal(i_id, st.ids)
    dpos = np.abs(periodic_diff(s_id, st.s, wl.H))
    dloga = np.max(np.abs(l_id - st.loga))
    report = {"errs": errs, "tols": tols, "dpos": float(dpos.max()), "dloga": float(dloga)}
    for k, e in errs.items():
        assert e <= tols[k], (k, report)
    assert dpos.max() <= max(pos_tol, position_tolerance(wl.H, wl.N, st.n)), report
    assert dloga <= loga_tol, report
    return errs


def compare_fields(f, st, wl, field_tol=FIELD_TOL):
    """Fields only (what a served request returns): u_bar, v, m, w and grad v
    of the CUDA path against the oracle state st."""
    ref = oracle_fields(st)
    errs = {k: rel_l2(f[k], ref[k]) for k in ref if k in f}
    tols = {k: field_tol for k in ("u", "v", "m", "w")}
    tols["u"] = max(field_tol, u_tolerance(st, wl.N))
    for axis, k in enumerate(("gx", "gy", "gz")):
        tols[k] = grad_tolerance(st, axis, wl.L)
    for k, e in errs.items():
        assert e <= tols[k], (k, errs, tols)
    return errs
