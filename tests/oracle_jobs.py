"""Long oracle runs computed in a background process while the other tests
run (started by conftest.py, with the 'spawn' start method, only when a test
that needs one is selected).  Each job is a plain function of seeded inputs:
it calls only the oracle and the input generators, never the CUDA path."""

import numpy as np

from oracle import sipf_oracle as O
from sipf_inputs import workload


def headline_run(steps, N=None):
    """The 128^3 headline workload (2^22 particles unless N is given) advanced
    `steps` steps by the FP64 oracle: fields, particles by id, diagnostics."""
    wl = workload("headline", N=N)
    st = O.make_state(wl.H, wl.L, wl.origin, wl.params, wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    st = O.run(st, wl.dt, steps)
    order = np.argsort(st.ids, kind="stable")
    return {"n": st.n, "t": st.t, "u": O.density(st), "v": st.v, "m": st.m, "w": st.w,
            "grad_v": st.grad_v, "s": st.s[order], "loga": st.loga[order],
            "ids": st.ids[order], "diag": O.diagnostics(st)}


JOBS = {"headline_100": (headline_run, (100,))}
