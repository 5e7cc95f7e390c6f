"""ctypes binding of libsipf.so (the C ABI declared in include/sipf.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Functions keep the C names; buffers are passed as raw
pointers (``int`` addresses, e.g. ``tensor.data_ptr()`` of a CUDA tensor
with ``where=SIPF_DEVICE``) or NumPy arrays (``where=SIPF_HOST``).  A missing
library raises immediately: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

SIPF_OK = 0
SIPF_EINVAL = -1
SIPF_ENOMEM = -2
SIPF_ECUDA = -3
SIPF_EUNSUPPORTED = -4
SIPF_ENONFINITE = -6
SIPF_EINTERNAL = -7

SIPF_HOST = 0
SIPF_DEVICE = 1

SIPF_ENSEMBLE_BATCHED = 0
SIPF_ENSEMBLE_STREAMS = 1

FIELD_U, FIELD_V, FIELD_M, FIELD_W, FIELD_GX, FIELD_GY, FIELD_GZ = (1, 2, 4, 8, 16, 32, 64)
FIELD_NAMES = ("u", "v", "m", "w", "gx", "gy", "gz")

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsipf.so")

EXPORTED = (
    "sipf_create", "sipf_set_state", "sipf_step", "sipf_fields", "sipf_particles",
    "sipf_particle_state", "sipf_cell_start", "sipf_diagnostics", "sipf_sync",
    "sipf_destroy", "sipf_strerror", "sipf_last_error", "sipf_brownian_normals",
    "sipf_profile", "sipf_profile_read", "sipf_profile_name",
    "sipf_deposit_noalloc", "sipf_save", "sipf_load",
    "sipf_describe", "sipf_resample", "sipf_ensemble_create", "sipf_ensemble_member",
    "sipf_ensemble_step", "sipf_ensemble_sync", "sipf_ensemble_last_error",
    "sipf_ensemble_destroy", "sipf_context_bytes", "sipf_device_bytes", "sipf_server_create",
    "sipf_server_submit", "sipf_server_advance", "sipf_server_poll", "sipf_server_collect",
    "sipf_server_stats", "sipf_server_last_error", "sipf_server_destroy",
    "sipf_server_set_limit", "sipf_server_fail_next_admission", "sipf_canonical_order",
    "sipf_ensemble_set_mode", "sipf_ensemble_last_path", "sipf_set_tuning", "sipf_get_tuning",
    "sipf_tuning_load", "sipf_tuning_lookup",
)
PROFILE_GROUPS = 4


class sipf_grid(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("L", ctypes.c_double), ("origin", ctypes.c_double * 3)]


class sipf_params(ctypes.Structure):
    _fields_ = [("chi", ctypes.c_double), ("Du", ctypes.c_double), ("Dm", ctypes.c_double),
                ("Dw", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("diffusion", ctypes.c_int32),
                ("v_update", ctypes.c_int32), ("H0", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("p2g_order", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sigma", ctypes.c_double)]


class sipf_tuning(ctypes.Structure):
    _fields_ = [("radix_plan", ctypes.c_int32), ("step_blocks_per_sm", ctypes.c_int32),
                ("bucket_slack_div", ctypes.c_int32), ("bucket_slack_add", ctypes.c_int32)]


class sipf_diag(ctypes.Structure):
    _fields_ = [("mass_particles", ctypes.c_double), ("mass_grid", ctypes.c_double),
                ("min_u", ctypes.c_double), ("min_v", ctypes.c_double),
                ("min_m", ctypes.c_double), ("min_w", ctypes.c_double),
                ("step", ctypes.c_int64), ("time", ctypes.c_double),
                ("nonfinite", ctypes.c_int64)]


class SipfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    """Load libsipf.so from the package directory (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, U32, U64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                             ctypes.c_uint64)
    sig = {
        "sipf_create": ([ctypes.POINTER(sipf_grid), I64, ctypes.POINTER(sipf_params), P,
                         ctypes.POINTER(P)], I32),
        "sipf_set_state": ([P, P, P, P, P, P, P, I32], I32),
        "sipf_step": ([P, ctypes.c_double, I64], I32),
        "sipf_fields": ([P, U32, P, I32], I32),
        "sipf_particles": ([P, P, P, P, I32], I32),
        "sipf_particle_state": ([P, P, P, P, I32], I32),
        "sipf_cell_start": ([P, P, I32], I32),
        "sipf_canonical_order": ([P, P, P, I32], I32),
        "sipf_diagnostics": ([P, ctypes.POINTER(sipf_diag)], I32),
        "sipf_sync": ([P], I32),
        "sipf_destroy": ([P], None),
        "sipf_strerror": ([I32], ctypes.c_char_p),
        "sipf_last_error": ([P], ctypes.c_char_p),
        "sipf_brownian_normals": ([P, I64, U32, U64, P, P, P], I32),
        "sipf_profile": ([P, I32], I32),
        "sipf_profile_read": ([P, P, P, I32], I32),
        "sipf_profile_name": ([I32], ctypes.c_char_p),
        "sipf_deposit_noalloc": ([ctypes.POINTER(sipf_grid), P, P, I64, P, P], I32),
        "sipf_save": ([P, ctypes.c_char_p], I32),
        "sipf_resample": ([P, ctypes.c_double, ctypes.POINTER(ctypes.c_int32)], I32),
        "sipf_ensemble_create": ([I32, P, P, P, ctypes.POINTER(P)], I32),
        "sipf_ensemble_member": ([P, I32], P),
        "sipf_ensemble_step": ([P, P, I64], I32),
        "sipf_ensemble_sync": ([P], I32),
        "sipf_ensemble_last_error": ([P], ctypes.c_char_p),
        "sipf_ensemble_destroy": ([P], None),
        "sipf_ensemble_set_mode": ([P, I32], I32),
        "sipf_set_tuning": ([P, ctypes.POINTER(sipf_tuning)], I32),
        "sipf_get_tuning": ([P, ctypes.POINTER(sipf_tuning)], I32),
        "sipf_tuning_load": ([ctypes.c_char_p], I32),
        "sipf_tuning_lookup": ([I32, I64, ctypes.POINTER(sipf_tuning)], I32),
        "sipf_ensemble_last_path": ([P], I32),
        "sipf_context_bytes": ([ctypes.POINTER(sipf_grid), I64, ctypes.POINTER(sipf_params)], I64),
        "sipf_device_bytes": ([P], I64),
        "sipf_server_create": ([I64, ctypes.POINTER(P)], I32),
        "sipf_server_submit": ([P, ctypes.POINTER(sipf_grid), I64, ctypes.POINTER(sipf_params),
                                P, P, P, P, P, ctypes.c_double, I64, ctypes.POINTER(I64)], I32),
        "sipf_server_advance": ([P, I64, ctypes.POINTER(I32)], I32),
        "sipf_server_poll": ([P, P, I32, ctypes.POINTER(I32)], I32),
        "sipf_server_collect": ([P, I64, U32, P], I32),
        "sipf_server_stats": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32),
                               ctypes.POINTER(I32)], I32),
        "sipf_server_last_error": ([P], ctypes.c_char_p),
        "sipf_server_destroy": ([P], None),
        "sipf_server_set_limit": ([P, I32], I32),
        "sipf_server_fail_next_admission": ([P, I32], I32),
        "sipf_describe": ([P, ctypes.POINTER(sipf_grid), ctypes.POINTER(I64),
                           ctypes.POINTER(sipf_params), ctypes.POINTER(I64),
                           ctypes.POINTER(ctypes.c_double)], I32),
        "sipf_load": ([ctypes.c_char_p, P, ctypes.POINTER(P)], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(buf):
    """Address of a NumPy array, a CUDA tensor, or an int address."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if hasattr(buf, "is_contiguous") and not buf.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _check(code: int, ctx=None):
    if code != SIPF_OK:
        lib = load()
        msg = lib.sipf_strerror(code).decode()
        if ctx:
            extra = lib.sipf_last_error(ctx).decode()
            if extra:
                msg = f"{msg}: {extra}"
        raise SipfError(code, msg)


# ---------------------------------------------------------------- C names

def sipf_create(grid: sipf_grid, N: int, params: sipf_params, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().sipf_create(ctypes.byref(grid), int(N), ctypes.byref(params),
                              ctypes.c_void_p(stream or None), ctypes.byref(out)))
    return out.value


def sipf_set_state(ctx, x, mass, id_, v, m, w, where=SIPF_HOST):
    _check(load().sipf_set_state(ctx, _ptr(x), _ptr(mass), _ptr(id_), _ptr(v), _ptr(m), _ptr(w),
                                 where), ctx)


def sipf_step(ctx, dt: float, k: int = 1):
    _check(load().sipf_step(ctx, float(dt), int(k)), ctx)


def sipf_fields(ctx, mask: int, dst, where=SIPF_HOST):
    _check(load().sipf_fields(ctx, mask, _ptr(dst), where), ctx)


def sipf_particles(ctx, x=None, mass=None, id_=None, where=SIPF_HOST):
    _check(load().sipf_particles(ctx, _ptr(x), _ptr(mass), _ptr(id_), where), ctx)


def sipf_particle_state(ctx, s=None, loga=None, id_=None, where=SIPF_HOST):
    _check(load().sipf_particle_state(ctx, _ptr(s), _ptr(loga), _ptr(id_), where), ctx)


def sipf_cell_start(ctx, dst, where=SIPF_HOST):
    _check(load().sipf_cell_start(ctx, _ptr(dst), where), ctx)


def sipf_canonical_order(ctx, cell_start=None, ids=None, where=SIPF_HOST):
    _check(load().sipf_canonical_order(ctx, _ptr(cell_start), _ptr(ids), where), ctx)


def sipf_set_tuning(ctx, radix_plan=0, step_blocks_per_sm=0, bucket_slack_div=8,
                    bucket_slack_add=32):
    t = sipf_tuning(radix_plan, step_blocks_per_sm, bucket_slack_div, bucket_slack_add)
    _check(load().sipf_set_tuning(ctx, ctypes.byref(t)), ctx)


def sipf_get_tuning(ctx) -> dict:
    t = sipf_tuning()
    _check(load().sipf_get_tuning(ctx, ctypes.byref(t)), ctx)
    return {k: getattr(t, k) for k, _ in sipf_tuning._fields_}


def sipf_tuning_load(path):
    _check(load().sipf_tuning_load(None if path is None else str(path).encode()))


def sipf_tuning_lookup(H: int, N: int):
    """The table's tuning for (H, N) as a dict, or None."""
    t = sipf_tuning()
    found = load().sipf_tuning_lookup(int(H), int(N), ctypes.byref(t))
    if found < 0:
        _check(found)
    return {k: getattr(t, k) for k, _ in sipf_tuning._fields_} if found == 1 else None


def sipf_diagnostics(ctx) -> dict:
    d = sipf_diag()
    _check(load().sipf_diagnostics(ctx, ctypes.byref(d)), ctx)
    return {k: getattr(d, k) for k, _ in sipf_diag._fields_}


def sipf_sync(ctx):
    _check(load().sipf_sync(ctx), ctx)


def sipf_destroy(ctx):
    if ctx:
        load().sipf_destroy(ctx)


def sipf_save(ctx, path: str):
    _check(load().sipf_save(ctx, os.fsencode(path)), ctx)


def sipf_load(path: str, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().sipf_load(os.fsencode(path), ctypes.c_void_p(stream or None), ctypes.byref(out)))
    return out.value


def sipf_resample(ctx, ratio: float = 0.0) -> bool:
    """Residual resampling (Alg. 4) when max/min mass > ratio; True if done."""
    done = ctypes.c_int32(0)
    _check(load().sipf_resample(ctx, float(ratio), ctypes.byref(done)), ctx)
    return bool(done.value)


def _check_ens(code: int, ens):
    if code != SIPF_OK:
        lib = load()
        msg = lib.sipf_strerror(code).decode()
        extra = lib.sipf_ensemble_last_error(ens).decode() if ens else ""
        raise SipfError(code, f"{msg}: {extra}" if extra else msg)


def sipf_ensemble_create(grids, Ns, params) -> int:
    n = len(grids)
    ga = (sipf_grid * n)(*grids)
    na = (ctypes.c_int64 * n)(*[int(x) for x in Ns])
    pa = (sipf_params * n)(*params)
    out = ctypes.c_void_p()
    _check(load().sipf_ensemble_create(n, ga, na, pa, ctypes.byref(out)))
    return out.value


def sipf_ensemble_member(ens, i: int) -> int:
    c = load().sipf_ensemble_member(ens, int(i))
    if not c:
        raise IndexError(i)
    return c


def sipf_ensemble_step(ens, dts, k: int = 1):
    d = np.ascontiguousarray(dts, dtype=np.float64)
    _check_ens(load().sipf_ensemble_step(ens, d.ctypes.data, int(k)), ens)


def sipf_ensemble_sync(ens):
    _check_ens(load().sipf_ensemble_sync(ens), ens)


def sipf_ensemble_destroy(ens):
    if ens:
        load().sipf_ensemble_destroy(ens)


def sipf_describe(ctx) -> dict:
    g, n, p = sipf_grid(), ctypes.c_int64(), sipf_params()
    step, time = ctypes.c_int64(), ctypes.c_double()
    _check(load().sipf_describe(ctx, ctypes.byref(g), ctypes.byref(n), ctypes.byref(p),
                                ctypes.byref(step), ctypes.byref(time)), ctx)
    return {"H": g.H, "L": g.L, "origin": tuple(g.origin), "N": n.value,
            "params": {k: getattr(p, k) for k, _ in sipf_params._fields_},
            "step": step.value, "time": time.value}


def sipf_brownian_normals(ids_dev, N: int, n: int, seed: int, z_dev, bits_dev=None, stream=0):
    _check(load().sipf_brownian_normals(_ptr(ids_dev), int(N), int(n), int(seed), _ptr(z_dev),
                                        _ptr(bits_dev), ctypes.c_void_p(stream or None)))


def sipf_deposit_noalloc(grid: sipf_grid, x_dev, mass_dev, N: int, u_dev, stream=0):
    """Deposit u_bar of N particles into u_dev without allocating device memory
    (for callers that may not allocate; grids up to 64^3).  Asynchronous on
    `stream`; overlapping calls on one GPU share the library's scratch and race."""
    _check(load().sipf_deposit_noalloc(ctypes.byref(grid), _ptr(x_dev), _ptr(mass_dev), int(N),
                                       _ptr(u_dev), ctypes.c_void_p(stream or None)))


def sipf_profile(ctx, enable: bool):
    _check(load().sipf_profile(ctx, int(bool(enable))), ctx)


def sipf_profile_read(ctx) -> dict:
    """{group name: (total ms, launches)} over the recorded steps."""
    ms = np.zeros(PROFILE_GROUPS, dtype=np.float64)
    n = np.zeros(PROFILE_GROUPS, dtype=np.int64)
    _check(load().sipf_profile_read(ctx, ms.ctypes.data, n.ctypes.data, PROFILE_GROUPS), ctx)
    return {load().sipf_profile_name(k).decode(): (float(ms[k]), int(n[k]))
            for k in range(PROFILE_GROUPS)}


# ---------------------------------------------------------------- convenience

def make_grid(H: int, L: float, origin=(0.0, 0.0, 0.0)) -> sipf_grid:
    g = sipf_grid()
    g.H = H
    g.L = L
    for k in range(3):
        g.origin[k] = origin[k]
    return g


def make_params(p) -> sipf_params:
    """From any object with chi, Du, Dm, Dw, alpha, beta, gamma (and optional
    diffusion, v_update, H0, seed) attributes."""
    q = sipf_params()
    for name in ("chi", "Du", "Dm", "Dw", "alpha", "beta", "gamma"):
        setattr(q, name, float(getattr(p, name)))
    q.diffusion = int(getattr(p, "diffusion", 0))
    q.v_update = int(getattr(p, "v_update", 0))
    q.H0 = float(getattr(p, "H0", 0.0))
    q.seed = int(getattr(p, "seed", 0))
    q.p2g_order = int(getattr(p, "p2g_order", 2))
    q.sigma = float(getattr(p, "sigma", 0.0))
    return q


class Simulation:
    """Owns one context; host NumPy in and out (SoA conversions included)."""

    def __init__(self, H, L, origin, N, params, stream: int = 0, _ctx=None):
        self.H, self.L, self.N = H, L, N
        self.stream = stream
        self.ctx = _ctx if _ctx is not None else sipf_create(make_grid(H, L, origin), N,
                                                             make_params(params), stream)

    @classmethod
    def load(cls, path: str, stream: int = 0) -> "Simulation":
        """A simulation resumed from a checkpoint written by save()."""
        ctx = sipf_load(path, stream)
        d = sipf_describe(ctx)
        return cls(d["H"], d["L"], d["origin"], d["N"], None, _ctx=ctx)

    def save(self, path: str):
        sipf_save(self.ctx, path)

    def resample(self, ratio: float = 0.0) -> bool:
        return sipf_resample(self.ctx, ratio)

    def close(self):
        if self.ctx:
            sipf_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, x, mass, ids, v, m, w):
        xs = np.ascontiguousarray(np.asarray(x, dtype=np.float32).T)
        sipf_set_state(self.ctx, xs, np.ascontiguousarray(mass, dtype=np.float64),
                       None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32),
                       np.ascontiguousarray(v, dtype=np.float32),
                       np.ascontiguousarray(m, dtype=np.float32),
                       np.ascontiguousarray(w, dtype=np.float32), SIPF_HOST)

    def step(self, dt, k=1):
        sipf_step(self.ctx, dt, k)

    def fields(self, mask=127) -> dict:
        nsel = bin(mask).count("1")
        H3 = self.H ** 3
        buf = np.empty(nsel * H3, dtype=np.float32)
        sipf_fields(self.ctx, mask, buf, SIPF_HOST)
        out, off = {}, 0
        for b, name in enumerate(FIELD_NAMES):
            if mask & (1 << b):
                out[name] = buf[off * H3:(off + 1) * H3].reshape(self.H, self.H, self.H)
                off += 1
        return out

    def particles(self):
        """(x (N, 3) float32 physical, mass (N,) float64, id (N,) uint32), storage order."""
        x = np.empty(3 * self.N, dtype=np.float32)
        mass = np.empty(self.N, dtype=np.float64)
        ids = np.empty(self.N, dtype=np.uint32)
        sipf_particles(self.ctx, x, mass, ids, SIPF_HOST)
        return x.reshape(3, self.N).T.copy(), mass, ids

    def particle_state(self):
        """(s (N, 3) float32 grid units, loga (N,) float64, id (N,) uint32), storage order."""
        s = np.empty(3 * self.N, dtype=np.float32)
        loga = np.empty(self.N, dtype=np.float64)
        ids = np.empty(self.N, dtype=np.uint32)
        sipf_particle_state(self.ctx, s, loga, ids, SIPF_HOST)
        return s.reshape(3, self.N).T.copy(), loga, ids

    def cell_start(self):
        cs = np.empty(self.H ** 3 + 1, dtype=np.int32)
        sipf_cell_start(self.ctx, cs, SIPF_HOST)
        return cs

    def canonical_order(self):
        """(cell_start, ids in (cell key, id) order) of the current particles."""
        cs = np.empty(self.H ** 3 + 1, dtype=np.int32)
        ids = np.empty(self.N, dtype=np.uint32)
        sipf_canonical_order(self.ctx, cs, ids, SIPF_HOST)
        return cs, ids

    def diagnostics(self) -> dict:
        return sipf_diagnostics(self.ctx)


class Ensemble:
    """Independent runs advanced together (batched launches across members,
    or one stream per member); members are Simulation views (owned by the
    ensemble)."""

    def __init__(self, specs, mode: int = SIPF_ENSEMBLE_BATCHED):
        """specs: sequence of (H, L, origin, N, params)."""
        grids = [make_grid(H, L, origin) for H, L, origin, _, _ in specs]
        self.ens = sipf_ensemble_create(grids, [N for _, _, _, N, _ in specs],
                                        [make_params(p) for *_, p in specs])
        self.members = [Simulation(H, L, origin, N, None, _ctx=sipf_ensemble_member(self.ens, i))
                        for i, (H, L, origin, N, _) in enumerate(specs)]
        self.set_mode(mode)

    def set_mode(self, mode: int):
        _check_ens(load().sipf_ensemble_set_mode(self.ens, int(mode)), self.ens)

    def last_path(self) -> int:
        return int(load().sipf_ensemble_last_path(self.ens))

    def step(self, dts, k=1):
        sipf_ensemble_step(self.ens, dts, k)

    def sync(self):
        sipf_ensemble_sync(self.ens)

    def close(self):
        if self.ens:
            for m in self.members:
                m.ctx = None          # owned by the ensemble
            sipf_ensemble_destroy(self.ens)
            self.ens = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sipf_context_bytes(grid: sipf_grid, N: int, params: sipf_params) -> int:
    return int(load().sipf_context_bytes(ctypes.byref(grid), int(N), ctypes.byref(params)))


def _check_srv(code: int, srv):
    if code != SIPF_OK:
        lib = load()
        msg = lib.sipf_strerror(code).decode()
        extra = lib.sipf_server_last_error(srv).decode() if srv else ""
        raise SipfError(code, f"{msg}: {extra}" if extra else msg)


class Server:
    """Continuous-batching request scheduler (host calls of one thread)."""

    def __init__(self, budget_bytes: int, max_live: int = 0):
        out = ctypes.c_void_p()
        _check(load().sipf_server_create(int(budget_bytes), ctypes.byref(out)))
        self.srv = out.value
        self.H = {}
        if max_live:
            _check_srv(load().sipf_server_set_limit(self.srv, int(max_live)), self.srv)

    def fail_next_admission(self, code: int):
        """Fault injection for tests: the next admission fails with `code`."""
        _check_srv(load().sipf_server_fail_next_admission(self.srv, int(code)), self.srv)

    def submit(self, H, L, origin, N, params, x, mass, v, m, w, dt, steps) -> int:
        xs = np.ascontiguousarray(np.asarray(x, dtype=np.float32).T)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        v, m, w = (np.ascontiguousarray(a, dtype=np.float32) for a in (v, m, w))
        rid = ctypes.c_int64()
        _check_srv(load().sipf_server_submit(
            self.srv, ctypes.byref(make_grid(H, L, origin)), int(N),
            ctypes.byref(make_params(params)), xs.ctypes.data, mass.ctypes.data, v.ctypes.data,
            m.ctypes.data, w.ctypes.data, float(dt), int(steps), ctypes.byref(rid)), self.srv)
        self.H[rid.value] = H
        return rid.value

    def advance(self, quantum: int = 2) -> int:
        pending = ctypes.c_int32()
        _check_srv(load().sipf_server_advance(self.srv, int(quantum), ctypes.byref(pending)),
                   self.srv)
        return pending.value

    def poll(self, capacity: int = 256) -> list:
        ids = np.zeros(capacity, dtype=np.int64)
        n = ctypes.c_int32()
        _check_srv(load().sipf_server_poll(self.srv, ids.ctypes.data, capacity, ctypes.byref(n)),
                   self.srv)
        return [int(i) for i in ids[:n.value]]

    def collect(self, rid: int, mask: int = 127) -> dict:
        H = self.H.pop(rid)
        nsel = bin(mask).count("1")
        buf = np.empty(max(nsel, 1) * H ** 3, dtype=np.float32)
        _check_srv(load().sipf_server_collect(self.srv, int(rid), mask, buf.ctypes.data),
                   self.srv)
        out, off = {}, 0
        for b, name in enumerate(FIELD_NAMES):
            if mask & (1 << b):
                out[name] = buf[off * H ** 3:(off + 1) * H ** 3].reshape(H, H, H)
                off += 1
        return out

    def stats(self) -> dict:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        q, l = ctypes.c_int32(), ctypes.c_int32()
        _check(load().sipf_server_stats(self.srv, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(q), ctypes.byref(l)))
        return {"in_use": a.value, "peak": b.value, "queued": q.value, "live": l.value}

    def close(self):
        if self.srv:
            load().sipf_server_destroy(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
