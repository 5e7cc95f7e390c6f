"""FP64 CPU oracle of one SIPF-W time step -- TEST INFRASTRUCTURE ONLY.

This is a plain, slow, obviously-correct restatement of the SIPF-W scheme
(Hu, Wang, Xin, Zhang, "A Novel Stochastic Particle-Field Algorithm for a
Reaction-Diffusion-Advection Cancer Invasion Model", Alg. 3) for the 3D
u/v/m/w haptotaxis system.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path (``paper_2605_20140_gb300``) and never imports it.

Everything is float64 NumPy.  Library primitives used as steps: ``np.fft``
(3D DFT), ``np.bincount`` (scatter-add), ``np.lexsort`` (sort).

Notation (paper Sec. 2): periodic box of side L, H nodes per axis, h = L/H,
nodes at x_min + q h.  Particle positions are kept in grid units
s = (X - x_min)/h in [0, H), the coordinate in which the paper's assignment
function is written (p_j = h^-1 |x_j - q_j h|, Sec. 2.2.1).  Fields are
arrays f[z, y, x].

Readings of the paper taken here (where it is silent or inconsistent):

* Jacobi ordering: deposit, gather, push and field update all read the
  step-(n-1) state (Eq. u_hat_update uses grad v^(n-1), w^(n-1) at X^(n-1);
  Eq. k_q_update uses the source at n-1).
* Diffusion solve: the implicit Fourier multiplier
  1/(1 + tau R + tau D |2 pi q / L|^2) that the convergence analysis states
  the algorithm maintains (Sec. 4, m and w updates); the exponential
  multiplier exp(-tau D |k|^2 - tau R) of Eq. k_q_update is a switch.
* v update: the implicit pointwise form v/(1 + alpha tau m) of Sec. 2.3.3
  (explicit v(1 - alpha tau m) from the source S of Eq. g_t is a switch).
* Wave numbers q in {-H/2, ..., H/2-1}; the Nyquist component of each
  spectral derivative is set to zero (Eq. gradv on an even grid).
* Low-pass filter exp(-2 pi^2 |q|^2 / H0^2) (Alg. 3): off unless 0 < H0 < H;
  when on it multiplies the m and w spectra and the v spectrum used for
  grad v, never the stored v.
* Regularised m source (Eq. m_reg): with sigma > 0 the source of m is
  K_sigma * u_bar, K_sigma the density of N(0, sigma I_3) (sigma a variance,
  in units of L^2), applied spectrally; the w source keeps u_bar.  Off by
  default (sigma = 0), like the paper's experiments.
* Deposit: u_bar(qh) = sum_p a_p R_h(X_p, qh) (Alg. 1; the extra factor
  u_hat(X_p) printed in Eq. def_u_overline is read as a typo).  R_h is the
  trilinear function, or (p2g_order = 4) the fourth-order R_h^(4) of
  Sec. 2.2.1, whose printed cases leave nodes with two or more distances above
  1 at weight 0; the grid-to-particle interpolation stays trilinear
  (Theorem overall: fourth-order P2G, second-order G2P).
* Mass update a <- a (1 + tau rho(w_H) - tau) (Eq. u_hat_update) held as
  log a <- log a + log1p(tau (rho(w_H) - 1)).
* Brownian increments: W = sqrt(2 Du tau) z, z from Philox4x32-10 (Salmon et
  al., SC'11) with key (seed mod 2^32, seed >> 32) and counter
  (n, 0, id, 0) for step n >= 1 and particle id, then Box-Muller.  Uniforms
  u = (2 (b >> 9) + 1) 2^-24 (exact in float32).
* Periodic wrap s <- s - H floor(s/H); a result equal to H becomes 0.
* Canonical particle order: by cell key, ties by particle id.  The cell key
  orders cells tile-major in 8^3-cell tiles (tile index, then local cell).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

TILE = 8

# Philox-4x32 multipliers and Weyl key increments (Salmon, Moraes, Dror,
# Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------

def mulhilo32(a: int, b: np.ndarray):
    """High and low 32-bit words of the 64-bit product a*b (b uint32)."""
    p = np.uint64(a) * b.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & _MASK32).astype(np.uint32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds (SC'11): each round multiplies words 0 and 2
    by M0 and M1, mixes the high halves into words 1 and 3 with the key, and
    the key is advanced by the Weyl constants between rounds."""
    c = [np.asarray(x, dtype=np.uint32).copy() for x in (c0, c1, c2, c3)]
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    for r in range(10):
        if r > 0:
            k0 = np.uint32((int(k0) + PHILOX_W0) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + PHILOX_W1) & 0xFFFFFFFF)
        hi0, lo0 = mulhilo32(PHILOX_M0, c[0])
        hi1, lo1 = mulhilo32(PHILOX_M1, c[2])
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def uniforms_from_bits(b: np.ndarray) -> np.ndarray:
    """(2 (b >> 9) + 1) * 2^-24: odd multiples of 2^-24 in (0, 1)."""
    return (2.0 * (b >> np.uint32(9)).astype(np.float64) + 1.0) * 2.0 ** -24


def brownian_normals(ids: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Three standard normals per particle for step n (Box-Muller on the four
    Philox words of counter (n, 0, id, 0)); shape (N, 3)."""
    ids = np.asarray(ids, dtype=np.uint32)
    zero = np.zeros_like(ids)
    step = np.full_like(ids, np.uint32(n & 0xFFFFFFFF))
    b = philox4x32_10(step, zero, ids, zero, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = [uniforms_from_bits(x) for x in b]
    r01 = np.sqrt(-2.0 * np.log(u[0]))
    r23 = np.sqrt(-2.0 * np.log(u[2]))
    z0 = r01 * np.cos(2.0 * np.pi * u[1])
    z1 = r01 * np.sin(2.0 * np.pi * u[1])
    z2 = r23 * np.cos(2.0 * np.pi * u[3])
    return np.stack([z0, z1, z2], axis=1)


# --------------------------------------------------------------------------
# Cells, canonical order
# --------------------------------------------------------------------------

def cells(s: np.ndarray) -> np.ndarray:
    """Integer cell index floor(s) per axis (grid units), shape (N, 3)."""
    return np.floor(s).astype(np.int64)


def cell_keys(s: np.ndarray, H: int) -> np.ndarray:
    """Tile-major cell key: (tile index) * 512 + (local cell index), tiles of
    8^3 cells, both indices ordered z, then y, then x."""
    c = cells(s)
    T = H // TILE
    cx, cy, cz = c[:, 0], c[:, 1], c[:, 2]
    tile = ((cz // TILE) * T + (cy // TILE)) * T + (cx // TILE)
    local = ((cz % TILE) * TILE + (cy % TILE)) * TILE + (cx % TILE)
    return tile * TILE ** 3 + local


def canonical_order(keys: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """Permutation sorting particles by (cell key, id)."""
    return np.lexsort((np.asarray(ids, dtype=np.int64), keys))


def cell_start(keys: np.ndarray, H: int) -> np.ndarray:
    """Offsets of each cell's run in the canonical order (length H^3 + 1)."""
    counts = np.bincount(keys, minlength=H ** 3)
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


# --------------------------------------------------------------------------
# Particle-in-cell operators (Sec. 2.2.1-2.2.2)
# --------------------------------------------------------------------------

def _corner_terms(s: np.ndarray, H: int):
    """For each of the 8 corners (dx, dy, dz) of the particle's cell: the flat
    node index and the trilinear weight prod_j max(1 - |s_j - q_j|, 0)."""
    c = cells(s)
    f = s - c
    out = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                wx = f[:, 0] if dx else 1.0 - f[:, 0]
                wy = f[:, 1] if dy else 1.0 - f[:, 1]
                wz = f[:, 2] if dz else 1.0 - f[:, 2]
                ix = (c[:, 0] + dx) % H
                iy = (c[:, 1] + dy) % H
                iz = (c[:, 2] + dz) % H
                out.append(((iz * H + iy) * H + ix, wx * wy * wz))
    return out


def deposit(s: np.ndarray, a: np.ndarray, H: int, h: float) -> np.ndarray:
    """Alg. 1 with the trilinear assignment function R_h (h^-3 times the
    product of hat functions): u_bar(qh) = sum_p a_p R_h(X_p, qh)."""
    u = np.zeros(H ** 3)
    for idx, wgt in _corner_terms(s, H):
        u += np.bincount(idx, weights=a * wgt, minlength=H ** 3)
    return (u / h ** 3).reshape(H, H, H)


def r4_weight(p1, p2, p3):
    """h^3 R_h^(4) (Sec. 2.2.1, the fourth-order assignment function) as a
    function of the per-axis distances p_j = |x_j - q_j h| / h, case by case:
    all p_j <= 1: prod_j (1 - p_j) (1 + sum_j p_j (1 - p_j) / 2);
    one p_j in (1, 2], the others <= 1:
        -(1/6) prod_{k != j} (1 - p_k) (p_j - 1)(2 - p_j)(3 - p_j);
    otherwise 0."""
    p = [np.asarray(x, dtype=np.float64) for x in (p1, p2, p3)]
    near = [x <= 1.0 for x in p]
    mid = [(x > 1.0) & (x <= 2.0) for x in p]
    w = np.zeros(np.broadcast(*p).shape)
    core = near[0] & near[1] & near[2]
    w = np.where(core, (1 - p[0]) * (1 - p[1]) * (1 - p[2]) *
                 (1 + (p[0] * (1 - p[0]) + p[1] * (1 - p[1]) + p[2] * (1 - p[2])) / 2), w)
    for j in range(3):
        k, l = [i for i in range(3) if i != j]
        arm = mid[j] & near[k] & near[l]
        w = np.where(arm, -(1 - p[k]) * (1 - p[l]) * (p[j] - 1) * (2 - p[j]) * (3 - p[j]) / 6, w)
    return w


def deposit4(s: np.ndarray, a: np.ndarray, H: int, h: float) -> np.ndarray:
    """Alg. 1 with the fourth-order assignment function R_h^(4): every node
    q with offset d in {-1, 0, 1, 2}^3 from the particle's cell is tried and
    weighted by r4_weight of its distances (32 of the 64 are non-zero)."""
    c = cells(s)
    u = np.zeros(H ** 3)
    for dz in (-1, 0, 1, 2):
        for dy in (-1, 0, 1, 2):
            for dx in (-1, 0, 1, 2):
                q = c + np.array([dx, dy, dz])
                d = np.abs(s - q)
                wgt = r4_weight(d[:, 0], d[:, 1], d[:, 2])
                qq = q % H
                idx = (qq[:, 2] * H + qq[:, 1]) * H + qq[:, 0]
                u += np.bincount(idx, weights=a * wgt, minlength=H ** 3)
    return (u / h ** 3).reshape(H, H, H)


def deposit_order(s: np.ndarray, a: np.ndarray, H: int, h: float, order: int) -> np.ndarray:
    """u_bar with the trilinear (order 2) or the fourth-order assignment."""
    if order == 4:
        return deposit4(s, a, H, h)
    if order != 2:
        raise ValueError("p2g_order must be 2 or 4")
    return deposit(s, a, H, h)


def gather(f: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Alg. 2 with K_h = h^3 R_h: f_H(X_p) = sum_q K_h(X_p, qh) f(qh)."""
    H = f.shape[0]
    flat = f.reshape(-1)
    out = np.zeros(s.shape[0])
    for idx, wgt in _corner_terms(s, H):
        out += wgt * flat[idx]
    return out


# --------------------------------------------------------------------------
# Spectral operators (Eqs. vmw_hat, k_q_update, gradv)
# --------------------------------------------------------------------------

def wavenumbers(H: int) -> np.ndarray:
    """Integer mode indices q in DFT order: 0..H/2-1, -H/2..-1."""
    return np.fft.fftfreq(H, d=1.0 / H)


def _q_grids(H: int):
    q = wavenumbers(H)
    return q[:, None, None], q[None, :, None], q[None, None, :]   # qz, qy, qx


def low_pass(H: int, H0: float):
    """exp(-2 pi^2 |q|^2 / H0^2) (Alg. 3), or None when off."""
    if not (H0 > 0 and H0 < H):
        return None
    qz, qy, qx = _q_grids(H)
    return np.exp(-2.0 * math.pi ** 2 * (qx ** 2 + qy ** 2 + qz ** 2) / H0 ** 2)


def diffusion_multiplier(H: int, L: float, D: float, R: float, tau: float,
                         mode: int = 0) -> np.ndarray:
    """Per-mode factor of the linear diffusion/decay solve for one component.
    mode 0: 1/(1 + tau R + tau D |k|^2) (implicit, Sec. 4);
    mode 1: exp(-tau D |k|^2 - tau R) (Eq. k_q_update); k = 2 pi q / L."""
    qz, qy, qx = _q_grids(H)
    k2 = (2.0 * math.pi / L) ** 2 * (qx ** 2 + qy ** 2 + qz ** 2)
    if mode == 0:
        return 1.0 / (1.0 + tau * R + tau * D * k2)
    if mode == 1:
        return np.exp(-tau * D * k2 - tau * R)
    raise ValueError("unknown diffusion mode")


def spectral_gradient(v: np.ndarray, L: float, H0: float = 0.0) -> np.ndarray:
    """grad v on the nodes (Eq. gradv): inverse DFT of (2 pi i q / L) v_hat per
    axis, Nyquist component zeroed; returns (3, H, H, H) ordered x, y, z."""
    H = v.shape[0]
    V = np.fft.fftn(v)
    filt = low_pass(H, H0)
    if filt is not None:
        V = V * filt
    q = wavenumbers(H)
    qd = np.where(q == -H // 2, 0.0, q)
    ik = 2j * math.pi / L * qd
    gx = np.fft.ifftn(V * ik[None, None, :]).real
    gy = np.fft.ifftn(V * ik[None, :, None]).real
    gz = np.fft.ifftn(V * ik[:, None, None]).real
    return np.stack([gx, gy, gz])


def diffuse(f_star: np.ndarray, L: float, D: float, R: float, tau: float,
            mode: int = 0, H0: float = 0.0) -> np.ndarray:
    """D_tau of Eq. g_hat_phy in Fourier space: multiply the DFT of the
    reacted field by the per-mode factor (and the optional filter)."""
    H = f_star.shape[0]
    F = np.fft.fftn(f_star) * diffusion_multiplier(H, L, D, R, tau, mode)
    filt = low_pass(H, H0)
    if filt is not None:
        F = F * filt
    return np.fft.ifftn(F).real


# --------------------------------------------------------------------------
# Reaction (Eq. g_t, R_tau of Eq. g_hat_phy, implicit v of Sec. 2.3.3)
# --------------------------------------------------------------------------

def rho(w):
    """Proliferation rho(w) = 2w/(1+w) (Eq. haptotaxis-system)."""
    return 2.0 * w / (1.0 + w)


def eta(u):
    """Oxygen consumption eta(u) = 2u/(1+u) (Eq. haptotaxis-system)."""
    return 2.0 * u / (1.0 + u)


def gaussian_smooth(f: np.ndarray, L: float, sigma: float) -> np.ndarray:
    """K_sigma * f on the periodic grid, K_sigma the density of N(0, sigma I_3)
    (Eq. m_reg): the DFT of f times the characteristic function
    exp(-sigma |k|^2 / 2), k = 2 pi q / L."""
    if sigma <= 0.0:
        return np.asarray(f, dtype=np.float64).copy()
    H = f.shape[0]
    q = wavenumbers(H)
    k2 = (2 * np.pi / L) ** 2 * (q[:, None, None] ** 2 + q[None, :, None] ** 2 +
                                  q[None, None, :] ** 2)
    return np.fft.ifftn(np.fft.fftn(f) * np.exp(-0.5 * sigma * k2)).real


def react(v, m, w, ubar, p, tau, L=1.0):
    """R_tau: explicit Euler of S(u, g) = (-alpha m v; u; gamma v - eta(u) w),
    with v taken implicitly as v/(1 + alpha tau m) (or explicitly).  With
    p.sigma > 0 the m source is the regularised K_sigma * u (Eq. m_reg); the
    w source keeps u itself."""
    m_star = m + tau * gaussian_smooth(ubar, L, getattr(p, "sigma", 0.0))
    w_star = w + tau * (p.gamma * v - eta(ubar) * w)
    if p.v_update == 0:
        v_new = v / (1.0 + p.alpha * tau * m)
    else:
        v_new = v * (1.0 - p.alpha * tau * m)
    return v_new, m_star, w_star


# --------------------------------------------------------------------------
# State and the step (Alg. 3)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class State:
    H: int
    L: float
    origin: np.ndarray
    p: object                 # parameters (chi, Du, Dm, Dw, alpha, beta, gamma, ...)
    s: np.ndarray             # (N, 3) grid units, float64
    loga: np.ndarray          # (N,) log particle mass
    ids: np.ndarray           # (N,) uint32
    v: np.ndarray             # (H, H, H)
    m: np.ndarray
    w: np.ndarray
    grad_v: np.ndarray        # (3, H, H, H)
    n: int = 0                # steps taken
    t: float = 0.0

    @property
    def h(self) -> float:
        return self.L / self.H

    @property
    def mass(self) -> np.ndarray:
        return np.exp(self.loga)


def wrap(s: np.ndarray, H: int) -> np.ndarray:
    s = s - H * np.floor(s / H)
    s[s >= H] = 0.0
    return s


def make_state(H, L, origin, p, x, mass, ids, v, m, w) -> State:
    """Alg. 3 initialisation from given samples X^(0), masses a^(0) and node
    values of g(., 0); grad v^(0) from the DFT of v^(0)."""
    if H % TILE:
        raise ValueError("H must be a multiple of 8")
    origin = np.asarray(origin, dtype=np.float64)
    h = L / H
    s = wrap((np.asarray(x, dtype=np.float64) - origin) / h, H)
    with np.errstate(divide="ignore"):
        loga = np.log(np.asarray(mass, dtype=np.float64))
    v = np.asarray(v, dtype=np.float64)
    return State(H, L, origin, p, s, loga, np.asarray(ids, dtype=np.uint32).copy(),
                 v.copy(), np.asarray(m, dtype=np.float64).copy(),
                 np.asarray(w, dtype=np.float64).copy(),
                 spectral_gradient(v, L, p.H0))


def density(st: State) -> np.ndarray:
    """u_bar of the current particles (Alg. 1)."""
    return deposit_order(st.s, st.mass, st.H, st.h, getattr(st.p, "p2g_order", 2))


def step(st: State, tau: float, normals: np.ndarray | None = None) -> State:
    """One step n-1 -> n of Alg. 3.  ``normals`` overrides the Philox normals
    (shape (N, 3)) for tests that share Brownian paths between step sizes."""
    p, H, h, L = st.p, st.H, st.h, st.L
    n = st.n + 1
    a = st.mass
    # Alg. 1: u_bar^(n-1) on the nodes from (X^(n-1), a^(n-1)); the gather
    # stays trilinear for either assignment order (Theorem overall).
    ubar = deposit_order(st.s, a, H, h, getattr(p, "p2g_order", 2))
    # Alg. 2 / Eq. g2ph: grad v_H^(n-1) and w_H^(n-1) at X^(n-1).
    g = np.stack([gather(st.grad_v[d], st.s) for d in range(3)], axis=1)
    w_H = gather(st.w, st.s)
    # Eq. u_hat_update: Euler-Maruyama push and the mass factor.
    z = brownian_normals(st.ids, n, p.seed) if normals is None else normals
    s_new = st.s + (p.chi * tau / h) * g + (math.sqrt(2.0 * p.Du * tau) / h) * z
    s_new = wrap(s_new, H)
    loga_new = st.loga + np.log1p(tau * (rho(w_H) - 1.0))
    # Eq. g_hat_phy / k_q_update: reaction at n-1, then the diffusion solve.
    v_new, m_star, w_star = react(st.v, st.m, st.w, ubar, p, tau, L)
    m_new = diffuse(m_star, L, p.Dm, p.beta, tau, p.diffusion, p.H0)
    w_new = diffuse(w_star, L, p.Dw, 1.0, tau, p.diffusion, p.H0)
    grad_new = spectral_gradient(v_new, L, p.H0)
    return State(H, L, st.origin, p, s_new, loga_new, st.ids, v_new, m_new, w_new,
                 grad_new, n, st.t + tau)


def advance_particles(st: State, tau: float, idx: np.ndarray):
    """The particle part of one step (Eq. u_hat_update) for the particles
    with indices idx only: new grid-unit positions and log-masses, from the
    gather of grad v^(n-1) and w^(n-1) at X^(n-1) and the step-n noise."""
    p, H, h = st.p, st.H, st.h
    s = st.s[idx]
    g = np.stack([gather(st.grad_v[d], s) for d in range(3)], axis=1)
    w_H = gather(st.w, s)
    z = brownian_normals(st.ids[idx], st.n + 1, p.seed)
    s_new = wrap(s + (p.chi * tau / h) * g + (math.sqrt(2.0 * p.Du * tau) / h) * z, H)
    return s_new, st.loga[idx] + np.log1p(tau * (rho(w_H) - 1.0))


def run(st: State, tau: float, k: int) -> State:
    for _ in range(k):
        st = step(st, tau)
    return st


def diagnostics(st: State) -> dict:
    """FP64 totals and minima (Lemma mass, Corollary mass, positivity lemma)."""
    u = density(st)
    a = st.mass
    fields = (u, st.v, st.m, st.w)
    return {
        "mass_particles": float(np.sum(a)),
        "mass_grid": float(np.sum(u) * st.h ** 3),
        "min_u": float(u.min()), "min_v": float(st.v.min()),
        "min_m": float(st.m.min()), "min_w": float(st.w.min()),
        "nonfinite": int(sum(np.count_nonzero(~np.isfinite(f)) for f in fields)
                         + np.count_nonzero(~np.isfinite(st.s))),
        "step": st.n, "time": st.t,
    }


# --------------------------------------------------------------------------
# Error metric of the convergence study (Sec. 5.1)
# --------------------------------------------------------------------------

def fourier_truncate(f: np.ndarray, K: int) -> np.ndarray:
    """Down-sample a periodic H^3 node field to K^3 nodes by keeping the DFT
    modes q in {-K/2, ..., K/2-1} per axis (K even, K <= H)."""
    H = f.shape[0]
    F = np.fft.fftn(f)
    keep = np.concatenate([np.arange(K // 2), np.arange(H - K // 2, H)])
    G = F[np.ix_(keep, keep, keep)]
    return np.fft.ifftn(G).real * (K / H) ** 3


def error_E(u1: np.ndarray, u2: np.ndarray, K: int = 16) -> float:
    """Relative L2 difference ||u1 - u2|| / max(||u1||, ||u2||) of two fields
    after Fourier truncation to K^3 nodes (the metric E of Sec. 5.1)."""
    a = fourier_truncate(u1, K)
    b = fourier_truncate(u2, K)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(a), np.linalg.norm(b)))
