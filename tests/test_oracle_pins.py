"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  None compares the oracle with itself: each
checks a closed form, an invariant stated in the paper, a brute-force
evaluation of the paper's formula, or an independent library.
"""

import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

from oracle import sipf_oracle as O
from sipf_inputs import Params, workload


def _state(H=16, L=1.0, N=64, p=None, x=None, mass=None, v=None, m=None, w=None, seed=0):
    rng = np.random.default_rng(seed)
    p = p or Params()
    if x is None:
        x = (rng.random((N, 3)) * L).astype(np.float32)
    N = x.shape[0]
    if mass is None:
        mass = np.full(N, 1.0 / N)
    shape = (H, H, H)
    v = np.ones(shape) if v is None else v
    m = np.zeros(shape) if m is None else m
    w = np.full(shape, 0.5) if w is None else w
    return O.make_state(H, L, (0.0, 0.0, 0.0), p, x, mass, np.arange(N, dtype=np.uint32), v, m, w)


def _grid(H, L=1.0):
    q = np.arange(H) * (L / H)
    return np.meshgrid(q, q, q, indexing="ij")   # Z, Y, X


# ---------------------------------------------------------------- Philox

def _load_curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host-side Philox4_32_10 generator (a CPU library routine)
    emits block j = Philox((j >> 16, 0, j & 0xffff, 0), key=seed); the
    oracle's Philox must reproduce those words exactly, which fixes the
    multipliers, the key schedule, the round count and the word order."""
    lib = _load_curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    seed = 0x0123456789ABCDEF
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    nblk = 3 * 65536 + 1000
    buf = np.zeros(4 * nblk, np.uint32)
    assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size)) == 0
    lib.curandDestroyGenerator(gen)
    j = np.arange(nblk, dtype=np.uint32)
    zero = np.zeros_like(j)
    b = O.philox4x32_10(j >> np.uint32(16), zero, j & np.uint32(0xFFFF), zero,
                        seed & 0xFFFFFFFF, seed >> 32)
    np.testing.assert_array_equal(np.stack(b, axis=1), buf.reshape(-1, 4))


def test_mulhilo_against_python_integers():
    rng = np.random.default_rng(1)
    b = rng.integers(0, 2 ** 32, size=1000, dtype=np.uint64).astype(np.uint32)
    for a in (O.PHILOX_M0, O.PHILOX_M1, 0xFFFFFFFF):
        hi, lo = O.mulhilo32(a, b)
        for bi, h, l in zip(b[:200], hi[:200], lo[:200]):
            prod = a * int(bi)
            assert int(h) == prod >> 32 and int(l) == prod & 0xFFFFFFFF


def test_uniforms_are_exact_float32_in_open_interval():
    b = np.array([0, 1, 511, 512, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = O.uniforms_from_bits(b)
    assert np.all(u > 0) and np.all(u < 1)
    np.testing.assert_array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 2.0 ** -24 and u[4] == 1.0 - 2.0 ** -24


def test_brownian_normals_moments_and_independence():
    N = 1 << 18
    z = O.brownian_normals(np.arange(N, dtype=np.uint32), 7, 42)
    se = 1.0 / math.sqrt(N)
    assert np.all(np.abs(z.mean(axis=0)) < 5 * se)
    assert np.all(np.abs(z.var(axis=0) - 1.0) < 5 * math.sqrt(2.0) * se)
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5 * se)
    # kurtosis of a normal is 3
    k = (z ** 4).mean(axis=0)
    assert np.all(np.abs(k - 3.0) < 0.05)
    # different steps are uncorrelated
    z2 = O.brownian_normals(np.arange(N, dtype=np.uint32), 8, 42)
    assert abs(np.mean(z[:, 0] * z2[:, 0])) < 5 * se


# ---------------------------------------------------------------- FFT / spectral

def _naive_dft3(f):
    H = f.shape[0]
    k = np.arange(H)
    E = np.exp(-2j * np.pi * np.outer(k, k) / H)
    out = np.zeros((H, H, H), dtype=complex)
    for kz in range(H):
        for ky in range(H):
            for kx in range(H):
                out[kz, ky, kx] = np.sum(f * E[kz][:, None, None] * E[ky][None, :, None]
                                         * E[kx][None, None, :])
    return out


@pytest.mark.parametrize("H", [8, 12])
def test_fft_convention_against_naive_dft(H):
    """The oracle uses np.fft for the DFT of Eq. vmw_hat; check its sign,
    ordering and scaling against the DFT written as an explicit sum."""
    rng = np.random.default_rng(H)
    f = rng.standard_normal((H, H, H))
    ref = _naive_dft3(f)
    np.testing.assert_allclose(np.fft.fftn(f), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    q = O.wavenumbers(H)
    assert list(q[: H // 2]) == list(range(H // 2)) and q[H // 2] == -H // 2


@pytest.mark.parametrize("L", [1.0, 6.0])
def test_spectral_gradient_of_a_sine_mode(L):
    """grad sin(2 pi q.x / L) = (2 pi q / L) cos(2 pi q.x / L) exactly for
    |q_j| < H/2 (Eq. gradv)."""
    H = 16
    Z, Y, X = _grid(H, L)
    q = np.array([3, -5, 2])   # x, y, z
    ph = 2 * np.pi * (q[0] * X + q[1] * Y + q[2] * Z) / L
    g = O.spectral_gradient(np.sin(ph), L)
    for d in range(3):
        np.testing.assert_allclose(g[d], 2 * np.pi * q[d] / L * np.cos(ph), atol=1e-11)


def test_spectral_gradient_zeroes_the_nyquist_mode():
    H = 16
    Z, Y, X = _grid(H)
    nyq = np.cos(np.pi * np.round(X * H))          # (-1)^ix
    g = O.spectral_gradient(nyq + np.sin(2 * np.pi * Y), 1.0)
    np.testing.assert_allclose(g[0], 0.0, atol=1e-11)
    np.testing.assert_allclose(g[1], 2 * np.pi * np.cos(2 * np.pi * Y), atol=1e-11)


@pytest.mark.parametrize("mode", [0, 1])
def test_single_fourier_mode_decay_in_a_step(mode):
    """With massless particles (no source), gamma = 0 and alpha = 0, one
    step multiplies a Fourier mode of m by 1/(1 + tau beta + tau Dm |k|^2)
    (implicit, Sec. 4) or exp(-tau Dm |k|^2 - tau beta) (Eq. k_q_update);
    w likewise with R = 1 and Dw."""
    H, L, tau = 16, 2.0, 0.01
    p = Params(chi=0.0, Du=0.0, Dm=0.03, Dw=0.07, alpha=0.0, beta=0.4, gamma=0.0,
               diffusion=mode)
    Z, Y, X = _grid(H, L)
    q = np.array([2, 1, -3])
    mode_f = np.cos(2 * np.pi * (q[0] * X + q[1] * Y + q[2] * Z) / L)
    st = _state(H, L, N=8, p=p, mass=np.zeros(8), m=1.5 * mode_f, w=0.25 * mode_f,
                v=np.ones((H, H, H)))
    k2 = (2 * np.pi / L) ** 2 * np.sum(q ** 2)
    if mode == 0:
        fm, fw = 1 / (1 + tau * p.beta + tau * p.Dm * k2), 1 / (1 + tau + tau * p.Dw * k2)
    else:
        fm, fw = math.exp(-tau * p.Dm * k2 - tau * p.beta), math.exp(-tau * p.Dw * k2 - tau)
    st1 = O.run(st, tau, 3)
    np.testing.assert_allclose(st1.m, 1.5 * mode_f * fm ** 3, atol=1e-13)
    np.testing.assert_allclose(st1.w, 0.25 * mode_f * fw ** 3, atol=1e-13)
    np.testing.assert_array_equal(st1.v, st.v)


def test_low_pass_filter_factor():
    """Alg. 3 filter exp(-2 pi^2 |q|^2 / H0^2) on a single mode of m."""
    H, L, tau, H0 = 16, 1.0, 0.01, 6.0
    p = Params(chi=0.0, Du=0.0, Dm=0.0, Dw=0.0, alpha=0.0, beta=0.0, gamma=0.0, H0=H0)
    Z, Y, X = _grid(H, L)
    q = np.array([1, 2, 0])
    f = np.cos(2 * np.pi * (q[0] * X + q[1] * Y))
    st = _state(H, L, N=4, p=p, mass=np.zeros(4), m=f, w=np.zeros((H, H, H)))
    st1 = O.step(st, tau)
    np.testing.assert_allclose(st1.m, f * math.exp(-2 * np.pi ** 2 * 5 / H0 ** 2), atol=1e-13)
    # the stored v is never filtered
    np.testing.assert_array_equal(st1.v, st.v)


# ---------------------------------------------------------------- PIC operators

def _hat_R(x, node, h, L):
    """R_h of Sec. 2.2.1 evaluated literally: h^-3 prod_j max(1 - |x_j - q_j h|/h, 0)
    with the periodic minimum-image distance."""
    d = x - node
    d = d - L * np.round(d / L)
    return h ** -3 * np.prod(np.maximum(1.0 - np.abs(d) / h, 0.0))


def test_deposit_against_bruteforce_assignment_function():
    H, L, N = 8, 1.5, 40
    rng = np.random.default_rng(3)
    x = (rng.random((N, 3)) * L).astype(np.float32)
    x[0] = [0.0, 0.0, 0.0]                      # on a node
    x[1] = np.float32(L) - np.float32(1e-6)     # next to the seam
    a = rng.random(N) + 0.1
    st = _state(H, L, x=x, mass=a)
    u = O.density(st)
    h = L / H
    ref = np.zeros((H, H, H))
    xs = np.asarray(x, dtype=np.float64)
    for iz in range(H):
        for iy in range(H):
            for ix in range(H):
                node = np.array([ix, iy, iz]) * h
                ref[iz, iy, ix] = sum(a[p] * _hat_R(xs[p], node, h, L) for p in range(N))
    np.testing.assert_allclose(u, ref, rtol=1e-12, atol=1e-12 * ref.max())


def test_deposit_partition_of_unity_and_sign():
    st = _state(32, 1.0, N=5000, seed=5)
    u = O.density(st)
    assert abs(u.sum() * st.h ** 3 - st.mass.sum()) < 1e-13 * st.mass.sum()
    assert u.min() >= 0.0


def test_particle_on_a_node_deposits_a_delta():
    H, L = 16, 1.0
    h = L / H
    x = np.array([[3 * h, 5 * h, 7 * h]], dtype=np.float32)
    st = _state(H, L, x=x, mass=np.array([0.3]))
    u = O.density(st)
    ref = np.zeros((H, H, H))
    ref[7, 5, 3] = 0.3 / h ** 3
    np.testing.assert_allclose(u, ref, atol=1e-12)


def test_gather_against_bruteforce_kernel():
    H, L, N = 8, 1.0, 30
    rng = np.random.default_rng(4)
    x = (rng.random((N, 3)) * L).astype(np.float32)
    f = rng.standard_normal((H, H, H))
    st = _state(H, L, x=x)
    got = O.gather(f, st.s)
    h = L / H
    ref = np.zeros(N)
    xs = np.asarray(x, dtype=np.float64)
    for p in range(N):
        for iz in range(H):
            for iy in range(H):
                for ix in range(H):
                    node = np.array([ix, iy, iz]) * h
                    ref[p] += h ** 3 * _hat_R(xs[p], node, h, L) * f[iz, iy, ix]
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_gather_reproduces_affine_fields_away_from_the_seam():
    H = 16
    rng = np.random.default_rng(6)
    s = 1.0 + (H - 3.0) * rng.random((500, 3))
    Z, Y, X = np.meshgrid(np.arange(H), np.arange(H), np.arange(H), indexing="ij")
    f = 0.3 + 1.1 * X - 0.7 * Y + 0.25 * Z
    np.testing.assert_allclose(O.gather(f, s), 0.3 + 1.1 * s[:, 0] - 0.7 * s[:, 1] + 0.25 * s[:, 2],
                               atol=1e-12)
    np.testing.assert_allclose(O.gather(np.full((H, H, H), 2.5), s), 2.5, atol=1e-14)


# ---------------------------------------------------------------- reaction terms

def test_m_source_from_a_particle_on_a_node():
    """m* = m + tau u_bar (Eq. g_t): with Dm = beta = 0 the multiplier is 1."""
    H, L, tau = 16, 1.0, 0.01
    h = L / H
    p = Params(chi=0.0, Du=0.0, Dm=0.0, Dw=0.0, alpha=0.0, beta=0.0, gamma=0.0)
    x = np.array([[2 * h, 9 * h, 4 * h]], dtype=np.float32)
    st = _state(H, L, x=x, mass=np.array([0.2]), p=p, m=np.full((H, H, H), 0.1))
    st1 = O.step(st, tau)
    ref = np.full((H, H, H), 0.1)
    ref[4, 9, 2] += tau * 0.2 / h ** 3
    np.testing.assert_allclose(st1.m, ref, atol=1e-12)


def test_w_source_closed_form_without_diffusion():
    """w^1 = (w + tau(gamma v - eta(u_bar) w)) / (1 + tau) when Dw = 0."""
    H, L, tau = 8, 1.0, 0.02
    p = Params(chi=0.0, Du=0.0, Dm=0.0, Dw=0.0, alpha=0.0, beta=0.0, gamma=3.0)
    rng = np.random.default_rng(7)
    v = 0.5 + rng.random((H, H, H))
    w = 0.2 + rng.random((H, H, H))
    st = _state(H, L, N=50, p=p, v=v, w=w, seed=7)
    u = O.density(st)
    st1 = O.step(st, tau)
    ref = (w + tau * (3.0 * v - 2 * u / (1 + u) * w)) / (1 + tau)
    np.testing.assert_allclose(st1.w, ref, atol=1e-12)


@pytest.mark.parametrize("v_update", [0, 1])
def test_v_update_closed_form(v_update):
    """Uniform m that stays fixed (beta = 0, no source): v^n = v0/(1+alpha tau m)^n
    (implicit, Sec. 2.3.3) or v0 (1 - alpha tau m)^n (explicit)."""
    H, tau, n = 8, 0.01, 5
    p = Params(chi=0.0, Du=0.0, Dm=0.0, beta=0.0, alpha=4.0, v_update=v_update)
    rng = np.random.default_rng(8)
    v0 = 0.5 + rng.random((H, H, H))
    st = _state(H, N=4, p=p, v=v0, m=np.full((H, H, H), 0.7), mass=np.zeros(4))
    stn = O.run(st, tau, n)
    fac = 1 / (1 + 4.0 * tau * 0.7) if v_update == 0 else 1 - 4.0 * tau * 0.7
    np.testing.assert_allclose(stn.v, v0 * fac ** n, rtol=1e-13)


def test_total_mass_ode_under_constant_oxygen():
    """Constant w = w0 (gamma v0 = w0, alpha = 0, negligible u): every particle
    sees rho(w0), so M_n = M_0 (1 + tau (rho(w0) - 1))^n (Eq. u_hat_update)."""
    H, tau, n, w0 = 16, 0.01, 20, 0.8
    p = Params(chi=0.3, Du=1e-3, Dm=1e-3, Dw=1e-2, alpha=0.0, beta=0.1, gamma=w0 / 0.5)
    M0 = 1e-22
    st = _state(H, N=300, p=p, v=np.full((H, H, H), 0.5), w=np.full((H, H, H), w0),
                mass=np.full(300, M0 / 300), seed=9)
    stn = O.run(st, tau, n)
    rho0 = 2 * w0 / (1 + w0)
    np.testing.assert_allclose(stn.mass.sum(), M0 * (1 + tau * (rho0 - 1)) ** n, rtol=1e-12)
    np.testing.assert_allclose(stn.w, w0, rtol=1e-12)


# ---------------------------------------------------------------- dynamics

def test_brownian_variance_with_zero_chemotaxis():
    """chi = 0: per-axis displacement variance 2 Du t (Eq. SDE), mean 0."""
    H, L, tau, n, Du = 32, 1.0, 1e-3, 20, 1e-3
    N = 1 << 16
    p = Params(chi=0.0, Du=Du, alpha=0.0, seed=11)
    x = np.full((N, 3), 0.5, dtype=np.float32)
    st = _state(H, L, x=x, p=p, mass=np.full(N, 1.0 / N))
    stn = O.run(st, tau, n)
    d = (stn.s - st.s) * (L / H)
    var = 2 * Du * tau * n
    assert np.all(np.abs(d.mean(axis=0)) < 4 * math.sqrt(var / N))
    assert np.all(np.abs(d.var(axis=0) - var) < 4 * math.sqrt(2.0 / N) * var)


def test_mass_lemma_and_corollary_on_the_small_workload():
    """(1-tau) a <= a' <= (1+tau) a per particle (Lemma mass) and
    M0 e^-t <= M <= M0 e^t (Corollary mass), plus positivity."""
    from sipf_inputs import workload
    wl = workload("small", N=4096, H=16)
    st = O.make_state(wl.H, wl.L, wl.origin, wl.params, wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    M0 = st.mass.sum()
    tau = wl.dt
    for _ in range(5):
        a_prev = st.mass
        st = O.step(st, tau)
        a = st.mass
        assert np.all(a >= (1 - tau) * a_prev * (1 - 1e-15))
        assert np.all(a <= (1 + tau) * a_prev * (1 + 1e-15))
    M = st.mass.sum()
    assert M0 * math.exp(-st.t) <= M <= M0 * math.exp(st.t)
    d = O.diagnostics(st)
    assert d["min_u"] >= 0 and d["min_v"] > 0 and np.all(st.mass > 0)
    # m and w: the truncated implicit multiplier is not a positive kernel
    # (its off-centre entries reach about -tau D / (2 h^2) per axis), so the
    # paper's positivity lemma holds for them only up to that undershoot.
    h2 = (wl.L / wl.H) ** 2
    for name, D in (("m", wl.params.Dm), ("w", wl.params.Dw)):
        f = getattr(st, name)
        assert d["min_" + name] >= -3 * st.n * tau * D / h2 * np.abs(f).max()
    assert d["nonfinite"] == 0


# ---------------------------------------------------------------- binning

def test_cell_keys_tile_major_bijection_and_order():
    H = 16
    c = np.stack(np.meshgrid(np.arange(H), np.arange(H), np.arange(H), indexing="ij"), -1)
    cz, cy, cx = c[..., 0].ravel(), c[..., 1].ravel(), c[..., 2].ravel()
    s = np.stack([cx, cy, cz], 1) + 0.5
    k = O.cell_keys(s, H)
    assert sorted(k.tolist()) == list(range(H ** 3))
    # brute force of the definition for a few cells
    for (x, y, z) in [(0, 0, 0), (7, 0, 0), (8, 0, 0), (0, 8, 0), (15, 15, 15), (9, 3, 12)]:
        tile = ((z // 8) * 2 + y // 8) * 2 + x // 8
        local = ((z % 8) * 8 + y % 8) * 8 + x % 8
        assert O.cell_keys(np.array([[x + 0.25, y + 0.25, z + 0.25]]), H)[0] == tile * 512 + local


def test_canonical_order_and_cell_start():
    H = 16
    rng = np.random.default_rng(12)
    s = rng.random((3000, 3)) * H
    s[:500] = np.floor(s[:500])                  # exactly on nodes
    ids = rng.permutation(3000).astype(np.uint32)
    k = O.cell_keys(s, H)
    order = O.canonical_order(k, ids)
    ks, is_ = k[order], ids[order].astype(np.int64)
    assert np.all((ks[1:] > ks[:-1]) | ((ks[1:] == ks[:-1]) & (is_[1:] > is_[:-1])))
    cs = O.cell_start(k, H)
    assert cs[0] == 0 and cs[-1] == 3000 and np.all(np.diff(cs) >= 0)
    for c in rng.integers(0, H ** 3, 50):
        assert np.all(ks[cs[c]:cs[c + 1]] == c)


def test_wrap_edge_cases():
    H = 8
    s = np.array([[-1e-300, 8.0, 3.5], [-8.0, 15.99, 16.0], [-0.5, 0.0, 7.999999]])
    r = O.wrap(s.copy(), H)
    assert np.all(r >= 0) and np.all(r < H)
    np.testing.assert_allclose(r[1], [0.0, 7.99, 0.0], atol=1e-12)
    assert r[2, 0] == 7.5


def test_advance_particles_is_the_particle_part_of_a_step():
    """The per-sample particle update equals the particles of a full step."""
    from sipf_inputs import workload
    wl = workload("small", N=2000, H=16)
    st = O.make_state(wl.H, wl.L, wl.origin, wl.params, wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    idx = np.array([0, 5, 17, 999, 1999])
    s_new, l_new = O.advance_particles(st, wl.dt, idx)
    st1 = O.step(st, wl.dt)
    np.testing.assert_array_equal(s_new, st1.s[idx])
    np.testing.assert_array_equal(l_new, st1.loga[idx])


# ---------------------------------------------------------------- fourth-order assignment R^(4)

def _single_particle_weights(x, H=16):
    """Node weights h^3 R^(4)(x, q) of one unit-mass particle at x (grid units)
    on an H^3 grid with h = 1, as an (H, H, H) array."""
    return O.deposit4(np.asarray([x], dtype=np.float64), np.ones(1), H, 1.0)


def test_r4_worked_values_at_a_cell_centre():
    # p = (1/2, 1/2, 1/2) at the 8 corners: (1/8)(1 + 3/8) = 0.171875;
    # at a star node p = (3/2, 1/2, 1/2): -(1/6)(1/4)(1/2)(1/2)(3/2) = -0.015625
    u = _single_particle_weights([7.5, 7.5, 7.5])
    assert u[7, 7, 7] == 0.171875 and u[8, 8, 8] == 0.171875
    assert u[7, 7, 6] == -0.015625 and u[8, 7, 9] == -0.015625
    assert u[6, 6, 7] == 0.0                      # two distances above 1
    assert np.count_nonzero(u) == 32


@pytest.mark.parametrize("seed", [0, 1])
def test_r4_reproduces_polynomials_up_to_degree_three(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        x = rng.uniform(6.0, 9.0, 3)
        u = _single_particle_weights(x)
        idx = np.nonzero(u)
        w = u[idx]
        dz, dy, dx = (np.asarray(i, dtype=np.float64) - x[k] for i, k in zip(idx, (2, 1, 0)))
        assert np.count_nonzero(u) == 32
        for a in range(5):
            for b in range(5 - a):
                for c in range(5 - a - b):
                    m = np.sum(w * dx ** a * dy ** b * dz ** c)
                    want = 1.0 if a + b + c == 0 else 0.0
                    if a + b + c <= 3:
                        assert abs(m - want) <= 1e-12, (a, b, c, m)
        # not an accident of degree 4: the fourth x-moment is non-zero
        assert abs(np.sum(w * dx ** 4)) > 1e-3


def test_r4_on_a_node_plane_is_cubic_lagrange_interpolation():
    nodes = np.array([-1.0, 0.0, 1.0, 2.0])
    for f in (0.1, 0.25, 0.5, 0.8):
        u = _single_particle_weights([7.0 + f, 7.0, 7.0])
        for i, xi in enumerate(nodes):
            others = np.delete(nodes, i)
            ell = np.prod((f - others) / (xi - others))
            assert abs(u[7, 7, 7 + int(xi)] - ell) <= 1e-14
        assert np.count_nonzero(np.abs(u) > 1e-15) == 4


def test_r4_deposit_conserves_mass():
    rng = np.random.default_rng(4)
    H = 16
    s = rng.uniform(0, H, (500, 3))
    a = rng.uniform(0.5, 2.0, 500)
    u = O.deposit4(s, a, H, 0.25)
    assert abs(u.sum() * 0.25 ** 3 - a.sum()) <= 1e-12 * a.sum()


# ---------------------------------------------------------------- K_sigma-regularised m source

def test_gaussian_smoothing_of_a_plane_wave_and_the_mean():
    H, L, sigma = 16, 2.0, 0.003
    q = np.arange(H) * (L / H)
    Z, Y, X = np.meshgrid(q, q, q, indexing="ij")
    qv = np.array([2, -3, 1])
    f = 0.7 + np.cos(2 * np.pi * (qv[0] * X + qv[1] * Y + qv[2] * Z) / L)
    g = O.gaussian_smooth(f, L, sigma)
    k2 = (2 * np.pi / L) ** 2 * np.sum(qv ** 2)
    want = 0.7 + np.exp(-0.5 * sigma * k2) * (f - 0.7)
    assert np.max(np.abs(g - want)) <= 1e-13
    np.testing.assert_array_equal(O.gaussian_smooth(f, L, 0.0), f)


def test_gaussian_smoothing_equals_the_periodised_kernel_in_real_space():
    """Brute force: u_s(x_i) = sum_j h^3 G(x_i - x_j) u(x_j) with G the density of
    N(0, sigma I_3) summed over periodic images; sigma = 4 h^2 keeps the
    aliasing of the sampled kernel below e^-19."""
    H, L = 8, 1.0
    h = L / H
    sigma = 4 * h * h
    rng = np.random.default_rng(0)
    u = rng.random((H, H, H))
    idx = np.arange(H)
    d1 = (idx[:, None] - idx[None, :]) * h                      # x_i - x_j per axis
    img = np.arange(-3, 4) * L
    g1 = np.exp(-((d1[:, :, None] + img) ** 2) / (2 * sigma)).sum(axis=2)
    g1 /= np.sqrt(2 * np.pi * sigma)                             # 1D factor of the density
    # separable 3D kernel h^3 G = prod_axes (h g1)
    K = h * g1
    want = np.einsum("ia,jb,kc,abc->ijk", K, K, K, u)
    got = O.gaussian_smooth(u, L, sigma)
    assert np.max(np.abs(got - want)) <= 1e-9 * np.abs(want).max()
    assert abs(got.mean() - u.mean()) <= 1e-14


def test_gather_error_is_second_order_on_smooth_fields():
    """Trilinear interpolation of a smooth periodic field at random points:
    the error falls as h^2 (ratio about 4 per halving of h)."""
    rng = np.random.default_rng(7)
    pts = rng.random((4000, 3))                      # physical positions in [0, 1)^3

    def f(x, y, z):
        return np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y) + 0.5 * np.sin(4 * np.pi * z)

    errs = []
    for H in (16, 32, 64):
        q = np.arange(H) / H
        Z, Y, X = np.meshgrid(q, q, q, indexing="ij")
        g = O.gather(f(X, Y, Z), pts * H)
        errs.append(np.max(np.abs(g - f(pts[:, 0], pts[:, 1], pts[:, 2]))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_positivity_on_the_small_workload():
    """The deposit is non-negative exactly (trilinear weights), v stays
    positive under the implicit update and w under its source (tau <= 1/2);
    m is positive up to the negative off-centre entries of the truncated
    implicit multiplier, bounded by 3 n tau Dm / h^2 of its maximum after n
    steps (measured -1.3e-5 after 20 steps, against the bound 6.1e-5)."""
    wl = workload("small", H=32, N=1 << 15)
    st = O.make_state(wl.H, wl.L, wl.origin, wl.params, wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    h = wl.L / wl.H
    for n in range(1, 21):
        st = O.step(st, wl.dt)
        assert O.density(st).min() >= 0.0
        assert st.v.min() > 0.0
        assert st.w.min() > 0.0
        assert st.m.min() >= -3 * n * wl.dt * wl.params.Dm / h ** 2 * np.abs(st.m).max()
