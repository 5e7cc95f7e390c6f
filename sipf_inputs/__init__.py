"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module only *generates* initial data (particle positions, masses, ids
and the v, m, w node fields) and names the workloads.  It contains none of
the SIPF-W step arithmetic: deposit, gather, push, mass update, reaction and
the spectral solve live in ``oracle/`` (CPU reference) and in the CUDA
kernels, which never share code.

Workloads (all periodic boxes, fields sampled on nodes x_min + q h):

* ``small``   -- unit cube, H=32, N=2**15, one Gaussian cloud (sigma 0.05)
                 about (0.5, 0.5, 0.5), total mass 1; v0 = 1 - 0.5 g,
                 m0 = 0.5 g, w0 = 0.5 with g = exp(-|x-c|^2/0.01) (periodic
                 minimum-image distance); chi=0.01, Du=1e-3, Dm=1e-3,
                 Dw=1e-2, alpha=10, beta=0.1, gamma=0.5, dt=1e-3, 100 steps.
* ``headline`` -- unit cube, H=128, N=2**22, three Gaussian seeds
                 (sigma 0.04) at centres drawn U[0.2, 0.8]^3, equal particle
                 masses (1/N each, total 1); v0 = prod_s (1 - 0.5 g_s),
                 m0 = 0.5 sum_s g_s, w0 = 0.5; same parameters, dt=5e-4,
                 1000 steps.
* ``large``    -- as ``headline`` at H=256, N=2**25, chi=0.02, dt=2.5e-4,
                 500 steps.
* ``paper3d``  -- the 3D experiment of the paper's Section 5.2: box [0,6]^3,
                 u0 = 3 on the ball |x-(3,3,3)| <= sqrt(0.3), m0 = u0 on nodes,
                 v0 = 0.05 cos(5 pi x1^2/18) sin(13 pi x2^2/72)
                 cos(pi x3^2/12) + 0.3, w0 = 4 v0, chi=0.4,
                 Du=Dm=Dw=0.01, alpha=5, beta=0.01, gamma=5, dt=1e-3.

Positions are returned as float32 physical coordinates in [x_min, x_min+L)
with shape (N, 3) (columns x, y, z); fields as float32 arrays of shape
(H, H, H) indexed [z, y, x] (x fastest in memory).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Params",
    "Workload",
    "ensemble_workloads",
    "gaussian_mixture_positions",
    "node_coordinates",
    "periodic_sq_distance",
    "workload",
    "uniform_positions",
]


@dataclasses.dataclass
class Params:
    """Model parameters of the u/v/m/w haptotaxis system (all >= 0)."""

    chi: float = 0.01
    Du: float = 1e-3
    Dm: float = 1e-3
    Dw: float = 1e-2
    alpha: float = 10.0
    beta: float = 0.1
    gamma: float = 0.5
    diffusion: int = 0      # 0 implicit multiplier, 1 exponential multiplier
    v_update: int = 0       # 0 implicit v/(1+alpha tau m), 1 explicit v(1-alpha tau m)
    H0: float = 0.0         # low-pass filter cut-off; 0 (or >= H) means off
    seed: int = 0           # Philox key for the Brownian increments
    p2g_order: int = 2      # particle-to-grid assignment: 2 trilinear, 4 the star stencil R^(4)
    sigma: float = 0.0      # variance of the Gaussian K_sigma regularising the m source; 0 = off


@dataclasses.dataclass
class Workload:
    name: str
    H: int
    L: float
    origin: tuple
    N: int
    dt: float
    steps: int
    params: Params
    x: np.ndarray           # (N, 3) float32 physical positions
    mass: np.ndarray        # (N,) float64 particle masses
    ids: np.ndarray         # (N,) uint32 persistent particle ids
    v: np.ndarray           # (H, H, H) float32
    m: np.ndarray
    w: np.ndarray


def node_coordinates(H: int, L: float, origin) -> tuple:
    """Physical coordinates (X, Y, Z) of the H^3 nodes, each shaped (H, H, H)
    and indexed [z, y, x]."""
    h = L / H
    q = np.arange(H, dtype=np.float64) * h
    z, y, x = np.meshgrid(q + origin[2], q + origin[1], q + origin[0], indexing="ij")
    return x, y, z


def periodic_sq_distance(x, y, z, c, L: float):
    """Squared minimum-image distance from (x, y, z) to the point c."""
    out = 0.0
    for comp, cc in zip((x, y, z), c):
        d = comp - cc
        d = d - L * np.round(d / L)
        out = out + d * d
    return out


def _wrap_f32(x: np.ndarray, L: float, origin) -> np.ndarray:
    """Wrap float64 positions into the box and round them to float32, keeping
    every coordinate strictly below origin + L after the rounding."""
    o = np.asarray(origin, dtype=np.float64)
    y = o + np.mod(x - o, L)
    y32 = y.astype(np.float32)
    hi = (o + L).astype(np.float32)
    bad = y32 >= hi
    if np.any(bad):
        y32[bad] = np.broadcast_to(o.astype(np.float32), y32.shape)[bad]
    return y32


def gaussian_mixture_positions(N: int, centres, sigma: float, L: float, origin,
                               rng: np.random.Generator) -> np.ndarray:
    """N i.i.d. samples of an equal-weight Gaussian mixture, wrapped into the
    periodic box, as float32 (N, 3)."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    comp = rng.integers(0, centres.shape[0], size=N)
    x = centres[comp] + sigma * rng.standard_normal((N, 3))
    return _wrap_f32(x, L, origin)


def uniform_positions(N: int, L: float, origin, rng: np.random.Generator) -> np.ndarray:
    o = np.asarray(origin, dtype=np.float64)
    return _wrap_f32(o + L * rng.random((N, 3)), L, origin)


def _gaussian_seed_fields(H, L, origin, centres):
    X, Y, Z = node_coordinates(H, L, origin)
    g = [np.exp(-periodic_sq_distance(X, Y, Z, c, L) / 0.01) for c in centres]
    v = np.ones((H, H, H))
    for gs in g:
        v = v * (1.0 - 0.5 * gs)
    m = 0.5 * sum(g)
    w = np.full((H, H, H), 0.5)
    return v.astype(np.float32), m.astype(np.float32), w.astype(np.float32)


def workload(name: str, seed: int = 0, H: int | None = None, N: int | None = None) -> Workload:
    """Build a named workload; ``H`` and ``N`` override the grid size and the
    particle count (the initial-data recipe is unchanged)."""
    rng = np.random.default_rng(np.random.PCG64(1000 + seed))
    if name == "small":
        H = H or 32
        N = N or 2 ** 15
        L, origin = 1.0, (0.0, 0.0, 0.0)
        centres = [(0.5, 0.5, 0.5)]
        x = gaussian_mixture_positions(N, centres, 0.05, L, origin, rng)
        v, m, w = _gaussian_seed_fields(H, L, origin, centres)
        p = Params(seed=seed)
        dt, steps = 1e-3, 100
    elif name in ("headline", "large"):
        H = H or (128 if name == "headline" else 256)
        N = N or (2 ** 22 if name == "headline" else 2 ** 25)
        L, origin = 1.0, (0.0, 0.0, 0.0)
        centres = 0.2 + 0.6 * rng.random((3, 3))
        x = gaussian_mixture_positions(N, centres, 0.04, L, origin, rng)
        v, m, w = _gaussian_seed_fields(H, L, origin, centres)
        if name == "headline":
            p = Params(seed=seed)
            dt, steps = 5e-4, 1000
        else:
            p = Params(chi=0.02, seed=seed)
            dt, steps = 2.5e-4, 500
    elif name == "paper3d":
        H = H or 64
        N = N or 2 ** 22
        L, origin = 6.0, (0.0, 0.0, 0.0)
        r0 = math.sqrt(0.3)
        # uniform samples in the ball by rejection from the bounding cube
        pts = []
        need = N
        while need > 0:
            cand = rng.uniform(-r0, r0, size=(2 * need + 16, 3))
            cand = cand[np.sum(cand * cand, axis=1) <= 0.3]
            pts.append(cand[:need])
            need -= min(need, cand.shape[0])
        x = _wrap_f32(np.concatenate(pts) + 3.0, L, origin)
        X, Y, Z = node_coordinates(H, L, origin)
        ball = (((X - 3.0) ** 2 + (Y - 3.0) ** 2 + (Z - 3.0) ** 2) <= 0.3).astype(np.float64)
        m = (3.0 * ball).astype(np.float32)
        v64 = (0.05 * np.cos(5 * np.pi * X ** 2 / 18) * np.sin(13 * np.pi * Y ** 2 / 72)
               * np.cos(np.pi * Z ** 2 / 12) + 0.3)
        v = v64.astype(np.float32)
        w = (4.0 * v64).astype(np.float32)
        p = Params(chi=0.4, Du=0.01, Dm=0.01, Dw=0.01, alpha=5.0, beta=0.01, gamma=5.0,
                   seed=seed)
        dt, steps = 1e-3, 6000
        M0 = 3.0 * 4.0 / 3.0 * math.pi * 0.3 ** 1.5
        mass = np.full(N, M0 / N)
        return Workload(name, H, L, origin, N, dt, steps, p, x, mass,
                        np.arange(N, dtype=np.uint32), v, m, w)
    else:
        raise ValueError(f"unknown workload {name!r}")
    mass = np.full(N, 1.0 / N)
    return Workload(name, H, L, origin, N, dt, steps, p, x, mass,
                    np.arange(N, dtype=np.uint32), v, m, w)


def ensemble_workloads(count: int = 64, seed: int = 0, max_log2_N: int = 20,
                       sizes=(32, 48, 64, 96)) -> list:
    """Uneven ensemble of independent runs: grid side H uniform over ``sizes``,
    particle count N = round(2^U[14, max_log2_N]), chi ~ U[0.005, 0.03],
    alpha ~ U[5, 20], Du ~ U[5e-4, 2e-3], one Philox key per run, 200 steps of
    dt 1e-3; initial data as in ``small`` (one Gaussian cloud of sigma 0.05 at
    the box centre, equal masses of total 1)."""
    rng = np.random.default_rng(np.random.PCG64(7000 + seed))
    runs = []
    for r in range(count):
        H = int(rng.choice(sizes))
        N = int(round(2.0 ** rng.uniform(14.0, max_log2_N)))
        chi = float(rng.uniform(0.005, 0.03))
        alpha = float(rng.uniform(5.0, 20.0))
        Du = float(rng.uniform(5e-4, 2e-3))
        wl = workload("small", seed=1000 * seed + r, H=H, N=N)
        wl.name = f"ensemble[{r}]"
        wl.params = dataclasses.replace(wl.params, chi=chi, alpha=alpha, Du=Du,
                                        seed=(seed << 32) | r)
        wl.steps = 200
        runs.append(wl)
    return runs
