"""The input recipe of the paper's 3D study (Sec. 5.2) against the values the
paper prints for it (tests/golden/paper_3d_study.json): domain, initial data
of u, m, v, w, parameters, time step and step count."""

import json
import math
import os

import numpy as np
import pytest

from sipf_inputs import node_coordinates, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_3d_study.json")


@pytest.fixture(scope="module")
def printed():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def wl():
    return workload("paper3d", H=32, N=1 << 16)


def test_domain_parameters_and_time(printed, wl):
    assert wl.L == printed["domain"]["L"]
    assert tuple(wl.origin) == tuple(printed["domain"]["origin"])
    for k, v in printed["parameters"].items():
        if k != "cite":
            assert getattr(wl.params, k) == v, k
    assert wl.dt == printed["time"]["tau"]
    assert wl.steps == printed["time"]["steps"]
    assert wl.steps * wl.dt == pytest.approx(printed["time"]["T"], rel=1e-12)
    assert workload("paper3d", H=16).N == printed["particles"]["P"]


def test_initial_u_particles_fill_the_ball_with_its_mass(printed, wl):
    iu = printed["initial_u"]
    c = np.asarray(iu["centre"])
    r2 = np.sum((wl.x.astype(np.float64) - c) ** 2, axis=1)
    # float32 rounding of the stored positions, at |x| <= 6
    assert r2.max() <= iu["radius_squared"] * (1 + 1e-6)
    # u0 = height on the ball: total mass height * (4/3) pi r0^3, equal weights
    M0 = iu["height"] * 4.0 / 3.0 * math.pi * iu["radius_squared"] ** 1.5
    assert wl.mass.sum() == pytest.approx(M0, rel=1e-12)
    assert np.all(wl.mass == wl.mass[0])
    # the radial law of a uniform ball: P(r <= s r0) = s^3
    s3 = (r2 / iu["radius_squared"]) ** 1.5
    assert abs(np.mean(s3 <= 0.5) - 0.5) < 4 * math.sqrt(0.25 / wl.N)


def test_initial_fields_on_the_nodes(printed, wl):
    X, Y, Z = node_coordinates(wl.H, wl.L, wl.origin)
    iu = printed["initial_u"]
    c = iu["centre"]
    ball = ((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) <= iu["radius_squared"]
    assert printed["initial_m_equals_initial_u"]
    np.testing.assert_array_equal(wl.m, np.where(ball, iu["height"], 0.0).astype(np.float32))
    iv = printed["initial_v"]
    fn = {"cos": np.cos, "sin": np.sin}
    ph = iv["phase_over_pi"]
    f = [fn[name] for name in iv["factors"]]
    v = (iv["amplitude"] * f[0](np.pi * ph["x1_squared"] * X ** 2)
         * f[1](np.pi * ph["x2_squared"] * Y ** 2) * f[2](np.pi * ph["x3_squared"] * Z ** 2)
         + iv["offset"])
    np.testing.assert_allclose(wl.v, v, rtol=0, atol=1e-7)
    np.testing.assert_allclose(wl.w, printed["initial_w_over_v"]["value"] * v, rtol=0, atol=4e-7)
