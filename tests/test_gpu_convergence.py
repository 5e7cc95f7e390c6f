"""The paper's 3D convergence study (Sec. 5.2) on the GPU path: the ball
initial data on [0, 6]^3 with 2^22 particles, run to t = 1 at H = 16, 32,
64, 128 and 256 with the same particles and Brownian paths, and the cell
density of each H compared with H = 256 by the Fourier-truncated relative
error E of Sec. 5.1.  The paper's fitted slope of log2 E against log2 H
(-1.407) comes from tests/golden/paper_3d_study.json; the test requires the
errors to fall from H = 32 on and the fitted slope to lie within 0.3 of the
printed one (measured here: about -1.42)."""

import json
import os

import numpy as np
import pytest

from oracle import sipf_oracle as O
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


def test_spatial_convergence_slope_of_the_3d_study():
    Hs = [16, 32, 64, 128, 256]
    stream = torch.cuda.Stream()
    u = {}
    for H in Hs:
        wl = workload("paper3d", H=H, N=2 ** 22)
        with sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params,
                             stream=stream.cuda_stream) as sim:
            sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
            sim.step(wl.dt, 1000)
            u[H] = sim.fields(sipf.FIELD_U)["u"].astype(np.float64)
    E = [O.error_E(u[H], u[256], 16) for H in Hs[:-1]]
    slope = np.polyfit(np.log2(Hs[:-1]), np.log2(E), 1)[0]
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_3d_study.json")) as f:
        printed = json.load(f)["convergence_slope"]
    assert printed["H"] == Hs[:-1] and printed["reference_H"] == Hs[-1]
    print("E", E, "slope", slope, "printed", printed["value"])
    assert E[1] > E[2] > E[3]
    assert abs(slope - printed["value"]) <= 0.3
