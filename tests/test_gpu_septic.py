"""Cubic B-spline basis functions on the GPU (the smoother basis of Sec. V's remark).

The deposit kernel is the septic B-spline B7 (8 taps per axis, Cox-de Boor weights on the GPU,
truncated powers in the oracle); the Galerkin mass matrix has 7 bands (a cyclic 3-pole
recursion along x and an LDL^T of the principal block along p on the GPU; a circulant DFT
solve and banded elimination in the oracle). The oracle is pinned to the dense integral
definitions (tests/test_oracle_pins.py).
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

FP64_TOL = 1e-12
FP32_TOL = 1e-5
PAPER = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "paper_parameters.json")))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def workload(kind, nx, np_, precision):
    if kind == "pendulum":
        g = I.Grid(nx, np_, -math.pi, math.pi, -3.0, 3.0)
        pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.1)
        return I.Workload("t", g, pu, I.BASIS_SEPTIC, precision, 0, "gaussian",
                          dict(xc=0.0, pc=0.8, sx=0.5, sp=0.5))
    if kind == "rotation":
        g = I.Grid(nx, np_, -5.0, 5.0, -5.0, 5.0)
        pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, 1.0, 0.2)
        return I.Workload("t", g, pu, I.BASIS_SEPTIC, precision, 0, "gaussian",
                          dict(xc=1.0, pc=0.0, sx=0.6, sp=0.6))
    g = I.Grid(nx, np_, 0.0, 2 * math.pi, -1.5, 1.5)
    k = I.PUSH_FEL if kind == "fel" else I.PUSH_FEL_RK4
    pu = I.Pusher(k, I.POT_FREE, 1.0, 1.0, 0.05, 0.05, 0.0, 0.2, 0.1)
    return I.Workload("t", g, pu, I.BASIS_SEPTIC, precision, 0, "fel_gaussian", dict(sp=0.1, eps=1e-2))


def run_pair(wl, steps, projection=I.PROJ_GALERKIN):
    f0 = I.make_f0(wl)
    if wl.precision == I.FP32:
        f0 = f0.astype(np.float32)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=wl.precision, projection=projection)
    sim.set_f(f0)
    sim.step(steps)
    got, hist, plan, mom = sim.get_f(), sim.field_history(), sim.plan(), sim.moments()
    sim.close()
    st = O.State(wl.grid, wl.pusher, wl.basis, projection, f0.astype(np.float64))
    ohist = st.run(steps, history=True)
    return got, hist, st, ohist, plan, mom


@pytest.mark.parametrize("kind", ["pendulum", "rotation", "fel", "fel_rk4"])
@pytest.mark.parametrize("proj", [I.PROJ_GALERKIN, I.PROJ_LUMPED])
def test_septic_fp64_matches_oracle(kind, proj):
    wl = workload(kind, 64, 48, I.FP64)
    got, hist, st, ohist, plan, mom = run_pair(wl, 12, proj)
    assert plan["kernel"] == V.VP_KERNEL_SCATTER
    assert np.max(np.abs(got - st.w)) <= FP64_TOL * np.max(np.abs(st.w))
    if kind.startswith("fel"):
        amp = np.max(np.hypot(ohist[:, 0], ohist[:, 1]))
        assert np.max(np.abs(hist - ohist)) <= FP64_TOL * amp
    om = st.moments()
    assert abs(mom["mass"] - om["mass"]) <= 1e-12 * abs(om["mass"])


def test_septic_fp32_matches_oracle():
    wl = workload("pendulum", 256, 128, I.FP32)
    got, _, st, _, _, _ = run_pair(wl, 10)
    assert np.abs(got - st.w).sum() / np.abs(st.w).sum() <= FP32_TOL


def test_smoother_basis_negative_weights_on_gpu():
    """The GPU reproduces the measured answer to Sec. V's remark: under the Galerkin projection
    the cubic B-spline basis leaves more negative weight in the flat-top FEL than the tent basis."""
    hw = PAPER["fel_flattop_half_width"]["value"]
    g = I.Grid(64, 128, 0.0, 2 * math.pi, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.05, 1e-2, 0.0)
    neg = {}
    for basis in (I.BASIS_CUBIC, I.BASIS_SEPTIC):
        wl = I.Workload("t", g, pu, basis, I.FP64, 0, "fel_flattop", dict(half_width=hw, eps=1e-2))
        sim = V.Sim(g, basis, pu, precision=V.VP_FP64)
        sim.set_f(I.make_f0(wl))
        sim.step(5)
        neg[basis] = sim.moments()["neg_mass"]
        sim.close()
    assert neg[I.BASIS_SEPTIC] < 1.2 * neg[I.BASIS_CUBIC] < 0.0


def test_septic_fused_requests_are_refused():
    wl = workload("pendulum", 64, 48, I.FP32)
    with pytest.raises(V.VlasovError) as ei:
        V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, kernel=V.VP_KERNEL_FUSED)
    assert ei.value.status == V.VP_ERR_UNSUPPORTED
