"""The paper's own numerical examples, run on the GPU and checked against the oracle.

The paper prints no numbers (its figures carry no data), so these runs check that the
GPU reproduces the oracle at the paper's stated parameters (tests/golden/paper_parameters.json),
at the paper's snapshot steps, together with the diagnostics its figures show: the phase-space
density, its line-outs, the negative weights and the entropy.

- Sec. IV.A linear oscillator: exact rotation by pi/10 per step, one revolution in 20 steps.
- Sec. IV.A nonlinear oscillator: H = p^2/2 + cos x (the paper's sign), step 2 pi / 20,
  snapshots after 10, 20, 30 and 80 steps, a distribution on the unstable point.
- Sec. IV.B FEL: flat-top energy distribution |p| < 0.1, snapshots after 50, 100, 150 steps.
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

HERE = os.path.dirname(os.path.abspath(__file__))
PAPER = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
FP64_TOL = 1e-12
FP32_TOL = 1e-5


def oracle_floor(k, grid):
    """Relative difference the oracle's own rounding allows after k steps: it pushes absolute
    FP64 coordinates, so each step moves a node by up to ulp(max |x|) / h_x cells of rounding
    (the GPU's integer + fraction displacements are finer); three times that per step."""
    hx = (grid.x1 - grid.x0) / grid.nx
    return 3.0 * k * np.spacing(max(abs(grid.x0), abs(grid.x1))) / hx


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def rel_linf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def snapshots(wl, steps, precision=I.FP64, projection=I.PROJ_GALERKIN):
    """GPU and oracle side by side; at each snapshot the weights and both sides' moments."""
    f0 = I.make_f0(wl)
    if precision == I.FP32:
        f0 = f0.astype(np.float32)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=precision, projection=projection)
    sim.set_f(f0)
    st = O.State(wl.grid, wl.pusher, wl.basis, projection, f0.astype(np.float64))
    out, done = [], 0
    for k in steps:
        sim.step(k - done)
        st.run(k - done)
        done = k
        mo = st.moments()
        mo["a_re"], mo["a_im"] = float(st.fel[0]), float(st.fel[1])
        out.append((k, sim.get_f(), st.w.copy(), sim.moments(), mo))
    sim.close()
    return out


@pytest.mark.parametrize("basis", [I.BASIS_TENT, I.BASIS_CUBIC])
def test_linear_oscillator_one_revolution(basis):
    """20 steps of pi/10: the push returns every node home; the projected density moves with it."""
    n = PAPER["oscillator_steps_per_revolution"]["value"]
    om = 1.0
    h = PAPER["oscillator_phase_advance_per_step"]["float"] / om
    g = I.Grid(128, 128, -4.0, 4.0, -4.0, 4.0)
    pu = I.Pusher(I.PUSH_ROTATION, I.POT_HARMONIC, 1.0, om, h)
    wl = I.Workload("t", g, pu, basis, I.FP64, n, "gaussian", dict(xc=1.5, pc=0.0, sx=0.4, sp=0.4))
    res = snapshots(wl, [5, 10, n])
    for k, got, want, mg, mo in res:
        assert rel_linf(got, want) <= FP64_TOL, k
        for q in ("mass", "mean_x", "mean_p", "var_x", "var_p", "entropy"):
            assert abs(mg[q] - mo[q]) <= 1e-10 * max(1.0, abs(mo[q])), (k, q)
    # after one revolution the centre of mass is back where it started
    k, got, want, mg, mo = res[-1]
    assert abs(mg["mean_x"] - 1.5) < 1e-3 and abs(mg["mean_p"]) < 1e-3


@pytest.mark.parametrize("basis", [I.BASIS_TENT, I.BASIS_CUBIC])
def test_pendulum_paper_sign_and_step_snapshots(basis):
    """H = p^2/2 + cos x, h = 2 pi / 20; a distribution on the unstable point (x = pi)."""
    g = I.Grid(128, 128, -math.pi, math.pi, -3.0, 3.0)
    h = PAPER["pendulum_step"]["float"]
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, PAPER["pendulum_hamiltonian"]["v_sign"], 1.0, h)
    wl = I.Workload("t", g, pu, basis, I.FP64, 80, "gaussian", dict(xc=math.pi, pc=0.0, sx=1.2, sp=1.0))
    for k, got, want, mg, mo in snapshots(wl, PAPER["pendulum_snapshots"]["value"]):
        tol = max(FP64_TOL, oracle_floor(k, g))
        assert rel_linf(got, want) <= tol, k
        # line-outs of the figures: the density along p through the X-point and along x at p = 0
        assert rel_linf(got[:, 0], want[:, 0]) <= tol and rel_linf(got[64], want[64]) <= tol
        assert abs(mg["entropy"] - mo["entropy"]) <= 1e-10 * abs(mo["entropy"]), k
        assert abs(mg["neg_mass"] - mo["neg_mass"]) <= 1e-10 * abs(mo["neg_mass"]) + 1e-15, k
        if basis == I.BASIS_TENT:
            assert mg["neg_mass"] == 0.0      # the tent deposit never makes a negative weight
    if basis == I.BASIS_CUBIC:
        assert mg["neg_mass"] < -1e-6          # the Galerkin (tent-basis) update does


def test_pendulum_paper_sign_fp32_fused():
    g = I.Grid(1024, 640, -math.pi, math.pi, -3.0, 3.0)
    h = PAPER["pendulum_step"]["float"]
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, PAPER["pendulum_hamiltonian"]["v_sign"], 1.0, h)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP32, 30, "gaussian",
                    dict(xc=math.pi, pc=0.0, sx=1.2, sp=1.0))
    for k, got, want, mg, mo in snapshots(wl, [10, 20, 30], precision=I.FP32):
        assert np.abs(got - want).sum() / np.abs(want).sum() <= FP32_TOL, k


def test_fel_flattop_snapshots():
    """Sec. IV.B: a flat top in energy, |p| < 0.1; negative weights appear at its hard edges."""
    hw = PAPER["fel_flattop_half_width"]["value"]
    g = I.Grid(64, 128, 0.0, 2 * math.pi, -0.5, 0.5)
    pu = I.Pusher(I.PUSH_FEL, I.POT_FREE, 1.0, 1.0, 0.05, 1e-2, 0.0)
    wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 150, "fel_flattop", dict(half_width=hw, eps=1e-2))
    a0 = pu.a0_re
    for k, got, want, mg, mo in snapshots(wl, PAPER["fel_snapshots"]["value"]):
        # the instability amplifies rounding-level differences as it amplifies the field itself
        growth = max(1.0, math.hypot(mo["a_re"], mo["a_im"]) / a0)
        assert rel_linf(got, want) <= FP64_TOL * growth, (k, growth)
        assert abs(mg["neg_mass"] - mo["neg_mass"]) <= 1e-10 * abs(mo["neg_mass"]), k
        assert mg["neg_mass"] < 0.0
        amp = math.hypot(mo["a_re"], mo["a_im"])
        assert math.hypot(mg["a_re"] - mo["a_re"], mg["a_im"] - mo["a_im"]) <= FP64_TOL * amp, k
