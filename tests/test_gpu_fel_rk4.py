"""The RK4 FEL integrator (Sec. IV.B's) on the GPU, against the oracle.

Each step reduces the bunching of all particles at each RK4 stage and deposits every node at
its RK4 end point (scatter kernel). The oracle's RK4 is pinned to fourth order and to the
dispersion relation (tests/test_oracle_pins.py); here the GPU matches it to 1e-12 (FP64) and
shows the same fourth-order drift of the <p> + |A|^2 invariant.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

FP64_TOL = 1e-12
FP32_TOL = 1e-5
FP32_FIELD_TOL = 5e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def fel(nth, np_, precision, delta=0.0, sigma2=0.0, dt=0.05, a0=0.05, sp=0.1, pr=(-1.5, 1.5),
        basis=I.BASIS_CUBIC):
    return I.Workload("t", I.Grid(nth, np_, 0.0, 2 * math.pi, *pr),
                      I.Pusher(I.PUSH_FEL_RK4, I.POT_FREE, 1.0, 1.0, dt, a0, 0.0, delta, sigma2), basis,
                      precision, 0, "fel_gaussian", dict(sp=sp, eps=1e-2))


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


@pytest.mark.parametrize("delta,sigma2", [(0.0, 0.0), (0.3, 0.2), (-0.5, 0.4)])
@pytest.mark.parametrize("basis,proj", [(I.BASIS_CUBIC, I.PROJ_GALERKIN), (I.BASIS_CUBIC, I.PROJ_LUMPED),
                                        (I.BASIS_TENT, I.PROJ_GALERKIN)], ids=["galerkin", "lumped", "tent"])
def test_rk4_fp64_matches_oracle(delta, sigma2, basis, proj):
    wl = fel(64, 96, I.FP64, delta, sigma2, basis=basis)
    got, hist, st, ohist, plan, _ = run_pair(wl, 25, projection=proj)
    assert plan["kernel"] == V.VP_KERNEL_SCATTER
    assert np.max(np.abs(got - st.w)) <= FP64_TOL * np.max(np.abs(st.w))
    amp = np.max(np.hypot(ohist[:, 0], ohist[:, 1]))
    assert np.max(np.abs(hist - ohist)) <= FP64_TOL * amp


def test_rk4_fp32_matches_oracle():
    wl = fel(512, 256, I.FP32, 0.2, 0.1, dt=0.02)
    got, hist, st, ohist, _, _ = run_pair(wl, 20)
    assert np.abs(got - st.w).sum() / np.abs(st.w).sum() <= FP32_TOL
    amp = np.hypot(ohist[:, 0], ohist[:, 1])
    assert np.max(np.abs(np.hypot(hist[:, 0], hist[:, 1]) - amp) / amp) <= FP32_FIELD_TOL


def test_rk4_on_gpu_is_fourth_order():
    """Drift of <p> + |A|^2 over tau = 1 falls ~16x per halving of dt (no edge loss)."""
    drift = []
    for dt in (0.2, 0.1, 0.05):
        g = I.Grid(64, 256, 0.0, 2 * math.pi, -2.5, 2.5)
        pu = I.Pusher(I.PUSH_FEL_RK4, I.POT_FREE, 1.0, 1.0, dt, 0.3, 0.0)
        wl = I.Workload("t", g, pu, I.BASIS_CUBIC, I.FP64, 0, "fel_gaussian", dict(sp=0.1, eps=1e-2))
        sim = V.Sim(g, wl.basis, pu, precision=V.VP_FP64)
        sim.set_f(I.make_f0(wl))
        e0 = sim.moments()["energy"]
        sim.step(int(round(1.0 / dt)))
        drift.append(abs(sim.moments()["energy"] - e0))
        sim.close()
    for a, b in zip(drift, drift[1:]):
        assert 12.0 < a / b < 20.0


def test_rk4_requests_for_the_fused_kernel_are_refused():
    wl = fel(64, 96, I.FP32)
    with pytest.raises(V.VlasovError) as ei:
        V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, kernel=V.VP_KERNEL_FUSED)
    assert ei.value.status == V.VP_ERR_UNSUPPORTED
