"""FP32 accuracy over whole runs: 2000 steps against the FP64 oracle.

The per-step parity tests bound the error of a few steps; these bound what
accumulates over the full step counts of the 8192 x 8192 pendulum and of the
FEL run to tau = 20, on meshes the oracle finishes in about half a minute.

- Pendulum (two-Gaussian initial state, leapfrog dt = 0.02, cubic Galerkin):
  rounding noise adds up like a random walk, so 2000 steps stay within the FP32
  bound of 1e-5 relative L1 only if no step carries a systematic bias (a mean
  excess of the tap weights, or a DC gain of the Lambda solves other than one,
  of even 1e-8 per step would already use up 2e-5).
- FEL (Sec. IV.B, universal scaling): the instability amplifies every
  perturbation of the theta modulation by ~1e4 up to saturation, FP32 rounding
  noise included. f is therefore within 1e-5 only in the linear regime; after
  saturation the bound stated for FP32 is 2e-3, and the field |A| (a global sum)
  stays within the FP32 field bound throughout.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

FP32_TOL = 1e-5
FP32_FIELD_TOL = 5e-4
FP32_SATURATED_TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def start(wl):
    f0 = I.make_f0(wl).astype(np.float32)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32)
    sim.set_f(f0)
    st = O.State(wl.grid, wl.pusher, wl.basis, I.PROJ_GALERKIN, f0.astype(np.float64))
    return sim, st


def test_pendulum_2000_steps_fp32():
    wl = I.pendulum_8192_fp32_cubic(384, 384)
    sim, st = start(wl)
    m0 = st.moments()["mass"]
    for done, upto in ((0, 500), (500, 2000)):
        sim.step(upto - done)
        st.run(upto - done)
        err = rel_l1(sim.get_f(), st.w)
        assert err <= FP32_TOL, (upto, err)
    mg, mo = sim.moments(), st.moments()
    # the mass itself: conserved by the oracle to round-off, by FP32 to rounding noise
    assert abs(mo["mass"] - m0) <= 1e-12 * m0
    assert abs(mg["mass"] - mo["mass"]) <= 5e-6 * mo["mass"]
    assert abs(mg["energy"] - mo["energy"]) <= 5e-5 * abs(mo["energy"])
    sim.close()


def test_fel_to_saturation_fp32():
    wl = I.fel_4096x2048_fp32_cubic(128, 1024)
    sim, st = start(wl)
    hist = []
    for done, upto, tol in ((0, 200, FP32_TOL), (200, 2000, FP32_SATURATED_TOL)):
        sim.step(upto - done)
        hist.append(st.run(upto - done, history=True))
        err = rel_l1(sim.get_f(), st.w)
        assert err <= tol, (upto, err)
    ah = np.hypot(*np.concatenate(hist).reshape(-1, 2).T)
    gh = np.hypot(*sim.field_history().T)
    assert gh.shape == ah.shape == (2000,)
    # the run reaches saturation: |A| grows from 1e-3 to order one
    assert ah.max() > 0.5
    assert np.max(np.abs(gh - ah) / ah) <= FP32_FIELD_TOL
    mg, mo = sim.moments(), st.moments()
    assert abs(mg["mass"] - mo["mass"]) <= 1e-5 * mo["mass"]
    sim.close()
