"""vp_moments_static: moments with no device allocation (its scratch is a static device array).

For callers that cannot allocate device memory when they want the diagnostics:
an application whose framework allocator already holds the device's memory, or
a latency-critical loop that must not take the synchronisation an allocation
can bring. The entry point must give what vp_moments gives, within the FP64
tolerance of the other moment tests, on two consecutive calls that share the
static array, and agree with the FP64 oracle's moments of the same weights.

The file name sorts last, so pytest collects it after every other test file: a
run that stops at the first failure (-x) has then already run all the other
tests if this one fails. It also runs on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

TOL = 1e-11   # FP64 reductions in another summation order


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def static_moments(w, grid, pusher, lost, a, stream):
    out = V.vp_moments_t()
    g = V.make_grid(grid)
    pu = V.make_pusher(pusher)
    aa = (C.c_double * 2)(*a)
    dt = V.VP_FP64 if w.dtype == torch.float64 else V.VP_FP32
    st = V.lib().vp_moments_static(C.c_void_p(w.data_ptr()), dt, C.byref(g), C.byref(pu),
                                   float(lost), aa, C.byref(out), C.c_void_p(stream.cuda_stream))
    assert st == V.VP_OK
    return out.as_dict()


@pytest.mark.parametrize("which", ["pendulum_fp32", "fel_fp32", "pendulum_fp64"])
def test_static_moments_equal_vp_moments_on_two_calls(which):
    stream = torch.cuda.Stream()
    if which == "fel_fp32":
        wl = I.fel_4096x2048_fp32_cubic(512, 256, sp=0.1, a0=0.05)
    elif which == "pendulum_fp64":
        wl = I.pendulum_8192_fp32_cubic(300, 200)
        wl.precision = I.FP64
    else:
        wl = I.pendulum_8192_fp32_cubic(700, 500)
    dtype = torch.float64 if wl.precision == I.FP64 else torch.float32
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=wl.precision, stream=stream)
    f0 = I.make_f0(wl)
    sim.set_f(f0 if wl.precision == I.FP64 else f0.astype(np.float32))
    for call in range(2):
        sim.step(5)
        want = sim.moments()
        w = torch.empty((wl.grid.np, wl.grid.nx), dtype=dtype, device="cuda")
        sim.get_f_device(w)
        torch.cuda.synchronize()
        got = static_moments(w, wl.grid, wl.pusher, want["lost_mass"], (want["a_re"], want["a_im"]),
                             stream)
        for k in ("sum_w", "mass", "mean_x", "mean_p", "var_x", "var_p", "cov_xp", "energy",
                  "trapped", "entropy", "neg_mass", "b_re", "b_im", "max_abs_w", "lost_mass"):
            scale = max(abs(want[k]), 1e-9 * abs(want["sum_w"]))
            assert abs(got[k] - want[k]) <= TOL * scale, (call, k, got[k], want[k])
        # the oracle's FP64 moments of the same weights (a serial sum: another order again).
        # Quantities that cancel to near zero are compared on the scale of their terms: the
        # coordinate range for the means, its square for the second moments, one for the
        # bunching and the energy, the mass for the partial masses.
        om = O.moments(wl.grid, wl.pusher, w.double().cpu().numpy(), (want["a_re"], want["a_im"]))
        L = max(abs(wl.grid.x0), abs(wl.grid.x1), abs(wl.grid.p0), abs(wl.grid.p1))
        floor = {"mean_x": L, "mean_p": L, "var_x": L * L, "var_p": L * L, "cov_xp": L * L,
                 "energy": 1.0, "entropy": 1.0, "b_re": 1.0, "b_im": 1.0, "trapped": om["mass"],
                 "neg_mass": om["mass"]}
        for k in ("sum_w", "mass", "mean_x", "mean_p", "var_x", "var_p", "cov_xp", "energy",
                  "trapped", "entropy", "neg_mass", "b_re", "b_im", "max_abs_w"):
            scale = max(abs(om[k]), floor.get(k, 0.0))
            assert abs(got[k] - om[k]) <= TOL * scale, (call, k, got[k], om[k])
    sim.close()


def test_static_moments_reject_meshes_above_the_limit():
    g = V.vp_grid(16384, 8192, -np.pi, np.pi, -4.0, 4.0)     # 2^27 nodes > 2^26
    pu = V.make_pusher(I.Pusher())
    out = V.vp_moments_t()
    dummy = torch.zeros(4, device="cuda")
    st = V.lib().vp_moments_static(C.c_void_p(dummy.data_ptr()), V.VP_FP32, C.byref(g), C.byref(pu),
                                   0.0, None, C.byref(out), None)
    assert st == V.VP_ERR_UNSUPPORTED
