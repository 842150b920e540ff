"""Bitwise reproducibility of the FP32 one-pass step.

The FP32 deposit sums integer (fixed-point) cells with integer atomics, so the
order in which CTAs and threads add into a cell cannot change a bit; the FEL
partial sums and the field update run in a fixed order. The same step on the
same state therefore gives identical bits run after run, and a simulation
advanced inside a batch gives the bits it gives alone (same tile shapes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def run(wl, steps, stream=None):
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, stream=stream)
    sim.set_f(I.make_f0(wl).astype(np.float32))
    sim.step(steps)
    f = sim.get_f(np.float32)
    h = sim.field_history()
    assert sim.kernel() == V.VP_KERNEL_FUSED
    sim.close()
    return f, h


@pytest.mark.parametrize("wl", [I.pendulum_8192_fp32_cubic(1024, 512),
                                I.fel_4096x2048_fp32_cubic(512, 256),
                                I.pendulum_8192_fp32_cubic(200, 160)],   # whole-period tiles
                         ids=["pendulum", "fel", "full_row"])
def test_repeated_runs_are_bitwise_identical(wl):
    f1, h1 = run(wl, 25)
    f2, h2 = run(wl, 25)
    assert np.array_equal(f1.view(np.uint32), f2.view(np.uint32))
    assert np.array_equal(h1, h2)


def test_batch_equals_alone_bitwise():
    stream = torch.cuda.Stream()
    wls = I.batch_256(count=6, steps=0, sizes=(64, 256, 512))
    batched = []
    for wl in wls:
        s = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, stream=stream)
        s.set_f(I.make_f0(wl).astype(np.float32))
        batched.append(s)
    b = V.Batch(batched, stream=stream)
    b.step(9, use_graph=True)
    for wl, sb in zip(wls, batched):
        fa, ha = run(wl, 9, stream=stream)
        assert np.array_equal(sb.get_f(np.float32).view(np.uint32), fa.view(np.uint32)), wl.name
        assert np.array_equal(sb.field_history(), ha), wl.name
    b.close()
    for s in batched:
        s.close()


@pytest.mark.parametrize("wl", [I.pendulum_8192_fp32_cubic(1024, 512),
                                I.fel_4096x2048_fp32_cubic(512, 256)])
def test_reading_the_weights_between_steps_changes_nothing(wl):
    """With the stored state s = Lambda_p w, vp_get_f, vp_moments and vp_state_device compute w
    into the idle ping-pong buffer, which the next step overwrites: reading between steps must
    leave every later step's bits as they are."""
    f_plain, h_plain = run(wl, 12)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32)
    assert sim.plan()["state_is_s"] == 1
    sim.set_f(I.make_f0(wl).astype(np.float32))
    for k in range(4):
        sim.step(3)
        sim.get_f(np.float32)
        sim.moments()
        sim.state_ptr()
    f = sim.get_f(np.float32)
    h = sim.field_history()
    sim.close()
    assert np.array_equal(f, f_plain)
    assert np.array_equal(h, h_plain)
