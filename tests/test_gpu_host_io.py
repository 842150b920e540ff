"""vp_set_f / vp_get_f with pinned host buffers.

When the stored state is s = Lambda_p w (the fused Galerkin step), the library reads a pinned
host source in place with the Lambda_p multiply and writes a pinned host destination in place
with the p solve, instead of staging the weights through a device copy. Both routes must give
the same bits as a pageable buffer, on ragged mesh sizes, and a pinned buffer that is not
aligned to its element size must take the staged route.
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


def pendulum(nx, np_, precision):
    g = I.Grid(nx, np_, -np.pi, np.pi, -3.0, 3.0)
    pu = I.Pusher(I.PUSH_KDK, I.POT_PENDULUM, 1.0, 1.0, 0.05)
    return I.Workload("t", g, pu, I.BASIS_CUBIC, precision, 0, "gaussian",
                      dict(xc=0.5, pc=0.0, sx=0.8, sp=0.7))


@pytest.mark.parametrize("precision", [I.FP32, I.FP64])
@pytest.mark.parametrize("shape", [(1000, 650), (256, 64), (300, 65)])
def test_pinned_matches_pageable(precision, shape):
    wl = pendulum(*shape, precision)
    npt = np.float32 if precision == I.FP32 else np.float64
    tdt = torch.float32 if precision == I.FP32 else torch.float64
    f0 = I.make_f0(wl).astype(npt)
    outs = []
    for pinned in (False, True):
        sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=precision, kernel=V.VP_KERNEL_FUSED)
        assert sim.kernel() == V.VP_KERNEL_FUSED
        if pinned:
            host_in = torch.from_numpy(f0.copy()).pin_memory()
            host_out = torch.zeros(f0.shape, dtype=tdt).pin_memory()
            sim.set_f_host_ptr(host_in.data_ptr(), precision)
            first = torch.zeros_like(host_out).pin_memory()
            sim.get_f_host_ptr(first.data_ptr(), precision)
            sim.step(3)
            sim.get_f_host_ptr(host_out.data_ptr(), precision)
            outs.append((first.numpy().copy(), host_out.numpy().copy()))
        else:
            sim.set_f(f0)
            first = sim.get_f(dtype=npt)
            sim.step(3)
            outs.append((first, sim.get_f(dtype=npt)))
        sim.close()
    (a0, a3), (b0, b3) = outs
    assert np.array_equal(a0, b0)
    if precision == I.FP32:
        # the FP32 step deposits through integer atomics: bit-reproducible
        assert np.array_equal(a3, b3)
    else:
        # FP64 shared-memory atomics add in arrival order: equal to rounding
        assert np.max(np.abs(a3 - b3)) <= 1e-13 * np.max(np.abs(b3))
    # round trip: Lambda_p then its inverse returns the weights to the solve's rounding
    tol = 1e-6 if precision == I.FP32 else 1e-14
    assert np.max(np.abs(b0 - f0)) <= tol * np.max(np.abs(f0))


def test_misaligned_pinned_buffer_is_staged():
    wl = pendulum(260, 70, I.FP32)
    f0 = I.make_f0(wl).astype(np.float32)
    n = f0.size
    ref = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32)
    ref.set_f(f0)
    ref.step(2)
    want = ref.get_f(dtype=np.float32)
    ref.close()
    # a pinned byte buffer; the weights start 2 bytes in, off their 4-byte alignment
    raw = torch.zeros(4 * n + 16, dtype=torch.uint8).pin_memory()
    base, off = raw.data_ptr(), 2
    assert base % 4 == 0
    view = raw.numpy()[off:off + 4 * n]
    view[:] = np.frombuffer(f0.tobytes(), dtype=np.uint8)
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32)
    sim.set_f_host_ptr(base + off, V.VP_FP32)
    sim.step(2)
    raw.zero_()
    sim.get_f_host_ptr(base + off, V.VP_FP32)
    got = np.frombuffer(raw.numpy()[off:off + 4 * n].tobytes(), dtype=np.float32).reshape(f0.shape)
    sim.close()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kernel", [V.VP_KERNEL_AUTO, V.VP_KERNEL_FUSED_XPASS])
@pytest.mark.parametrize("precision", [I.FP32, I.FP64])
def test_async_transfers_match_the_synchronous_calls(kernel, precision):
    """vp_set_f_async / vp_get_f_async (copy engine on the sim's stream, no wait) give what
    vp_set_f / vp_get_f give; two simulations on two streams interleaved from one thread, as the
    benchmark's end-to-end loop runs them, give what one simulation gives. FP32 sums integer
    window cells: the same bits. FP64 deposits with floating-point atomics, whose order varies
    from run to run: equal to within a few roundings."""
    wl = pendulum(1000, 650, precision)
    npt = np.float32 if precision == I.FP32 else np.float64
    tdt = torch.float32 if precision == I.FP32 else torch.float64
    f0 = I.make_f0(wl).astype(npt)
    ref = V.Sim(wl.grid, wl.basis, wl.pusher, precision=precision, kernel=kernel)
    ref.set_f(f0)
    ref.step(2)
    want = ref.get_f(npt)
    ref.close()
    pipes = []
    for _ in range(2):
        sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=precision, kernel=kernel,
                    stream=torch.cuda.Stream())
        hin = torch.from_numpy(f0.reshape(-1)).pin_memory()
        hout = torch.zeros(f0.size, dtype=tdt).pin_memory()
        pipes.append((sim, hin, hout))
    for k in range(4):
        sim, hin, hout = pipes[k % 2]
        if k >= 2:
            sim.sync()
        sim.set_f_async_ptr(hin.data_ptr(), precision)
        sim.step(2)
        sim.get_f_async_ptr(hout.data_ptr(), precision)
    for sim, _, hout in pipes:
        sim.sync()
        got = hout.numpy().reshape(want.shape)
        if precision == I.FP32:
            assert np.array_equal(got, want)
        else:
            assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
        other = V.VP_FP64 if precision == I.FP32 else V.VP_FP32
        with pytest.raises(V.VlasovError) as ei:
            sim.get_f_async_ptr(hout.data_ptr(), other)
        assert ei.value.status == V.VP_ERR_ARG
        sim.close()
