"""Batched stepping: many ragged simulations in one persistent launch (CUDA graph).

Each simulation advanced inside a batch must equal the same simulation stepped on
its own (same kernel, same arithmetic; only the order of shared-memory atomic
additions may differ), and agree with the FP64 oracle within the FP32 bound.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

FP32_TOL = 1e-5
SAME_TOL = 2e-6   # batched vs alone: same arithmetic up to summation order


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def mixed_workloads(steps=0):
    wls = I.batch_256(count=10, steps=steps, sizes=(64, 128, 256, 512, 1024))
    return wls


def make_sims(wls, stream):
    sims = []
    for wl in wls:
        s = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, stream=stream)
        s.set_f(I.make_f0(wl).astype(np.float32))
        sims.append(s)
    return sims


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_individual_steps(use_graph):
    stream = torch.cuda.Stream()
    wls = mixed_workloads()
    batched = make_sims(wls, stream)
    alone = make_sims(wls, stream)
    b = V.Batch(batched, stream=stream)
    b.step(7, use_graph=use_graph)
    b.step(6, use_graph=use_graph)
    for s in alone:
        s.step(13)
    for wl, sb, sa in zip(wls, batched, alone):
        fb, fa = sb.get_f(), sa.get_f()
        assert rel_l1(fb, fa) <= SAME_TOL, wl.name
        mb, ma = sb.moments(), sa.moments()
        assert mb["step"] == ma["step"] == 13
        if wl.pusher.kind == I.PUSH_FEL:
            # the order of shared-memory atomic additions changes f at FP32 rounding level,
            # and the early bunching magnifies that ~1e3 times (it is a 1e-4 modulation)
            hb, ha = sb.field_history(), sa.field_history()
            assert np.max(np.abs(hb - ha)) <= 1e-5 * np.max(np.abs(ha)), wl.name
    b.close()


def test_batch_matches_oracle():
    stream = torch.cuda.Stream()
    wls = [w for w in mixed_workloads() if w.grid.nx <= 256][:4]
    sims = make_sims(wls, stream)
    b = V.Batch(sims, stream=stream)
    b.step(12)
    for wl, s in zip(wls, sims):
        st = O.State(wl.grid, wl.pusher, wl.basis, wl.projection,
                     I.make_f0(wl).astype(np.float32).astype(np.float64))
        st.run(12)
        assert rel_l1(s.get_f(), st.w) <= FP32_TOL, wl.name
    b.close()


def _batch_vs_oracle(wls, tiles, steps):
    stream = torch.cuda.Stream()
    sims = []
    for wl, (tx, tp) in zip(wls, tiles):
        s = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, tile_x=tx, tile_p=tp,
                  stream=stream)
        s.set_f(I.make_f0(wl).astype(np.float32))
        sims.append(s)
    b = V.Batch(sims, stream=stream)
    b.step(steps)
    for wl, s in zip(wls, sims):
        st = O.State(wl.grid, wl.pusher, wl.basis, wl.projection,
                     I.make_f0(wl).astype(np.float32).astype(np.float64))
        hist = st.run(steps, history=True)
        assert rel_l1(s.get_f(), st.w) <= FP32_TOL, (wl.name, s.plan())
        if wl.pusher.kind == I.PUSH_FEL:
            gh, ah = np.hypot(*s.field_history().T), np.hypot(*hist.T)
            assert np.max(np.abs(gh - ah) / ah) <= 5e-4, wl.name
        s.close()
    b.close()


@pytest.mark.parametrize("tx", [64, 128, 224, 256])
def test_batch_tile_shapes_match_oracle(tx):
    """The tile shapes the batched autotuner picks for the 256-instance workload (widths 64,
    128, 224, 256 at height 64), each applied to pendulum and FEL instances of the batch."""
    wls = [w for w in I.batch_256(count=24, steps=0) if w.grid.nx <= 512]
    wls = [w for w in wls if w.pusher.kind == I.PUSH_KDK][:2] + \
        [w for w in wls if w.pusher.kind == I.PUSH_FEL][:2]
    _batch_vs_oracle(wls, [(tx, 64)] * len(wls), 12)


def test_batch_autotuned_shapes_match_oracle():
    """Shapes from vp_autotune(batched=1), as the benchmark's batch uses them."""
    wls = [w for w in I.batch_256(count=24, steps=0) if w.grid.nx <= 512][:6]
    tuned = V.autotune(wls, batched=True, stream=torch.cuda.Stream())
    _batch_vs_oracle(wls, [(r["tile_x"], r["tile_p"]) for r in tuned], 10)


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_step_each_stops_every_simulation_at_its_own_count(use_graph):
    """vp_batch_step_each: in one call of n steps simulation k takes min(n, max_steps[k]) steps
    (0 and negative: none) and gives the same bits as stepping it alone that many times; a
    second call continues from there."""
    stream = torch.cuda.Stream()
    wls = mixed_workloads()[:6]
    batched = make_sims(wls, stream)
    alone = make_sims(wls, stream)
    b = V.Batch(batched, stream=stream)
    first = [9, 0, 4, 12, -3, 9]
    b.step_each(9, first, use_graph=use_graph)
    second = [2, 5, 0, 1, 3, 9]
    b.step_each(5, second, use_graph=use_graph)
    for k, (wl, sb, sa) in enumerate(zip(wls, batched, alone)):
        n = max(0, min(9, first[k])) + max(0, min(5, second[k]))
        if n:
            sa.step(n)
        assert sb.moments()["step"] == sa.moments()["step"] == n, wl.name
        assert np.array_equal(sb.get_f(), sa.get_f()), wl.name
        if wl.pusher.kind == I.PUSH_FEL:
            assert np.array_equal(sb.field_history(), sa.field_history()), wl.name
    b.close()


def test_batch_graph_on_the_legacy_stream_steps_directly():
    """The legacy default stream cannot be captured: use_graph there launches the steps
    directly and gives the same weights as the graph on a created stream."""
    wls = [w for w in I.batch_256(count=24, steps=0) if w.grid.nx <= 256][:3]
    legacy = torch.cuda.default_stream()
    assert legacy.cuda_stream == 0
    a = make_sims(wls, legacy)
    s2 = torch.cuda.Stream()
    c = make_sims(wls, s2)
    ba, bc = V.Batch(a, stream=legacy), V.Batch(c, stream=s2)
    ba.step(5, use_graph=True)
    bc.step(5, use_graph=True)
    for x, y in zip(a, c):
        assert np.array_equal(x.get_f(), y.get_f())
    ba.close()
    bc.close()


def test_batch_rejects_mixed_precision():
    stream = torch.cuda.Stream()
    wl = mixed_workloads()[0]
    s32 = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, stream=stream)
    s64 = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP64, stream=stream)
    with pytest.raises(V.VlasovError):
        V.Batch([s32, s64], stream=stream)
