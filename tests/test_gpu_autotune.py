"""The tile-shape autotuner (vp_autotune) and the plans it picks.

A tile shape only decides which CTA computes a node, so a simulation built
with the tuned shape must give the default plan's step up to the order of
shared-memory atomic additions, and the FP64 oracle's within the FP32 bound.
A single configuration tuned for the planner's choice may also pick the
separate-x-pass plan, whose exact row solve differs from the in-tile one by
the in-tile truncation |z|^16 and rounding order: within the same bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

FP32_TOL = 1e-5
SAME_TOL = 2e-6   # same arithmetic, other summation order


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def run(wl, steps, tile=(0, 0), stream=None, kernel=V.VP_KERNEL_AUTO):
    sim = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, kernel=kernel, tile_x=tile[0], tile_p=tile[1],
                stream=stream)
    sim.set_f(I.make_f0(wl).astype(np.float32))
    sim.step(steps)
    plan = sim.plan()
    f = sim.get_f()
    sim.close()
    return f, plan


def test_single_tuning_picks_a_valid_faster_shape_and_caches_it():
    V.autotune_clear_cache()
    wl = I.pendulum_8192_fp32_cubic(1536, 768)
    r, = V.autotune([wl])
    assert r["from_cache"] == 0 and r["candidates"] >= 2
    assert r["kernel"] in (V.VP_KERNEL_FUSED, V.VP_KERNEL_FUSED_XPASS)
    assert r["ms_per_step"] <= r["default_ms_per_step"] * 1.0001
    r2, = V.autotune([wl])
    assert r2["from_cache"] == 1
    assert (r2["tile_x"], r2["tile_p"]) == (r["tile_x"], r["tile_p"])
    # the tuned shape plans to itself and computes the same step
    f_tuned, plan = run(wl, 8, (r["tile_x"], r["tile_p"]), kernel=r["kernel"])
    assert (plan["tile_x"], plan["tile_p"], plan["kernel"]) == (r["tile_x"], r["tile_p"], r["kernel"])
    f_default, _ = run(wl, 8)
    assert rel_l1(f_tuned, f_default) <= SAME_TOL


def test_tuned_shape_matches_the_oracle():
    wl = I.fel_4096x2048_fp32_cubic(768, 256)
    r, = V.autotune([wl], use_cache=False)
    f, _ = run(wl, 6, (r["tile_x"], r["tile_p"]), kernel=r["kernel"])
    f0 = I.make_f0(wl).astype(np.float32).astype(np.float64)
    st = O.State(wl.grid, wl.pusher, wl.basis, I.PROJ_GALERKIN, f0)
    st.run(6)
    assert rel_l1(f, st.w) <= FP32_TOL


def test_batched_tuning_gives_every_instance_a_plan():
    stream = torch.cuda.Stream()
    wls = I.batch_256(count=8, steps=0, sizes=(64, 256, 512, 1024))
    res = V.autotune(wls, batched=True, use_cache=False, stream=stream)
    assert len(res) == len(wls)
    assert all(r["kernel"] == V.VP_KERNEL_FUSED for r in res)
    assert res[0]["ms_per_step"] <= res[0]["default_ms_per_step"] * 1.0001
    sims, alone = [], []
    for wl, r in zip(wls, res):
        for lst in (sims, alone):
            s = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, tile_x=r["tile_x"],
                      tile_p=r["tile_p"], stream=stream)
            s.set_f(I.make_f0(wl).astype(np.float32))
            lst.append(s)
    b = V.Batch(sims, stream=stream)
    b.step(5)
    for s in alone:
        s.step(5)
    for wl, sb, sa in zip(wls, sims, alone):
        assert rel_l1(sb.get_f(), sa.get_f()) <= SAME_TOL, wl.name
    b.close()
    for s in sims + alone:
        s.close()
