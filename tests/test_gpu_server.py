"""Serving with continuous batching: each result is the same alone and in the mix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

SAME_TOL = 2e-6   # FP32: same arithmetic up to the order of shared-memory atomic additions


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_12227_gb300 import build as B
    B.build()


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def small_trace(n=8):
    reqs = I.serving_trace(count=n, nmin=64, nmax=700, smin=5, smax=40)
    return reqs


def run_alone(wl, f0, steps, stream):
    s = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, stream=stream)
    s.set_f(f0)
    s.step(steps)
    out = s.get_f()
    s.close()
    return out


def drain(srv, want):
    got = {}
    for _ in range(10000):
        q, a = srv.run(1)
        for r in srv.poll():
            got[r["id"]] = r
        if len(got) >= want and q == 0 and a == 0:
            break
    return got


def test_each_result_is_the_same_alone_and_in_the_mix():
    stream = torch.cuda.Stream()
    reqs = small_trace()
    srv = V.Server(2 << 30, slice_steps=7, stream=stream)
    f0s = {}
    for r in reqs:
        f0 = I.make_f0(r.workload).astype(np.float32)
        f0s[r.rid] = f0
        srv.submit(r.rid, r.workload.grid, r.workload.basis, r.workload.pusher, f0,
                   r.workload.steps, keep_f=True)
    got = drain(srv, len(reqs))
    assert set(got) == {r.rid for r in reqs}
    assert any(g["batched"] for g in got.values())
    for r in reqs:
        res = got[r.rid]
        assert res["status"] == V.VP_OK
        assert res["moments"]["step"] == r.workload.steps
        f_mix = srv.take_f(r.rid, (r.workload.grid.np, r.workload.grid.nx))
        f_alone = run_alone(r.workload, f0s[r.rid], r.workload.steps, stream)
        assert rel_l1(f_mix, f_alone) <= SAME_TOL, r.workload.name
    srv.close()


def test_budget_admission_is_fifo_and_bounded():
    stream = torch.cuda.Stream()
    # ten equal requests; the budget holds three of them (the batch tables also take room)
    base = I.pendulum_8192_fp32_cubic(300, 300, steps=12)
    reqs = [I.Request(k, 0.0, base) for k in range(10)]
    one = V.vp_workspace_size(V.make_grid(base.grid), base.basis, V.make_pusher(base.pusher),
                              V.vp_opts(0, 0, 0, 0, 0, 0, None))
    srv = V.Server(4 * one, budget_bytes=3 * one + 4096, slice_steps=5, stream=stream)
    for r in reqs:
        srv.submit(r.rid, r.workload.grid, r.workload.basis, r.workload.pusher,
                   I.make_f0(r.workload).astype(np.float32), r.workload.steps)
    max_active = 0
    got = {}
    for _ in range(10000):
        q, a = srv.run(1)
        max_active = max(max_active, a)
        for res in srv.poll():
            got[res["id"]] = res
        if q == 0 and a == 0:
            break
    assert len(got) == len(reqs) and all(g["status"] == V.VP_OK for g in got.values())
    assert max_active <= 3
    admits = [got[r.rid]["t_admit"] for r in reqs]
    assert admits == sorted(admits)
    for g in got.values():
        assert g["t_submit"] <= g["t_admit"] <= g["t_finish"]
    srv.close()


def test_invalid_request_finishes_with_its_status():
    stream = torch.cuda.Stream()
    srv = V.Server(64 << 20, stream=stream)
    g = I.Grid(3, 8, -np.pi, np.pi, -1.0, 1.0)
    srv.submit(7, g, V.VP_BASIS_CUBIC_BSPLINE, I.Pusher(), np.zeros((8, 3), np.float32), 5)
    got = drain(srv, 1)
    assert got[7]["status"] == V.VP_ERR_ARG
    srv.close()
