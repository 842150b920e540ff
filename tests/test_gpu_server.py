"""Serving with continuous batching: each result is the same alone and in the mix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2007_12227_gb300 import inputs as I  # noqa: E402
from paper_2007_12227_gb300 import vlasov as V  # noqa: E402

SAME_TOL = 2e-6   # FP32: same arithmetic up to the order of shared-memory atomic additions
FP32_TOL = 1e-5   # FP32 against the FP64 oracle (relative L1 of f)
FP32_FIELD_TOL = 5e-4   # FP32 |A| against the oracle (the theta modulation of f0 is 1e-4)


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


def run_alone(wl, f0, steps, stream, dtype=np.float64):
    s = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, stream=stream)
    s.set_f(f0)
    s.step(steps)
    out = s.get_f(dtype=dtype)
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


def test_served_results_match_the_oracle():
    """Served results (pendulum and FEL) against the FP64 oracle run of the same request:
    f within the FP32 bound, the field A at completion within the FP32 field bound."""
    stream = torch.cuda.Stream()
    reqs = small_trace(12)
    fel = [r for r in reqs if r.workload.pusher.kind == I.PUSH_FEL][:2]
    pend = [r for r in reqs if r.workload.pusher.kind == I.PUSH_KDK][:2]
    chosen = fel + pend
    assert len(fel) == 2 and len(pend) == 2
    srv = V.Server(2 << 30, slice_steps=6, stream=stream)
    f0s = {}
    for r in reqs:
        f0 = I.make_f0(r.workload).astype(np.float32)
        f0s[r.rid] = f0
        srv.submit(r.rid, r.workload.grid, r.workload.basis, r.workload.pusher, f0,
                   r.workload.steps, keep_f=True)
    got = drain(srv, len(reqs))
    for r in chosen:
        wl = r.workload
        res = got[r.rid]
        assert res["status"] == V.VP_OK and res["batched"]
        f = srv.take_f(r.rid, (wl.grid.np, wl.grid.nx))
        st = O.State(wl.grid, wl.pusher, wl.basis, wl.projection, f0s[r.rid].astype(np.float64))
        st.run(wl.steps)
        assert rel_l1(f, st.w) <= FP32_TOL, wl.name
        if wl.pusher.kind == I.PUSH_FEL:
            a_gpu = np.hypot(res["moments"]["a_re"], res["moments"]["a_im"])
            a_or = np.hypot(st.fel[0], st.fel[1])
            assert abs(a_gpu - a_or) <= FP32_FIELD_TOL * a_or, wl.name
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


def test_cancel_a_running_and_a_queued_request():
    """Six requests run as one batch; one is cancelled mid-run, and a seventh that is still
    queued (the budget has no room for it) is cancelled too. Both report VP_ERR_CANCELLED;
    the other five finish and give the same bits as when each runs alone."""
    stream = torch.cuda.Stream()
    reqs = small_trace(6)
    reqs = [I.Request(r.rid, r.arrival, I.with_steps(r.workload, 30)) for r in reqs]
    big = I.Request(99, 0.0, I.pendulum_8192_fp32_cubic(1024, 1024, steps=30))
    sizes = [V.vp_workspace_size(V.make_grid(r.workload.grid), r.workload.basis,
                                 V.make_pusher(r.workload.pusher), V.vp_opts(0, 0, 0, 0, 0, 0, None))
             for r in reqs]
    budget = sum(sizes) + (8 << 20)   # the six and their batch tables; not the 1024^2 request
    srv = V.Server(budget + (64 << 20), budget_bytes=budget, slice_steps=5, stream=stream)
    f0s = {}
    for r in reqs + [big]:
        f0 = I.make_f0(r.workload).astype(np.float32)
        f0s[r.rid] = f0
        srv.submit(r.rid, r.workload.grid, r.workload.basis, r.workload.pusher, f0,
                   r.workload.steps, keep_f=True)
    q, a = srv.run(2)          # 10 of 30 steps done
    assert a == 6 and q == 1
    victim = reqs[2].rid
    srv.cancel(victim)
    srv.cancel(big.rid)
    with pytest.raises(V.VlasovError) as ei:
        srv.cancel(12345)
    assert ei.value.status == V.VP_ERR_STATE
    got = drain(srv, 7)
    assert set(got) == {r.rid for r in reqs} | {big.rid}
    assert got[big.rid]["status"] == V.VP_ERR_CANCELLED
    assert got[victim]["status"] == V.VP_ERR_CANCELLED
    assert got[victim]["moments"]["step"] == 10
    with pytest.raises(V.VlasovError):
        srv.take_f(victim, (reqs[2].workload.grid.np, reqs[2].workload.grid.nx))
    for r in reqs:
        if r.rid == victim:
            continue
        assert got[r.rid]["status"] == V.VP_OK and got[r.rid]["moments"]["step"] == 30
        f_mix = srv.take_f(r.rid, (r.workload.grid.np, r.workload.grid.nx), dtype=np.float32)
        f_alone = run_alone(r.workload, f0s[r.rid], 30, stream, dtype=np.float32)
        assert np.array_equal(f_mix, f_alone), r.workload.name
    srv.close()


def test_invalid_request_finishes_with_its_status():
    stream = torch.cuda.Stream()
    srv = V.Server(64 << 20, stream=stream)
    g = I.Grid(3, 8, -np.pi, np.pi, -1.0, 1.0)
    srv.submit(7, g, V.VP_BASIS_CUBIC_BSPLINE, I.Pusher(), np.zeros((8, 3), np.float32), 5)
    got = drain(srv, 1)
    assert got[7]["status"] == V.VP_ERR_ARG
    srv.close()
