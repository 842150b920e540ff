"""The N-replica path of bench.py, on CPU with the gloo backend (world size 2).

Each rank runs an independent replica of the step (the workloads shard by
instance and need no exchange), so the only cross-rank operations are the
barrier and the max of the ranks' times; the reported value is the units of
all replicas over the slowest replica's time. The reference arm runs on rank 0
only; other ranks exit without work.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = [12.5, 20.0][rank]            # a slow and a fast replica
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 1000 * 10, ms * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, rate))


def test_two_gloo_replicas_report_the_slowest_time_and_the_whole_job_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    # 2 replicas x 10,000 node-updates in 20 ms
    assert all(abs(r[2] - 2 * 10_000 / 0.020) < 1e-6 for r in res)


def test_reference_arm_does_no_work_off_rank_0(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(bench.parse()) == 0
    assert capsys.readouterr().out == ""


def test_single_process_rate_has_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 100, 0.5) == 200.0
