#!/usr/bin/env python
"""Benchmark of the phase-space Vlasov step on GB300.

Default workload: pendulum H = p^2/2 - cos x on an 8192 x 8192 mesh, FP32
weights, cubic B-spline deposit with the Galerkin mass-matrix solve
(tent basis), leapfrog dt = 0.02; one benchmark step = one vp_step(1):
push + deposit + Lambda^{-1} (x and p solves) + step bookkeeping, on the plan
the library's autotuner picks (the one-pass kernel, or its tile pass without
the x solve followed by the x-solve row pass).

Prints one JSON line. value = node-updates/s over all ranks (each rank runs
an independent replica: the step has no cross-GPU exchange at this size).
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2007_12227_gb300 import inputs as I  # noqa: E402

METRIC = "phase-space node-updates/s (push+deposit) and HBM GB/s vs peak; batched/served vs plain"
UNIT = "node-updates/s"
FALLBACK_HBM_GBS = 6800.0
# sources of the one-pass step kernel: the committed ncu traffic applies only to these bytes
FUSED_SOURCES = ["paper_2007_12227_gb300/csrc/vp_fused.cu", "paper_2007_12227_gb300/csrc/vp_internal.h",
                 "paper_2007_12227_gb300/csrc/vp_sum.cuh", "paper_2007_12227_gb300/csrc/vp_fel.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--workload", default="pendulum", choices=["pendulum", "fel"],
                    help="pendulum: 8192^2 two-Gaussian pendulum (the headline); fel: 4096 x 2048 FEL")
    ap.add_argument("--size", type=int, default=0,
                    help="mesh side (pendulum, default 8192) or theta points (fel, default 4096)")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=40)
    ap.add_argument("--serve-count", type=int, default=60,
                    help="requests of the serving trace to run (the whole fixed trace is 2000)")
    ap.add_argument("--tile", default="", help="TX,TP: fixed tile shape instead of the autotuner's")
    ap.add_argument("--kernel", default="auto", choices=["auto", "fused", "xpass"],
                    help="step plan: the planner's, the one-pass kernel, or the one-pass tile with a "
                         "separate x-solve row pass")
    ap.add_argument("--projection", default="galerkin", choices=["galerkin", "lumped"],
                    help="the timed workload's treatment of Lambda: the Galerkin solve (the headline) "
                         "or its row sum (the deposit alone)")
    ap.add_argument("--e2e-pipes", type=int, default=3,
                    help="simulations (each on its own stream) the end-to-end loop interleaves")
    ap.add_argument("--skip-late", action="store_true",
                    help="skip timing the last 20 steps of the workload's run")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """The largest of x over all ranks (the replicas' slowest time), x on every rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size, units_per_rank, seconds_max):
    """Units processed by all replicas divided by the slowest replica's time."""
    return world_size * units_per_rank / seconds_max


def workload(size, kind="pendulum"):
    if kind == "fel":
        size = size or 4096
        return I.fel_4096x2048_fp32_cubic(size, size // 2)
    size = size or 8192
    return I.pendulum_8192_fp32_cubic(size, size)


L2_BYTES = 129 * 2**20   # GB300 L2


class L2Flush:
    """Writes a buffer twice the size of L2 on the stream, so that the next kernel starts cold."""

    def __init__(self, torch, stream):
        self.buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        self.stream = stream
        self.n = 0

    def __call__(self):
        import torch
        with torch.cuda.stream(self.stream):
            self.buf.fill_(float(self.n & 1))
        self.n += 1


def flushed_steps(sim, steps, flush, stream):
    """steps single steps, each after an L2 flush: (total step ms, summed per-phase ms).
    Each step is bracketed by two CUDA events on the sim's stream (so its time excludes the flush);
    the per-phase times come from a second flushed pass of step_profiled(1), whose events between
    the phases take time of their own (about 2 us each) and are kept out of the step time."""
    import torch
    total = 0.0
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(1)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    phases = None
    nprof = min(steps, 50)
    for _ in range(nprof):
        flush()
        ph = sim.step_profiled(1)
        phases = ph if phases is None else [a + b for a, b in zip(phases, ph)]
    return total, [p * steps / nprof for p in phases]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def traffic_from_profile(kernel_file, source_files, tile=None, key="traffic_bytes_per_launch"):
    """Per-launch DRAM bytes (or another per-launch figure, by key) from the committed ncu summary,
    if the kernel is unchanged and the summary was taken with the same tile shape."""
    path = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(key + r":\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    digest = hashlib.sha256()
    for sf in source_files:
        digest.update(open(os.path.join(ROOT, sf), "rb").read())
    if digest.hexdigest() != h.group(1):
        return None
    t = re.search(r"^tile:\s*(\d+)x(\d+)", text, re.M)
    if tile is not None and (not t or (int(t.group(1)), int(t.group(2))) != tuple(tile)):
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def bench_batch(V, torch, stream, batch_steps=40, seq_rounds=5):
    """256 ragged instances (pendulum / FEL, 64^2 .. 2048^2): one persistent launch per
    step replayed from a CUDA graph, against the same instances stepped one by one.
    Tile shapes: the library's autotuner, timing candidate shapes on the whole batch."""
    wls = I.batch_256()
    t0 = time.perf_counter()
    tuned = V.autotune(wls, batched=True, stream=stream)
    tune_s = time.perf_counter() - t0
    sims = []
    for wl, r in zip(wls, tuned):
        sm = V.Sim(wl.grid, wl.basis, wl.pusher, precision=V.VP_FP32, tile_x=r["tile_x"],
                   tile_p=r["tile_p"], stream=stream)
        sm.set_f(I.make_f0(wl).astype(np.float32))
        sims.append(sm)
    nodes = sum(w.grid.nodes for w in wls)
    batch = V.Batch(sims, stream=stream)
    batch.step(3)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / batch_steps
    # sequential plain solves: every instance advanced by its own vp_step calls
    for sm in sims:
        sm.step(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(seq_rounds):
        for sm in sims:
            sm.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    sms = e0.elapsed_time(e1) / seq_rounds
    batch.close()
    for sm in sims:
        sm.close()
    return {"instances": len(wls), "nodes_per_step": nodes,
            "batched_node_updates_per_s": nodes / (bms * 1e-3), "batched_ms_per_step": bms,
            "sequential_node_updates_per_s": nodes / (sms * 1e-3), "sequential_ms_per_step": sms,
            "speedup": sms / bms, "graph": True, "steps_timed": batch_steps,
            "autotune": {"seconds": tune_s, "candidates": tuned[0]["candidates"],
                         "tuned_ms_per_step": tuned[0]["ms_per_step"],
                         "default_ms_per_step": tuned[0]["default_ms_per_step"],
                         "shapes": sorted({(r["tile_x"], r["tile_p"]) for r in tuned})}}


def sequential_plain(V, torch, stream, reqs, f0s):
    """The same requests solved one after another with plain vp_step calls (each: create,
    set the weights, step, read the moments, destroy): the baseline the served form must beat."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, f0 in zip(reqs, f0s):
        sim = V.Sim(r.workload.grid, r.workload.basis, r.workload.pusher, precision=V.VP_FP32,
                    stream=stream)
        sim.set_f(f0)
        sim.step(r.workload.steps)
        sim.moments()
        sim.close()
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def bench_serve(V, torch, stream, count=60, budget_gb=150.0, rate=500.0, sequential=False):
    """Served form: the first `count` requests of the Poisson trace (meshes 128^2 .. 4096^2
    log-uniform, 100 .. 5000 steps, pendulum / FEL) arriving in real time at `rate` per
    second; continuous batching under an HBM budget. Latency = finish - arrival."""
    reqs = I.serving_trace(count=count, rate=rate)
    f0s = [I.make_f0(r.workload).astype(np.float32) for r in reqs]
    free = torch.cuda.mem_get_info()[0]
    arena = int(min(budget_gb * 1e9, 0.8 * free))
    srv = V.Server(arena, budget_bytes=arena, slice_steps=100, stream=stream)
    t0 = srv.clock()
    nxt = 0
    done = {}
    while len(done) < len(reqs):
        now = srv.clock() - t0
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            r = reqs[nxt]
            srv.submit(r.rid, r.workload.grid, r.workload.basis, r.workload.pusher, f0s[nxt],
                       r.workload.steps)
            nxt += 1
        q, a = srv.run(1)
        for res in srv.poll():
            done[res["id"]] = res
        if q == 0 and a == 0 and nxt < len(reqs):
            time.sleep(max(0.0, reqs[nxt].arrival - (srv.clock() - t0)))
    wall = srv.clock() - t0
    srv.close()
    lat = sorted(done[r.rid]["t_finish"] - (t0 + r.arrival) for r in reqs)
    work = sum(r.workload.grid.nodes * r.workload.steps for r in reqs)
    part = "full" if count >= 2000 else "prefix"
    seq = None
    if sequential:
        seq_s = sequential_plain(V, torch, stream, reqs, f0s)
        seq = {"wall_s": seq_s, "node_updates_per_s": work / seq_s,
               "served_over_sequential": (work / wall) / (work / seq_s)}
    return {"requests": count, "trace": f"Poisson {rate:.3g}/s, seed 2007122272 ({part})",
            "sequential_plain": seq,
            "rate_per_s": rate, "offered_node_updates_per_s": rate * work / count,
            "node_updates": work, "wall_s": wall, "node_updates_per_s": work / wall,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "budget_bytes": arena,
            "batched_fraction": sum(1 for d in done.values() if d["batched"]) / len(done)}


def oracle_fel_state(wl, f):
    if wl.pusher.kind != I.PUSH_FEL:
        return None
    from oracle import oracle as O
    br, bi = O.bunching(wl.grid, f)
    return [wl.pusher.a0_re, wl.pusher.a0_im, br, bi]


def cpu_baseline(wl, steps=2):
    """The FP64 oracle on a bounded sample (`steps` steps of the full mesh): its band-parallel
    mode over all host cores (bitwise the serial step), and the serial step on one core."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    f0 = I.make_f0(wl)
    O.lib()
    f, fel = f0, oracle_fel_state(wl, f0)
    t0 = time.perf_counter()
    for _ in range(steps):
        f, fel, _ = O.step_par(wl.grid, wl.basis, I.PROJ_GALERKIN, wl.pusher, f, fel, threads=cores)
    dpar = time.perf_counter() - t0
    f, fel = f0, oracle_fel_state(wl, f0)
    t0 = time.perf_counter()
    for _ in range(steps):
        f, fel, _ = O.step(wl.grid, wl.basis, I.PROJ_GALERKIN, wl.pusher, f, fel)
    dser = time.perf_counter() - t0
    return {"value": wl.grid.nodes * steps / dpar, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of the full {wl.grid.nx}x{wl.grid.np} mesh, FP64 C oracle in its "
                      f"band-parallel mode on {cores} threads (bitwise the serial step), {dpar:.2f} s",
            "serial": {"value": wl.grid.nodes * steps / dser, "cores": 1,
                       "sample": f"the same {steps} steps, serial, {dser:.2f} s"}}


def g_str(wl):
    return f"{wl.grid.nx}x{wl.grid.np}"


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    side = 2048
    cores = os.cpu_count() or 1
    wl = workload(side, args.workload)
    full = workload(0, args.workload)
    f = I.make_f0(wl)
    fel = oracle_fel_state(wl, f)
    O.lib()
    for _ in range(args.warmup):
        f, fel, _ = O.step_par(wl.grid, wl.basis, I.PROJ_GALERKIN, wl.pusher, f, fel, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, fel, _ = O.step_par(wl.grid, wl.basis, I.PROJ_GALERKIN, wl.pusher, f, fel, threads=cores)
    dt = time.perf_counter() - t0
    value = wl.grid.nodes * args.steps / dt
    sample = (f"{args.steps} steps of the same physics on a {g_str(wl)} mesh "
              f"(FP64 C oracle, band-parallel on {cores} threads, bitwise the serial step; "
              f"full mesh is {g_str(full)})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": full.name, "sample_mesh": g_str(wl), "steps": args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2007_12227_gb300 import build as B
    from paper_2007_12227_gb300 import vlasov as V

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    wl = workload(args.size, args.workload)
    kernel = {"auto": V.VP_KERNEL_AUTO, "fused": V.VP_KERNEL_FUSED,
              "xpass": V.VP_KERNEL_FUSED_XPASS}[args.kernel]
    proj = V.VP_PROJ_LUMPED if args.projection == "lumped" else V.VP_PROJ_GALERKIN
    g = wl.grid
    N = g.nodes
    f0 = I.make_f0(wl).astype(np.float32)
    stream = torch.cuda.Stream()
    # working set of a step: two state buffers, and the deposit buffer of the separate-x-pass plan
    # (counted either way here). Below twice the L2, each
    # timed step runs after an L2 flush; above it, the steps run back to back.
    working = 3 * 4 * N
    cold = working < 2 * L2_BYTES
    flush = L2Flush(torch, stream) if cold else None
    # tile shape from the library's autotuner (timed candidates; outside the timed region)
    t_tune = time.perf_counter()
    if args.tile:
        tx, tp = (int(v) for v in args.tile.split(","))
        tuned = {"tile_x": tx, "tile_p": tp, "candidates": 0, "ms_per_step": None,
                 "default_ms_per_step": None}
    else:
        tuned = V.autotune([wl], projection=proj, kernel=kernel, stream=stream)[0]
    t_tune = time.perf_counter() - t_tune
    # the tuner's plan: its kernel (the one-pass kernel or its separate-x-pass form) and shape
    plan_kernel = tuned.get("kernel", kernel) if not args.tile else kernel
    sim = V.Sim(g, wl.basis, wl.pusher, precision=V.VP_FP32, projection=proj, kernel=plan_kernel,
                tile_x=tuned["tile_x"],
                tile_p=tuned["tile_p"], stream=stream)
    sim.set_f(f0)
    sim.step(args.warmup)
    sim.sync()

    # ---- timed region: exactly K steps, events on the sim's stream
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if cold:
        ms, cold_phase = flushed_steps(sim, args.steps, flush, stream)
    else:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    if not cold:
        ms = ev0.elapsed_time(ev1)
    sim.sync()
    ms = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms / args.steps
    value = whole_job_rate(ws, N * args.steps, ms * 1e-3)
    # kernels per vp_step on this plan, as the library reports it (the one-pass kernel finishes
    # the step in its last CTA: one launch per step)
    plan = sim.plan()
    launches_per_step = plan["launches_per_step"]

    # ---- per-phase device time (same stream, events between the kernels)
    if cold:
        phase_ms = [p / args.steps for p in cold_phase]
    else:
        nprof = min(args.steps, 500)
        phase = sim.step_profiled(nprof)
        phase_ms = [p / nprof for p in phase]
    names = ["push_deposit", "lambda_inv_x", "lambda_inv_p", "field_or_count"]
    dom = int(np.argmax(phase_ms))
    bytes_per_node = {"push_deposit": 8, "lambda_inv_x": 8, "lambda_inv_p": 8,
                      "field_or_count": 0}
    peak, peak_kind = peaks()
    alg_bytes = bytes_per_node[names[dom]] * N
    achieved = alg_bytes / (phase_ms[dom] * 1e-3) / 1e9
    xpass = plan["kernel"] == V.VP_KERNEL_FUSED_XPASS
    step_profile = {"pendulum_8192x8192_fp32_cubic": "step_fused_pendulum_8192.md",
                    "fel_4096x2048_fp32_cubic": "step_fused_fel_4096x2048.md"}.get(wl.name, "none.md")
    if xpass:
        step_profile = step_profile.replace("step_fused_", "step_fused_xpass_")
    if args.projection == "lumped":
        step_profile = step_profile.replace("step_fused_", "step_fused_lumped_")
    kernel_files = {"push_deposit": (step_profile, FUSED_SOURCES),
                    "lambda_inv_x": ("xsolve_rows_pendulum_8192.md", FUSED_SOURCES) if xpass else
                                    ("filter_x_pendulum_8192.md", ["paper_2007_12227_gb300/csrc/vp_filter.cu"]),
                    "lambda_inv_p": ("filter_p_pendulum_8192.md",
                                     ["paper_2007_12227_gb300/csrc/vp_filter.cu"])}
    traffic = inst = None
    if names[dom] in kernel_files:
        ptile = (plan["tile_x"], plan["tile_p"]) if names[dom] == "push_deposit" else None
        traffic = traffic_from_profile(*kernel_files[names[dom]], tile=ptile)
        inst = traffic_from_profile(*kernel_files[names[dom]], tile=ptile, key="inst_executed_per_launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": names[dom],
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": alg_bytes,
                "phase_ms": dict(zip(names, phase_ms)),
                "step_algorithmic_gbs": 8 * N / (ms_per_step * 1e-3) / 1e9,
                "step_frac": 8 * N / (ms_per_step * 1e-3) / 1e9 / peak}
    # instruction-issue roofline of the same kernel: warp instructions per launch (committed ncu
    # count, same source and tile) over its live time, against 4 issue slots per SM and cycle at the
    # median SM clock sampled during the timed region
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if inst and mhz:
        issue_peak = sms * 4 * mhz * 1e6
        issue_rate = inst / (phase_ms[dom] * 1e-3)
        roofline["issue"] = {"inst_per_launch": inst, "unit": "warp instructions/s",
                             "achieved": issue_rate, "peak": issue_peak, "frac": issue_rate / issue_peak,
                             "thread_inst_per_node": inst * 32 / N, "sms": sms, "sm_mhz": mhz,
                             "source": "ncu smsp__inst_executed.sum of the committed profile"}

    # ---- late in the run: the last 20 of the workload's 2000 steps (the state filaments, the
    #      kernel's work depends on it), timed the same way outside the headline region
    late = None
    done = args.warmup + args.steps + (min(args.steps, 500) if not cold else 0)
    if wl.steps >= 40 and not args.skip_late:
        target = wl.steps - 20
        if done < target:
            sim.step(target - done)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(20)
        ev1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        late = {"steps": f"{max(done, target) + 1}-{max(done, target) + 20}",
                "ms_per_step": ev0.elapsed_time(ev1) / 20,
                "node_updates_per_s": N * 20 / (ev0.elapsed_time(ev1) * 1e-3),
                "l2": "steps back to back" if not cold else "steps back to back (working set in L2)"}

    # ---- end to end through the C ABI with pinned host buffers. Every step uploads its whole input
    #      and downloads its whole output. Simulations of the same plan on their own streams (three
    #      by default) are driven from this thread with the asynchronous transfer calls, so one's
    #      upload overlaps another's step and download (a host buffer is reused once its simulation
    #      has synchronised). The one-simulation loop with the synchronous calls is reported beside it.
    e2e = None
    if not args.skip_e2e:
        npipe = max(1, args.e2e_pipes)
        ke = max(2 * npipe, min(20, args.steps))
        ke += (-ke) % npipe
        host_in = torch.from_numpy(f0).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        sim.set_f_host_ptr(host_in.data_ptr(), V.VP_FP32)
        sim.step(1)
        sim.get_f_host_ptr(host_out.data_ptr(), V.VP_FP32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            sim.set_f_host_ptr(host_in.data_ptr(), V.VP_FP32)
            sim.step(1)
            sim.get_f_host_ptr(host_out.data_ptr(), V.VP_FP32)
        wall_seq = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        pipes = [(sim, host_in, host_out)]
        for _ in range(npipe - 1):
            pipes.append((V.Sim(g, wl.basis, wl.pusher, precision=V.VP_FP32, projection=proj, kernel=plan_kernel,
                                tile_x=tuned["tile_x"], tile_p=tuned["tile_p"], stream=torch.cuda.Stream()),
                          torch.from_numpy(f0).pin_memory(), torch.empty_like(host_in).pin_memory()))

        def e2e_step(k):
            s_, hin, hout = pipes[k % npipe]
            s_.set_f_async_ptr(hin.data_ptr(), V.VP_FP32)
            s_.step(1)
            s_.get_f_async_ptr(hout.data_ptr(), V.VP_FP32)

        for k in range(npipe):
            e2e_step(k)
        for p_ in pipes:
            p_[0].sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(ke):
            if k >= npipe:
                pipes[k % npipe][0].sync()   # the step that used these host buffers has finished
            e2e_step(k)
        for p_ in pipes:
            p_[0].sync()
        wall = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        # the pipelined output equals the one-simulation output of the same input
        same = all(bool(torch.equal(pipes[0][2], p_[2])) for p_ in pipes[1:])
        for p_ in pipes[1:]:
            p_[0].close()
        e2e = {"value": whole_job_rate(ws, N * ke, wall), "unit": UNIT, "h2d_bytes_per_step": 4 * N,
               "d2h_bytes_per_step": 4 * N, "steps": ke,
               "note": "per step: vp_set_f_async from pinned host + vp_step(1) + vp_get_f_async to pinned "
                       f"host; {npipe} simulations on their own streams, one host thread",
               "simulations": npipe,
               "outputs_agree": same,
               "sequential": {"value": whole_job_rate(ws, N * ke, wall_seq), "unit": UNIT,
                              "note": "one simulation: vp_set_f + vp_step(1) + vp_get_f per step"}}

    # ---- other workloads on the same GPU (context lines, not the headline)
    extra = {}
    if not args.skip_extra and rank == 0:
        fel = I.fel_4096x2048_fp32_cubic()
        # the autotuner's plan (kernel and tile shape), as for the headline workload
        ftuned = V.autotune([fel], stream=stream)[0]
        fsim = V.Sim(fel.grid, fel.basis, fel.pusher, precision=V.VP_FP32, kernel=ftuned["kernel"],
                     tile_x=ftuned["tile_x"], tile_p=ftuned["tile_p"], stream=stream)
        fsim.set_f(I.make_f0(fel).astype(np.float32))
        fsim.step(20)
        fsim.sync()
        # its working set (~100 MiB) fits in L2: each timed step follows an L2 flush
        nf = 200
        fl = flush if flush is not None else L2Flush(torch, stream)
        fms, fph = flushed_steps(fsim, nf, fl, stream)
        fms /= nf
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fsim.step(nf)
        e1.record(stream)
        torch.cuda.synchronize()
        warm = e0.elapsed_time(e1) / nf
        fplan = fsim.plan()
        extra[fel.name] = {"node_updates_per_s": fel.grid.nodes / (fms * 1e-3),
                           "ms_per_step": fms, "steps_timed": nf,
                           "tile": [fplan["tile_x"], fplan["tile_p"]],
                           "plan": "separate x pass" if fplan["kernel"] == V.VP_KERNEL_FUSED_XPASS else "one pass",
                           "l2": "flushed before every timed step",
                           "phase_ms": dict(zip(names, [p / nf for p in fph])),
                           "warm_l2_ms_per_step": warm}
        fsim.close()

    if not args.skip_extra and rank == 0 and args.workload == "pendulum" and args.projection == "galerkin":
        # the same mesh with the lumped projection (Lambda replaced by its row sum: the step is the
        # deposit alone, no solves), on the autotuner's plan for it
        ltuned = V.autotune([wl], projection=V.VP_PROJ_LUMPED, stream=stream)[0]
        lsim = V.Sim(g, wl.basis, wl.pusher, precision=V.VP_FP32, projection=V.VP_PROJ_LUMPED,
                     kernel=ltuned["kernel"], tile_x=ltuned["tile_x"], tile_p=ltuned["tile_p"], stream=stream)
        lsim.set_f(f0)
        lsim.step(10)
        lsim.sync()
        nl = 200
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lsim.step(nl)
        e1.record(stream)
        torch.cuda.synchronize()
        lms = e0.elapsed_time(e1) / nl
        lplan = lsim.plan()
        extra[wl.name + "_lumped"] = {"node_updates_per_s": N / (lms * 1e-3), "ms_per_step": lms,
                                      "steps_timed": nl, "tile": [lplan["tile_x"], lplan["tile_p"]],
                                      "launches_per_step": lplan["launches_per_step"],
                                      "algorithmic_gbs": 8 * N / (lms * 1e-3) / 1e9,
                                      "frac_of_hbm_peak": 8 * N / (lms * 1e-3) / 1e9 / peak,
                                      "l2": "steps back to back (inputs larger than L2)"}
        lsim.close()

    if not args.skip_extra and rank == 0 and not args.skip_batch:
        extra["batch_256"] = bench_batch(V, torch, stream, args.batch_steps)
    if not args.skip_extra and rank == 0 and not args.skip_serve:
        extra["served"] = bench_serve(V, torch, stream, count=args.serve_count, sequential=True)
        # the same requests at ~70% of the batched throughput: a queue that stays bounded
        cap = extra.get("batch_256", {}).get("batched_node_updates_per_s", 4e10)
        reqs = I.serving_trace(count=args.serve_count)
        mean_work = sum(r.workload.grid.nodes * r.workload.steps for r in reqs) / len(reqs)
        extra["served_rho0.7"] = bench_serve(V, torch, stream, count=args.serve_count,
                                             rate=0.7 * cap / mean_work)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        cpu = cpu_baseline(wl)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "mesh": f"{g.nx}x{g.np}", "dt": wl.pusher.dt,
                           "basis": f"cubic_bspline_{args.projection}", "parallelism": f"replicas{ws}",
                           "tile": [plan["tile_x"], plan["tile_p"]],
                           "plan": ("one-pass tile kernel without the x solve + exact x-solve row pass"
                                    if xpass else "one-pass step kernel"),
                           "launches_per_step": launches_per_step,
                           "autotune": {"seconds": t_tune, "candidates": tuned["candidates"],
                                        "tuned_ms_per_step": tuned["ms_per_step"],
                                        "default_ms_per_step": tuned["default_ms_per_step"]},
                           "l2": (f"working set {working / 2**20:.0f} MiB below twice the L2: an L2 flush "
                                  f"({2 * L2_BYTES / 2**20:.0f} MiB written) before every timed step, "
                                  f"the step timed by its own events"
                                  if cold else
                                  f"inputs larger than L2 (workspace {plan['workspace_bytes'] / 2**20:.0f} MiB: "
                                  f"two {4 * N / 2**20:.0f} MiB state buffers"
                                  + (f" + the {4 * N / 2**20:.0f} MiB deposit between the tile and row passes"
                                     if xpass else "") + ")")},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "late_window": late,
                "gpu_launches": launches_per_step * args.steps, "extra": extra}
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
