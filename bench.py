#!/usr/bin/env python3
"""Benchmark of the batched sparse-permanent estimator on one B300.

Workload (one step): 64 Erdos-Renyi bipartite matrices with a planted
permutation, n ~ U{100..2000}, average degree ~ U[4, 8] (generator seed 2),
estimated together in one persistent launch with the schedule "two-sided
minimum degree + initial DM + SK(K0=100, K=10) Adaptive, no inner DM", FP32
proposal / FP64 log-weights.  Each step runs a fresh, disjoint slice of
trajectory ids (T per matrix), the whole hot path: preprocessing (CSC build,
initial DM, outer SK), trajectories, statistics.

metric: effective samples per second, sum over matrices of
(sum X)^2 / sum X^2 per step, divided by the device time of the steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica (independent trajectory ids);
value = all ranks' effective samples / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_15390_b300 import inputs as G  # noqa: E402

METRIC = "effective samples/s at fixed rel. error, learned+batched vs plain, 1 B300"
UNIT = "effective samples/s"
N_MATS, N_LO, N_HI, D_LO, D_HI, GEN_SEED = 64, 100, 2000, 4.0, 8.0, 2
WORKLOAD = ("64 ER+planted-permutation matrices, n~U{100..2000}, avg degree~U[4,8] "
            "(generator seed 2); two-sided MD, initial DM, SK(K0=100,K=10) Adaptive, no inner DM; "
            "FP32 proposal, FP64 log-weights; one persistent launch per step")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--traj", type=int, default=256, help="trajectories per matrix per step")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-compare", action="store_true",
                   help="skip the learned-batched vs plain-unbatched comparison")
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--mats", type=int, default=N_MATS,
                   help="use the first K matrices (profiling of a smaller case)")
    p.add_argument("--nmax", type=int, default=N_HI,
                   help="draw n from U{100..nmax} instead (profiling of a smaller case)")
    return p.parse_args()


def schedule_fields():
    # vertex_rule, initial_dm, K0, K, sk (ADAPTIVE=2), dm (NONE=0), precision (FP32=0), theta
    return dict(vertex_rule=0, initial_dm=1, K0=100, K=10, sk=2, dm=0, precision=0, theta=0.33)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_2608_15390_b300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_2608_15390_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic_per_byte():
    """DRAM bytes per algorithmic byte of the trajectory kernel from the
    committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traj_kernel_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_alg_byte")


def cpu_baseline(mats, T_gpu_ess_per_traj, seconds_budget=20.0):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    same workload: one trajectory of every 4th matrix, repeated until about
    `seconds_budget` of CPU work; reported as effective samples/s through the
    GPU run's effective samples per trajectory."""
    import oracle as O
    sched = O.Schedule(**{k: v for k, v in schedule_fields().items()})
    threads = os.cpu_count() or 1
    sample = mats[::4]
    t0 = time.perf_counter()
    done = 0
    rounds = 0
    while True:
        for k, m in enumerate(sample):
            P = O.Prepared(m, sched)
            P.run(seed=99, count=threads, first_traj=rounds * threads, matrix=4 * k, threads=threads)
            done += threads
        rounds += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    dt = time.perf_counter() - t0
    tps = done / dt
    return {"value": tps * T_gpu_ess_per_traj, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{done} trajectories ({threads} per matrix per round, {rounds} rounds) on "
                      f"matrices 0,4,...,60 of the workload incl. preprocessing, {dt:.1f} s; "
                      f"{tps:.3f} traj/s x the GPU run's effective samples per trajectory"}


def compare_learned_vs_plain(ctx, B, dev, args, T):
    """The metric's comparison on the same 64 matrices and trajectory counts:
    the learned proposal (network trained here, untimed, on pairs recorded
    from an SK-scheduled run on 16 training matrices of the same family,
    generator seed 7) run batched in one launch, against the plain estimator
    (outer SK only, no inner scaling) run one matrix per launch.  Device time
    from CUDA events on the launching stream, effective samples summed."""
    import torch
    stream = torch.cuda.current_stream()
    train = [G.er_planted(m.n, 6.0, seed=7_000 + k) for k, m in
             enumerate(G.batch_er(16, N_LO, N_HI, D_LO, D_HI, seed=7))]
    teacher = B.Schedule(initial_dm=1, K0=100, K=10, sk=B.SK_FIXED, precision=B.PREC_FP32_PROPOSAL)
    model = ctx.model(seed=11)
    t0 = time.perf_counter()
    rep = model.train(train, teacher, n_pairs=2_000_000, epochs=4, batch=8192, lr=2e-3, seed=12)
    t_train = time.perf_counter() - t0
    learned = B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL, learned=model)
    plain = B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL)
    nt = [T] * len(dev)
    ctx.estimate_batch_ex(dev, nt, args.seed, learned, first_traj=1 << 40)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res, _ = ctx.estimate_batch_ex(dev, nt, args.seed, learned, first_traj=(1 << 40) + T)
    e1.record(stream)
    torch.cuda.synchronize()
    t_l = e0.elapsed_time(e1) / 1e3
    ess_l = sum(r["ess"] for r in res)
    e0.record(stream)
    ess_p = 0.0
    for k, m in enumerate(dev):
        r, _ = ctx.estimate_batch_ex([m], [T], args.seed, plain, first_traj=(1 << 41) + k * T)
        ess_p += r[0]["ess"]
    e1.record(stream)
    torch.cuda.synchronize()
    t_p = e0.elapsed_time(e1) / 1e3
    model.close()
    return {"learned_batched_ess_per_s": ess_l / t_l, "plain_unbatched_ess_per_s": ess_p / t_p,
            "ratio": (ess_l / t_l) / (ess_p / t_p),
            "learned_traj_per_s": len(dev) * T / t_l, "plain_traj_per_s": len(dev) * T / t_p,
            "train": {"pairs": rep["n_pairs"], "loss_first": rep["loss_first"], "loss_last": rep["loss_last"],
                      "seconds": t_train}}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, timed as it stands on the host cores."""
    if rank != 0:
        return
    import oracle as O
    mats = G.batch_er(N_MATS, N_LO, N_HI, D_LO, D_HI, seed=GEN_SEED)
    sched = O.Schedule(**schedule_fields())
    threads = os.cpu_count() or 1
    per_step = mats[::8]  # bounded sample: 8 matrices x `threads` trajectories per step

    def step(i):
        ess = 0.0
        ntraj = 0
        for k, m in enumerate(per_step):
            P = O.Prepared(m, sched)
            r = P.run(seed=args.seed, count=threads, first_traj=i * threads, matrix=8 * k,
                      threads=threads)
            st = O.stats(r["log_x"])
            ess += st["ess"]
            ntraj += threads
        return ess, ntraj

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    tot_ess = 0.0
    tot_traj = 0
    for i in range(args.steps):
        e, n = step(args.warmup + i)
        tot_ess += e
        tot_traj += n
    dt = time.perf_counter() - t0
    val = tot_ess / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "8 of the 64 matrices (every 8th), "
                       f"{threads} trajectories each per step"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{tot_traj} trajectories over {args.steps} steps"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "traj_per_s": tot_traj / dt}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2608_15390_b300 import binding as B

    mats = G.batch_er(N_MATS, N_LO, args.nmax, D_LO, D_HI, seed=GEN_SEED)[: args.mats]
    dev = [G.Csr(m.n, torch.from_numpy(m.row_ptr).cuda(), torch.from_numpy(m.col_idx).cuda())
           for m in mats]
    pinned = [G.Csr(m.n, torch.from_numpy(m.row_ptr).pin_memory(), torch.from_numpy(m.col_idx).pin_memory())
              for m in mats]
    stream = torch.cuda.current_stream()
    ctx = B.Context(local, stream.cuda_stream)
    sched = B.Schedule(**schedule_fields())
    T = args.traj
    nt = [T] * len(mats)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(i, host=False):
        first = ((rank * 1_000_000 + i) * T) % (1 << 47)
        res, _ = ctx.estimate_batch_ex(pinned if host else dev, nt, args.seed, sched, first_traj=first)
        return res

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    tot_ess = 0.0
    tot_traj = 0
    alg_bytes = 0
    kern_ms = 0.0
    prep_ms = 0.0
    rse = []
    launches = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))  # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        res = step(args.warmup + i)
        ev[i][1].record(stream)
        info = ctx.last_call_info()
        kern_ms += info["traj_kernel_ms"]
        prep_ms += info["prep_kernel_ms"]
        launches += 4  # prepare, trajectories, stats partial, stats merge
        for r in res:
            tot_ess += r["ess"]
            tot_traj += r["n_traj"]
            alg_bytes += r["alg_bytes"]
            rse.append(r["rse"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    # e2e: the same steps through the public API from pinned host buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_ess = 0.0
    for i in range(args.steps):
        res = step(10_000 + i, host=True)
        e2e_ess += sum(r["ess"] for r in res)
    t_e2e = time.perf_counter() - t0
    info = ctx.last_call_info()
    h2d, d2h = info["h2d_bytes"], info["d2h_bytes"]

    if dist:
        t = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        s = torch.tensor([tot_ess, float(tot_traj), e2e_ess], dtype=torch.float64, device="cuda")
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        t_dev, t_e2e = float(t[0]), float(t[1])
        tot_ess, tot_traj, e2e_ess = float(s[0]), int(s[1]), float(s[2])

    value = tot_ess / t_dev
    ess_per_traj = tot_ess / max(1, tot_traj)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = (alg_bytes / args.steps) / (kern_ms / args.steps / 1e3) / 1e9
    tpb = ncu_traffic_per_byte()
    traffic = None if tpb is None else tpb * alg_bytes / args.steps
    if args.mats != N_MATS or args.nmax != N_HI:
        line_cfg_note = f"reduced case: first {args.mats} matrices, n<={args.nmax} (not a bench value)"
    else:
        line_cfg_note = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "traj_per_matrix_per_step": T,
                   "l2": "flushed between timed steps (256 MB write outside the step events)",
                   "parallelism": f"replicas{world}", "note": line_cfg_note},
        "traj_per_s": tot_traj / t_dev,
        "ess_per_traj": ess_per_traj,
        "median_rse_per_step": statistics.median(rse) if rse else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "traj_kernel<float>", "peak_source": "measured" if peaks else "fallback",
                     "kernel_ms_per_step": kern_ms / args.steps,
                     "prep_ms_per_step": prep_ms / args.steps},
        "gpu_launches": launches * world,
        "clocks": clk,
        "e2e": {"value": e2e_ess / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
    }
    if not args.no_compare:
        line["compare"] = compare_learned_vs_plain(ctx, B, dev, args, T)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mats, ess_per_traj)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
