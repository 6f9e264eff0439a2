#!/usr/bin/env python3
"""Benchmark of the batched sparse-permanent estimator on one B300.

Workload: 64 Erdos-Renyi bipartite matrices with a planted permutation,
n ~ U{100..2000}, average degree ~ U[4, 8] (generator seed 2).

A step is one whole job at fixed relative error: every matrix of the batch
estimated until its RSE (Sec. 4 "Metrics") is at most eps (default 0.1;
--eps), through the public call estimate_permanent_batch with rse_target =
eps and a time budget (default 4 s; --budget): preprocessing once (CSC
build, initial DM, outer SK), then rounds of one persistent launch over the
matrices still short of the target (consecutive trajectory ids per matrix,
statistics merged after each round).  A matrix the budget stops first is
censored: it keeps the ESS it reached, and the line counts the matrices at
target.  Steps use disjoint trajectory ids.

value: effective samples per second of the learned proposal run batched
(the metric's "learned+batched"): the Sec. 2 ESS of every matrix at its stop,
summed over the matrices and steps, over the device time of the steps (CUDA
events on the launching stream).  At a fixed RSE a matrix ends with
ESS ~ 1/eps^2, so no matrix dominates the sum.  The network is trained before
the timed region (time reported) on pairs recorded from an SK-scheduled run
on 16 training matrices of the same family (seed 7).

compare: the metric's "plain" (outer SK only) run batched and one matrix per
call, and SK(100,10)-Adaptive run batched, each as one job at the same eps and
budget; per matrix, ESS/s over its attributed device time (pm_result.dev_ms),
and the learned/arm ratios over the matrices that reached the target in both.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--eps E] [--impl ours|reference]

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
from paper_2608_15390_b300.merge import merge  # noqa: E402

METRIC = "effective samples/s at fixed rel. error, learned+batched vs plain, 1 B300"
UNIT = "effective samples/s"
N_MATS, N_LO, N_HI, D_LO, D_HI, GEN_SEED = 64, 100, 2000, 4.0, 8.0, 2
EPS = 0.1
STEP_BUDGET_S = 4.0  # device-side time budget of one job (a step)
TRAJ_CAP = 1 << 26  # per matrix and job: an upper bound the target or the budget ends first
WORKLOAD_CORE = ("64 ER+planted-permutation matrices, n~U{100..2000}, avg degree~U[4,8] "
                 "(generator seed 2); learned proposal (8-64-64-1 BF16 network) with two-sided MD, "
                 "initial DM, outer SK(100), FP32 proposal, FP64 log-weights")
WORKLOAD = (WORKLOAD_CORE + "; a step estimates every matrix to RSE <= eps within a time budget "
            "(estimate_permanent_batch with rse_target and time_budget_s: preprocessing, then rounds of one "
            "persistent launch over the unfinished matrices), layouts autotuned")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--eps", type=float, default=EPS, help="RSE target of every matrix in a job")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the comparison arms")
    p.add_argument("--budget", type=float, default=STEP_BUDGET_S,
                   help="time budget of one job (a step, and each comparison arm), seconds")
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--mats", type=int, default=N_MATS,
                   help="use the first K matrices (profiling of a smaller case)")
    p.add_argument("--study-budget", type=float, default=2.0, help="seconds per run of the e4 / theta studies")
    p.add_argument("--theta", type=float, default=0.33, help="large workload: theta of the filtering preset")
    p.add_argument("--large-preset", default="local_threshold", choices=list(PRESETS),
                   help="large workload: the filtering preset")
    p.add_argument("--skip-plain", action="store_true", help="large workload: only the filtering run")
    p.add_argument("--large-budget", type=float, default=60.0, help="large workload: seconds of the filtering run")
    p.add_argument("--train-mats", type=int, default=100, help="learned workload: training matrices (n = 1e4)")
    p.add_argument("--train-pairs", type=int, default=10_000_000, help="learned workload: training pairs")
    p.add_argument("--workload", default="batch",
                   choices=["batch", "serving", "large", "e4", "theta", "ablation", "learned", "grad"],
                   help="batch: the 64-matrix batch (the metric); serving: the Poisson request stream; "
                        "large: one n = 1e5 band matrix (state in global memory)")
    p.add_argument("--serve-seconds", type=float, default=20.0, help="arrival window of each serving load")
    p.add_argument("--serve-estimator", default="learned", choices=["learned", "local", "local_capped"],
                   help="estimator of the serving workload")
    p.add_argument("--nmax", type=int, default=N_HI,
                   help="draw n from U{100..nmax} instead (profiling of a smaller case)")
    return p.parse_args()


def schedule_fields():
    """The SK-scheduled estimator of the batched workload: two-sided MD, initial
    DM, SK(K0=100, K=10) Adaptive, no inner DM, FP32 proposal."""
    return dict(vertex_rule=0, initial_dm=1, K0=100, K=10, sk=2, dm=0, precision=0, theta=0.33)


TEACHER = dict(vertex_rule=0, initial_dm=1, K0=100, K=10, sk=1, dm=0, precision=0, theta=0.33)
LEARNED = dict(vertex_rule=0, initial_dm=1, K0=100, K=0, sk=0, dm=0, precision=0, theta=0.33)
TRAIN_SEED, N_TRAIN = 7, 16


def training_matrices():
    return [G.er_planted(m.n, 6.0, seed=7_000 + k)
            for k, m in enumerate(G.batch_er(N_TRAIN, N_LO, N_HI, D_LO, D_HI, seed=TRAIN_SEED))]


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


def ncu_traffic_per_launch(eps, n_mats):
    """DRAM bytes (read + write) per trajectory-kernel launch of this workload
    from the committed one-pass ncu capture, if it was taken on the current
    kernel source and workload (else None)."""
    path = os.path.join(ROOT, "profiles", "traj_kernel_learned_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    if d.get("eps") != eps or d.get("matrices") != n_mats:
        return None
    return d.get("dram_bytes_per_launch")


def bf16_params(p):
    a = np.asarray(p, dtype=np.float32).copy()
    u = a.view(np.uint32)
    w = ((u.astype(np.uint64) + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = a.astype(np.float64)
    for lo, hi in ((0, 512), (576, 4672), (4736, 4800)):  # weights are BF16 on the device
        out[lo:hi] = w[lo:hi].view(np.float32)
    return out


def cpu_baseline(mats, params, gpu_ess_per_traj, seconds_budget=20.0):
    """The oracle as it stands (the learned proposal computed on the CPU with
    the same network), on the host cores, on a bounded sample of the same
    workload: every 4th matrix, one trajectory per host thread per round,
    until about `seconds_budget` of CPU work; reported as effective samples/s
    through the GPU run's effective samples per trajectory (same estimator)."""
    import oracle as O
    sched = O.Schedule(**LEARNED)
    threads = os.cpu_count() or 1
    sample = mats[::4]
    preps = [O.Prepared(m, sched) for m in sample]
    t0 = time.perf_counter()
    done = rounds = 0
    while True:
        for k, P in enumerate(preps):
            P.run_model(seed=99, count=threads, params=params, first_traj=rounds * threads, matrix=4 * k,
                        threads=threads)
            done += threads
        rounds += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    dt = time.perf_counter() - t0
    tps = done / dt
    return {"value": tps * gpu_ess_per_traj, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{done} learned-proposal trajectories ({threads} per matrix per round, {rounds} "
                      f"rounds) on matrices 0,4,...,60 of the workload, {dt:.1f} s, preprocessing "
                      f"excluded; {tps:.2f} traj/s x the GPU jobs' effective samples per trajectory"}


def timed(ctx, stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def job_summary(res, t_job):
    """A job's figures from its per-matrix results and device time t_job:
    effective samples (Sec. 2 ESS at each matrix's stop), trajectories, and
    per matrix its attributed device time (pm_result.dev_ms), ESS and
    whether it stopped at the RSE target."""
    return {"ess": float(sum(r["ess"] for r in res)), "traj": int(sum(r["n_traj"] for r in res)),
            "t_k": np.array([r["dev_ms"] / 1e3 for r in res]), "ess_k": np.array([r["ess"] for r in res]),
            "rse_k": np.array([r["rse"] for r in res]), "met_k": np.array([r["stop"] == 1 for r in res]),
            "rounds": int(max(r["rounds"] for r in res)), "met": int(sum(r["stop"] == 1 for r in res)),
            "t_job": t_job}


def arm_figures(js):
    """An arm's job at eps: its ESS/s over the whole job, over the matrices
    that reached the target, and the count of matrices the budget stopped."""
    m = js["met_k"]
    return {"ess_per_s": js["ess"] / js["t_job"], "job_seconds": js["t_job"], "matrices_at_target": int(m.sum()),
            "ess_per_s_at_target": float(js["ess_k"][m].sum() / js["t_k"][m].sum()) if m.any() else None,
            "traj_per_s": js["traj"] / js["t_job"], "median_rse": float(np.nanmedian(js["rse_k"]))}


def compare_arms(ctx, B, dev, args, learned):
    """The metric's "plain" (outer SK only) run batched and one matrix per
    call, and SK(100,10)-Adaptive batched, each one job at the same eps and
    time budget as a learned step (one matrix per call: 1/64 of the budget
    each); per-matrix ratios of ESS/s over the matrices that reached the
    target in both arms."""
    import torch
    stream = torch.cuda.current_stream()
    first = (1 << 44)
    out = {}
    arms = {"plain_batched": B.Schedule(**LEARNED, rse_target=args.eps, time_budget_s=args.budget),
            "adaptive_sk_batched": B.Schedule(**schedule_fields(), rse_target=args.eps, time_budget_s=args.budget)}
    for name, sched in arms.items():
        (res, _), dt = timed(ctx, stream, lambda: ctx.estimate_batch_ex(dev, [TRAJ_CAP] * len(dev), args.seed, sched,
                                                                       first_traj=first))
        out[name] = job_summary(res, dt)
        print(f"compare {name}: {dt:.2f} s, {out[name]['met']} at target", file=sys.stderr, flush=True)
    sched = B.Schedule(**LEARNED, rse_target=args.eps, time_budget_s=args.budget / len(dev))
    res_u, t_u = [], 0.0
    for k, m in enumerate(dev):
        (r, _), dt = timed(ctx, stream, lambda: ctx.estimate_batch_ex([m], [TRAJ_CAP], args.seed, sched,
                                                                     first_traj=first + k))
        res_u.append(r[0])
        t_u += dt
    out["plain_unbatched"] = job_summary(res_u, t_u)
    print(f"compare plain_unbatched: {t_u:.2f} s", file=sys.stderr, flush=True)
    cmp = {}
    lr = learned["ess_k"] / learned["t_k"]
    for name, js in out.items():
        cmp[name] = arm_figures(js)
        both = learned["met_k"] & js["met_k"]
        cmp[name]["matrices_at_target_in_both"] = int(both.sum())
        if both.any():
            ratio = lr[both] / (js["ess_k"][both] / js["t_k"][both])
            cmp[name]["learned_vs_this_per_matrix_median"] = float(np.median(ratio))
            cmp[name]["learned_vs_this_per_matrix_geomean"] = float(np.exp(np.mean(np.log(ratio))))
    return cmp


def oracle_train(seed=5, pairs=40000, steps=300, batch=512, lr=2e-3):
    """The network trained by the oracle alone: pairs recorded by the oracle
    from the SK-scheduled teacher on 4 training matrices, Adam on the FP64
    gradient of the per-step centred loss over minibatches of whole steps."""
    import oracle as O
    mats = training_matrices()[:4]
    feats, targs, grps = [], [], []
    for k, m in enumerate(mats):
        f, t, _, g = O.Prepared(m, O.Schedule(**TEACHER)).record(seed=seed, count=2, cap=pairs // 4, matrix=k)
        feats.append(f)
        targs.append(t)
        grps.append(g)
    X = np.concatenate(feats).astype(np.float64)
    Y = np.concatenate(targs).astype(np.float64)
    Gc = np.concatenate(grps)
    starts = np.nonzero((Gc >> 16) == 0)[0]
    sizes = (Gc[starts] & 0xFFFF).astype(np.int64)
    rng = np.random.default_rng(seed)
    p = np.zeros(O.N_PARAM)
    p[:512] = rng.normal(size=512) * np.sqrt(2 / 8)
    p[576:4672] = rng.normal(size=4096) * np.sqrt(2 / 64)
    p[4736:4800] = rng.normal(size=64) * np.sqrt(1 / 64)
    p[4800] = Y.mean()
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    per_batch = max(1, int(batch / sizes.mean()))
    for it in range(1, steps + 1):
        pick = rng.integers(0, len(starts), size=per_batch)
        idx = np.concatenate([np.arange(starts[q], starts[q] + sizes[q]) for q in pick])
        _, g = O.mlp_grad(p, X[idx], Y[idx], Gc[idx])
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        p -= lr * (m1 / (1 - 0.9 ** it)) / (np.sqrt(m2 / (1 - 0.999 ** it)) + 1e-8)
    return bf16_params(p.astype(np.float32))


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands on the host cores, running
    the learned proposal (network trained by the oracle itself, untimed) as
    the GPU arm's jobs do, on a bounded sample of the workload (every 8th
    matrix): a step runs rounds of trajectories over the sampled matrices
    still short of RSE <= eps (at least 1024 trajectories) until all reach it
    or the step's time budget ends; value = the sampled matrices' ESS at their
    stop, summed over the steps, over the CPU time of the steps."""
    if rank != 0:
        return
    import oracle as O
    mats = G.batch_er(N_MATS, N_LO, N_HI, D_LO, D_HI, seed=GEN_SEED)
    t0 = time.perf_counter()
    params = oracle_train()
    t_train = time.perf_counter() - t0
    sched = O.Schedule(**LEARNED)
    threads = os.cpu_count() or 1
    sample = list(range(0, N_MATS, 8))
    preps = [O.Prepared(mats[k], sched) for k in sample]
    per = 4 * threads

    def job(i):
        t_start = time.perf_counter()
        logs = [[] for _ in sample]
        done = [False] * len(sample)
        rnd = 0
        while not all(done) and time.perf_counter() - t_start < args.budget:
            for q, (k, P) in enumerate(zip(sample, preps)):
                if done[q]:
                    continue
                first = (i << 30) + rnd * per
                logs[q].append(P.run_model(seed=args.seed, count=per, params=params, first_traj=first, matrix=k,
                                           threads=threads)["log_x"])
                st = O.stats(np.concatenate(logs[q]))
                done[q] = st["n_traj"] >= 1024 and st["n_alive"] >= 2 and st["rse"] <= args.eps
            rnd += 1
        sts = [O.stats(np.concatenate(lx)) for lx in logs]
        return sum(st["ess"] for st in sts), sum(st["n_traj"] for st in sts), sum(done), \
            time.perf_counter() - t_start

    for i in range(args.warmup):
        job(i)
    tot_ess = tot_traj = 0
    met = []
    dt = 0.0
    for i in range(args.steps):
        e, n, d, t = job(args.warmup + i)
        tot_ess += e
        tot_traj += n
        met.append(d)
        dt += t
    val = tot_ess / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_CORE + "; the CPU oracle on the host cores", "eps": args.eps,
                       "step_budget_s": args.budget,
                       "sample": f"8 of the 64 matrices (every 8th), rounds of {per} trajectories per "
                                 "unfinished matrix, preprocessing excluded",
                       "matrices_at_target_mean": float(np.mean(met)),
                       "network": f"trained by the oracle ({t_train:.1f} s, untimed)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{tot_traj} learned-proposal trajectories over {args.steps} steps"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "traj_per_s": tot_traj / dt}
    print(json.dumps(line), flush=True)


SERVE_N_LO, SERVE_N_HI, SERVE_SEED, SERVE_RSE = 50, 50_000, 5, 1e-2
SERVE_MAX_STEPS = 1 << 26  # work budget of a request: trajectory steps (n per trajectory)


def serve_budget(m):
    """trajectories a request may use: 2^26 steps, between 1024 and 2^16"""
    return int(min(1 << 16, max(1024, SERVE_MAX_STEPS // m.n)))


def serving_request(i):
    """Request i of the serving stream: n = floor(exp U[ln 50, ln 5e4]), power-law
    row degrees (exponent 2.5, minimum 2), planted permutation."""
    rng = np.random.default_rng([SERVE_SEED, i])
    n = int(math.exp(rng.uniform(math.log(SERVE_N_LO), math.log(SERVE_N_HI))))
    return G.powerlaw_planted(n, seed=SERVE_SEED * 1_000_003 + i)


def run_serving(args, local):
    """The serving configuration: a capacity run (all requests present at
    once), then Poisson arrivals at 0.3 / 0.6 / 0.9 of that capacity for
    --serve-seconds each; every request asks for RSE <= 1e-2 with a work
    budget of 2^26 trajectory steps (1024 to 2^16 trajectories); latency =
    finish time - arrival time on the server
    clock.  The learned proposal is trained first (untimed) on power-law
    matrices of the same family."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    model = None
    if args.serve_estimator == "learned":
        model = ctx.model(seed=21)
        train = [G.powerlaw_planted(n, seed=900 + k) for k, n in enumerate(np.geomspace(50, 3000, 16).astype(int))]
        model.train(train, B.Schedule(**TEACHER), n_pairs=1_000_000, epochs=4, batch=8192, lr=2e-3, seed=22,
                    objective=B.OBJ_CENTRED)
        sched = B.Schedule(**LEARNED, learned=model)
    else:  # Local SK repair after every step (no inner DM), exact or with the bounded-work cap
        sched = B.Schedule(initial_dm=1, K0=100, K=10, sk=B.SK_LOCAL, dm=B.DM_NONE, precision=B.PREC_FP32_PROPOSAL,
                           local_cap=32 if args.serve_estimator == "local_capped" else 0)

    def make_server():
        return ctx.server(sched, seed=args.seed, device_budget_bytes=32 << 30, steps_per_round=1 << 22,
                          traj_min=32, traj_max=1 << 15, min_traj_done=1024)

    def summarise(done, arrivals, t_span):
        lat = np.array([d["done_time"] - arrivals[d["id"]] for d in done])
        ok = [d for d in done if d["status"] == B.REQ_DONE]
        return {"requests": len(done), "throughput_req_per_s": len(done) / t_span,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "target_met_frac": len(ok) / max(1, len(done)),
                "budget_spent_frac": sum(d["status"] == B.REQ_BUDGET for d in done) / max(1, len(done)),
                "median_rse": float(np.median([d["result"]["rse"] for d in done if d["result"]["n_alive"] > 1]))}

    # capacity: 48 requests present at once, served to completion
    reqs = [serving_request(i) for i in range(48)]
    sv = make_server()
    arrivals = {}
    for m in reqs:
        arrivals[sv.submit(m, SERVE_RSE, serve_budget(m))] = sv.clock()
    t_start = sv.clock()
    done = []
    while len(done) < len(reqs):
        out, _, _ = sv.round()
        done += out
    t_cap = sv.clock() - t_start
    capacity = len(reqs) / t_cap
    cap_line = summarise(done, arrivals, t_cap)
    sv.close()
    loads = []
    for frac in (0.3, 0.6, 0.9):
        rate = frac * capacity
        rng = np.random.default_rng([SERVE_SEED, int(frac * 10)])
        times = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * args.serve_seconds * 2) + 8))
        times = times[times < args.serve_seconds]
        base = 10_000 * int(frac * 10)
        pending = [(t, serving_request(base + i)) for i, t in enumerate(times)]
        sv = make_server()
        t0 = sv.clock()
        arrivals, done, nxt = {}, [], 0
        while nxt < len(pending) or len(done) < len(pending):
            now = sv.clock() - t0
            while nxt < len(pending) and pending[nxt][0] <= now:
                arrivals[sv.submit(pending[nxt][1], SERVE_RSE, serve_budget(pending[nxt][1]))] = t0 + pending[nxt][0]
                nxt += 1
            out, na, nq = sv.round()
            done += out
            if na == 0 and nq == 0 and nxt < len(pending):
                time.sleep(max(0.0, min(0.05, pending[nxt][0] - (sv.clock() - t0))))
        t_span = sv.clock() - t0
        line = summarise(done, arrivals, t_span)
        line.update({"load": frac, "arrival_rate_req_per_s": rate, "arrivals": len(pending)})
        loads.append(line)
        sv.close()
    if model is not None:
        model.close()
    out = {"metric": "serving: p50 / p99 latency and throughput at RSE <= 1e-2", "workload": "serving",
           "config": {"requests": "n = floor(exp U[ln 50, ln 5e4]), power-law rows (2.5, min 2) + planted "
                                  "permutation, RSE target 1e-2, budget 2^26 trajectory steps each "
                                  "(1024 to 2^16 trajectories)",
                      "estimator": {"learned": "learned proposal, two-sided MD, initial DM, outer SK(100)",
                                    "local": "Local SK repair after every step (Eq. 5, exact), initial DM, "
                                             "outer SK(100), no inner DM",
                                    "local_capped": "the same with the bounded-work Local repair, cap 32"
                                    }[args.serve_estimator],
                      "admission": "device bytes of admitted requests <= 32 GiB, first come first served",
                      "arrival_window_s": args.serve_seconds},
           "capacity_req_per_s": capacity, "capacity_run": cap_line, "loads": loads, "data": "synthetic"}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_large(args, local):
    """The large sparse configuration: n = 1e5, width-3 band (|i-j| <= 1) plus a
    planted permutation plus uniform off-band entries up to m = 5e5 (generator
    seed 3).  Each trajectory's degrees and tree live in global memory (the
    group's slot).  Two estimators:
      plain             two-sided MD, initial DM, outer SK(100): --steps waves
                        of one trajectory per group slot of the GPU (a resident
                        batch replayed from a CUDA graph);
      local_threshold   the filtering schedule of Sec. 3.3 (Local SK repair,
                        Thrs DM at theta = --theta) on a time budget of
                        --large-budget seconds, up to 2^20 trajectories: a
                        16-warp group per trajectory shares each DM call's
                        component step.
    Each line reports trajectories, p_match, RSE, ESS and the algorithmic
    bytes against the measured HBM copy peak."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    m = G.band_random(100_000, 500_000, seed=3)
    dev = G.Csr(m.n, torch.from_numpy(m.row_ptr).cuda(), torch.from_numpy(m.col_idx).cuda())
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6400.0
    matrix = ("n=1e5, |i-j|<=1 band + planted permutation + uniform off-band entries to m=5e5 (generator seed 3)")
    out = []
    # plain
    sched = B.Schedule(**LEARNED)
    if args.skip_plain:
        args.steps = 0
    props = torch.cuda.get_device_properties(local)
    T = props.multi_processor_count * 16
    bt = ctx.batch([dev], [T], sched, graph=True, autotune=False)
    bt.run(0, args.seed)  # warm-up (and the one-time preprocessing timing)
    prep_ms = ctx.last_call_info()["prep_kernel_ms"]
    runs, kern, alg = [], 0.0, 0
    for i in range(args.steps):
        res, _ = bt.run((i + 1) * T, args.seed)
        kern += ctx.last_call_info()["traj_kernel_ms"]
        runs.append(res[0])
        alg += res[0]["alg_bytes"]
    plan = bt.plan(0)
    bt.close()
    if runs:
        mrg = merge(runs)
        ach = alg / (kern / 1e3) / 1e9
        out.append({"estimator": "plain: two-sided MD, initial DM, outer SK(100)", "layout": plan,
                    "traj": mrg["n_traj"], "traj_per_s": mrg["n_traj"] / (kern / 1e3), "p_match": mrg["p_match"],
                    "rse": mrg["rse"], "ess": mrg["ess"], "prep_ms": prep_ms, "kernel_s": kern / 1e3,
                    "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": ach / hbm_peak}})
        print(f"plain: {mrg['n_traj']} trajectories, p_match {mrg['p_match']}", file=sys.stderr, flush=True)
    # the filtering schedule on a time budget
    s = B.preset(args.large_preset)
    s.theta = args.theta
    s.time_budget_s = args.large_budget
    t0 = time.perf_counter()
    r = ctx.estimate_batch_ex([dev], [1 << 20], args.seed, s, first_traj=1 << 30)[0][0]
    wall = time.perf_counter() - t0
    info = ctx.last_call_info()
    ks = info["traj_kernel_ms"] / 1e3
    ach = r["alg_bytes"] / ks / 1e9 if ks > 0 else 0.0
    out.append({"estimator": f"{args.large_preset} (theta {args.theta}), time budget {args.large_budget} s",
                "traj": r["n_traj"], "status": r["status"], "stop": r["stop"],
                "traj_per_s": r["n_traj"] / ks if ks > 0 else None, "p_match": r["p_match"], "rse": r["rse"],
                "ess": r["ess"], "log_estimate": r["log_estimate"],
                "dm_calls_per_traj": r["n_dm_calls"] / max(1, r["n_traj"]),
                "local_repairs_per_traj": r["n_local_sk"] / max(1, r["n_traj"]), "kernel_s": ks, "wall_s": wall,
                "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                             "frac": ach / hbm_peak}})
    print(f"{args.large_preset}: {r['n_traj']} trajectories, p_match {r['p_match']}", file=sys.stderr, flush=True)
    line = {"metric": "n = 1e5 band matrix: plain and filtering estimators", "workload": "large", "data": "synthetic",
            "config": {"matrix": matrix, "peak_source": "measured copy (MEASURED_PEAKS.json)" if peaks else "fallback",
                       "bytes": "algorithmic, counted per trajectory on the device (pm_result.alg_bytes)"},
            "runs": out}
    print(json.dumps(line), flush=True)
    ctx.close()


PRESETS = ("fixed_all", "adaptive_threshold", "local_threshold", "adaptive_tracked", "local_tracked")


# the E4 study's grid (as tests/golden/make_e4_log_permanents.py): order,
# deletion probability, weights; generator seed 4000 + index
E4_GRID = [(n, p, w) for n in (100, 500, 1000, 2000) for p in (0.1, 0.5, 0.9) for w in (False, True)]


def e4_matrices(with_permanents=True):
    """The E4 study's block-diagonal matrices (Sec. 4 known-permanent family),
    with their exact ln per(A) as stored by
    tests/golden/make_e4_log_permanents.py when with_permanents."""
    pers = {}
    if with_permanents:
        d = json.load(open(os.path.join(ROOT, "tests", "golden", "e4_log_permanents.json")))
        pers = {r["index"]: r for r in d["matrices"]}
    out = []
    for i, (n, p, w) in enumerate(E4_GRID):
        m = G.block_diagonal(n, p, seed=4000 + i, weighted=w)
        info = {"index": i, "n": n, "p": p, "weighted": w, "seed": 4000 + i}
        if with_permanents:
            assert pers[i]["nnz"] == m.nnz and pers[i]["n"] == n
            info["log_per"] = pers[i]["log_per"]
        out.append((info, m))
    return out


def budget_run(ctx, B, m, sched, budget, seed, first=0, cap=1 << 22):
    """One estimate of m on a time budget (the paper's runs stop at a time
    cap, Sec. 4): the trajectories started within `budget` seconds."""
    sched.time_budget_s = budget
    t0 = time.perf_counter()
    r = ctx.estimate_permanent_batch([m], [cap], seed, sched)[0] if first == 0 else \
        ctx.estimate_batch_ex([m], [cap], seed, sched, first_traj=first)[0][0]
    r["wall_s"] = time.perf_counter() - t0
    return r


def run_e4(args, local):
    """NEXT-1: the five presets of Sec. 4 on the known-permanent block-diagonal
    family (binary and U[1, 1.5] weights, n in {100, 500, 1000, 2000},
    deletion probability p in {0.1, 0.5, 0.9}) with equal GPU-time budgets,
    FP32 proposal.  Per preset: trajectories in the budget, RSE, p_match,
    the realised relative error against the exact permanent, and the trend
    of the local_threshold / fixed_all trajectory ratio with p (Table 2 and
    the discussion of Figs. 4-5)."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    mats = e4_matrices()
    rows = []
    for name in PRESETS:
        for info, m in mats:
            r = budget_run(ctx, B, m, B.preset(name), args.study_budget, args.seed)
            le = r["log_estimate"]
            err = abs(math.expm1(le - info["log_per"])) if le > -math.inf else 1.0
            rows.append({"preset": name, "n": info["n"], "p": info["p"], "weighted": info["weighted"],
                         "traj": r["n_traj"], "rse": r["rse"], "p_match": r["p_match"], "rel_err": err,
                         "within_3rse": bool(err <= 3 * r["rse"]) if r["rse"] == r["rse"] else False,
                         "dm_per_traj": r["n_dm_calls"] / max(1, r["n_traj"]),
                         "sk_iter_per_traj": r["n_full_sk"] / max(1, r["n_traj"]),
                         "local_per_traj": r["n_local_sk"] / max(1, r["n_traj"])})
    summary = {}
    for name in PRESETS:
        rs = [x for x in rows if x["preset"] == name]
        summary[name] = {"median_traj": float(np.median([x["traj"] for x in rs])),
                         "median_rse": float(np.nanmedian([x["rse"] for x in rs])),
                         "min_p_match": float(min(x["p_match"] for x in rs)),
                         "median_rel_err": float(np.median([x["rel_err"] for x in rs])),
                         "within_3rse": sum(x["within_3rse"] for x in rs), "runs": len(rs)}
    by_p = {}
    for p in (0.1, 0.5, 0.9):
        ratio = [l["traj"] / max(1, f["traj"]) for l in rows if l["preset"] == "local_threshold" and l["p"] == p
                 for f in rows if f["preset"] == "fixed_all" and f["p"] == p and f["n"] == l["n"]
                 and f["weighted"] == l["weighted"]]
        by_p[str(p)] = float(np.median(ratio))
    out = {"workload": "e4", "metric": "five presets on equal GPU-time budgets, known-permanent family",
           "config": {"budget_s_per_run": args.study_budget, "matrices": len(mats),
                      "grid": "n in {100,500,1000,2000} x p in {0.1,0.5,0.9} x {binary, U[1,1.5]} "
                              "(generator seeds 4000+i)", "precision": "FP32 proposal, FP64 log-weights"},
           "summary": summary, "local_threshold_over_fixed_all_traj_by_p": by_p, "runs": rows,
           "data": "synthetic"}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_theta(args, local):
    """NEXT-2: sensitivity of the Thrs and Trck DM policies to theta (the
    paper leaves Trck's open, Sec. 4): the four adaptive / local presets with
    theta in {0.1, 0.2, 0.33, 0.5, 0.7, 0.9} on a time budget each, on three
    E4 matrices (n = 1000, binary, p = 0.1 / 0.5 / 0.9) and two ER+planted
    matrices (n = 500 / 1000, d = 6).  Figure of merit: the work-normalised
    relative variance RSE^2 x seconds (lower is better; ESS/s ~ 1/that)."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    mats = [(f"e4 n=1000 p={i['p']}", m) for i, m in e4_matrices(False) if i["n"] == 1000 and not i["weighted"]]
    mats += [(f"er n={n} d=6", G.er_planted(n, 6.0, seed=3100 + n)) for n in (500, 1000)]
    thetas = (0.1, 0.2, 0.33, 0.5, 0.7, 0.9)
    rows = []
    for name in ("adaptive_threshold", "local_threshold", "adaptive_tracked", "local_tracked"):
        for label, m in mats:
            for th in thetas:
                s = B.preset(name)
                s.theta = th
                r = budget_run(ctx, B, m, s, args.study_budget, args.seed)
                wv = r["rse"] ** 2 * r["wall_s"] if r["rse"] == r["rse"] else math.inf
                rows.append({"preset": name, "matrix": label, "theta": th, "traj": r["n_traj"], "rse": r["rse"],
                             "p_match": r["p_match"], "dm_per_traj": r["n_dm_calls"] / max(1, r["n_traj"]),
                             "work_norm_var": wv})
    best = {}
    for name in ("adaptive_threshold", "local_threshold", "adaptive_tracked", "local_tracked"):
        for label, _ in mats:
            rs = [x for x in rows if x["preset"] == name and x["matrix"] == label]
            b = min(rs, key=lambda x: x["work_norm_var"])
            ref = [x for x in rs if x["theta"] == 0.33][0]
            best[f"{name} | {label}"] = {"best_theta": b["theta"],
                                         "gain_vs_0.33": ref["work_norm_var"] / b["work_norm_var"]
                                         if b["work_norm_var"] > 0 else None}
    out = {"workload": "theta", "metric": "RSE^2 x seconds per (preset, matrix, theta); lower is better",
           "config": {"budget_s_per_run": args.study_budget, "thetas": thetas}, "best": best, "runs": rows,
           "data": "synthetic"}
    print(json.dumps(out), flush=True)
    ctx.close()


def first_infeasible_steps(m, chosen):
    """For each traced path, the first step whose child (the residual after
    removing the chosen pair) has no perfect matching, or -1 (Sec. 2: a
    residual without a perfect matching contributes X = 0).  A perfect
    matching of the residual is kept and repaired after each elimination by
    one alternating breadth-first search (host code)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_bipartite_matching
    n = m.n
    rp, ci = np.asarray(m.row_ptr), np.asarray(m.col_idx)
    A = csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    base = maximum_bipartite_matching(A, perm_type="column")  # row i -> its column
    out = []
    for path in chosen:
        mr = base.copy()
        mc = np.full(n, -1)
        mc[mr] = np.arange(n)
        arow = np.ones(n, bool)
        acol = np.ones(n, bool)
        bad = -1
        for t, (v, u) in enumerate(path):
            if v < 0:
                break
            R, Cc = (v, u - n) if v < n else (u, v - n)
            arow[R] = False
            acol[Cc] = False
            if mr[R] == Cc:
                continue
            c_free, r_free = mr[R], mc[Cc]  # their partners lose them
            mc[c_free] = -1
            mr[r_free] = -1
            par = {}
            frontier, found = [r_free], False
            while frontier and not found:
                nxt = []
                for i in frontier:
                    for j in ci[rp[i]:rp[i + 1]]:
                        if not acol[j] or j in par:
                            continue
                        par[j] = i
                        if j == c_free:
                            found = True
                            break
                        nxt.append(mc[j])
                    if found:
                        break
                frontier = nxt
            if not found:
                bad = t
                break
            j = c_free
            while True:  # flip the alternating path
                i = par[j]
                nj = mr[i]
                mr[i] = j
                mc[j] = i
                if i == r_free:
                    break
                j = nj
        out.append(bad)
    return out


def run_ablation(args, local):
    """NEXT-4: the row-order vertex rule of Alg. 1 against the two-sided
    minimum-degree rule (Sec. 3.2, Fig. 2) on ER+planted matrices and E4
    matrices, plain (outer SK only) and SK(100,10) Adaptive without inner DM,
    1000 trajectories each (p_match and relative spread, as the paper's
    sphere3 / Trefethen comparison); and the z-bucket histogram of the first
    infeasible child along plain two-sided-MD paths (z = r_v c_u of the
    chosen edge from the outer scaling)."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    mats = [(f"er n={n} d=6", G.er_planted(n, 6.0, seed=3200 + n)) for n in (200, 500, 1000)]
    mats += [(f"e4 n={i['n']} p={i['p']}", m) for i, m in e4_matrices(False)
             if i["n"] == 500 and not i["weighted"]]
    rows = []
    for label, m in mats:
        for sk_name, sk in (("plain", B.SK_NONE), ("adaptive_sk", B.SK_ADAPTIVE)):
            for vr_name, vr in (("row_order", B.VR_ROW_ORDER), ("two_sided_md", B.VR_MIN_DEGREE_2SIDED)):
                s = B.Schedule(vertex_rule=vr, initial_dm=1, K0=100, K=10, sk=sk, precision=B.PREC_FP32_PROPOSAL)
                t0 = time.perf_counter()
                r = ctx.estimate_permanent(m, 1000, args.seed, s)
                rows.append({"matrix": label, "schedule": sk_name, "vertex_rule": vr_name,
                             "p_match": r["p_match"], "rel_spread": r["rel_spread"],
                             "traj_per_s": 1000 / (time.perf_counter() - t0)})
    # z-bucket histogram of infeasible children (plain two-sided MD, outer SK)
    edges = np.linspace(0, 1, 11)
    steps = np.zeros(11)
    fails = np.zeros(11)
    s = B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL)
    for label, m in mats:
        if m.n > 500:
            continue
        pre = ctx.preprocess(m, s)
        r0, c0 = pre["r"], pre["c"]
        tr = ctx.trace(m, 100, args.seed, s)
        bad = first_infeasible_steps(m, tr["chosen"])
        for q in range(100):
            for t in range(m.n):
                v, u = tr["chosen"][q, t]
                if v < 0:
                    break
                R, Cc = (v, u - m.n) if v < m.n else (u, v - m.n)
                z = float(np.float32(r0[R]) * np.float32(c0[Cc]))
                b = min(10, int(z * 10))
                steps[b] += 1
                if t == bad[q]:
                    fails[b] += 1
                    break
    hist = [{"z_lo": float(edges[b]) if b < 10 else 1.0, "steps": int(steps[b]), "first_infeasible": int(fails[b]),
             "rate": float(fails[b] / steps[b]) if steps[b] else None} for b in range(11)]
    out = {"workload": "ablation", "metric": "p_match and relative spread: row order vs two-sided MD; "
           "z-bucket rate of first infeasible children", "vertex_rule": rows, "z_histogram": hist,
           "config": {"trajectories": 1000, "histogram": "100 traced plain two-sided-MD paths per matrix "
                      "with n <= 500; bucket 10 holds z >= 1"}, "data": "synthetic"}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_learned_scale(args, local):
    """Configuration 4 at its stated scale: the learned proposal trained on
    pairs recorded from the SK(100,10) Fixed teacher on 100 ER+planted
    matrices (n = 1e4, d = 6, generator seeds 1000-1099), evaluated on
    held-out seeds (2000+) at n = 1e4 and n = 1e5 against the plain estimator
    (outer SK only, same vertex rule), each matrix run to RSE <= eps within a
    time budget through estimate_permanent (rse_target, time_budget_s)."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    train = [G.er_planted(10_000, 6.0, seed=1000 + k) for k in range(args.train_mats)]
    model = ctx.model(seed=31)
    t0 = time.perf_counter()
    rep = model.train(train, B.Schedule(**TEACHER), n_pairs=args.train_pairs, epochs=2, batch=8192, lr=2e-3,
                      seed=32, objective=B.OBJ_CENTRED)
    t_train = time.perf_counter() - t0
    print(f"trained on {rep['n_pairs']} pairs in {t_train:.1f} s", file=sys.stderr, flush=True)
    rows = []
    for n, count in ((10_000, 4), (100_000, 2)):
        for q in range(count):
            m = G.er_planted(n, 6.0, seed=2000 + q + (100 if n > 10_000 else 0))
            for arm, s in (("plain", B.Schedule(**LEARNED)), ("learned", B.Schedule(**LEARNED, learned=model))):
                s.rse_target = args.eps
                s.time_budget_s = args.study_budget
                r = ctx.estimate_batch_ex([m], [TRAJ_CAP], args.seed, s)[0][0]
                t = r["dev_ms"] / 1e3
                rows.append({"n": n, "matrix_seed": 2000 + q + (100 if n > 10_000 else 0), "arm": arm,
                             "traj": r["n_traj"], "p_match": r["p_match"], "rse": r["rse"], "ess": r["ess"],
                             "device_s": t, "ess_per_s": r["ess"] / t if t > 0 else None,
                             "at_target": r["stop"] == 1, "traj_per_s": r["n_traj"] / t if t > 0 else None})
                print(f"n={n} #{q} {arm}: {r['n_traj']} traj, p_match {r['p_match']:.3f}, rse {r['rse']:.3g}",
                      file=sys.stderr, flush=True)
    ratios = {}
    for n in (10_000, 100_000):
        rs = []
        for q in range(4):
            a = [x for x in rows if x["n"] == n and x["matrix_seed"] % 100 == q and x["arm"] == "learned"]
            b = [x for x in rows if x["n"] == n and x["matrix_seed"] % 100 == q and x["arm"] == "plain"]
            if a and b and a[0]["ess_per_s"] and b[0]["ess_per_s"]:
                rs.append(a[0]["ess_per_s"] / b[0]["ess_per_s"])
        ratios[str(n)] = {"learned_vs_plain_ess_per_s": rs, "median": float(np.median(rs)) if rs else None}
    out = {"workload": "learned", "metric": "effective samples/s at fixed RSE (budgeted), learned vs plain",
           "config": {"train": f"{args.train_mats} ER+planted matrices n=1e4 d=6 (seeds 1000+), teacher "
                               "SK(100,10) Fixed, per-step centred loss, 2 epochs, batch 8192",
                      "eval": "held-out ER+planted d=6: 4 at n=1e4 (seeds 2000-2003), 2 at n=1e5 (seeds 2100-2101)",
                      "eps": args.eps, "budget_s_per_run": args.study_budget},
           "train": {"pairs": rep["n_pairs"], "seconds": t_train, "record_s": rep["seconds_record"],
                     "train_s": rep["seconds_train"], "loss_first": rep["loss_first"], "loss_last": rep["loss_last"]},
           "ratios": ratios, "runs": rows, "data": "synthetic"}
    print(json.dumps(out), flush=True)
    model.close()
    ctx.close()


def run_grad(args, local):
    """The learned proposal's training gradient (the tcgen05 kernel, with the
    residual pass and the fixed-order reduction) on synthetic rows: standard-
    normal features and targets, mean squared error, B = 8,192 (one training
    batch), 2^20 and 2^22 rows.  Device time of the kernels per call
    (pm_call_info.grad_kernel_ms, median of the calls) against the bf16 tensor
    peak, at 3 x 9,344 flop per row (the 8-64-64-1 network's forward and the
    two backward products)."""
    import torch
    from paper_2608_15390_b300 import binding as B
    torch.cuda.set_device(local)
    ctx = B.Context(local, torch.cuda.current_stream().cuda_stream)
    model = ctx.model(seed=1)
    peaks = measured_peaks()
    tc_peak = peaks["bf16_tflops"] if peaks else 1800.0
    rng = np.random.default_rng(0)
    out = []
    for n in (8192, 1 << 20, 1 << 22):
        X = rng.normal(size=(n, 8)).astype(np.float32)
        T = rng.normal(size=n).astype(np.float32)
        model.gradient(X, T)
        ms = []
        for _ in range(max(3, args.steps)):
            model.gradient(X, T)
            ms.append(ctx.last_call_info()["grad_kernel_ms"])
        med = float(np.median(ms))
        tflops = 3 * 9344 * n / (med * 1e-3) / 1e12
        out.append({"rows": n, "kernel_ms": med, "rows_per_s": n / (med * 1e-3), "tflops": tflops,
                    "frac_of_bf16_peak": tflops / tc_peak})
        print(f"rows {n}: {med:.3f} ms, {tflops:.1f} TFLOP/s", file=sys.stderr, flush=True)
    print(json.dumps({"workload": "grad", "metric": "training-gradient rows/s (device time)", "runs": out,
                      "peak": {"bf16_tflops": tc_peak,
                               "source": "measured (MEASURED_PEAKS.json)" if peaks else "fallback"},
                      "data": "synthetic"}), flush=True)
    model.close()
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serving":
        if rank == 0:
            run_serving(args, local)
        return
    if args.workload == "large":
        if rank == 0:
            run_large(args, local)
        return
    if args.workload in ("e4", "theta", "ablation", "learned", "grad"):
        if rank == 0:
            {"e4": run_e4, "theta": run_theta, "ablation": run_ablation,
             "learned": run_learned_scale, "grad": run_grad}[args.workload](args, local)
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
    bw = ctx.probe_bandwidth()
    model = ctx.model(seed=11)
    t0 = time.perf_counter()
    train_rep = model.train(training_matrices(), B.Schedule(**TEACHER), n_pairs=2_000_000, epochs=4,
                            batch=8192, lr=2e-3, seed=12, objective=B.OBJ_CENTRED)
    t_train = time.perf_counter() - t0
    sched = B.Schedule(**LEARNED, learned=model, rse_target=args.eps, time_budget_s=args.budget)
    nt = [TRAJ_CAP] * len(mats)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # layouts: the autotuner times each size class once and caches its choice
    # in the context, where every later call of the same schedule finds it
    t0 = time.perf_counter()
    tb = ctx.batch(dev, [1024] * len(mats), B.Schedule(**LEARNED, learned=model), graph=False, autotune=True)
    plans = [tb.plan(k) for k in range(len(mats))]
    tb.close()
    t_tune = time.perf_counter() - t0

    def job(i, host=False):
        first = ((rank * 4096 + i) << 30) % (1 << 47)
        return ctx.estimate_batch_ex(pinned if host else dev, nt, args.seed, sched, first_traj=first)[0]

    for i in range(args.warmup):
        res = job(i)
        print(f"warm-up {i}: {max(r['rounds'] for r in res)} rounds", file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    jobs = []
    kern_ms = prep_ms = 0.0
    alg_bytes = mlp_rows = 0
    launches = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))  # L2 flush between timed steps (outside the events)
        ev[i][0].record(stream)
        res = job(args.warmup + i)
        ev[i][1].record(stream)
        info = ctx.last_call_info()
        kern_ms += info["traj_kernel_ms"]
        prep_ms += info["prep_kernel_ms"]
        rounds = max(r["rounds"] for r in res)
        launches += 1 + 3 * rounds  # prepare; per round: trajectories, statistics partial + merge
        alg_bytes += sum(r["alg_bytes"] for r in res)
        mlp_rows += sum(r["mlp_rows"] for r in res)
        jobs.append(res)
        print(f"step {i}: {sum(r['stop'] == 1 for r in res)} of {len(res)} matrices at target, "
              f"{max(r['rounds'] for r in res)} rounds", file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_s = [a.elapsed_time(b) / 1e3 for a, b in ev]
    t_dev = sum(step_s)
    summ = [job_summary(res, t) for res, t in zip(jobs, step_s)]
    tot_ess = sum(js["ess"] for js in summ)
    tot_traj = sum(js["traj"] for js in summ)
    # e2e: the same jobs through the public call from pinned host CSR
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_ess = 0.0
    for i in range(args.steps):
        e2e_ess += sum(r["ess"] for r in job(10_000 + i, host=True))
    t_e2e = time.perf_counter() - t0
    info = ctx.last_call_info()
    h2d, d2h = info["h2d_bytes"], info["d2h_bytes"]

    if dist:
        t = torch.tensor([t_dev, t_e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, t_e2e = float(t[0]), float(t[1])
        s = torch.tensor([tot_ess, e2e_ess, float(tot_traj)], dtype=torch.float64, device="cuda")
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        tot_ess, e2e_ess, tot_traj = float(s[0]), float(s[1]), int(s[2])

    value = tot_ess / t_dev
    ess_per_traj = tot_ess / max(1, tot_traj)
    note = None
    if args.mats != N_MATS or args.nmax != N_HI:
        note = f"reduced case: first {args.mats} matrices, n<={args.nmax} (not a bench value)"
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6400.0
    tc_peak = peaks["bf16_tflops"] if peaks else 1800.0
    kern_s = kern_ms / 1e3
    achieved_gb = alg_bytes / kern_s / 1e9
    achieved_tf = mlp_rows * 9344.0 / kern_s / 1e12
    rounds_per_job = statistics.median(js["rounds"] for js in summ)
    traffic = ncu_traffic_per_launch(args.eps, len(mats))
    ess_k = np.concatenate([js["ess_k"] for js in summ])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "eps": args.eps, "step_budget_s": args.budget,
                   "traj_cap_per_matrix": TRAJ_CAP,
                   "l2": "flushed between timed steps (256 MB write outside the step events)",
                   "parallelism": f"replicas{world}", "note": note},
        "traj_per_s": tot_traj / t_dev,
        "ess_per_traj": ess_per_traj,
        "job": {"seconds_median": statistics.median(step_s), "rounds_median": rounds_per_job,
                "matrices_at_target_mean": float(np.mean([js["met"] for js in summ])),
                "ess_per_s_at_target": float(sum(js["ess_k"][js["met_k"]].sum() for js in summ)
                                             / max(1e-12, sum(js["t_k"][js["met_k"]].sum() for js in summ))),
                "ess_per_matrix_median": float(np.median(ess_k)),
                "traj_per_job": tot_traj / args.steps,
                "ess_definition": "Sec. 2 ESS of each matrix at its stop (RSE <= eps, or the step's time "
                                  "budget for the matrices it censors), summed over matrices and steps"},
        "roofline": {"bound": "hbm", "achieved": achieved_gb, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved_gb / hbm_peak, "traffic": traffic,
                     "kernel": "traj_kernel<float, learned>",
                     "peak_source": "measured copy (MEASURED_PEAKS.json)" if peaks else "fallback",
                     "bytes": "algorithmic, counted per trajectory on the device (pm_result.alg_bytes: "
                              "16 B/vertex init; per step 8 B per adjacency entry of v and u + 16 B pointers, "
                              "32 B per degree decrement; features 8 B per entry of each candidate's list "
                              "+ 16 B per candidate); per launch = summed over the step's launches",
                     "kernel_ms_per_step": kern_ms / args.steps, "prep_ms_per_step": prep_ms / args.steps,
                     "l2": {"achieved": achieved_gb, "peak": bw["l2_read_gbs"], "unit": "GB/s",
                            "frac": achieved_gb / bw["l2_read_gbs"], "peak_source": "pm_probe_bandwidth"},
                     "smem_peak_gbs": bw["smem_read_gbs"],
                     "tensor": {"achieved": achieved_tf, "peak": tc_peak, "unit": "TFLOP/s",
                                "frac": achieved_tf / tc_peak,
                                "flops": "9344 per live candidate evaluated by the network"}},
        "gpu_launches": launches * world,
        "layouts": {"autotune_seconds": t_tune, "staged": sum(p["staged"] for p in plans),
                    "gstate": sum(p["gstate"] for p in plans), "tuned": sum(p["tuned"] for p in plans),
                    "groups_per_sm_median": statistics.median(p["groups"] for p in plans)},
        "clocks": clk,
        "e2e": {"value": e2e_ess / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "the same jobs through estimate_permanent_batch from pinned host CSR, host wall clock"},
    }
    line["train"] = {"objective": "per-step centred squared error", "pairs": train_rep["n_pairs"],
                     "loss_first": train_rep["loss_first"],
                     "loss_last": train_rep["loss_last"], "seconds": t_train,
                     "where": "before the timed region"}
    if not args.no_compare:
        cmp = compare_arms(ctx, B, dev, args, summ[0])
        for name in ("plain_unbatched", "plain_batched", "adaptive_sk_batched"):
            cmp[f"learned_batched_vs_{name}"] = value / cmp[name]["ess_per_s"]
        line["compare"] = cmp
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mats, bf16_params(model.params()), ess_per_traj)
    model.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
