"""Parity at the full sizes of the workloads, in the launch configurations
the bench uses.

- The n = 20 planted-permutation workload: all 1e5 trajectories (Philox seed
  1, two-sided MD, no scaling, initial DM off) against the oracle trajectory by
  trajectory (ln X within 1e-12), the statistics against the oracle's, and the
  estimate against the exact permanent (Ryser) within the reported RSE.
- The 64-matrix bench batch run as one persistent launch with Adaptive SK:
  sampled trajectories of several matrices replayed by the oracle.
- The bench's own learned schedule on the same batch, as the bench runs it
  (a resident batch, CUDA graph, autotuned layouts): on the largest matrices
  the chosen edges of sampled trajectories, traced in the same layout, are
  replayed bit-exact by the oracle, and the batch run's ln X of those
  trajectories agrees with the oracle's."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import ctx, binding, logx_close

pytestmark = pytest.mark.gpu


def test_planted_bernoulli_n20_all_1e5_trajectories():
    B = binding()
    m = G.planted_bernoulli(20, 0.3, seed=1)
    M = 100_000
    res, lx = ctx().estimate_batch_ex([m], [M], 1, B.Schedule(precision=B.PREC_FP64), want_log_x=True)
    o = O.Prepared(m, O.Schedule(precision=O.PREC_FP64)).run(seed=1, count=M, threads=16)
    assert logx_close(lx, o["log_x"], 1e-12) <= 1e-12
    st = O.stats(o["log_x"])
    r = res[0]
    assert r["n_alive"] == st["n_alive"]
    assert r["log_estimate"] == pytest.approx(st["log_estimate"], rel=1e-12, abs=1e-12)
    assert r["ess"] == pytest.approx(st["ess"], rel=1e-10)
    per = O.ryser(m.to_dense())
    rel = abs(math.exp(r["log_estimate"]) / per - 1)
    assert rel < 5 * r["rse"], (rel, r["rse"])


def test_bench_batch_sampled_against_the_oracle():
    B = binding()
    mats = G.batch_er(64, 100, 2000, 4.0, 8.0, seed=2)
    sched = B.Schedule(initial_dm=1, K0=100, K=10, sk=B.SK_ADAPTIVE, precision=B.PREC_FP32_PROPOSAL)
    T = 32
    _, lx = ctx().estimate_batch_ex(mats, [T] * 64, 1, sched, first_traj=5000, want_log_x=True)
    osched = O.Schedule(initial_dm=1, K0=100, K=10, sk=O.SK_ADAPTIVE, precision=O.PREC_FP32)
    small = [k for k in np.argsort([m.n for m in mats])[:4]]  # the oracle replays the smallest matrices
    for k in small:
        o = O.Prepared(mats[k], osched).run(seed=1, count=8, first_traj=5000, matrix=int(k), threads=8)
        assert logx_close(lx[T * k:T * k + 8], o["log_x"], 1e-12) <= 1e-12, k


def test_bench_learned_batch_largest_matrices():
    B = binding()
    rng = np.random.default_rng(21)
    p = (rng.normal(size=O.N_PARAM) * 0.3).astype(np.float32)
    model = ctx().model(p)
    mats = G.batch_er(64, 100, 2000, 4.0, 8.0, seed=2)
    sched = B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL, learned=model)
    T, first, seed = 256, 3 << 20, 1
    bt = ctx().batch(mats, [T] * 64, sched, graph=True, autotune=True)
    _, lx = bt.run(first, seed, want_log_x=True)
    osched = O.Schedule(initial_dm=1, K0=100, precision=O.PREC_FP32)
    largest = [int(k) for k in np.argsort([m.n for m in mats])[-3:]]
    for k in largest:
        c = 6
        g = ctx().trace(mats[k], c, seed, sched, first_traj=first, matrix_index=k)
        plan = bt.plan(k)
        used = ctx().last_call_info()["first_plan"]
        # a trace runs one trajectory per warp: a pair layout's trace takes
        # its one-per-warp counterpart (same staging), whose ln X bits the
        # pair layout reproduces (test_gpu_pair)
        fields = ("staged", "rc_smem", "gstate", "dm_smem") if plan["pair"] else \
            ("g", "groups", "staged", "rc_smem", "gstate", "dm_smem")
        assert used["pair"] == 0
        for f in fields:
            assert used[f] == plan[f], (k, f, used, plan)
        o = O.Prepared(mats[k], osched).run_ext(seed=seed, count=c, logits=g["logits"], first_traj=first,
                                                matrix=k, threads=8)
        assert np.array_equal(g["chosen"], o["chosen"]), k
        assert np.array_equal(g["dead_step"], o["dead_step"]), k
        assert logx_close(lx[T * k:T * k + c], o["log_x"], 1e-12) <= 1e-12, k
        assert np.array_equal(g["log_x"], lx[T * k:T * k + c]), k
    bt.close()
    model.close()
