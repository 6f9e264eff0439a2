"""Large orders: trajectory state in global memory (n above what shared
memory holds), against the oracle (whole trajectories at n = 20000; the first
steps of every trajectory at the n = 100000 band + random configuration) and
against an exactly known permanent (block-diagonal family of Sec. 4)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import compare_trace, ctx, binding, to_gpu_sched, logx_close

pytestmark = pytest.mark.gpu


def test_global_state_whole_trajectories_n20000():
    m = G.er_planted(20000, 3.0, seed=5)
    compare_trace(m, O.Schedule(initial_dm=1, K0=20, precision=O.PREC_FP32), count=16, seed=3)


def _prefix_compare(m, sched, count, steps, seed=1):
    g = ctx().trace(m, count, seed, to_gpu_sched(sched))
    P = O.Prepared(m, sched)
    P.set_max_steps(steps)
    o = P.run(seed=seed, count=count, threads=8, trace=True)
    assert np.array_equal(g["chosen"][:, :steps], o["chosen"][:, :steps])
    assert np.array_equal(g["deg_v"][:, :steps], o["deg_v"][:, :steps])
    return g


@pytest.mark.parametrize("sk", [O.SK_LOCAL, O.SK_ADAPTIVE])
def test_global_state_prefixes_n20000(sk):
    m = G.er_planted(20000, 4.0, seed=6)
    _prefix_compare(m, O.Schedule(initial_dm=1, K0=20, K=4, sk=sk, precision=O.PREC_FP32), count=8, steps=400)


def test_band_random_n100000_prefixes():
    # the large sparse configuration: n = 100000, nnz = 500000 from a |i-j| <= 1
    # band, a planted permutation and uniform off-band entries; Local SK
    m = G.band_random(100000, 500000, seed=3)
    sched = O.Schedule(initial_dm=1, K0=100, sk=O.SK_LOCAL, precision=O.PREC_FP32)
    g = _prefix_compare(m, sched, count=4, steps=1500)
    assert np.all(g["chosen"][:, 1500:2000] >= 0) or np.any(g["dead_step"] >= 0)


def test_block_diagonal_known_permanent_n5000():
    m = G.block_diagonal(5000, 0.5, seed=9, orders=(20,))
    log_per = sum(math.log(O.ryser(b)) for b in m.blocks)
    B = binding()
    s = B.Schedule(initial_dm=1, K0=100, sk=B.SK_LOCAL, precision=B.PREC_FP32_PROPOSAL)
    r = ctx().estimate_permanent(m, 4096, 4, s)
    assert r["p_match"] > 0
    assert abs(r["log_estimate"] - log_per) < 5 * r["rse"] + 0.05, (r["log_estimate"], log_per, r["rse"])


def _trace_in_layout(m, sched, count, seed, **layout):
    """pm_trace of `count` trajectories in a pinned layout (a context of its
    own, so the pin reaches no other test), against the oracle."""
    B = binding()
    c = B.Context(0)
    gs = to_gpu_sched(sched)
    c.layout_set(gs, m.n, m.nnz, **layout)
    g = c.trace(m, count, seed, gs)
    plan = c.last_call_info()["first_plan"]
    c.close()
    o = O.Prepared(m, sched).run(seed=seed, count=count, threads=8, trace=True)
    assert np.array_equal(g["dead_step"], o["dead_step"])
    assert np.array_equal(g["deg_v"], o["deg_v"])
    assert np.array_equal(g["chosen"], o["chosen"])
    assert logx_close(g["log_x"], o["log_x"], 1e-12) <= 1e-12
    return g, plan


@pytest.mark.parametrize("g", [4, 16])
@pytest.mark.parametrize("case", [("band", "local_threshold", O.PREC_FP32), ("er", "local_tracked", O.PREC_FP64),
                                  ("er", "adaptive_threshold", O.PREC_FP32)])
def test_group_dm_pinned_layout(case, g):
    """DM schedules with the trajectory state in global memory and a group of
    g warps sharing the DM's component step (trimming, one forward-backward
    search from the smallest undone vertex, Tarjan on the leader warp for the
    rest), pinned with pm_layout_set at n = 3000 where the oracle's DM is
    fast.  The supported-edge set is unique (Sec. 2), so masks, and with them
    paths, degrees and death steps, are bit-exact against the oracle's
    matching + Tarjan; the full-SK schedule also runs its sweeps on the group."""
    kind, name, prec = case
    m = G.band_random(3000, 15000, seed=3) if kind == "band" else G.er_planted(3000, 5.0, seed=78)
    g_out, plan = _trace_in_layout(m, O.preset(name, prec), 6, 3, g=g, gstate=1)
    assert plan["gstate"] == 1 and plan["g"] == g, plan


def test_group_dm_heuristic_layout_n16000():
    """At n = 16000 four trajectory states no longer fit in shared memory: the
    heuristic layout of a DM schedule is global state with a 16-warp group
    (local_threshold at theta = 0.1, FP64; whole trajectories)."""
    s = O.preset("local_threshold", O.PREC_FP64)
    s.theta = 0.1
    m = G.er_planted(16000, 5.0, seed=78)
    compare_trace(m, s, count=2, seed=3)
    plan = ctx().last_call_info()["first_plan"]
    assert plan["gstate"] == 1 and plan["g"] == 16, plan
