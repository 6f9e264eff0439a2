"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: chosen edges, picked-vertex degrees and death steps bit-exact; ln X
within 1e-12 * max(1, |ln X|) in both precision modes (the proposal
arithmetic is replayed exactly, so only the last bits of the log-weight
accumulation differ); statistics within 1e-12 relative.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import compare_trace, ctx, binding, to_gpu_sched, logx_close

pytestmark = pytest.mark.gpu

TOL = 1e-12
FP = [O.PREC_FP64, O.PREC_FP32]


def test_philox_device_known_answers():
    gold = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(gold):
        if not line.strip() or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        out = ctx().philox_blocks(v[:4], v[4:6], 1)
        assert [int(x) for x in out[0]] == v[6:10]
    # and a run of counters against the oracle's generator
    out = ctx().philox_blocks([5, 77, 3, 9], [0xDEADBEEF, 0x12345], 257)
    for i in range(0, 257, 16):
        assert [int(x) for x in out[i]] == O.philox4x32_10([5 + i, 77, 3, 9], [0xDEADBEEF, 0x12345])


@pytest.mark.parametrize("prec", FP)
def test_plain_md_planted_bernoulli_n20(prec):
    # the n = 20, p = 0.3 planted-permutation workload, plain (no scaling)
    m = G.planted_bernoulli(20, 0.3, seed=1)
    compare_trace(m, O.Schedule(precision=prec), count=3001, seed=1)


def test_row_order_rule():
    m = G.planted_bernoulli(24, 0.3, seed=2)
    compare_trace(m, O.Schedule(vertex_rule=O.VR_ROW_ORDER), count=777, seed=5)


@pytest.mark.parametrize("prec", FP)
def test_outer_sk_weighted(prec):
    m = G.random_weighted(40, 0.2, seed=3)
    compare_trace(m, O.Schedule(K0=100, precision=prec), count=513, seed=11)


@pytest.mark.parametrize("prec", FP)
def test_initial_dm_and_outer_sk(prec):
    m = G.er_planted(150, 3.0, seed=7)
    compare_trace(m, O.Schedule(initial_dm=1, K0=50, precision=prec), count=300, seed=3, first=1000)


@pytest.mark.parametrize("prec", FP)
@pytest.mark.parametrize("sk", [O.SK_FIXED, O.SK_ADAPTIVE])
def test_inner_full_sk(prec, sk):
    m = G.er_planted(90, 4.0, seed=9)
    compare_trace(m, O.Schedule(initial_dm=1, K0=20, K=4, sk=sk, precision=prec), count=97, seed=2)


@pytest.mark.parametrize("prec", FP)
@pytest.mark.parametrize("name", ["local_threshold", "local_tracked", "adaptive_threshold",
                                  "adaptive_tracked", "fixed_all"])
def test_paper_presets(prec, name):
    m = G.er_planted(60, 4.0, seed=13)
    compare_trace(m, O.preset(name, prec), count=65, seed=4)


@pytest.mark.parametrize("prec", FP)
def test_presets_weighted_block_diagonal(prec):
    m = G.block_diagonal(100, 0.5, seed=21, weighted=True)
    for name in ("local_threshold", "adaptive_tracked"):
        compare_trace(m, O.preset(name, prec), count=33, seed=6)


def test_long_adjacency_lists():
    # rows and columns with more than 32 entries take the multi-chunk path
    m = G.planted_bernoulli(90, 0.55, seed=4)
    compare_trace(m, O.Schedule(), count=200, seed=8)
    compare_trace(m, O.Schedule(K0=10, precision=O.PREC_FP32), count=200, seed=8)
    w = G.random_weighted(80, 0.6, seed=5)
    compare_trace(w, O.Schedule(K0=5, K=2, sk=O.SK_LOCAL, precision=O.PREC_FP32), count=64, seed=9)


@pytest.mark.parametrize("prec", FP)
@pytest.mark.parametrize("cap", [4, 16, 64])
def test_bounded_local_repair_power_law_hubs(prec, cap):
    """The bounded-work Local repair (a reading of the variant Sec. 3.3
    leaves open): power-law rows with hubs of 60-360 entries, so hubs are
    neither expanded nor summed exactly but sampled with the step's Philox
    offset; local_threshold and local_tracked, both precisions."""
    for name, n, seed in (("local_threshold", 400, 2), ("local_tracked", 800, 1)):
        s = O.preset(name, prec)
        s.local_cap = cap
        compare_trace(G.powerlaw_planted(n, seed=seed), s, 24, seed=5)


@pytest.mark.parametrize("prec", FP)
def test_two_level_degree_tree(prec):
    # 2n > 1024 leaves: the minimum-degree tree has two stored levels
    m = G.er_planted(700, 5.0, seed=17)
    compare_trace(m, O.Schedule(initial_dm=1, K0=20, precision=prec), count=40, seed=12)


@pytest.mark.parametrize("prec", FP)
def test_preprocess_matches_oracle(prec):
    for m in (G.er_planted(300, 4.0, seed=31), G.random_weighted(50, 0.15, seed=32),
              G.block_diagonal(100, 0.7, seed=33, weighted=True)):
        sched = O.Schedule(initial_dm=1, K0=100, precision=prec)
        g = ctx().preprocess(m, to_gpu_sched(sched))
        P = O.Prepared(m, sched)
        assert g["ok"] == P.ok
        assert np.array_equal(g["keep"], P.mask())
        r, c = P.scaling()
        assert np.array_equal(g["r"], r) and np.array_equal(g["c"], c)


def test_statistics_match_oracle():
    m = G.planted_bernoulli(20, 0.3, seed=1)
    sched = O.Schedule(precision=O.PREC_FP32)
    T = 40000
    res = ctx().estimate_permanent(m, T, 1, to_gpu_sched(sched))
    o = O.Prepared(m, sched).run(seed=1, count=T, threads=8)
    st = O.stats(o["log_x"])
    assert res["n_traj"] == T and res["n_alive"] == st["n_alive"]
    for key in ("log_estimate", "ess", "p_match", "rel_spread", "rse", "log_sum_x", "log_sum_x2"):
        assert res[key] == pytest.approx(st[key], rel=1e-12, abs=1e-12), key
    per = O.ryser(m.to_dense())
    assert abs(math.exp(res["log_estimate"]) / per - 1) < 5 * res["rse"]


def test_batch_matches_per_matrix_replay():
    mats = [G.er_planted(n, 4.0, seed=40 + n) for n in (37, 120, 64)]
    sched = O.Schedule(initial_dm=1, K0=30, K=3, sk=O.SK_ADAPTIVE, precision=O.PREC_FP32)
    T = [70, 33, 101]
    res, lx = ctx().estimate_batch_ex(mats, T, 7, to_gpu_sched(sched), want_log_x=True)
    off = 0
    for k, m in enumerate(mats):
        o = O.Prepared(m, sched).run(seed=7, count=T[k], matrix=k, threads=8)
        assert logx_close(lx[off:off + T[k]], o["log_x"], TOL) <= TOL
        st = O.stats(o["log_x"])
        assert res[k]["log_estimate"] == pytest.approx(st["log_estimate"], rel=1e-12)
        assert res[k]["n_full_sk"] == o["n_full_sk"]
        off += T[k]


def test_operation_counts_match_oracle():
    m = G.er_planted(80, 4.0, seed=50)
    for name in ("local_threshold", "adaptive_tracked", "fixed_all"):
        sched = O.preset(name, O.PREC_FP32)
        res = ctx().estimate_permanent(m, 48, 3, to_gpu_sched(sched))
        o = O.Prepared(m, sched).run(seed=3, count=48, threads=8)
        assert (res["n_dm_calls"], res["n_full_sk"], res["n_local_sk"]) == \
            (o["n_dm"], o["n_full_sk"], o["n_local_sk"])


def test_all_ones_and_degenerate_cases():
    J = G.all_ones(9)
    res = ctx().estimate_permanent(J, 500, 2, binding().Schedule())
    assert res["log_estimate"] == pytest.approx(math.log(math.factorial(9)), rel=1e-13)
    assert res["rel_spread"] == pytest.approx(0.0, abs=1e-12) and res["ess"] == pytest.approx(500)
    one = G.csr_from_dense(np.ones((1, 1)))
    res = ctx().estimate_permanent(one, 10, 2, binding().Schedule())
    assert res["log_estimate"] == 0.0 and res["p_match"] == 1.0
    # per(A) = 0: the initial DM finds no perfect matching
    d = np.zeros((4, 4)); d[0, :] = 1; d[1:, 0] = 1
    z = G.csr_from_dense(d)
    s = binding().Schedule(initial_dm=1, K0=10)
    res = ctx().estimate_permanent(z, 100, 1, s)
    assert res["log_estimate"] == -math.inf and res["p_match"] == 0.0
    compare_trace(z, O.Schedule(initial_dm=1, K0=10), count=10)
    compare_trace(z, O.Schedule(), count=50)


def test_malformed_input_is_rejected():
    B = binding()
    m = G.er_planted(30, 3.0, seed=1)
    bad = G.Csr(m.n, m.row_ptr.copy(), m.col_idx[::-1].copy())   # unsorted rows
    with pytest.raises(B.PmError) as e:
        ctx().estimate_permanent(bad, 10, 1, B.Schedule())
    assert e.value.status == B.PM_EINVAL
    bad2 = G.Csr(m.n, m.row_ptr.copy(), np.full_like(m.col_idx, 40))  # out of range
    with pytest.raises(B.PmError):
        ctx().estimate_permanent(bad2, 10, 1, B.Schedule())
    # the context stays usable after a rejected call
    res = ctx().estimate_permanent(m, 64, 1, B.Schedule())
    assert res["n_traj"] == 64


def test_device_resident_inputs_match_host_inputs():
    import torch
    m = G.er_planted(200, 5.0, seed=61)
    sched = binding().Schedule(initial_dm=1, K0=20, K=2, sk=binding().SK_ADAPTIVE, precision=0)
    host = ctx().estimate_permanent(m, 256, 9, sched)
    dev = G.Csr(m.n, torch.from_numpy(m.row_ptr).cuda(), torch.from_numpy(m.col_idx).cuda())
    gpu = ctx().estimate_permanent(dev, 256, 9, sched)
    for key in ("log_estimate", "ess", "p_match", "rel_spread", "n_full_sk"):
        assert host[key] == gpu[key]
