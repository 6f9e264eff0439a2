"""Pair layout: two trajectories per warp, one per 16-lane half, for the
schedules without inner SK, DM or Local repair (plain scaled, uniform and
learned proposals).  Every trajectory takes the same picks, integer weights,
draws and corrections as in the one-trajectory-per-warp layout, whose paths
the oracle checks bit-exactly (test_gpu_parity, test_gpu_learned), so ln X
must be the same bits, trajectory by trajectory; so must the per-matrix work
counters (algorithmic bytes and network rows), which both layouts sum from
the same per-step terms."""
import numpy as np
import pytest

from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import binding

pytestmark = pytest.mark.gpu


def _run(mats, ntraj, seed, sched, pins):
    """ln X of every trajectory and the results, in a context of its own with
    each (n, nnz, layout) of `pins` pinned."""
    B = binding()
    c = B.Context(0)
    try:
        for n, nnz, lay in pins:
            c.layout_set(sched, n, nnz, **lay)
        res, lx = c.estimate_batch_ex(mats, [ntraj] * len(mats), seed, sched, want_log_x=True)
        plan = c.last_call_info()["first_plan"]
    finally:
        c.close()
    return lx, res, plan


def _same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


def _compare(m, sched, ntraj=512, seed=7, staged=1):
    lx_p, res_p, plan_p = _run([m], ntraj, seed, sched, [(m.n, m.nnz, dict(pair=1, staged=staged))])
    lx_s, res_s, plan_s = _run([m], ntraj, seed, sched, [(m.n, m.nnz, dict(pair=0, staged=staged))])
    assert plan_p["pair"] == 1 and plan_p["groups"] % 2 == 0 and plan_p["groups"] >= 4, plan_p
    assert plan_s["pair"] == 0, plan_s
    fin = np.isfinite(lx_s)
    assert _same_bits(lx_p, lx_s), (np.count_nonzero(lx_p != lx_s), np.abs(lx_p[fin] - lx_s[fin]).max())
    for key in ("log_estimate", "n_alive", "alg_bytes", "mlp_rows"):
        assert res_p[0][key] == res_s[0][key] or (np.isnan(res_p[0][key]) and np.isnan(res_s[0][key])), key
    return lx_p, res_p[0]


def _model(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    from tests._gpu_common import ctx
    return ctx().model((rng.normal(size=4801) * scale).astype(np.float32))


@pytest.mark.parametrize("staged", [1, 0])
def test_pair_scaled_proposal(staged):
    m = G.er_planted(300, 4.0, seed=11)
    B = binding()
    _compare(m, B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL), staged=staged)


def test_pair_fp64_and_weighted():
    B = binding()
    m = G.random_weighted(120, 0.06, seed=4)
    _compare(m, B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP64))
    _compare(m, B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL))


def test_pair_uniform_proposal():
    # binary input with no scaling: every proposal is uniform over the live candidates
    B = binding()
    m = G.planted_bernoulli(64, 0.15, seed=2)
    lx, r = _compare(m, B.Schedule(), ntraj=2048)
    assert r["n_alive"] > 0


def test_pair_row_order_rule():
    B = binding()
    m = G.er_planted(200, 5.0, seed=8)
    _compare(m, B.Schedule(vertex_rule=B.VR_ROW_ORDER, initial_dm=1, K0=40, precision=B.PREC_FP32_PROPOSAL))


def test_pair_powerlaw_hubs():
    # lists longer than 16 and 32 entries: several candidate chunks per half-warp
    B = binding()
    m = G.powerlaw_planted(2000, seed=5, exponent=2.1)
    deg = np.diff(m.row_ptr)
    assert deg.max() > 48
    _compare(m, B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL), ntraj=256, staged=1)
    _compare(m, B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL), ntraj=256, staged=0)


@pytest.mark.parametrize("kind", ["er", "hubs", "weighted"])
def test_pair_learned(kind):
    B = binding()
    model = _model(21)
    if kind == "er":
        m = G.er_planted(250, 4.0, seed=13)
    elif kind == "hubs":
        m = G.powerlaw_planted(1500, seed=6, exponent=2.1)
    else:
        m = G.random_weighted(100, 0.08, seed=9)
    s = B.Schedule(initial_dm=1, K0=60, precision=B.PREC_FP32_PROPOSAL, learned=model)
    lx, r = _compare(m, s, ntraj=256)
    assert r["mlp_rows"] > 0


def test_pair_learned_unit_scale():
    # a learned schedule on a binary matrix without scaling: the proposal stays uniform
    B = binding()
    model = _model(22)
    m = G.planted_bernoulli(48, 0.2, seed=3)
    _compare(m, B.Schedule(learned=model, precision=B.PREC_FP32_PROPOSAL), ntraj=512)


def test_pair_no_perfect_matching():
    B = binding()
    d = np.zeros((4, 4)); d[0, :] = 1; d[1:, 0] = 1
    z = G.csr_from_dense(d)
    lx, r = _compare(z, B.Schedule(initial_dm=1, K0=10), ntraj=64)
    assert np.all(np.isneginf(lx)) and r["p_match"] == 0.0


def test_pair_mixed_batch():
    """One launch over matrices of two size classes, one pinned to the pair
    layout and one to the one-trajectory-per-warp layout: both kinds of chunk
    run in the same kernel; each matrix's ln X matches its all-standard run."""
    B = binding()
    s = B.Schedule(initial_dm=1, K0=80, precision=B.PREC_FP32_PROPOSAL)
    small = [G.er_planted(100 + 3 * i, 4.0, seed=40 + i) for i in range(3)]
    large = [G.er_planted(700 + 5 * i, 4.0, seed=60 + i) for i in range(3)]
    mats = [small[0], large[0], small[1], large[1], small[2], large[2]]
    pins_mixed = [(100, small[0].nnz, dict(pair=1, staged=1)), (700, large[0].nnz, dict(pair=0, staged=1))]
    pins_std = [(100, small[0].nnz, dict(pair=0, staged=1)), (700, large[0].nnz, dict(pair=0, staged=1))]
    lx_m, _, plan = _run(mats, 300, 5, s, pins_mixed)
    lx_s, _, _ = _run(mats, 300, 5, s, pins_std)
    assert plan["pair"] == 1
    assert _same_bits(lx_m, lx_s)


def test_pair_plan_rules():
    """The pair layout exists only for schedules without inner SK or DM, and
    traces fall back to one trajectory per warp."""
    B = binding()
    c = B.Context(0)
    try:
        m = G.er_planted(200, 4.0, seed=1)
        with pytest.raises(B.PmError):
            c.layout_set(B.preset("local_threshold"), m.n, m.nnz, pair=1, staged=1)
        s = B.Schedule(initial_dm=1, K0=20, precision=B.PREC_FP32_PROPOSAL)
        c.layout_set(s, m.n, m.nnz, pair=1, staged=1)
        c.trace(m, 8, 3, s)
        assert c.last_call_info()["first_plan"]["pair"] == 0
        c.estimate_permanent(m, 64, 3, s)
        assert c.last_call_info()["first_plan"]["pair"] == 1
    finally:
        c.close()
