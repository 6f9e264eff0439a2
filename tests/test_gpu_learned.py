"""GPU parity of the learned proposal (an extension; the paper has
no learned part) against the CPU oracle, and what training gains.

Bars:
  forward    BF16 weights/inputs and BF16 hidden activations on tensor cores,
             GELU through the hardware tanh approximation (relative error up
             to 2^-11), vs an FP64 network with the same rounding of weights,
             inputs and activations and an exact tanh: a hidden unit can be
             off by one BF16 ulp (2^-8) plus the tanh error; through two
             64-wide layers with weights of size ~0.4 that is a few 1e-2 at
             most, so |dy| <= 6e-2 * max(1, |y|), median <= 5e-3
  gradient   cosine > 0.999 per parameter block, relative norm error < 5e-2
             (mean squared error and the per-step centred loss)
  features   recorded pairs: same keys, step groups, features and targets
             within 1e-5
  in-path    the network inside the trajectory kernel, on the states the
             device visited, against the oracle's network on its own features
             of those states: the forward bar above
  replay     with the GPU's logits supplied, the oracle's paths are
             bit-exact and ln X agrees within 1e-12
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import binding, ctx, logx_close

pytestmark = pytest.mark.gpu

BLOCKS = {"W1": (0, 512), "b1": (512, 576), "W2": (576, 4672), "b2": (4672, 4736), "W3": (4736, 4800),
          "b3": (4800, 4801)}


def bf16(x):
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32)
    u[:] = ((u.astype(np.uint64) + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return a


def oracle_params(p):
    """The GPU keeps weights in BF16 and biases in FP32."""
    q = np.asarray(p, dtype=np.float32).astype(np.float64)
    for name in ("W1", "W2", "W3"):
        a, b = BLOCKS[name]
        q[a:b] = bf16(p[a:b])
    return q


def rand_params(rng, scale=0.4):
    return (rng.normal(size=O.N_PARAM) * scale).astype(np.float32)


def test_mlp_forward_matches_oracle():
    rng = np.random.default_rng(3)
    for trial in range(3):
        p = rand_params(rng)
        m = ctx().model(p)
        X = rng.normal(size=(1003, 8)).astype(np.float32)
        y = m.forward(X)
        ref = O.mlp_forward(oracle_params(p), bf16(X).astype(np.float64), round_act=True)
        err = np.abs(y - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() < 6e-2, err.max()
        assert np.median(err) < 5e-3, np.median(err)
        m.close()


def step_groups(rng, B):
    """group codes (index << 16 | size) of consecutive steps of 1..9 rows"""
    codes = []
    while len(codes) < B:
        s = int(min(rng.integers(1, 10), B - len(codes)))
        codes += [(k << 16) | s for k in range(s)]
    return np.array(codes, dtype=np.uint32)


@pytest.mark.parametrize("centred", [False, True])
def test_mlp_gradient_matches_oracle(centred):
    rng = np.random.default_rng(4)
    p = rand_params(rng, 0.3)
    m = ctx().model(p)
    X = rng.normal(size=(4099, 8)).astype(np.float32)
    T = rng.normal(size=4099).astype(np.float32)
    grp = step_groups(rng, 4099) if centred else None
    loss, g = m.gradient(X, T, grp)
    ref_loss, ref = O.mlp_grad(oracle_params(p), bf16(X).astype(np.float64), T.astype(np.float64), grp)
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    for name, (a, b) in BLOCKS.items():
        u, v = g[a:b].astype(np.float64), ref[a:b]
        if name == "b3":
            if centred:  # a step-wide offset has no gradient
                assert abs(u[0]) < 1e-4 and abs(v[0]) < 1e-12
            else:
                assert u[0] == pytest.approx(v[0], rel=2e-2, abs=1e-4)
            continue
        cos = float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))
        rel = float(np.linalg.norm(u - v) / np.linalg.norm(v))
        assert cos > 0.999 and rel < 5e-2, (name, cos, rel)
    m.close()


@pytest.mark.parametrize("centred", [False, True])
def test_mlp_gradient_many_tiles_per_cta(centred):
    """50,003 rows: 391 row tiles of 128 over at most two CTAs per SM, so most
    CTAs accumulate several tiles in tensor memory before their partial sums
    are read out, and the last tile is ragged; the result is reproducible
    (fixed-order reduction over the CTAs)."""
    rng = np.random.default_rng(14)
    p = rand_params(rng, 0.3)
    m = ctx().model(p)
    n = 50_003
    X = rng.normal(size=(n, 8)).astype(np.float32)
    T = rng.normal(size=n).astype(np.float32)
    grp = step_groups(rng, n) if centred else None
    loss, g = m.gradient(X, T, grp)
    loss2, g2 = m.gradient(X, T, grp)
    assert loss == loss2 and np.array_equal(g, g2)
    ref_loss, ref = O.mlp_grad(oracle_params(p), bf16(X).astype(np.float64), T.astype(np.float64), grp)
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    for name, (a, b) in BLOCKS.items():
        if name == "b3":
            continue
        u, v = g[a:b].astype(np.float64), ref[a:b]
        cos = float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))
        rel = float(np.linalg.norm(u - v) / np.linalg.norm(v))
        assert cos > 0.999 and rel < 5e-2, (name, cos, rel)
    m.close()


def test_mlp_gradient_rejects_torn_groups():
    rng = np.random.default_rng(5)
    m = ctx().model(rand_params(rng))
    X = rng.normal(size=(6, 8)).astype(np.float32)
    T = rng.normal(size=6).astype(np.float32)
    bad = np.array([(0 << 16) | 3, (1 << 16) | 3, (2 << 16) | 3, (0 << 16) | 4, (1 << 16) | 4, (2 << 16) | 4],
                   dtype=np.uint32)  # the second step runs past the rows
    with pytest.raises(Exception):
        m.gradient(X, T, bad)
    m.close()


def test_recorded_pairs_match_oracle():
    B = binding()
    m = G.er_planted(80, 5.0, seed=21)
    teacher = O.Schedule(initial_dm=1, K0=20, K=3, sk=O.SK_FIXED, precision=O.PREC_FP32)
    gt = B.Schedule(initial_dm=1, K0=20, K=3, sk=B.SK_FIXED, precision=B.PREC_FP32_PROPOSAL)
    f, t, k, g = ctx().record_pairs(m, 8, 7, gt, cap=100000)
    of, ot, ok, og = O.Prepared(m, teacher).record(seed=7, count=8, cap=100000)
    assert len(k) == len(ok) and len(k) > 100
    order = np.argsort(k)
    assert np.array_equal(k[order], ok)
    assert np.array_equal(g[order], og)
    # on the device a step's pairs are consecutive as well
    start = np.arange(len(g)) - (g >> 16).astype(np.int64)
    assert np.array_equal(k[start] >> 14, k >> 14)
    assert np.allclose(f[order], of, rtol=1e-5, atol=1e-6)
    assert np.allclose(t[order], ot, rtol=1e-5, atol=1e-6)


def test_learned_trajectories_replay_bit_exact():
    B = binding()
    rng = np.random.default_rng(5)
    for mat in (G.er_planted(120, 5.0, seed=31), G.random_weighted(40, 0.15, seed=32)):
        p = rand_params(rng, 0.3)
        model = ctx().model(p)
        sched = B.Schedule(initial_dm=1, K0=30, precision=B.PREC_FP32_PROPOSAL, learned=model)
        T = 100
        g = ctx().trace(mat, T, 9, sched)
        P = O.Prepared(mat, O.Schedule(initial_dm=1, K0=30, precision=O.PREC_FP32))
        o = P.run_ext(seed=9, count=T, logits=g["logits"], threads=8)
        assert np.array_equal(g["dead_step"], o["dead_step"])
        assert np.array_equal(g["chosen"], o["chosen"])
        assert np.array_equal(g["deg_v"], o["deg_v"])
        assert logx_close(g["log_x"], o["log_x"], 1e-12) <= 1e-12
        model.close()


def test_training_reduces_the_loss():
    B = binding()
    mats = [G.er_planted(200, 6.0, seed=100 + i) for i in range(4)]
    teacher = B.Schedule(initial_dm=1, K0=100, K=10, sk=B.SK_FIXED, precision=B.PREC_FP32_PROPOSAL)
    for objective in (B.OBJ_MSE, B.OBJ_CENTRED):
        model = ctx().model(seed=1)
        rep = model.train(mats, teacher, n_pairs=200000, epochs=4, batch=4096, lr=2e-3, seed=2,
                          objective=objective)
        assert 199000 < rep["n_pairs"] <= 200000  # whole steps only
        assert rep["loss_last"] < 0.5 * rep["loss_first"], (objective, rep)
        model.close()


def test_learned_proposal_gains_over_the_plain_estimator():
    """Trained on ER+permutation matrices (n = 150, average degree 6), evaluated
    on held-out seeds: the learned proposal (no inner SK) must beat the plain
    estimator (outer SK only, same vertex rule) in effective samples per
    trajectory, and agree with the low-variance Fixed-SK estimate."""
    B = binding()
    train = [G.er_planted(150, 6.0, seed=1000 + i) for i in range(8)]
    teacher = B.Schedule(initial_dm=1, K0=100, K=10, sk=B.SK_FIXED, precision=B.PREC_FP32_PROPOSAL)
    model = ctx().model(seed=3)
    model.train(train, teacher, n_pairs=300000, epochs=6, batch=4096, lr=2e-3, seed=4)
    plain = B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL)
    learned = B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL, learned=model)
    gains = []
    for i in range(3):
        m = G.er_planted(150, 6.0, seed=2000 + i)
        a = ctx().estimate_permanent(m, 100000, 11, plain)
        b = ctx().estimate_permanent(m, 100000, 11, learned)
        ref = ctx().estimate_permanent(m, 20000, 11, teacher)
        gains.append(b["ess"] / a["ess"])
        assert abs(b["log_estimate"] - ref["log_estimate"]) < 5 * (b["rse"] + ref["rse"]) + 0.01
    assert np.median(gains) > 5.0, gains
    model.close()


def test_network_inside_the_trajectory_kernel_matches_oracle():
    """The logits the trajectory kernel computed for the live candidates of
    every step (features from the device's residual state, the in-kernel
    tensor-core network) against the oracle's features and FP64 network on the
    same states, with the oracle following the device's paths."""
    B = binding()
    rng = np.random.default_rng(8)
    m = G.er_planted(150, 6.0, seed=41)
    p = rand_params(rng, 0.3)
    model = ctx().model(p)
    sched = B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL, learned=model)
    T = 40
    g = ctx().trace(m, T, 13, sched)
    P = O.Prepared(m, O.Schedule(initial_dm=1, K0=50, precision=O.PREC_FP32))
    o = P.run_ext_model(seed=13, count=T, logits=g["logits"], params=oracle_params(p), threads=8)
    assert np.array_equal(o["chosen"], g["chosen"])
    # compare the candidates of steps with at least two (a single candidate
    # is taken with probability 1, whatever its logit)
    dv = g["deg_v"]
    sel = np.zeros(g["logits"].shape, dtype=bool)
    for q in range(T):
        for t in range(m.n):
            if dv[q, t] >= 2:
                sel[q, t, :dv[q, t]] = True
    y, ref = g["logits"][sel], o["model_logits"][sel].astype(np.float64)
    assert y.size > 1000
    err = np.abs(y - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < 6e-2, err.max()
    assert np.median(err) < 5e-3, np.median(err)
    model.close()


def test_training_is_reproducible():
    """The same matrices, teacher, seed and settings give bit-identical
    parameters: the recorded set, its order and the gradient reduction do not
    depend on how the device schedules its warps."""
    B = binding()
    mats = [G.er_planted(120, 6.0, seed=300 + i) for i in range(3)]
    teacher = B.Schedule(initial_dm=1, K0=50, K=5, sk=B.SK_FIXED, precision=B.PREC_FP32_PROPOSAL)
    out = []
    for _ in range(2):
        model = ctx().model(seed=5)
        rep = model.train(mats, teacher, n_pairs=60000, epochs=2, batch=2048, lr=2e-3, seed=6)
        out.append((model.params().copy(), rep["loss_last"], rep["n_pairs"]))
        model.close()
    assert out[0][2] == out[1][2] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def _replay_learned(mat, p, seed, T, K0=100):
    """Trace T learned-proposal trajectories on the device (every live
    candidate's logit kept) and replay them in the oracle with those logits
    while it evaluates its own network on the visited states."""
    B = binding()
    model = ctx().model(p)
    sched = B.Schedule(initial_dm=1, K0=K0, precision=B.PREC_FP32_PROPOSAL, learned=model)
    g = ctx().trace(mat, T, seed, sched)
    P = O.Prepared(mat, O.Schedule(initial_dm=1, K0=K0, precision=O.PREC_FP32))
    o = P.run_ext_model(seed=seed, count=T, logits=g["logits"], params=oracle_params(p), threads=8)
    model.close()
    return g, o


def _assert_replay(g, o):
    assert np.array_equal(g["dead_step"], o["dead_step"])
    assert np.array_equal(g["deg_v"], o["deg_v"])
    assert np.array_equal(g["chosen"], o["chosen"])
    assert logx_close(g["log_x"], o["log_x"], 1e-12) <= 1e-12


def _network_err(g, o, min_cands):
    """Relative error of the in-kernel network against the oracle's on every
    candidate of the steps with at least min_cands live candidates."""
    dv = g["deg_v"]
    sel = np.zeros(g["logits"].shape, dtype=bool)
    for q, t in zip(*np.nonzero(dv >= max(2, min_cands))):
        sel[q, t, :dv[q, t]] = True
    y, ref = g["logits"][sel], o["model_logits"][sel].astype(np.float64)
    return y, np.abs(y - ref) / np.maximum(1.0, np.abs(ref))


def test_learned_power_law_hubs_replay_bit_exact():
    """Power-law rows (exponent 2.5, minimum 2) with hub rows of 150 to 360
    entries: the picked vertex's adjacency runs over several 32-entry chunks,
    so the kernel keeps the logits of long lists in the group's global slot
    and evaluates the network on several candidate tiles per chunk.  Paths,
    degrees and death steps bit-exact, ln X within 1e-12, every logit on the
    forward bar."""
    rng = np.random.default_rng(12)
    hubs = 0
    for n, seed in ((800, 1), (1500, 1)):
        mat = G.powerlaw_planted(n, seed=seed)
        rows = np.diff(mat.row_ptr)
        assert rows.max() >= 150
        g, o = _replay_learned(mat, rand_params(rng, 0.3), seed=17, T=16)
        _assert_replay(g, o)
        # steps whose picked vertex is a hub row (adjacency longer than 32)
        v = g["chosen"][:, :, 0]
        hubs += int(np.sum((v >= 0) & (v < n) & (rows[np.clip(v, 0, n - 1)] > 32)))
        y, err = _network_err(g, o, 2)
        assert y.size > 1000 and err.max() < 6e-2 and np.median(err) < 5e-3, (err.max(), np.median(err))
    assert hubs >= 16, hubs  # about one hub pick per trajectory


def test_learned_more_than_32_live_candidates():
    """A dense planted matrix (n = 120, entries Bernoulli(0.45)): the first
    steps pick vertices with 40 to 60 live candidates, so one step's logits
    span two network chunks and the selection scans several chunks.  The
    oracle replays every candidate's logit (no 32-candidate cap)."""
    rng = np.random.default_rng(13)
    mat = G.planted_bernoulli(120, 0.45, seed=5)
    g, o = _replay_learned(mat, rand_params(rng, 0.3), seed=19, T=24, K0=50)
    _assert_replay(g, o)
    big = g["deg_v"] > 32
    assert big.sum() >= 24 * 5, big.sum()
    y, err = _network_err(g, o, 33)
    assert y.size > 24 * 5 * 33 and err.max() < 6e-2 and np.median(err) < 5e-3, (err.max(), np.median(err))
