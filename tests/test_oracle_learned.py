"""Pins of the oracle's learned-proposal parts (an extension: the
paper has no learned proposal, so these pin the pieces against mathematics
and against the paper's own unscaled estimator)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G


def test_exp_score_accuracy_and_special_values():
    # error budget: rounding y = x log2(e) to binary32 costs |y| ln2 2^-24
    # relative, the polynomial and its eight roundings a few 2^-24
    xs = np.linspace(-20, 20, 4001).astype(np.float32)
    u = 2.0 ** -24
    for x in xs:
        got = O.exp_score(float(x))
        want = math.exp(float(x))
        bound = abs(float(x)) * u + 10 * u
        assert abs(got / want - 1) < bound, x
    assert O.exp_score(0.0) == 1.0
    assert O.exp_score(100.0) == O.exp_score(20.0)
    assert O.exp_score(-100.0) == O.exp_score(-20.0)
    assert O.exp_score(float("nan")) == O.exp_score(-20.0)


def _rand_params(rng, scale=0.3):
    return rng.normal(size=O.N_PARAM) * scale


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = _rand_params(rng)
    X = rng.normal(size=(37, 8))
    T = rng.normal(size=37)
    loss, g = O.mlp_grad(P, X, T)
    yhat = O.mlp_forward(P, X)
    assert loss == pytest.approx(np.mean((yhat - T) ** 2), rel=1e-13)
    idx = rng.choice(O.N_PARAM, size=60, replace=False)
    idx = np.concatenate([idx, [0, 511, 512, 575, 576, 4671, 4672, 4735, 4736, 4799, 4800]])
    for i in idx:
        h = 1e-6
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (O.mlp_grad(Pp, X, T)[0] - O.mlp_grad(Pm, X, T)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_mlp_forward_closed_form():
    # with W1 = W2 = 0 every hidden unit is GELU(b): y = b3 + W3 . GELU(b2)
    # (GELU in its tanh form)
    P = np.zeros(O.N_PARAM)
    P[4672:4736] = 0.5          # b2
    P[4736:4800] = 2.0          # W3
    P[4800] = -1.0              # b3
    g05 = 0.5 * 0.5 * (1 + math.tanh(math.sqrt(2 / math.pi) * (0.5 + 0.044715 * 0.125)))
    y = O.mlp_forward(P, np.ones((3, 8)))
    assert np.allclose(y, -1.0 + 64 * 2.0 * g05, rtol=1e-14)


def test_features_hand_worked():
    # matrix A of tests/golden/md_paths.txt; step 0 picks row 1 (degree 2)
    # with candidates col 0 (degree 2, neighbours row0 (3) row1 (2)) and
    # col 1 (degree 3, neighbours row0 (3) row1 (2) row2 (3)); no scaling
    A = G.csr_from_coo(4, [0, 0, 0, 1, 1, 2, 2, 2, 3, 3], [0, 1, 2, 0, 1, 1, 2, 3, 2, 3])
    P = O.Prepared(A, O.Schedule(precision=O.PREC_FP32))
    f, t, k, _ = P.record(seed=1, count=1, cap=64)
    l1p = lambda x: np.float32(math.log1p(x))
    want0 = [l1p(2), l1p(2), l1p(5), l1p(5), 0, 0, 0, 0]
    want1 = [l1p(2), l1p(3), l1p(5), l1p(8), 0, 0, 0, 0]
    assert k[0] == 0 and k[1] == 1          # trajectory 0, step 0, candidates 0 and 1
    assert np.array_equal(f[0], np.float32(want0)) and np.array_equal(f[1], np.float32(want1))
    assert t[0] == 0 and t[1] == 0          # log(r_v c_l) with r = c = 1
    # the depth feature of step t is t / n
    steps = (k >> 14) & 0x3FFF
    assert np.allclose(f[:, 4], steps / 4.0)


def test_constant_logits_reproduce_the_unscaled_estimator():
    # equal scores give equal integer weights, i.e. the unscaled proposal
    for m in (G.planted_bernoulli(20, 0.3, seed=1), G.er_planted(60, 4.0, seed=2)):
        P = O.Prepared(m, O.Schedule(precision=O.PREC_FP32))
        a = P.run(seed=3, count=64, trace=True)
        lg = np.full((64, m.n, 32), 0.7, dtype=np.float32)
        b = P.run_ext(seed=3, count=64, logits=lg)
        assert np.array_equal(a["chosen"], b["chosen"])
        assert np.array_equal(a["log_x"], b["log_x"])


def test_logit_replay_is_unbiased_by_enumeration():
    # any positive scores keep E[X] = per(A): enumerate every path of the
    # replay with arbitrary logits and sum P(path) X(path) exactly
    from fractions import Fraction
    rng = np.random.default_rng(1)
    for seed, weighted in ((5, False), (6, True), (7, False)):
        m = G.random_weighted(6, 0.45, seed) if weighted else G.planted_bernoulli(6, 0.45, seed)
        d = m.to_dense()
        per = O.ryser_real(d)
        P = O.Prepared(m, O.Schedule(precision=O.PREC_FP32))
        lg = (rng.normal(size=(m.n, 32)) * 3).astype(np.float32)
        total, stack = 0.0, [([], Fraction(1))]
        while stack:
            prefix, prob = stack.pop()
            r = P.forced(prefix, logits=lg)
            if r[0] == "need":
                _, w, W, _, _ = r
                for k, wk in enumerate(w):
                    stack.append((prefix + [k], prob * Fraction(wk, W)))
            elif r[2] < 0:
                total += float(prob) * math.exp(r[1])
        assert total == pytest.approx(per, rel=1e-12)


def test_model_run_with_zero_network_is_the_unscaled_estimator():
    # a network that outputs a constant gives equal scores: the unscaled proposal
    m = G.er_planted(60, 4.0, seed=2)
    P = O.Prepared(m, O.Schedule(precision=O.PREC_FP32))
    params = np.zeros(O.N_PARAM)
    params[-1] = 0.3
    a = P.run(seed=5, count=40)
    b = P.run_model(seed=5, count=40, params=params)
    assert np.array_equal(a["log_x"], b["log_x"])


def _groups(sizes):
    """group codes (index << 16 | size) of consecutive groups of these sizes"""
    return np.concatenate([(np.arange(s, dtype=np.uint32) << 16) | s for s in sizes]).astype(np.uint32)


def test_centred_loss_is_the_within_step_variance_of_the_residual():
    # sum_i (e_i - mean e)^2 = (1/s) sum_{i<j} (e_i - e_j)^2 for a group of s
    # residuals: the loss from pairwise differences of plain forward outputs
    rng = np.random.default_rng(2)
    P = _rand_params(rng)
    sizes = [2, 5, 3, 7, 2, 4]
    grp = _groups(sizes)
    B = len(grp)
    X = rng.normal(size=(B, 8))
    T = rng.normal(size=B)
    e = O.mlp_forward(P, X) - T
    want, r0 = 0.0, 0
    for s in sizes:
        blk = e[r0:r0 + s]
        want += sum((blk[i] - blk[j]) ** 2 for i in range(s) for j in range(i + 1, s)) / s
        r0 += s
    loss, _ = O.mlp_grad(P, X, T, grp)
    assert loss == pytest.approx(want / B, rel=1e-12)


def test_centred_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    P = _rand_params(rng)
    grp = _groups([3, 2, 6, 4, 1, 5])
    B = len(grp)
    X = rng.normal(size=(B, 8))
    T = rng.normal(size=B)
    loss, g = O.mlp_grad(P, X, T, grp)
    idx = rng.choice(O.N_PARAM, size=50, replace=False)
    idx = np.concatenate([idx, [0, 511, 512, 575, 576, 4671, 4672, 4735, 4736, 4799]])
    for i in idx:
        h = 1e-6
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (O.mlp_grad(Pp, X, T, grp)[0] - O.mlp_grad(Pm, X, T, grp)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i
    # the output bias moves every prediction of a step alike: no gradient
    assert abs(g[4800]) < 1e-14


def test_centred_loss_ignores_a_per_step_offset():
    # adding a constant to a step's targets (a common factor of that step's
    # proposal scores, which Eq. 3 normalises away) changes nothing
    rng = np.random.default_rng(4)
    P = _rand_params(rng)
    sizes = [4, 2, 3, 5]
    grp = _groups(sizes)
    X = rng.normal(size=(len(grp), 8))
    T = rng.normal(size=len(grp))
    T2 = T + np.repeat(rng.normal(size=len(sizes)) * 5, sizes)
    l1, g1 = O.mlp_grad(P, X, T, grp)
    l2, g2 = O.mlp_grad(P, X, T2, grp)
    assert l2 == pytest.approx(l1, rel=1e-10)
    assert np.allclose(g1, g2, rtol=1e-8, atol=1e-12)
    # singleton groups carry no information
    l0, g0 = O.mlp_grad(P, X, T, _groups([1] * len(grp)))
    assert l0 == 0.0 and not g0.any()


def test_recorded_steps_form_contiguous_groups():
    # every step with at least two live candidates is recorded (finite
    # targets here), as one contiguous group in candidate order; no other
    m = G.er_planted(50, 4.0, seed=9)
    sched = O.Schedule(initial_dm=1, K0=20, K=3, sk=O.SK_FIXED, precision=O.PREC_FP32)
    P = O.Prepared(m, sched)
    f, t, k, g = P.record(seed=2, count=6, cap=1 << 20)
    tr = P.run(seed=2, count=6, trace=True)
    traj, step, cand = k >> 28, (k >> 14) & 0x3FFF, k & 0x3FFF
    r = 0
    want_steps = [(q, s) for q in range(6) for s in range(m.n) if tr["deg_v"][q, s] >= 2]
    for q, s in want_steps:
        d = tr["deg_v"][q, s]
        assert np.array_equal(traj[r:r + d], np.full(d, q)) and np.array_equal(step[r:r + d], np.full(d, s))
        assert np.array_equal(cand[r:r + d], np.arange(d))
        assert np.array_equal(g[r:r + d], (np.arange(d, dtype=np.uint32) << 16) | d)
        r += d
    assert r == len(k)
    # a capacity that cuts a step stops the recording before that step
    first = int(g[0] & 0xFFFF)
    f2, _, k2, g2 = P.record(seed=2, count=6, cap=first + 1)
    assert len(k2) == first and np.array_equal(k2, k[:first])


def test_network_logits_along_supplied_paths():
    # with K0 = 0 the features' scale terms vanish and zero logits give the
    # unscaled proposal, so the recorded pairs of a no-SK teacher walk the same
    # paths: the network's logits there are f(bf16(features)) pair by pair
    m = G.er_planted(40, 4.0, seed=10)
    P = O.Prepared(m, O.Schedule(precision=O.PREC_FP32))
    rng = np.random.default_rng(6)
    params = _rand_params(rng)
    T = 5
    out = P.run_ext_model(seed=4, count=T, logits=np.zeros((T, m.n, 32), np.float32), params=params, threads=2)
    base = P.run(seed=4, count=T, trace=True)
    assert np.array_equal(out["chosen"], base["chosen"])
    f, _, k, _ = P.record(seed=4, count=T, cap=1 << 20)
    bf = lambda a: np.asarray(a, np.float32).view(np.uint32)
    fb = ((bf(f).astype(np.uint64) + 0x7FFF + ((bf(f) >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)
    want = O.mlp_forward(params, fb.astype(np.float64), round_act=True).astype(np.float32)
    traj, step, cand = k >> 28, (k >> 14) & 0x3FFF, k & 0x3FFF
    got = out["model_logits"][traj.astype(int), step.astype(int), cand.astype(int)]
    assert len(k) > 20 and np.array_equal(got, want)


def test_ideal_proposal_gives_the_permanent_on_every_path():
    # Eq. 4: proposing the partner u of the picked vertex v with probability
    # proportional to B_vu per(minor without v's and u's lines) gives X = per(A)
    # on every completed trajectory.  The logits are ln per(minor), computed
    # here from the residual of each enumerated path (the pick re-derived: least
    # live degree, then lowest unified id; candidates in adjacency order), so
    # this also checks the pick rule, the candidate order and the correction.
    for seed in (3, 4, 8):
        m = G.planted_bernoulli(6, 0.5, seed)
        D = m.to_dense().astype(np.float64)
        n = m.n
        per = O.ryser_real(D)
        P = O.Prepared(m, O.Schedule(precision=O.PREC_FP64))

        def ideal_step_logits(pairs):
            rows = [i for i in range(n) if all(i != (a if a < n else b) for a, b in pairs)]
            cols = [j for j in range(n) if all(j != (b - n if b >= n else a - n) for a, b in pairs)]
            deg = {i: sum(D[i, j] != 0 for j in cols) for i in rows}
            deg.update({n + j: sum(D[i, j] != 0 for i in rows) for j in cols})
            v = min(deg, key=lambda x: (deg[x], x))
            if v < n:
                cand = [(v, j) for j in cols if D[v, j] != 0]
            else:
                cand = [(i, v - n) for i in rows if D[i, v - n] != 0]
            out = []
            for (i, j) in cand:
                r2 = [x for x in rows if x != i]
                c2 = [y for y in cols if y != j]
                pm = O.ryser_real(D[np.ix_(r2, c2)]) if r2 else 1.0
                out.append(math.log(pm) if pm > 0 else -30.0)
            return out

        completed = 0
        stack = [([], np.zeros((n, 32), dtype=np.float32))]
        while stack:
            prefix, lg = stack.pop()
            r = P.forced(prefix, logits=lg)
            if r[0] == "need":
                pairs = [tuple(x) for x in r[4]["chosen"][:len(prefix)]]
                lg = lg.copy()
                vals = ideal_step_logits(pairs)
                lg[len(prefix), :len(vals)] = vals
                r = P.forced(prefix, logits=lg)  # the step's weights under the ideal logits
                for k in range(len(r[1])):
                    stack.append((prefix + [k], lg))
            elif r[2] < 0:  # completed: X = per(A) up to binary32 rounding of the scores
                completed += 1
                assert math.exp(r[1]) == pytest.approx(per, rel=1e-5), (seed, prefix)
        assert completed >= 1
