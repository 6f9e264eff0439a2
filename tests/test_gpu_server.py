"""The serving loop (pm_server): requests estimated in rounds of one
persistent launch each.  A request's statistics must be exactly those of its
trajectories (the same trajectories pm_estimate_batch_ex runs for the round's
range and position), merged over its rounds; the finish rules (target,
budget, refusal, per = 0) must hold; and the estimates must agree with exact
permanents."""
import math

import numpy as np
import pytest

from paper_2608_15390_b300 import inputs as G
from paper_2608_15390_b300.merge import merge
from tests._gpu_common import binding, ctx
import oracle as O

pytestmark = pytest.mark.gpu


def _sched(B):
    return B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL)


def _drain(sv, max_rounds=1000):
    out = []
    for _ in range(max_rounds):
        done, na, nq = sv.round()
        out += done
        if na == 0 and nq == 0:
            return out
    raise AssertionError("server did not drain")


def test_one_round_equals_the_batch_call():
    B = binding()
    mats = [G.er_planted(60, 5.0, seed=1), G.er_planted(90, 4.0, seed=2)]
    T = 256
    sv = ctx().server(_sched(B), seed=5, steps_per_round=1 << 30, traj_min=T, traj_max=T, min_traj_done=1)
    ids = [sv.submit(m, 1e9, T) for m in mats]
    done = _drain(sv)
    assert sorted(d["id"] for d in done) == sorted(ids)
    want, _ = ctx().estimate_batch_ex(mats, [T, T], 5, _sched(B), first_traj=0)
    for d in done:
        k = ids.index(d["id"])
        r, w = d["result"], want[k]
        assert d["status"] == B.REQ_DONE and d["rounds"] == 1
        for key in ("n_traj", "n_alive", "log_sum_x", "log_sum_x2"):
            assert r[key] == w[key], key
        assert r["ess"] == pytest.approx(w["ess"], rel=1e-12)
    sv.close()


def test_rounds_merge_exactly():
    # traj_max = 100 per round and a budget of 350: rounds of 100, 100, 100, 50,
    # each the batch call's trajectories of range round << 24 at position 0
    B = binding()
    m = G.er_planted(70, 5.0, seed=3)
    sv = ctx().server(_sched(B), seed=9, steps_per_round=1 << 30, traj_min=1, traj_max=100, min_traj_done=1)
    sv.submit(m, 1e-9, 350)
    (d,) = _drain(sv)
    assert d["status"] == B.REQ_BUDGET and d["rounds"] == 4 and d["result"]["n_traj"] == 350
    parts = []
    for rnd, T in enumerate((100, 100, 100, 50)):
        r, _ = ctx().estimate_batch_ex([m], [T], 9, _sched(B), first_traj=rnd << 24)
        parts.append(r[0])
    want = merge(parts)
    assert d["result"]["log_sum_x"] == pytest.approx(want["log_sum_x"], rel=1e-13, abs=1e-13)
    assert d["result"]["log_sum_x2"] == pytest.approx(want["log_sum_x2"], rel=1e-13, abs=1e-13)
    assert d["result"]["rse"] == pytest.approx(want["rse"], rel=1e-10)
    sv.close()


def test_finish_rules_and_exact_permanents():
    B = binding()
    sv = ctx().server(_sched(B), seed=2, device_budget_bytes=64 << 20, steps_per_round=1 << 22, traj_min=64,
                      traj_max=1 << 15, min_traj_done=2048)
    # no perfect matching: per(A) = 0, finished at admission
    z = G.csr_from_coo(4, [0, 1, 2, 3], [0, 0, 2, 3])
    # exact permanents by Ryser
    small = [G.planted_bernoulli(14, 0.3, seed=s) for s in (1, 2, 3)]
    per = [O.ryser(m.to_dense()) for m in small]
    # far above the budget: refused
    big = G.er_planted(400_000, 4.0, seed=4)
    ids = {sv.submit(z, 1e-2, 1 << 20): "zero", sv.submit(big, 1e-2, 1 << 20): "big"}
    for k, m in enumerate(small):
        ids[sv.submit(m, 2e-3, 1 << 22)] = k
    done = {ids[d["id"]]: d for d in _drain(sv)}
    assert done["zero"]["status"] == B.REQ_DONE and done["zero"]["result"]["log_estimate"] == -math.inf
    assert done["big"]["status"] == B.REQ_REFUSED
    for k in range(3):
        d = done[k]
        assert d["status"] == B.REQ_DONE and d["result"]["rse"] <= 2e-3 and d["result"]["n_traj"] >= 2048
        rel = abs(math.exp(d["result"]["log_estimate"]) / per[k] - 1)
        assert rel < 6 * d["result"]["rse"] + 1e-3, (k, rel, d["result"]["rse"])
    sv.close()
