"""Resident batches (pm_batch): one persistent launch per run, captured as a
CUDA graph, layouts chosen by the autotuner.  Whatever the layout and the
launch route, every trajectory's ln X must be identical to the one
pm_estimate_batch_ex produces (each trajectory depends only on the seed, its
id and its matrix), and every trajectory must match the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import binding, ctx, logx_close

pytestmark = pytest.mark.gpu


def _mats():
    return [G.er_planted(n, d, seed=300 + i) for i, (n, d) in enumerate([(40, 4.0), (130, 6.0), (75, 5.0),
                                                                         (260, 4.5), (33, 7.0)])]


def _schedules(B):
    return {
        "plain": B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL),
        "adaptive": B.Schedule(initial_dm=1, K0=50, K=5, sk=B.SK_ADAPTIVE, precision=B.PREC_FP32_PROPOSAL),
        "local_threshold": B.preset("local_threshold"),
        "fp64_fixed_trck": B.Schedule(initial_dm=1, K0=20, K=2, sk=B.SK_FIXED, dm=B.DM_TRCK,
                                      precision=B.PREC_FP64),
    }


@pytest.mark.parametrize("name", ["plain", "adaptive", "local_threshold", "fp64_fixed_trck"])
@pytest.mark.parametrize("graph,autotune", [(True, False), (False, True), (True, True)])
def test_batch_runs_equal_the_one_shot_call(name, graph, autotune):
    B = binding()
    mats = _mats()
    sched = _schedules(B)[name]
    nt = [70, 33, 129, 40, 5]
    bt = ctx().batch(mats, nt, sched, graph=graph, autotune=autotune)
    for first, seed in ((0, 7), (1000, 7), (55, 123456789)):
        got, lx = bt.run(first, seed, want_log_x=True)
        want, lx_ref = ctx().estimate_batch_ex(mats, nt, seed, sched, first_traj=first, want_log_x=True)
        assert np.array_equal(np.isneginf(lx), np.isneginf(lx_ref))
        ok = np.isfinite(lx_ref)
        assert np.array_equal(lx[ok], lx_ref[ok]), "ln X differs from the one-shot call"
        for a, b in zip(got, want):
            for key in ("n_traj", "n_alive", "n_dm_calls", "n_full_sk", "n_local_sk"):
                assert a[key] == b[key], key
            assert a["log_sum_x"] == pytest.approx(b["log_sum_x"], rel=1e-12, abs=1e-12)
    if autotune:
        for k in range(len(mats)):
            info = bt.plan(k)
            assert info["groups"] >= 1 and info["g"] in (1, 2, 4, 8, 16)
            if info["probe_traj_per_s"] > 0 and info["heuristic_traj_per_s"] > 0:
                assert info["probe_traj_per_s"] >= info["heuristic_traj_per_s"]
    bt.close()


def test_batch_trajectories_match_the_oracle():
    B = binding()
    mats = _mats()[:3]
    sched = _schedules(B)["local_threshold"]
    osched = O.preset("local_threshold", precision=O.PREC_FP32)
    nt = [24, 24, 24]
    bt = ctx().batch(mats, nt, sched, graph=True, autotune=True)
    _, lx = bt.run(500, 3, want_log_x=True)
    for k, m in enumerate(mats):
        o = O.Prepared(m, osched).run(seed=3, count=24, first_traj=500, matrix=k, threads=8)
        assert logx_close(lx[24 * k:24 * (k + 1)], o["log_x"], 1e-12) <= 1e-12
    bt.close()


def test_batch_with_the_learned_proposal_and_host_inputs():
    B = binding()
    mats = _mats()
    rng = np.random.default_rng(2)
    model = ctx().model((rng.normal(size=4801) * 0.3).astype(np.float32))
    sched = B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL, learned=model)
    nt = [50] * len(mats)
    bt = ctx().batch(mats, nt, sched, graph=True, autotune=True)  # host CSR: copied at creation
    _, lx = bt.run(9, 11, want_log_x=True)
    _, lx_ref = ctx().estimate_batch_ex(mats, nt, 11, sched, first_traj=9, want_log_x=True)
    ok = np.isfinite(lx_ref)
    assert np.array_equal(np.isneginf(lx), np.isneginf(lx_ref)) and np.array_equal(lx[ok], lx_ref[ok])
    bt.close()
    model.close()


def test_batch_rejects_bad_arguments():
    B = binding()
    with pytest.raises(B.PmError):
        ctx().batch(_mats()[:1], [1 << 49], _schedules(B)["plain"])


def test_closing_the_context_first_is_safe():
    B = binding()
    c = B.Context(0)
    bt = c.batch(_mats()[:2], [8, 8], _schedules(B)["plain"], graph=True)
    bt.run(0, 1)
    c.close()      # closes the batch first
    bt.close()     # no-op
    del bt
