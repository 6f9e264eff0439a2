"""Run control of the estimate calls (Sec. 4: runs end at a relative-error
target or a time cap): RSE targets reached in rounds of consecutive
trajectory ids, a device-side time budget that runs out, cancellation from
another host thread, and the model file round trip.

A stopped launch starts no further trajectory and lets the started ones
finish, so every trajectory it reports is bit-identical to the same
trajectory id of an unstopped run; the ones it never started carry
ln X = NaN and are not part of the sample."""
import math
import threading
import time

import numpy as np
import pytest

import oracle as O
from paper_2608_15390_b300 import inputs as G
from tests._gpu_common import binding, ctx

pytestmark = pytest.mark.gpu


def plain(**kw):
    B = binding()
    return B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL, **kw)


def test_rse_target_stops_each_matrix_in_rounds():
    B = binding()
    # plain relative spreads (oracle, 2e4 trajectories): about 1.0-1.3 for the
    # n = 20 matrices (the first round meets the target), 3.6-4.3 for the
    # n = 40 ones (several rounds, about 5e3-7e3 trajectories), 0 for J_8
    mats = [G.planted_bernoulli(20, 0.3, seed=1), G.er_planted(40, 4.0, seed=60), G.er_planted(40, 4.0, seed=61),
            G.all_ones(8)]
    target = 0.05
    res, lx = ctx().estimate_batch_ex(mats, [1 << 22] * 4, 5, plain(rse_target=target), want_log_x=True)
    for k, r in enumerate(res):
        assert r["status"] == B.PM_OK
        assert r["stop"] == B.STOP_TARGET, (k, r)
        assert r["rse"] <= target and r["n_traj"] >= 1024 and r["rounds"] >= 1
    assert max(r["rounds"] for r in res[1:3]) >= 2
    # J_8: zero spread, stops at the first round with X = 8! on every trajectory
    assert res[3]["rse"] < 1e-6 and res[3]["log_estimate"] == pytest.approx(math.log(math.factorial(8)), rel=1e-12)
    # the rounds ran trajectories 0 .. M_k - 1 of each matrix
    for k in range(4):
        M = res[k]["n_traj"]
        seg = lx[(1 << 22) * k:(1 << 22) * (k + 1)]
        assert not np.isnan(seg[:M]).any() and np.isnan(seg[M:]).all()
    # one launch over the same ids of matrix 0 gives the same ln X, bit for
    # bit, and the same statistics
    M = res[0]["n_traj"]
    one, lx1 = ctx().estimate_batch_ex([mats[0]], [M], 5, plain(), want_log_x=True)
    assert np.array_equal(lx1, lx[:M])
    assert one[0]["log_estimate"] == pytest.approx(res[0]["log_estimate"], rel=1e-12, abs=1e-12)
    assert one[0]["ess"] == pytest.approx(res[0]["ess"], rel=1e-10)


def test_budgeted_target_serves_cheapest_to_finish_first():
    """An RSE target with a time budget over matrices of very different cost:
    after the first round the budget goes to the matrices it can bring to the
    target first (priced by their measured launch time per trajectory), the
    rest get what is left.  The small matrices reach the target (their
    samples are ids 0 .. M_k - 1), the large ones stop on the budget (a cut
    round leaves some of its ids unstarted, NaN); every trajectory that ran is
    bit-identical to the same id of one plain launch."""
    B = binding()
    easy = [G.planted_bernoulli(20, 0.3, seed=1), G.er_planted(40, 4.0, seed=60), G.er_planted(40, 4.0, seed=61)]
    hard = [G.er_planted(1500, 6.0, seed=71), G.er_planted(1400, 6.0, seed=72)]
    mats = [hard[0], easy[0], easy[1], hard[1], easy[2]]
    cap = 1 << 22
    res, lx = ctx().estimate_batch_ex(mats, [cap] * len(mats), 5, plain(rse_target=0.05, time_budget_s=1.5),
                                      want_log_x=True)
    for k in (1, 2, 4):
        assert res[k]["stop"] == B.STOP_TARGET and res[k]["rse"] <= 0.05, (k, res[k])
    for k in (0, 3):
        assert res[k]["stop"] == B.STOP_TIME and res[k]["n_traj"] > 0, (k, res[k])
    assert res[0]["status"] == B.PM_ETIMEOUT
    for k in range(len(mats)):
        M = res[k]["n_traj"]
        seg = lx[cap * k:cap * (k + 1)]
        assert int((~np.isnan(seg)).sum()) == M, k
        if res[k]["stop"] == B.STOP_TARGET:  # every round of it ran whole: ids 0 .. M - 1
            assert not np.isnan(seg[:M]).any(), k
    # matrix 3's first ids (its index in the batch keys its draws) in one plain launch
    M = 4096
    ref, lxr = ctx().estimate_batch_ex(mats, [0, 0, 0, M, 0], 5, plain(), want_log_x=True)
    seg = lx[cap * 3:cap * 3 + M]
    ran = ~np.isnan(seg)
    assert ran.sum() > 0 and np.array_equal(lxr[ran], seg[ran])


def _long_plain_workload(seconds=1.5):
    """A plain single-matrix run that takes about `seconds` on this device."""
    m = G.er_planted(1500, 6.0, seed=71)
    t0 = time.perf_counter()
    ctx().estimate_permanent(m, 4096, 3, plain())
    rate = 4096 / (time.perf_counter() - t0)
    return m, int(max(8192, rate * seconds))


def test_device_time_budget_runs_out():
    B = binding()
    m, n_traj = _long_plain_workload()
    t0 = time.perf_counter()
    res, lx = ctx().estimate_batch_ex([m], [n_traj], 3, plain(time_budget_s=0.1), want_log_x=True)
    t_stop = time.perf_counter() - t0
    r = res[0]
    assert r["status"] == B.PM_ETIMEOUT and r["stop"] == B.STOP_TIME, r
    ran = ~np.isnan(lx)
    assert 0 < r["n_traj"] == ran.sum() < n_traj
    t0 = time.perf_counter()
    full, lxf = ctx().estimate_batch_ex([m], [n_traj], 3, plain(), want_log_x=True)
    t_full = time.perf_counter() - t0
    assert full[0]["status"] == B.PM_OK and full[0]["n_traj"] == n_traj
    assert np.array_equal(lx[ran], lxf[ran])  # the trajectories that ran are the unstopped run's
    assert t_stop < 0.5 * t_full, (t_stop, t_full)
    # the statistics are those of the trajectories that ran
    st = O.stats(lx[ran])
    assert r["log_estimate"] == pytest.approx(st["log_estimate"], rel=1e-12, abs=1e-12)


def test_time_budget_of_a_resident_batch_run():
    B = binding()
    m, n_traj = _long_plain_workload()
    bt = ctx().batch([m], [n_traj], plain(time_budget_s=0.1), graph=True)
    res, lx = bt.run(0, 3, want_log_x=True)
    assert res[0]["status"] == B.PM_ETIMEOUT and 0 < res[0]["n_traj"] < n_traj
    assert res[0]["n_traj"] == int((~np.isnan(lx)).sum())
    bt.close()
    with pytest.raises(B.PmError):
        ctx().batch([m], [64], plain(rse_target=0.1))


def test_cancel_from_another_thread():
    B = binding()
    m, n_traj = _long_plain_workload(3.0)
    out = {}

    def run():
        t0 = time.perf_counter()
        out["r"] = ctx().estimate_permanent(m, n_traj, 4, plain())
        out["t"] = time.perf_counter() - t0

    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.3)
    ctx().cancel()
    th.join(timeout=60)
    assert not th.is_alive()
    r = out["r"]
    assert r["status"] == B.PM_ECANCELLED and r["stop"] == B.STOP_CANCELLED, r
    assert 0 < r["n_traj"] < n_traj and out["t"] < 2.0, (r["n_traj"], out["t"])
    # the next call starts with the flag cleared
    again = ctx().estimate_permanent(m, 256, 4, plain())
    assert again["status"] == B.PM_OK and again["n_traj"] == 256


def test_model_save_load_round_trip(tmp_path):
    B = binding()
    rng = np.random.default_rng(3)
    p = (rng.normal(size=O.N_PARAM) * 0.3).astype(np.float32)
    m1 = ctx().model(p)
    path = str(tmp_path / "net.pmmodel")
    m1.save(path)
    m2 = ctx().model_load(path)
    assert np.array_equal(m1.params(), m2.params())
    mat = G.er_planted(200, 6.0, seed=9)
    s1 = B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL, learned=m1)
    s2 = B.Schedule(initial_dm=1, K0=50, precision=B.PREC_FP32_PROPOSAL, learned=m2)
    a = ctx().estimate_batch_ex([mat], [512], 2, s1, want_log_x=True)[1]
    b = ctx().estimate_batch_ex([mat], [512], 2, s2, want_log_x=True)[1]
    assert np.array_equal(a, b)
    raw = bytearray(open(path, "rb").read())
    raw[40] ^= 1  # one flipped bit in the parameters: the checksum rejects it
    bad = str(tmp_path / "bad.pmmodel")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(B.PmError):
        ctx().model_load(bad)
    open(bad, "wb").write(bytes(raw[:100]))
    with pytest.raises(B.PmError):
        ctx().model_load(bad)
    with pytest.raises(B.PmError):
        ctx().model_load(str(tmp_path / "missing"))
    m1.close()
    m2.close()


def test_tune_theta_picks_the_lowest_work_normalised_variance():
    """pm_tune_theta: one budgeted probe per candidate theta (Thrs / Trck, the
    threshold Sec. 4 leaves to tuning); the schedule comes back with the
    candidate of least RSE^2 x device seconds."""
    B = binding()
    m = G.er_planted(400, 6.0, seed=91)
    s = B.preset("local_threshold")
    thetas = [0.1, 0.33, 0.7]
    best, scores = ctx().tune_theta(m, s, thetas, probe_s=0.3, seed=4)
    assert np.isfinite(scores).all(), scores
    assert best == thetas[int(np.argmin(scores))]
    with pytest.raises(B.PmError):
        ctx().tune_theta(m, B.Schedule(initial_dm=1, K0=100, precision=B.PREC_FP32_PROPOSAL), thetas)
