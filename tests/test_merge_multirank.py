"""Merging runs over disjoint trajectory ranges (ranks, or rounds of a
request): the host merge of the sufficient statistics equals the statistics
of all trajectories at once.  Two gloo ranks on the CPU each run the oracle
on their own range; rank 0 merges."""
import math
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2608_15390_b300 import inputs as G
from paper_2608_15390_b300.merge import merge


def _as_result(st):
    return {"n_traj": st["n_traj"], "n_alive": st["n_alive"], "log_sum_x": st["log_sum_x"],
            "log_sum_x2": st["log_sum_x2"]}


def test_merge_equals_whole_run():
    m = G.planted_bernoulli(20, 0.3, seed=1)
    P = O.Prepared(m, O.Schedule(K0=10, precision=O.PREC_FP32))
    lx = P.run(seed=3, count=3000, threads=4)["log_x"]
    whole = O.stats(lx)
    parts = [O.stats(lx[a:b]) for a, b in ((0, 1000), (1000, 1700), (1700, 3000))]
    got = merge(_as_result(p) for p in parts)
    for key in ("log_estimate", "ess", "p_match", "rel_spread", "rse"):
        assert got[key] == pytest.approx(whole[key], rel=1e-10), key
    assert got["n_traj"] == 3000 and got["n_alive"] == whole["n_alive"]


def test_merge_sums_counts_and_keeps_the_largest_stop_reason():
    a = {"n_traj": 10, "n_alive": 4, "log_sum_x": 1.0, "log_sum_x2": 2.5, "n_dm_calls": 3, "n_full_sk": 7,
         "n_local_sk": 11, "alg_bytes": 100, "mlp_rows": 9, "rounds": 1, "stop": 0}
    b = {"n_traj": 6, "n_alive": 0, "log_sum_x": -math.inf, "log_sum_x2": -math.inf, "n_dm_calls": 1,
         "n_full_sk": 2, "n_local_sk": 3, "alg_bytes": 50, "mlp_rows": 1, "rounds": 2, "stop": 2}
    r = merge([a, b])
    assert (r["n_traj"], r["n_alive"], r["n_dm_calls"], r["n_full_sk"], r["n_local_sk"]) == (16, 4, 4, 9, 14)
    assert (r["alg_bytes"], r["mlp_rows"], r["rounds"], r["stop"]) == (150, 10, 3, 2)
    assert r["log_estimate"] == pytest.approx(1.0 - math.log(16), rel=1e-15)
    assert r["ess"] == pytest.approx(math.exp(2 * 1.0 - 2.5), rel=1e-15)


def test_merge_all_dead_and_single():
    d = {"n_traj": 5, "n_alive": 0, "log_sum_x": -math.inf, "log_sum_x2": -math.inf}
    r = merge([d, d])
    assert r["log_estimate"] == -math.inf and r["p_match"] == 0.0
    one = merge([{"n_traj": 1, "n_alive": 1, "log_sum_x": 2.0, "log_sum_x2": 4.0}])
    assert one["log_estimate"] == 2.0 and math.isnan(one["rse"])


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = G.planted_bernoulli(20, 0.3, seed=1)
    P = O.Prepared(m, O.Schedule(K0=10, precision=O.PREC_FP32))
    per = 1500
    lx = P.run(seed=3, count=per, first_traj=rank * per)["log_x"]
    mine = _as_result(O.stats(lx))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        merged = merge(gathered)
        whole = O.stats(P.run(seed=3, count=per * world)["log_x"])
        np.save(out_path, np.array([merged["log_estimate"], whole["log_estimate"], merged["ess"], whole["ess"],
                                    merged["rse"], whole["rse"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_single_run(tmp_path):
    out = str(tmp_path / "merged.npy")
    port = 29500 + (os.getpid() % 2000)
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    a = np.load(out)
    assert a[0] == pytest.approx(a[1], rel=1e-12)
    assert a[2] == pytest.approx(a[3], rel=1e-10)
    assert a[4] == pytest.approx(a[5], rel=1e-10)
