"""The allocation-free statistics entry point (pm_log_weight_stats_noalloc)
against the statistics estimate_permanent reports for the same
log-weights.  This file is collected last so that a failure here leaves
every other test already run."""
import numpy as np
import pytest

from paper_2608_15390_b300 import inputs as G

pytestmark = pytest.mark.gpu


def _noalloc(B, torch, lx_host):
    lx = torch.from_numpy(lx_host).cuda()
    out = torch.zeros(9, dtype=torch.float64, device="cuda")
    st = B.log_weight_stats_noalloc(lx.data_ptr(), lx.numel(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == B.PM_OK
    torch.cuda.synchronize()
    raw = out.cpu().numpy()
    d = dict(zip(B.WEIGHT_STATS_FIELDS[:7], raw[:7].tolist()))
    d["n_traj"], d["n_alive"] = (int(x) for x in raw[7:9].view(np.uint64))
    return d


def test_noalloc_stats_match_estimate_twice():
    import torch
    from paper_2608_15390_b300 import binding as B
    ctx = B.Context(0)
    sched = B.Schedule(initial_dm=1, K0=20, precision=B.PREC_FP32_PROPOSAL)
    cases = [(G.planted_bernoulli(20, 0.3, seed=1), 70000), (G.er_planted(300, 5.0, seed=3), 9001)]
    for m, T in cases:  # two calls in a row share the fixed scratch
        res, lx = ctx.estimate_batch_ex([m], [T], 5, sched, want_log_x=True)
        ref = res[0]
        got = _noalloc(B, torch, lx)
        assert got["n_traj"] == ref["n_traj"] == T
        assert got["n_alive"] == ref["n_alive"]
        for key in ("log_estimate", "ess", "p_match", "rel_spread", "rse", "log_sum_x", "log_sum_x2"):
            assert got[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-12), key
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2608_15390_b300 import binding as B
    lx = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(9, dtype=torch.float64, device="cuda")
    assert B.log_weight_stats_noalloc(lx.data_ptr(), (1 << 26) + 1, out.data_ptr()) == B.PM_EUNSUPPORTED
    assert B.log_weight_stats_noalloc(lx.data_ptr(), 0, out.data_ptr()) == B.PM_EINVAL
