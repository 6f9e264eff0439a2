"""Host-side merge of estimator results from disjoint trajectory sets.

Trajectories are independent and their Philox counters disjoint, so runs over
disjoint trajectory ranges (other ranks, earlier rounds of a request) combine
exactly through their sufficient statistics: M, #alive, ln sum X and
ln sum X^2 (pm_result.n_traj, n_alive, log_sum_x, log_sum_x2).  The merged
values follow the definitions of Sec. 2 (ESS, p_match) and Sec. 4 "Metrics"
(mean, s_X with M - 1, relative spread, RSE), evaluated in log space so
that nothing overflows.  Pure arithmetic on a handful of scalars per run.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List


def _lse(values: List[float]) -> float:
    finite = [v for v in values if v > -math.inf]
    if not finite:
        return -math.inf
    c = max(finite)
    return c + math.log(sum(math.exp(v - c) for v in finite))


def merge(results: Iterable[Dict]) -> Dict:
    """Merge result dicts (as returned by the binding) of disjoint runs."""
    rs = list(results)
    M = sum(int(r["n_traj"]) for r in rs)
    alive = sum(int(r["n_alive"]) for r in rs)
    ls1 = _lse([r["log_sum_x"] for r in rs])
    ls2 = _lse([r["log_sum_x2"] for r in rs])
    out = {"n_traj": M, "n_alive": alive, "log_sum_x": ls1, "log_sum_x2": ls2,
           "p_match": alive / M if M else 0.0}
    if M == 0 or ls1 == -math.inf:
        out.update(log_estimate=-math.inf, estimate=0.0, ess=0.0, rel_spread=math.nan, rse=math.nan)
        return out
    log_mean = ls1 - math.log(M)
    out["log_estimate"] = log_mean
    out["estimate"] = math.exp(log_mean) if log_mean < 709 else math.inf
    out["ess"] = math.exp(2 * ls1 - ls2)
    # s_X^2 = (sum X^2 - M mean^2) / (M - 1); relative to mean^2:
    # (M sum X^2 / (sum X)^2 - 1) * M / (M - 1)
    if M > 1:
        ratio = M * math.exp(ls2 - 2 * ls1)
        var_rel = max(0.0, ratio - 1.0) * M / (M - 1)
        out["rel_spread"] = math.sqrt(var_rel)
        out["rse"] = out["rel_spread"] / math.sqrt(M)
    else:
        out["rel_spread"] = math.nan
        out["rse"] = math.nan
    return out
