"""Merge of estimator results from disjoint trajectory sets.

Trajectories are independent and their Philox counters disjoint, so runs over
disjoint trajectory ranges (other ranks, earlier rounds of a request, resumed
runs) combine exactly through their sufficient statistics: M, #alive,
ln sum X and ln sum X^2 (pm_result.n_traj, n_alive, log_sum_x, log_sum_x2).
The arithmetic is the library's pm_merge_results (host code, no device),
which evaluates the definitions of Sec. 2 (ESS, p_match) and Sec. 4
"Metrics" (mean, s_X with M - 1, relative spread, RSE) in log space.
"""
from __future__ import annotations

from typing import Dict, Iterable

from .binding import merge_results


def merge(results: Iterable[Dict]) -> Dict:
    """Merge result dicts (as returned by the binding) of disjoint runs of
    one matrix; fields absent from a dict count as 0."""
    return merge_results(list(results))
