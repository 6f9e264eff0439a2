"""CPU checks of the bench's host-side analysis: the first-infeasible-child
scan used by the z-bucket histogram (a kept perfect matching repaired by one
alternating search per elimination) against a fresh maximum matching of
every child, on oracle paths of the row-order rule, whose deaths always
follow an infeasible child."""
import importlib.util
import os

import numpy as np
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import maximum_bipartite_matching

import oracle as O
from paper_2608_15390_b300 import inputs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_first_infeasible_child_matches_fresh_matchings():
    bench = _bench()
    found = 0
    for seed in range(12):
        m = G.planted_bernoulli(10, 0.15, seed=seed)
        tr = O.Prepared(m, O.Schedule(precision=O.PREC_FP64, vertex_rule=O.VR_ROW_ORDER)).run(
            seed=seed, count=30, trace=True)
        got = bench.first_infeasible_steps(m, tr["chosen"])
        d = m.to_dense() != 0
        n = m.n
        for q in range(30):
            rows, cols, want = list(range(n)), list(range(n)), -1
            for t in range(n - 1):
                v, u = tr["chosen"][q, t]
                if v < 0:
                    break
                R, C = (v, u - n) if v < n else (u, v - n)
                rows.remove(R)
                cols.remove(C)
                mm = maximum_bipartite_matching(csr_matrix(d[np.ix_(rows, cols)].astype(float)), perm_type="column")
                if (mm < 0).any():
                    want = t
                    break
            assert got[q] == want, (seed, q)
            if tr["dead_step"][q] >= 0:
                assert 0 <= want < tr["dead_step"][q]
            found += want >= 0
    assert found > 50
