"""Write e4_log_permanents.json: the exact ln per(A) of the block-diagonal
matrices of the Sec. 4 known-permanent family that the E4 preset study runs
(bench.py --workload e4).

per(A) of a block-diagonal matrix under independent row and column
permutations is the product of its blocks' permanents (Eq. 1: a permutation
with a nonzero product stays inside the blocks), so ln per(A) is the sum of
the blocks' ln per, each computed by the oracle's Ryser formula (exact
integers for binary blocks, binary64 for weighted ones).  Calls nothing but
the oracle and the seeded input generator.

    python tests/golden/make_e4_log_permanents.py
"""
import json
import math
import os
import sys
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# the study's grid: order, deletion probability, weights; generator seed 4000 + index
GRID = [(n, p, w) for n in (100, 500, 1000, 2000) for p in (0.1, 0.5, 0.9) for w in (False, True)]


def one(i):
    import oracle as O
    from paper_2608_15390_b300 import inputs as G
    n, p, w = GRID[i]
    m = G.block_diagonal(n, p, seed=4000 + i, weighted=w)
    lp = 0.0
    for b in m.blocks:
        v = O.ryser(b) if not w else O.ryser_real(b)
        lp += math.log(v)
    return {"index": i, "n": n, "p": p, "weighted": w, "seed": 4000 + i, "nnz": int(m.nnz),
            "blocks": len(m.blocks), "log_per": lp}


if __name__ == "__main__":
    with ProcessPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        rows = list(ex.map(one, range(len(GRID))))
    out = {"family": "Sec. 4 block-diagonal, blocks of order 20 or 25, entries off the block diagonal "
                     "deleted with probability p, weights U[1, 1.5] when weighted, random row and column "
                     "permutations (paper_2608_15390_b300.inputs.block_diagonal)",
           "method": "sum over blocks of ln per(block), the oracle's Ryser formula",
           "matrices": rows}
    with open(os.path.join(HERE, "e4_log_permanents.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(len(rows), "matrices written")
