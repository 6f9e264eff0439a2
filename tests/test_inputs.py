"""The seeded input generators produce the workloads their recipes state:
CSR well formed (sorted, distinct columns), the planted permutation present
(so a perfect matching exists), the requested sizes, and the same matrix for
the same seed.  They hold none of the method's arithmetic."""
import numpy as np

from paper_2608_15390_b300 import inputs as G


def _check_csr(m):
    rp, ci = np.asarray(m.row_ptr), np.asarray(m.col_idx)
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    assert np.all((ci >= 0) & (ci < m.n))
    for i in range(m.n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0), i  # strictly increasing: sorted, distinct


def _has_perfect_matching(m):
    """Kuhn's augmenting paths on the bipartite graph of the pattern."""
    rp, ci = np.asarray(m.row_ptr), np.asarray(m.col_idx)
    match_col = -np.ones(m.n, dtype=np.int64)

    def augment(i, seen):
        for j in ci[rp[i]:rp[i + 1]]:
            if seen[j]:
                continue
            seen[j] = True
            if match_col[j] < 0 or augment(match_col[j], seen):
                match_col[j] = i
                return True
        return False

    return all(augment(i, np.zeros(m.n, dtype=bool)) for i in range(m.n))


def test_generators_are_well_formed_and_reproducible():
    cases = [
        lambda: G.planted_bernoulli(20, 0.3, seed=1),
        lambda: G.er_planted(300, 6.0, seed=4),
        lambda: G.band_random(500, 2500, seed=3),
        lambda: G.powerlaw_planted(400, seed=5),
        lambda: G.block_diagonal(100, 0.3, seed=6),
    ]
    for make in cases:
        a, b = make(), make()
        _check_csr(a)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
        assert _has_perfect_matching(a)


def test_stated_sizes_and_shapes():
    band = G.band_random(1000, 5000, seed=3)
    assert band.nnz == 5000
    rp, ci = np.asarray(band.row_ptr), np.asarray(band.col_idx)
    rows = np.repeat(np.arange(1000), np.diff(rp))
    for off in (-1, 0, 1):  # the width-3 band is present
        i = np.arange(max(0, -off), min(1000, 1000 - off))
        keys = set((rows * 1000 + ci).tolist())
        assert all(int(x) * 1000 + int(x) + off in keys for x in i)
    er = G.er_planted(2000, 6.0, seed=9)
    assert 6.0 <= er.nnz / 2000 <= 8.0  # average degree d plus the planted entry
    batch = G.batch_er(64, 100, 2000, 4.0, 8.0, seed=2)
    assert len(batch) == 64 and all(100 <= m.n <= 2000 for m in batch)
    pl = G.powerlaw_planted(5000, seed=5)
    deg = np.diff(np.asarray(pl.row_ptr))
    assert np.median(deg) >= 2 and deg.max() > 50  # minimum 2 plus a heavy tail
