"""Seeded synthetic matrix generators.

This module only builds input matrices; it holds none of the estimator's
arithmetic, and both the CUDA path and the CPU oracle consume what it returns.
Every generator is deterministic in its ``seed`` (numpy's PCG64 stream) and
returns a :class:`Csr` with sorted, duplicate-free column indices per row.

Families (the shapes of the paper's workloads and of the scaled-up targets):

* ``planted_bernoulli``  -- n x n, each entry Bernoulli(p), plus a planted
  random permutation (guarantees a perfect matching).
* ``er_planted``         -- Erdos-Renyi bipartite, average degree d, plus a
  planted permutation.
* ``band_random``        -- |i-j| <= 1 band, plus a planted permutation, plus
  uniform off-band entries until nnz reaches a target.
* ``powerlaw_planted``   -- row degrees from P(d) ~ d^-a (d >= dmin), distinct
  uniform columns, plus a planted permutation.
* ``block_diagonal``     -- the known-permanent family of Sec. 4 (blocks of
  order 20/25 with the diagonal kept, off-diagonal entries deleted with
  probability p, optional U[1,1.5] weights, rows and columns permuted).
* small structured matrices for closed-form checks (all-ones, tridiagonal,
  permutation, upper triangular, circulant k-regular).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Csr:
    """Compressed sparse row matrix (int64 row_ptr, int32 col_idx, optional
    float32 values; ``values is None`` means a 0/1 matrix)."""

    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    values: Optional[np.ndarray] = None
    # exact-permanent helpers for block-structured generators: the dense
    # blocks (before permutation) whose permanents multiply to per(A)
    blocks: List[np.ndarray] = field(default_factory=list)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col_idx] = 1.0 if self.values is None else self.values
        return d


def csr_from_coo(n: int, rows, cols, vals=None) -> Csr:
    """Build a Csr from (row, col[, val]) triples; duplicates keep the first."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * n + cols
    key, first = np.unique(key, return_index=True)
    r = key // n
    c = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    v = None
    if vals is not None:
        v = np.asarray(vals, dtype=np.float32)[first]
    return Csr(n, row_ptr, c, v)


def csr_from_dense(d: np.ndarray, weighted: bool = False) -> Csr:
    d = np.asarray(d)
    n = d.shape[0]
    r, c = np.nonzero(d)
    return csr_from_coo(n, r, c, d[r, c] if weighted else None)


# ----------------------------------------------------------------------------
# workload families
# ----------------------------------------------------------------------------

def planted_bernoulli(n: int, p: float, seed: int) -> Csr:
    """Each entry Bernoulli(p) plus a planted uniform permutation."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    dense = rng.random((n, n)) < p
    dense[np.arange(n), perm] = True
    return csr_from_dense(dense)


def er_planted(n: int, d: float, seed: int) -> Csr:
    """Erdos-Renyi-like bipartite graph of average degree ``d`` plus a planted
    permutation.  Row i draws Binomial(n, d/n) columns uniformly (repeats
    merged), then (i, perm[i]) is added."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    k = rng.binomial(n, min(1.0, d / n), size=n)
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = rng.integers(0, n, size=int(k.sum()), dtype=np.int64)
    rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([cols, perm.astype(np.int64)])
    return csr_from_coo(n, rows, cols)


def band_random(n: int, nnz: int, seed: int, half_width: int = 1) -> Csr:
    """Band |i-j| <= half_width, planted permutation, then uniform off-band
    entries until the matrix holds ``nnz`` nonzeros."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    rows, cols = [], []
    for off in range(-half_width, half_width + 1):
        i = np.arange(max(0, -off), min(n, n - off), dtype=np.int64)
        rows.append(i)
        cols.append(i + off)
    rows.append(np.arange(n, dtype=np.int64))
    cols.append(perm.astype(np.int64))
    key = np.unique(np.concatenate(rows) * n + np.concatenate(cols))
    while key.size < nnz:
        extra = nnz - key.size
        rr = rng.integers(0, n, size=extra + extra // 8 + 16, dtype=np.int64)
        cc = rng.integers(0, n, size=rr.size, dtype=np.int64)
        new = np.setdiff1d(np.unique(rr * n + cc), key, assume_unique=True)
        new = rng.permutation(new)[:extra]
        key = np.union1d(key, new)
    return csr_from_coo(n, key // n, key % n)


def powerlaw_planted(n: int, seed: int, exponent: float = 2.5, dmin: int = 2) -> Csr:
    """Row degrees from the discrete power law P(d) ~ d^-exponent, d >= dmin,
    capped at n; uniform columns per row (a repeated draw is dropped, so a hub
    row can hold slightly fewer than d); plus a planted permutation."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    support = np.arange(dmin, n + 1, dtype=np.float64)
    pmf = support ** (-exponent)
    pmf /= pmf.sum()
    deg = rng.choice(support.astype(np.int64), size=n, p=pmf)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([cols, perm.astype(np.int64)])
    key = np.unique(rows * n + cols)
    return csr_from_coo(n, key // n, key % n)


def block_diagonal(n: int, p: float, seed: int, weighted: bool = False, orders=(20, 25)) -> Csr:
    """Known-permanent family of Sec. 4: dense diagonal blocks of order 20 or
    25 summing to n, every off-diagonal block entry deleted with probability
    p, the diagonal kept, weights U[1, 1.5] when ``weighted``; rows and
    columns are then permuted independently.  ``blocks`` holds the blocks."""
    rng = np.random.default_rng(seed)
    if tuple(orders) == (20,):
        if n % 20:
            raise ValueError(f"n={n} is not a sum of 20s")
        a, b = 0, n // 20
    else:
        comps = [(a, (n - 25 * a) // 20) for a in range(n // 25 + 1)
                 if (n - 25 * a) >= 0 and (n - 25 * a) % 20 == 0]
        if not comps:
            raise ValueError(f"n={n} is not a sum of 20s and 25s")
        a, b = comps[rng.integers(len(comps))]
    orders = rng.permutation([25] * a + [20] * b)
    blocks, rows, cols, vals = [], [], [], []
    base = 0
    for k in orders:
        keep = rng.random((k, k)) >= p
        np.fill_diagonal(keep, True)
        w = rng.uniform(1.0, 1.5, size=(k, k)) if weighted else np.ones((k, k))
        blk = np.where(keep, w, 0.0).astype(np.float32).astype(np.float64)
        blocks.append(blk)
        r, c = np.nonzero(keep)
        rows.append(r + base)
        cols.append(c + base)
        vals.append(blk[r, c])
        base += k
    pr = rng.permutation(n)
    pc = rng.permutation(n)
    m = csr_from_coo(n, pr[np.concatenate(rows)], pc[np.concatenate(cols)],
                     np.concatenate(vals) if weighted else None)
    m.blocks = blocks
    return m


def batch_er(count: int, n_lo: int, n_hi: int, d_lo: float, d_hi: float,
             seed: int) -> List[Csr]:
    """``count`` ER+permutation matrices, n ~ U{n_lo..n_hi}, d ~ U[d_lo, d_hi];
    matrix k is generated from its own stream (seed, k)."""
    out = []
    for k in range(count):
        rng = np.random.default_rng([seed, k])
        n = int(rng.integers(n_lo, n_hi + 1))
        d = float(rng.uniform(d_lo, d_hi))
        out.append(er_planted(n, d, int(rng.integers(1 << 62))))
    return out


# ----------------------------------------------------------------------------
# small structured matrices with closed-form permanents
# ----------------------------------------------------------------------------

def all_ones(n: int) -> Csr:
    return csr_from_dense(np.ones((n, n)))


def tridiagonal(n: int) -> Csr:
    i = np.arange(n)
    d = (np.abs(i[:, None] - i[None, :]) <= 1)
    return csr_from_dense(d)


def permutation(n: int, seed: int) -> Csr:
    perm = np.random.default_rng(seed).permutation(n)
    return csr_from_coo(n, np.arange(n), perm)


def upper_triangular(n: int) -> Csr:
    i = np.arange(n)
    return csr_from_dense(i[:, None] <= i[None, :])


def circulant(n: int, k: int) -> Csr:
    """Row i has ones in columns i, i+1, ..., i+k-1 (mod n): k-regular."""
    rows = np.repeat(np.arange(n), k)
    cols = (rows + np.tile(np.arange(k), n)) % n
    return csr_from_coo(n, rows, cols)


def random_weighted(n: int, p: float, seed: int, lo=1.0, hi=1.5) -> Csr:
    """planted_bernoulli support with U[lo, hi] float32 weights."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    dense = rng.random((n, n)) < p
    dense[np.arange(n), perm] = True
    w = rng.uniform(lo, hi, size=(n, n)).astype(np.float32)
    r, c = np.nonzero(dense)
    return csr_from_coo(n, r, c, w[r, c])
