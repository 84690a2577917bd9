"""Seeded synthetic inputs for the LOOPS SpMM workloads.

This module only draws inputs: sparse matrices in CSR form and dense operands. It holds
none of the SpMM arithmetic, so both the CPU oracle and the GPU library can be fed from it
without sharing any part of the method. Every generator takes an explicit seed and uses
numpy's PCG64 ``Generator``; the recipes follow the workloads the paper evaluates on
(SuiteSparse-like structure at N = 32, Sec. 4.1; GCN aggregation, Sec. 4.5), which are not
available here and are replaced by these synthetic stand-ins:

* ``uniform_rows``    fixed nonzeros per row at distinct uniform columns (plain CSR case).
* ``laplacian_blocks`` 2D 5-point Laplacian with dense 8x8 diagonal blocks added (the
  clustered structure a BCSR part is meant for, Sec. 3.2.1).
* ``rmat_graph``      R-MAT power-law graph, symmetrised, no self loops or duplicates.
* ``gcn_graph``       R-MAT + identity with D^-1/2 (A+I) D^-1/2 values (GCN layer input).
* ``batched_mix``     many matrices of log-uniform size with uniform/banded/block structure.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A sparse matrix in CSR form. ``row_ptr`` int64[n_rows + 1], ``col_idx`` int32[nnz],
    ``vals`` float64[nnz]. Columns inside a row may be unsorted or repeated."""

    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n_rows, self.n_cols), dtype=np.float64)
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col_idx.astype(np.int64)), self.vals)
        return d

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_rows, dtype=np.int64), np.diff(self.row_ptr))


def csr_from_coo(n_rows: int, n_cols: int, rows: np.ndarray, cols: np.ndarray,
                 vals: np.ndarray, sort_cols: bool = True) -> CSR:
    """Build CSR from coordinate triples (stable by row; by column inside a row if asked)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    # one stable sort of the combined key gives the (row, column) order of a two-key lexsort;
    # inputs already in that order (banded patterns) are taken as they are
    key = rows * max(int(n_cols), 1) + cols if sort_cols else rows
    if key.size > 1 and not np.all(key[1:] >= key[:-1]):
        order = np.argsort(key, kind="stable")
        rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n_rows)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n_rows, n_cols, row_ptr, cols.astype(np.int32), vals)


def _distinct_cols_per_row(rng: np.random.Generator, counts: np.ndarray, n_cols: int) -> np.ndarray:
    """For row i draw counts[i] distinct columns uniform on [0, n_cols), by rejection: draw,
    find repeats inside a row, redraw only those, until none remain. Returns int64 columns in
    row order (unsorted within a row)."""
    counts = np.asarray(counts, dtype=np.int64)
    if np.any(counts > n_cols):
        raise ValueError("more distinct columns requested than exist")
    rows = np.repeat(np.arange(counts.size, dtype=np.int64), counts)
    cols = rng.integers(0, n_cols, size=rows.size, dtype=np.int64)
    while True:
        key = rows * n_cols + cols
        order = np.argsort(key, kind="stable")   # the order of lexsort((cols, rows))
        k_s = key[order]
        dup = np.zeros(rows.size, dtype=bool)
        dup[1:] = k_s[1:] == k_s[:-1]
        if not dup.any():
            return cols
        bad = order[dup]
        cols[bad] = rng.integers(0, n_cols, size=bad.size, dtype=np.int64)


def uniform_rows(n: int, per_row: int, N: int, seed: int):
    """Square n x n matrix, ``per_row`` distinct uniform columns per row, values U[-1, 1];
    then a dense n x N operand U[-1, 1]. One generator draws A first, then B."""
    rng = np.random.default_rng(seed)
    counts = np.full(n, per_row, dtype=np.int64)
    cols = _distinct_cols_per_row(rng, counts, n)
    vals = rng.uniform(-1.0, 1.0, size=cols.size)
    rows = np.repeat(np.arange(n, dtype=np.int64), counts)
    A = csr_from_coo(n, n, rows, cols, vals, sort_cols=False)
    B = rng.uniform(-1.0, 1.0, size=(n, N))
    return A, B


def laplacian_blocks(grid: int = 512, n_blocks: int = 4096, block: int = 8, seed: int = 1,
                     N: int = 64, with_dense: bool = True):
    """2D 5-point Laplacian on a grid x grid mesh (4 on the diagonal, -1 on the four
    neighbours, Dirichlet boundary, natural ordering), plus ``n_blocks`` distinct aligned
    block x block diagonal blocks chosen uniformly, each receiving N(0, 1) added to all of
    its entries (the pattern is the union). Returns (A, B) with B (grid^2 x N) ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    n = grid * grid
    idx = np.arange(n, dtype=np.int64)
    gx, gy = idx % grid, idx // grid
    r_list = [idx]
    c_list = [idx]
    v_list = [np.full(n, 4.0)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (gx + dx >= 0) & (gx + dx < grid) & (gy + dy >= 0) & (gy + dy < grid)
        r_list.append(idx[ok])
        c_list.append(idx[ok] + dx + dy * grid)
        v_list.append(np.full(int(ok.sum()), -1.0))
    n_diag = n // block
    chosen = np.sort(rng.choice(n_diag, size=n_blocks, replace=False))
    br = np.repeat(chosen * block, block * block) + np.tile(np.repeat(np.arange(block), block), n_blocks)
    bc = np.repeat(chosen * block, block * block) + np.tile(np.tile(np.arange(block), block), n_blocks)
    bv = rng.standard_normal(br.size)
    rows = np.concatenate(r_list + [br])
    cols = np.concatenate(c_list + [bc])
    vals = np.concatenate(v_list + [bv])
    # merge coincident coordinates: Laplacian value + added block value
    key = rows * n + cols
    uk, inv = np.unique(key, return_inverse=True)
    mv = np.zeros(uk.size)
    np.add.at(mv, inv, vals)
    A = csr_from_coo(n, n, uk // n, uk % n, mv)
    B = rng.standard_normal((n, N)) if with_dense else None
    return A, B


def rmat_edges(rng: np.random.Generator, scale: int, n_samples: int,
               a: float = 0.57, b: float = 0.19, c: float = 0.19):
    """R-MAT edge samples: at each of ``scale`` levels pick a quadrant with probabilities
    (a, b, c, d = 1 - a - b - c) and append one bit to the source and target ids."""
    src = np.zeros(n_samples, dtype=np.int64)
    dst = np.zeros(n_samples, dtype=np.int64)
    for _ in range(scale):
        r = rng.random(n_samples)
        s_bit = (r >= a + b).astype(np.int64)                      # quadrants c, d
        d_bit = (((r >= a) & (r < a + b)) | (r >= a + b + c)).astype(np.int64)  # b, d
        src = (src << 1) | s_bit
        dst = (dst << 1) | d_bit
    return src, dst


def _symmetric_pattern(n: int, src: np.ndarray, dst: np.ndarray, self_loops: bool):
    keep = src != dst
    s, d = src[keep], dst[keep]
    u = np.concatenate([s, d])
    v = np.concatenate([d, s])
    key = np.unique(u * n + v)
    rows, cols = key // n, key % n
    if self_loops:
        diag = np.arange(n, dtype=np.int64)
        key = np.unique(np.concatenate([rows * n + cols, diag * n + diag]))
        rows, cols = key // n, key % n
    return rows, cols


def rmat_graph(scale: int = 20, samples_per_node: int = 8, seed: int = 3, N: int = 128,
               with_dense: bool = True):
    """R-MAT(0.57, 0.19, 0.19, 0.05) graph with 2^scale nodes from samples_per_node * 2^scale
    undirected edge samples; symmetrised, self loops and duplicates dropped. Values
    1/sqrt(d_i d_j) (symmetric normalisation by the pattern degrees). B ~ N(0, 1), n x N."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    src, dst = rmat_edges(rng, scale, samples_per_node * n)
    rows, cols = _symmetric_pattern(n, src, dst, self_loops=False)
    deg = np.bincount(rows, minlength=n).astype(np.float64)
    vals = 1.0 / np.sqrt(deg[rows] * deg[cols])
    A = csr_from_coo(n, n, rows, cols, vals)
    B = rng.standard_normal((n, N)) if with_dense else None
    return A, B


def gcn_graph(scale: int = 18, samples_per_node: int = 16, seed: int = 4, N: int = 256,
              with_dense: bool = True):
    """GCN aggregation matrix: R-MAT pattern (as ``rmat_graph``) plus the identity, values
    D^-1/2 (A + I) D^-1/2 computed in float64. Returns (A, X, dY), X and dY ~ N(0, 1), n x N."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    src, dst = rmat_edges(rng, scale, samples_per_node * n)
    rows, cols = _symmetric_pattern(n, src, dst, self_loops=True)
    deg = np.bincount(rows, minlength=n).astype(np.float64)
    vals = 1.0 / np.sqrt(deg[rows] * deg[cols])
    A = csr_from_coo(n, n, rows, cols, vals)
    if not with_dense:
        return A, None, None
    X = rng.standard_normal((n, N))
    dY = rng.standard_normal((n, N))
    return A, X, dY


def banded(n: int, half_band: int, rng: np.random.Generator) -> CSR:
    """All entries with |i - j| <= half_band, values N(0, 1)."""
    i = np.repeat(np.arange(n, dtype=np.int64), 2 * half_band + 1)
    j = i + np.tile(np.arange(-half_band, half_band + 1, dtype=np.int64), n)
    ok = (j >= 0) & (j < n)
    i, j = i[ok], j[ok]
    return csr_from_coo(n, n, i, j, rng.standard_normal(i.size))


def dense_blocks(n: int, blocks_per_row_block: int, bs: int, rng: np.random.Generator) -> CSR:
    """For each bs-row block, ``blocks_per_row_block`` distinct random bs-aligned column
    blocks, each a dense bs x bs block of N(0, 1) values."""
    n_rb = (n + bs - 1) // bs
    n_cb = (n + bs - 1) // bs
    k = min(blocks_per_row_block, n_cb)
    cb = _distinct_cols_per_row(rng, np.full(n_rb, k, dtype=np.int64), n_cb)
    rb = np.repeat(np.arange(n_rb, dtype=np.int64), k)
    r = np.repeat(rb * bs, bs * bs) + np.tile(np.repeat(np.arange(bs), bs), rb.size)
    c = np.repeat(cb * bs, bs * bs) + np.tile(np.tile(np.arange(bs), bs), rb.size)
    ok = (r < n) & (c < n)
    r, c = r[ok], c[ok]
    return csr_from_coo(n, n, r, c, rng.standard_normal(r.size))


def block_mix(n: int = 1 << 20, dense_fraction: float = 0.5, blocks_per_row_block: int = 2, bs: int = 16,
              per_row: int = 16, seed: int = 6, N: int = 64):
    """One square matrix mixing the two structures the hybrid split separates: a random
    ``dense_fraction`` of the bs-row blocks hold ``blocks_per_row_block`` dense bs x bs blocks
    at distinct random bs-aligned columns (bs entries per B_r x 1 tile), the other row blocks
    ``per_row`` distinct uniform columns per row (about one entry per tile). Values N(0, 1);
    then B, n x N, N(0, 1). One generator draws everything in that order."""
    rng = np.random.default_rng(seed)
    n_rb = (n + bs - 1) // bs
    dense_rb = rng.random(n_rb) < dense_fraction
    D = dense_blocks(n, blocks_per_row_block, bs, rng)
    d_rows = D.row_ids()
    keep_d = dense_rb[d_rows // bs]
    sparse_rows = np.flatnonzero(~dense_rb[np.arange(n) // bs])
    counts = np.full(sparse_rows.size, min(per_row, n), dtype=np.int64)
    s_cols = _distinct_cols_per_row(rng, counts, n)
    s_rows = np.repeat(sparse_rows, counts)
    rows = np.concatenate([d_rows[keep_d], s_rows])
    cols = np.concatenate([D.col_idx.astype(np.int64)[keep_d], s_cols])
    vals = np.concatenate([D.vals[keep_d], rng.standard_normal(s_rows.size)])
    A = csr_from_coo(n, n, rows, cols, vals)
    B = rng.standard_normal((n, N))
    return A, B


def batched_mix(count: int = 512, seed: int = 5, min_rows: int = 1000, max_rows: int = 65536,
                Ns=(16, 32, 64, 128)):
    """``count`` square matrices with rows = floor(exp(U[ln min_rows, ln max_rows])); the
    structure cycles by index mod 3: uniform (U{8..64} distinct columns per row, values
    N(0, 1)), banded (|i - j| <= 16), dense 16 x 16 blocks (two per 16-row block). Each
    matrix gets N drawn uniformly from ``Ns``. Returns a list of (A, N)."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(count):
        n = int(math.floor(math.exp(rng.uniform(math.log(min_rows), math.log(max_rows)))))
        N = int(Ns[int(rng.integers(0, len(Ns)))])
        kind = m % 3
        if kind == 0:
            counts = rng.integers(8, 65, size=n).astype(np.int64)
            counts = np.minimum(counts, n)
            cols = _distinct_cols_per_row(rng, counts, n)
            rows = np.repeat(np.arange(n, dtype=np.int64), counts)
            A = csr_from_coo(n, n, rows, cols, rng.standard_normal(cols.size))
        elif kind == 1:
            A = banded(n, 16, rng)
        else:
            A = dense_blocks(n, 2, 16, rng)
        out.append((A, N))
    return out


def dense_normal(rows: int, cols: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((rows, cols))


def dense_uniform(rows: int, cols: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=(rows, cols))


def random_csr(n_rows: int, n_cols: int, density: float, seed: int, integer_values: bool = False,
               duplicates: bool = False, unsorted: bool = False, explicit_zeros: bool = False) -> CSR:
    """Small irregular test matrix: Bernoulli(density) pattern, optionally with repeated
    (i, j) entries, shuffled columns inside rows, or some stored zeros. Integer values are
    drawn from {-3..3} so that every product and sum is exact in any float format."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n_rows, n_cols)) < density
    r, c = np.nonzero(mask)
    r = r.astype(np.int64)
    c = c.astype(np.int64)
    if duplicates and r.size:
        pick = rng.integers(0, r.size, size=max(1, r.size // 5))
        r = np.concatenate([r, r[pick]])
        c = np.concatenate([c, c[pick]])
    if integer_values:
        v = rng.integers(-3, 4, size=r.size).astype(np.float64)
    else:
        v = rng.standard_normal(r.size)
    if explicit_zeros and r.size:
        v[rng.random(r.size) < 0.1] = 0.0
    A = csr_from_coo(n_rows, n_cols, r, c, v, sort_cols=not unsorted)
    if unsorted:
        # shuffle entries within each row
        for i in range(n_rows):
            s, e = A.row_ptr[i], A.row_ptr[i + 1]
            p = rng.permutation(e - s) + s
            A.col_idx[s:e] = A.col_idx[p]
            A.vals[s:e] = A.vals[p]
    return A
