"""Pins for the CPU oracle: each check ties it to something other than itself -- a brute-force
loop or numpy's own routines, exact integer arithmetic, closed forms (identity, permutation,
diagonal), a hand-worked Algorithm 1 example, and the closed-form structure of the Laplacian
workload. A plausible slip in the oracle (a dropped term, a transposed operand, a wrong index
or sign, a mis-rounded format) fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W


def _int_csr(n_rows, n_cols, density, seed, **kw):
    return W.random_csr(n_rows, n_cols, density, seed, integer_values=True, **kw)


def _int_dense(rows, cols, seed):
    return np.random.default_rng(seed).integers(-4, 5, size=(rows, cols)).astype(np.float64)


# ------------------------------------------------------------------ SpMM definition (Sec. 2.1)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spmm_matches_bruteforce_dense(seed):
    A = W.random_csr(37, 29, 0.2, seed, duplicates=True, unsorted=True)
    B = W.dense_normal(29, 13, seed + 10)
    C = oracle.spmm(A, B)
    Ad = A.to_dense()
    np.testing.assert_allclose(C, oracle.gemm_dense(Ad, B), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(C, Ad @ B, rtol=1e-13, atol=1e-13)


def test_gemm_dense_matches_numpy():
    rng = np.random.default_rng(7)
    Ad = rng.standard_normal((11, 17))
    B = rng.standard_normal((17, 5))
    np.testing.assert_allclose(oracle.gemm_dense(Ad, B), Ad @ B, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed", [3, 4])
def test_spmm_exact_on_small_integers(seed):
    # every product and partial sum is an integer far below 2^53: exact in any order
    A = _int_csr(64, 48, 0.3, seed, duplicates=True, unsorted=True, explicit_zeros=True)
    B = _int_dense(48, 24, seed)
    C = oracle.spmm(A, B)
    exact = A.to_dense().astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C, exact.astype(np.float64))


def test_identity_permutation_diagonal_closed_forms():
    n, N = 50, 9
    B = W.dense_normal(n, N, 11)
    I = W.csr_from_coo(n, n, np.arange(n), np.arange(n), np.ones(n))
    assert np.array_equal(oracle.spmm(I, B), B)
    perm = np.random.default_rng(5).permutation(n)
    P = W.csr_from_coo(n, n, np.arange(n), perm, np.ones(n))
    assert np.array_equal(oracle.spmm(P, B), B[perm])
    d = np.random.default_rng(6).standard_normal(n)
    D = W.csr_from_coo(n, n, np.arange(n), np.arange(n), d)
    assert np.array_equal(oracle.spmm(D, B), d[:, None] * B)


def test_spmm_empty_rows_and_empty_matrix():
    A = W.csr_from_coo(6, 4, np.array([1, 1, 4]), np.array([0, 3, 2]), np.array([2.0, -1.0, 0.5]))
    B = W.dense_normal(4, 3, 1)
    C = oracle.spmm(A, B)
    assert np.all(C[[0, 2, 3, 5]] == 0.0)
    np.testing.assert_array_equal(C[1], 2.0 * B[0] - B[3])
    E = W.csr_from_coo(0, 4, np.zeros(0), np.zeros(0), np.zeros(0))
    assert oracle.spmm(E, B).shape == (0, 3)


def test_spmm_threads_bit_identical_to_one_thread():
    # the threaded timing leg runs the same row loop on row ranges; any thread count, empty
    # rows and an empty matrix give the single-threaded result bit for bit
    rng = np.random.default_rng(4)
    A = W.random_csr(700, 300, 0.02, 2, duplicates=True, unsorted=True)
    B = rng.standard_normal((300, 9))
    for t in (1, 2, 5, 16, 1000):
        assert np.array_equal(oracle.spmm_threads(A, B, t), oracle.spmm(A, B))
    E = W.CSR(0, 300, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.spmm_threads(E, B, 4).shape == (0, 9)


def test_spmm_rows_equals_full():
    A = W.random_csr(40, 40, 0.15, 9)
    B = W.dense_normal(40, 7, 2)
    rows = np.array([39, 0, 17, 17, 5])
    assert np.array_equal(oracle.spmm_rows(A, B, rows), oracle.spmm(A, B)[rows])


# ------------------------------------------------------------------ backward pieces
@pytest.mark.parametrize("seed", [0, 1])
def test_spmm_t_exact_integers(seed):
    A = _int_csr(33, 21, 0.25, seed, duplicates=True)
    dC = _int_dense(33, 10, seed + 1)
    exact = A.to_dense().astype(np.int64).T @ dC.astype(np.int64)
    assert np.array_equal(oracle.spmm_t(A, dC), exact.astype(np.float64))


def test_sddmm_exact_integers_and_definition():
    A = _int_csr(25, 31, 0.2, 8, duplicates=True, unsorted=True)
    dC = _int_dense(25, 6, 2)
    B = _int_dense(31, 6, 3)
    full = dC.astype(np.int64) @ B.astype(np.int64).T       # (dC B^T)[i, j]
    expect = full[A.row_ids(), A.col_idx.astype(np.int64)].astype(np.float64)
    assert np.array_equal(oracle.sddmm(A, dC, B), expect)


def test_gradients_of_sum_loss_by_finite_differences():
    # L = sum(W * (A.B)); dL/dB = A^T W, dL/dvals[k] = <W[i_k], B[j_k]>  (central differences)
    A = W.random_csr(12, 9, 0.3, 21)
    B = W.dense_normal(9, 4, 22)
    Wt = W.dense_normal(12, 4, 23)
    loss = lambda AA, BB: float(np.sum(Wt * oracle.spmm(AA, BB)))
    h = 1e-6
    gB = oracle.spmm_t(A, Wt)
    for (j, n) in [(0, 0), (3, 2), (8, 3)]:
        Bp, Bm = B.copy(), B.copy()
        Bp[j, n] += h
        Bm[j, n] -= h
        assert abs((loss(A, Bp) - loss(A, Bm)) / (2 * h) - gB[j, n]) < 1e-6
    gv = oracle.sddmm(A, Wt, B)
    for k in [0, A.nnz // 2, A.nnz - 1]:
        Ap = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.vals.copy())
        Am = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.vals.copy())
        Ap.vals[k] += h
        Am.vals[k] -= h
        assert abs((loss(Ap, B) - loss(Am, B)) / (2 * h) - gv[k]) < 1e-6


# ------------------------------------------------------------------ number formats
def test_round_to_f16_matches_numpy_cast():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-9, 6, 20000),
                        [65504.0, 65519.99, 65520.0, 1e6, -7e-8, 3e-8, 2.0 ** -25, 2.0 ** -24 * 1.5]])
    with np.errstate(over="ignore"):  # values past the binary16 range round to infinity on purpose
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(oracle.round_to(x, "f16"), ref)


def test_round_to_f32_matches_numpy_cast():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000) * 10.0 ** rng.integers(-44, 38, 20000)
    assert np.array_equal(oracle.round_to(x, "f32"), x.astype(np.float32).astype(np.float64))


def _bf16_via_f32_bits(x32: np.ndarray) -> np.ndarray:
    # independent bfloat16 rounding of binary32 inputs: add the round-to-nearest-even bias to
    # the 32-bit pattern and keep the high 16 bits (valid for finite inputs)
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_round_to_bf16_matches_bit_trick_and_known_ties():
    rng = np.random.default_rng(2)
    x32 = (rng.standard_normal(50000) * 10.0 ** rng.integers(-40, 37, 50000)).astype(np.float32)
    x32 = x32[np.isfinite(x32)]
    assert np.array_equal(oracle.round_to(x32.astype(np.float64), "bf16"), _bf16_via_f32_bits(x32))
    # quantum at 1.0 is 2^-7: 1 + 2^-8 ties to 1 (even), 1 + 3*2^-8 ties up to 1 + 2^-6
    got = oracle.round_to(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)]), "bf16")
    assert list(got) == [1.0, 1 + 2.0 ** -6, -1.0]


def test_scales():
    assert oracle.plan_scale([1.0, -0.25], "f16") == 2.0 ** 14
    assert oracle.plan_scale([3.0], "bf16") == 2.0 ** 12
    assert oracle.plan_scale([0.0], "f16") == 1.0
    assert oracle.plan_scale([5.0], "f32") == 1.0
    B = np.array([[0.3, 4.0, 0.0, -3.0], [-0.1, 1.0, 0.0, 2.5]])
    assert list(oracle.col_scales(B)) == [0.5, 4.0, 1.0, 4.0]
    B16, s = oracle.scale_round_columns(B, "f16")
    assert np.all(np.abs(B16) <= 1.0)
    # a column maximum above 2^127 (binary32 range) keeps the largest binary32 power of two
    big = np.array([[3.0e38], [1.0]])
    assert oracle.col_scales(big)[0] == 2.0 ** 127


# ------------------------------------------------------------------ Algorithm 1 partition
def _check_case(part, case):
    for key in ("csr_rows", "csr_ptr", "csr_col", "csr_val", "rb_ids", "rb_ptr", "tile_col"):
        assert list(part[key]) == case[key], key
    tv = np.asarray(case["tile_val"], dtype=np.float64).reshape(-1, case["block_rows"])
    assert np.array_equal(part["tile_val"], tv)


def test_partition_hand_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "alg1_tiny.json")))
    m = g["matrix"]
    A = W.CSR(m["n_rows"], m["n_cols"], np.array(m["row_ptr"], np.int64),
              np.array(m["col_idx"], np.int32), np.array(m["vals"], np.float64))
    for case in g["cases"]:
        tau = math.inf if case["tau"] == "inf" else float(case["tau"])
        part = oracle.partition(A, "f64", block_rows=case["block_rows"], k_pad=case["k_pad"], tau=tau)
        _check_case(part, case)
    c = g["contiguous"]
    part = oracle.partition(A, "f64", block_rows=c["block_rows"], k_pad=c["k_pad"], contiguous=True,
                            r_boundary=c["r_boundary"])
    _check_case(part, c)
    c = g["tile_split"]
    part = oracle.partition(A, "f64", block_rows=c["block_rows"], k_pad=c["k_pad"], tau=c["tau"],
                            tile_min=c["tile_min"])
    _check_case(part, c)


@pytest.mark.parametrize("tau", [0.0, 1.0, 1.5, 2.0, 4.0, math.inf])
@pytest.mark.parametrize("br,kpad", [(8, 4), (16, 16), (16, 1)])
@pytest.mark.parametrize("tile_min", [0, 2, 3])
def test_partition_invariant_exact(tau, br, kpad, tile_min):
    # any split: expanding the partition gives A back, and C from the parts equals C (exact)
    A = _int_csr(45, 40, 0.12, int(br + kpad), duplicates=True, unsorted=True, explicit_zeros=True)
    B = _int_dense(40, 5, 3)
    part = oracle.partition(A, "f64", block_rows=br, k_pad=kpad, tau=tau, tile_min=tile_min)
    assert np.array_equal(oracle.expand_partition(part, A.n_rows, A.n_cols), A.to_dense())
    assert np.array_equal(oracle.spmm_partitioned(part, A.n_rows, B), oracle.spmm(A, B))
    # structure: every row is covered; without the tile split each row is in exactly one
    # part; kept tiles hold at least tile_min entries; tiles per block are a multiple of k_pad
    rows = set(int(r) for r in part["csr_rows"])
    for b in part["rb_ids"]:
        blk = set(range(int(b) * br, min(int(b) * br + br, A.n_rows)))
        if tile_min <= 1:
            assert not (rows & blk)
        rows |= blk
    assert rows == set(range(A.n_rows))
    if tile_min > 1:
        D = A.to_dense()
        for x, b in enumerate(part["rb_ids"]):
            for t in range(part["rb_ptr"][x], part["rb_ptr"][x + 1]):
                c = part["tile_col"][t]
                if c >= 0:
                    r0 = int(b) * br
                    stored = sum(int(np.sum(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]] == c))
                                 for i in range(r0, min(r0 + br, A.n_rows)))
                    assert stored >= tile_min
    assert np.all(np.diff(part["rb_ptr"]) % kpad == 0)
    if tau == math.inf:
        assert part["rb_ids"].size == 0
    if tau == 0.0:
        nonempty = {i // br for i in range(A.n_rows) if A.row_ptr[i + 1] > A.row_ptr[i]}
        assert set(int(b) for b in part["rb_ids"]) == nonempty


def test_partition_16bit_values_are_scaled_and_rounded():
    A = W.random_csr(30, 30, 0.2, 4)
    A.vals = A.vals * 1e-3
    for fmt in ("f16", "bf16", "f32"):
        part = oracle.partition(A, fmt, tau=0.0, k_pad=1)
        s = oracle.plan_scale(A.vals, fmt)
        assert part["scale"] == s
        v = part["tile_val"][part["tile_col"] >= 0]
        assert np.array_equal(v, oracle.round_to(v, fmt))
        D = oracle.expand_partition(part, A.n_rows, A.n_cols)
        # each stored value is within half a quantum of s * a
        tol = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "f32": 2.0 ** -24}[fmt]
        Ad = A.to_dense()
        assert np.all(np.abs(D - Ad) <= tol * np.abs(Ad) + 1e-30)


def test_laplacian_blocks_closed_form_split():
    # 512 x 512 five-point Laplacian; 4,096 aligned 8 x 8 diagonal blocks densified with N(0,1).
    # An interior plain row block has 8 rows x 5 entries = 40 nnz over 26 columns (d = 1.54;
    # edge blocks reach 31/17 = 1.82 < 2); an augmented interior block has 64 + 16 + 2 = 82
    # nnz over 26 columns (d = 3.15; edge blocks more). So tau = 2 selects exactly the 4,096
    # augmented blocks.
    A, _ = W.laplacian_blocks(grid=512, n_blocks=4096, block=8, seed=1, with_dense=False)
    n = 512 * 512
    lap_nnz = 5 * n - 4 * 512
    assert A.nnz == lap_nnz + 4096 * (64 - 22)   # 22 of the 64 block entries are Laplacian ones
    assert A.nnz == 1_480_704
    part = oracle.partition(A, "f64", block_rows=8, k_pad=1, tau=2.0)
    assert part["rb_ids"].size == 4096
    assert part["csr_rows"].size == n - 4096 * 8
    tiles = np.diff(part["rb_ptr"])
    assert tiles.max() == 26 and tiles.min() >= 17
    # tiles of a fully interior augmented block: 8 dense + 8 up + 8 down + left + right
    nnz_bcsr = int(np.count_nonzero(part["tile_val"]))
    assert nnz_bcsr <= 4096 * 82


def test_block_mix_split_selects_exactly_the_dense_row_blocks():
    # A dense row block holds two 16 x 16 blocks: 512 nnz over 32 distinct columns (d = 16);
    # a sparse one 16 rows x 16 distinct uniform columns: 256 nnz over at most 256 columns
    # (d = 1 unless columns collide, which needs > 128 collisions to reach d = 2). So tau = 2
    # selects exactly the dense row blocks, and every tile of them holds 16 entries.
    A, B = W.block_mix(n=1 << 13, N=4, seed=6)
    rb_nnz = np.add.reduceat(np.diff(A.row_ptr), np.arange(0, A.n_rows, 16))
    dense = np.flatnonzero(rb_nnz == 512)
    assert set(np.unique(rb_nnz)) == {256, 512} and 0 < dense.size < rb_nnz.size
    part = oracle.partition(A, "f64", block_rows=16, k_pad=1, tau=2.0)
    assert np.array_equal(part["rb_ids"], dense)
    assert np.array_equal(np.diff(part["rb_ptr"]), np.full(dense.size, 32))
    assert np.count_nonzero(part["tile_val"]) == dense.size * 512
    ref = oracle.spmm(A, B)  # the parts sum in another order: equal up to rounding
    assert np.allclose(oracle.spmm_partitioned(part, A.n_rows, B), ref, rtol=1e-12, atol=1e-12)
