"""Planted mistakes: copies of the oracle's C file with one plausible slip each (a dropped
term, a wrong sign, a transposed index, an off-by-one bound, duplicates assigned instead of
summed, tiles in the wrong order, a padding tile pointing at a real column) are compiled on
the CPU, and the pin checks must reject every one of them. This shows the pins constrain the
oracle rather than restate it."""
import ctypes
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W

SRC = os.path.join(os.path.dirname(oracle.__file__), "loops_oracle.c")

MUTATIONS = {
    "dropped_term": ("for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {\n      const double a = vals[k];\n      const double* b = B + (int64_t)col_idx[k] * ldb;\n      for (int64_t n = 0; n < N; ++n) acc[n] += a * b[n];",
                     "for (int64_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k) {\n      const double a = vals[k];\n      const double* b = B + (int64_t)col_idx[k] * ldb;\n      for (int64_t n = 0; n < N; ++n) acc[n] += a * b[n];"),
    "wrong_sign": ("for (int64_t n = 0; n < N; ++n) acc[n] += a * b[n];",
                   "for (int64_t n = 0; n < N; ++n) acc[n] -= a * b[n];"),
    "transposed_operand": ("const double* b = B + (int64_t)col_idx[k] * ldb;\n      for (int64_t n = 0; n < N; ++n) acc[n] += a * b[n];",
                           "const double* b = B + (int64_t)i * ldb;\n      for (int64_t n = 0; n < N; ++n) acc[n] += a * b[n];"),
    "sddmm_wrong_row": ("const double* g = dC + i * lddc;\n      const double* b = B + (int64_t)col_idx[k] * ldb;\n      double s = 0.0;",
                        "const double* g = dC + (int64_t)col_idx[k] * lddc;\n      const double* b = B + i * ldb;\n      double s = 0.0;"),
    "spmm_t_no_scatter": ("double* d = dB + (int64_t)col_idx[k] * lddb;",
                          "double* d = dB + i * lddb;"),
    "duplicates_assigned": ("if (fill) tile_val[(tc - 1) * block_rows + e[y].r] += vals[e[y].k];",
                            "if (fill) tile_val[(tc - 1) * block_rows + e[y].r] = vals[e[y].k];"),
    "tiles_descending": ("if (a->col != b->col) return a->col < b->col ? -1 : 1;",
                         "if (a->col != b->col) return a->col > b->col ? -1 : 1;"),
    "padding_real_column": ("          tile_col[tc] = -1;\n",
                            "          tile_col[tc] = 0;\n"),
    "density_strict": ("kind[b] = ((double)nnz_rb >= tau * (double)u_rb) ? 1 : 0;",
                       "kind[b] = ((double)nnz_rb > tau * (double)u_rb) ? 1 : 0;"),
}


def _build_mutant(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert old in src, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    lib = tmp_path / f"lib_{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(lib),
                           str(path), "-lm"])
    return str(lib)


def _with_lib(path):
    """A copy of the oracle's bindings on another compiled library."""
    saved = oracle._lib
    oracle._lib = None
    real = oracle._load()           # sets the argtypes on the real library object
    mut = ctypes.CDLL(path)
    for name in ("oracle_spmm", "oracle_spmm_rows", "oracle_spmm_t", "oracle_sddmm", "oracle_gemm_dense",
                 "oracle_partition_sizes", "oracle_partition_fill"):
        getattr(mut, name).argtypes = getattr(real, name).argtypes
        getattr(mut, name).restype = getattr(real, name).restype
    oracle._lib = mut
    return saved


def _pins_fail():
    """Run a compact set of the pins; return the list of those that fail."""
    failed = []
    rng = np.random.default_rng(0)
    # square, so that a mutant indexing rows by columns (or back) stays inside its arrays
    A = W.random_csr(40, 40, 0.2, 5, integer_values=True, duplicates=True, unsorted=True)
    Bi = rng.integers(-4, 5, size=(40, 7)).astype(np.float64)
    Ad = A.to_dense()
    if not np.array_equal(oracle.spmm(A, Bi), (Ad.astype(np.int64) @ Bi.astype(np.int64)).astype(float)):
        failed.append("spmm_exact_integers")
    dC = rng.integers(-4, 5, size=(40, 7)).astype(np.float64)
    if not np.array_equal(oracle.spmm_t(A, dC), (Ad.astype(np.int64).T @ dC.astype(np.int64)).astype(float)):
        failed.append("spmm_t_exact_integers")
    full = dC.astype(np.int64) @ Bi.astype(np.int64).T
    if not np.array_equal(oracle.sddmm(A, dC, Bi), full[A.row_ids(), A.col_idx.astype(np.int64)].astype(float)):
        failed.append("sddmm_exact_integers")
    for tau, br, kpad in ((0.0, 8, 4), (1.5, 16, 16), (2.0, 8, 1)):
        part = oracle.partition(A, "f64", block_rows=br, k_pad=kpad, tau=tau)
        try:
            ok = np.array_equal(oracle.expand_partition(part, A.n_rows, A.n_cols), Ad) and \
                np.array_equal(oracle.spmm_partitioned(part, A.n_rows, Bi), oracle.spmm(A, Bi))
        except AssertionError:
            ok = False
        if not ok:
            failed.append(f"partition_invariant_{tau}")
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "alg1_tiny.json")))
    m = g["matrix"]
    T = W.CSR(m["n_rows"], m["n_cols"], np.array(m["row_ptr"], np.int64), np.array(m["col_idx"], np.int32),
              np.array(m["vals"], np.float64))
    for case in g["cases"]:
        tau = math.inf if case["tau"] == "inf" else float(case["tau"])
        part = oracle.partition(T, "f64", block_rows=case["block_rows"], k_pad=case["k_pad"], tau=tau)
        same = all(list(part[k]) == case[k] for k in ("csr_rows", "csr_ptr", "csr_col", "rb_ids", "rb_ptr",
                                                          "tile_col"))
        same = same and np.array_equal(part["tile_val"],
                                       np.asarray(case["tile_val"], float).reshape(-1, case["block_rows"]))
        if not same:
            failed.append("golden_" + str(case["tau"]))
            break
    return failed


def test_unmutated_oracle_passes():
    assert _pins_fail() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    saved = _with_lib(_build_mutant(tmp_path, name))
    try:
        failed = _pins_fail()
    finally:
        oracle._lib = saved
    assert failed, f"mutation {name} was not caught by any pin"
