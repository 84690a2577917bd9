"""C-ABI host logic, no GPU: the library loads and exports every declared symbol, its host
partitioner matches the independent oracle partitioner bit for bit (rounding included), and
invalid inputs come back as status codes."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "loops.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(loops_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(loops_lib):
    L = loops_lib.load()
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(loops_lib.EXPORTED)
    assert L.loops_version() >= 10000
    assert L.loops_status_str(3) == b"LOOPS_ERR_UNSUPPORTED"


def _compare(lib_part, ora_part):
    for k in ("csr_rows", "csr_ptr", "csr_col", "rb_ids", "rb_ptr", "tile_col"):
        assert np.array_equal(lib_part[k], ora_part[k]), k
    # values: bit-exact f64 images of the stored (rounded) values
    assert np.array_equal(lib_part["csr_val"].view(np.uint64), ora_part["csr_val"].view(np.uint64))
    assert np.array_equal(lib_part["tile_val"].view(np.uint64), ora_part["tile_val"].view(np.uint64))
    assert lib_part["scale"] == ora_part["scale"]


CASES = [
    dict(n=45, m=40, d=0.12, dup=True, uns=True, zeros=True),
    dict(n=67, m=33, d=0.3, dup=False, uns=False, zeros=False),
    dict(n=16, m=16, d=1.0, dup=False, uns=True, zeros=False),
    dict(n=5, m=70, d=0.05, dup=True, uns=False, zeros=True),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("dtype", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("tau", [0.0, 1.0, 1.5, 2.5, math.inf])
@pytest.mark.parametrize("tile_min", [0, 2, 3])
def test_partition_host_matches_oracle(loops_lib, case, dtype, tau, tile_min):
    c = CASES[case]
    A = W.random_csr(c["n"], c["m"], c["d"], 100 + case, duplicates=c["dup"], unsorted=c["uns"],
                     explicit_zeros=c["zeros"])
    A.vals = A.vals * 10.0 ** np.random.default_rng(case).integers(-7, 3, A.vals.size)
    kpad = {"f64": 4, "f32": 1, "f16": 16, "bf16": 16}[dtype]
    lib = loops_lib.partition_host(A, dtype, tau=tau, tile_min=tile_min)
    ora = oracle.partition(A, dtype, k_pad=kpad, tau=tau, tile_min=tile_min)
    assert lib["k_pad"] == kpad and lib["block_rows"] == oracle.default_block_rows(dtype)
    _compare(lib, ora)


@pytest.mark.parametrize("r_b", [0, 1, 7, 8, 9, 30, 1000])
def test_partition_host_contiguous_matches_oracle(loops_lib, r_b):
    A = W.random_csr(37, 29, 0.2, 7, duplicates=True)
    lib = loops_lib.partition_host(A, "f64", contiguous_split=True, r_boundary=r_b)
    ora = oracle.partition(A, "f64", k_pad=4, contiguous=True, r_boundary=r_b)
    _compare(lib, ora)


def test_partition_host_f32_block_rows_8(loops_lib):
    A = W.random_csr(50, 50, 0.2, 3)
    lib = loops_lib.partition_host(A, "f32", tau=1.2, block_rows=8)
    ora = oracle.partition(A, "f32", block_rows=8, k_pad=1, tau=1.2)
    _compare(lib, ora)


def test_partition_host_laplacian_closed_form(loops_lib):
    A, _ = W.laplacian_blocks(grid=64, n_blocks=64, block=8, seed=2, with_dense=False)
    lib = loops_lib.partition_host(A, "f64", tau=2.0)
    ora = oracle.partition(A, "f64", k_pad=4, tau=2.0)
    _compare(lib, ora)
    assert lib["rb_ids"].size == 64


def test_rounding_extremes_bit_exact(loops_lib):
    # values around the 16-bit formats' subnormal, tie and overflow boundaries (after s_A)
    v = np.array([1.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 2.0 ** -14 * (1 - 2.0 ** -11),
                  1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 2.0 ** -8), 1e-30, -2.5e-6])
    n = v.size
    A = W.CSR(1, n, np.array([0, n], np.int64), np.arange(n, dtype=np.int32), v)
    for dtype in ("f16", "bf16", "f32"):
        _compare(loops_lib.partition_host(A, dtype, tau=math.inf),
                 oracle.partition(A, dtype, k_pad={"f32": 1}.get(dtype, 16), tau=math.inf))


def _raw_csr(loops_lib, n_rows, n_cols, rp, ci, v):
    rp = np.asarray(rp, np.int64)
    ci = np.asarray(ci, np.int32)
    v = np.asarray(v, np.float64)
    return W.CSR(n_rows, n_cols, rp, ci, v)


@pytest.mark.parametrize("bad", ["non_monotone", "col_oob", "neg_col", "nnz_mismatch", "first_nonzero"])
def test_invalid_csr_is_rejected(loops_lib, bad):
    rp, ci = [0, 2, 3], [0, 1, 2]
    if bad == "non_monotone":
        rp = [0, 3, 2]
    elif bad == "col_oob":
        ci = [0, 1, 3]
    elif bad == "neg_col":
        ci = [0, -1, 2]
    elif bad == "nnz_mismatch":
        rp = [0, 2, 2]
    elif bad == "first_nonzero":
        rp = [1, 2, 3]
    A = _raw_csr(loops_lib, 2, 3, rp, ci, [1.0, 2.0, 3.0])
    L = loops_lib.load()
    cs, keep = loops_lib._csr_struct(A)
    cs.nnz = 3
    part = loops_lib._Part()
    st = L.loops_partition_host(ctypes.byref(cs), 0, None, ctypes.byref(part))
    assert st == 2, L.loops_last_error()
    assert L.loops_last_error()


def test_bad_arguments_are_status_codes(loops_lib):
    L = loops_lib.load()
    A = W.random_csr(10, 10, 0.3, 1)
    cs, keep = loops_lib._csr_struct(A)
    part = loops_lib._Part()
    assert L.loops_partition_host(None, 0, None, ctypes.byref(part)) == 1          # NULL A
    assert L.loops_partition_host(ctypes.byref(cs), 9, None, ctypes.byref(part)) == 1  # bad dtype
    o = loops_lib._opts(tau=2.0, block_rows=12)
    assert L.loops_partition_host(ctypes.byref(cs), 0, ctypes.byref(o), ctypes.byref(part)) == 3
    o = loops_lib._opts(tau=-1.0)
    assert L.loops_partition_host(ctypes.byref(cs), 0, ctypes.byref(o), ctypes.byref(part)) == 1
    # a destroyed / bogus plan handle is rejected without touching the GPU
    assert L.loops_plan_destroy(ctypes.c_void_p(0)) == 0
    info = loops_lib._Info()
    assert L.loops_plan_info_get(ctypes.c_void_p(0), ctypes.byref(info)) == 7
    bogus = (ctypes.c_uint64 * 64)()
    assert L.loops_plan_info_get(ctypes.cast(bogus, ctypes.c_void_p), ctypes.byref(info)) == 7


def test_plan_device_argument_checks_need_no_gpu(loops_lib):
    # every check below returns before the first CUDA call (the arrays are never read)
    L = loops_lib.load()
    A = W.random_csr(10, 10, 0.3, 1)
    cs, keep = loops_lib._csr_struct(A)
    h = ctypes.c_void_p()
    o = loops_lib._opts(tau=2.0)
    assert L.loops_plan_device(ctypes.byref(cs), 8, 0, ctypes.byref(o), None, None) == 1        # NULL out
    assert L.loops_plan_device(None, 8, 0, ctypes.byref(o), None, ctypes.byref(h)) == 1         # NULL A
    assert L.loops_plan_device(ctypes.byref(cs), 8, 9, ctypes.byref(o), None, ctypes.byref(h)) == 1  # dtype
    assert L.loops_plan_device(ctypes.byref(cs), -1, 0, ctypes.byref(o), None, ctypes.byref(h)) == 1  # N < 0
    assert L.loops_plan_device(ctypes.byref(cs), 1 << 21, 0, ctypes.byref(o), None, ctypes.byref(h)) == 3
    bad_br = loops_lib._opts(tau=2.0, block_rows=12)
    assert L.loops_plan_device(ctypes.byref(cs), 8, 0, ctypes.byref(bad_br), None, ctypes.byref(h)) == 3
    nan_tau = loops_lib._opts(tau=float("nan"))
    assert L.loops_plan_device(ctypes.byref(cs), 8, 0, ctypes.byref(nan_tau), None, ctypes.byref(h)) == 1
    both = loops_lib._opts(tau=2.0, want_backward=True, tile_min=2)
    assert L.loops_plan_device(ctypes.byref(cs), 8, 0, ctypes.byref(both), None, ctypes.byref(h)) == 3
    assert b"tile-level split" in L.loops_last_error()
    f16_vals = loops_lib._Csr(cs.n_rows, cs.n_cols, cs.nnz, cs.row_ptr, cs.col_idx, cs.vals, 2)
    assert L.loops_plan_device(ctypes.byref(f16_vals), 8, 0, ctypes.byref(o), None, ctypes.byref(h)) == 3
    assert h.value is None


def test_binding_rejects_inconsistent_arrays_before_reading_them(loops_lib):
    A = W.random_csr(30, 30, 0.2, 3)
    # row_ptr claims more entries than col_idx holds: the library's validation rejects it
    rp = A.row_ptr.copy()
    rp[-1] += 5
    with pytest.raises(loops_lib.LoopsError) as ei:
        loops_lib.Plan(W.CSR(30, 30, rp, A.col_idx, A.vals), 8, "f64", tau=2.0)
    assert ei.value.status == 2 and "row_ptr[n_rows] != nnz" in str(ei.value)
    with pytest.raises(ValueError):
        loops_lib.Plan(W.CSR(30, 30, A.row_ptr, A.col_idx, A.vals[:-1]), 8, "f64", tau=2.0)
    with pytest.raises(ValueError):
        loops_lib.Plan(W.CSR(31, 30, A.row_ptr, A.col_idx, A.vals), 8, "f64", tau=2.0)
