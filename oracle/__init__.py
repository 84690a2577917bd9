"""CPU oracle for the LOOPS hybrid SpMM (arxiv 2511.08158) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The GPU library never calls it and shares no code with it.

The arithmetic lives in ``loops_oracle.c`` (plain C loops in IEEE binary64, compiled with
gcc on first use); this module only marshals numpy arrays into it and adds the
number-format readings, written out with numpy:

* ``round_to(x, fmt)``: round-to-nearest-even of a float64 array into binary32, binary16 or
  bfloat16, from the formats' definitions (significand bits, minimum exponent, largest
  finite value), returned as float64.
* ``plan_scale(vals, fmt)``: the power of two s_A with max|a| * s_A <= 2^14 applied to A
  before a 16-bit cast (1 when A is all zero or the format is not 16-bit).
* ``col_scales(B)``: s_j = 2^ceil(log2 max_i |B_ij|) per column (1 for an all-zero column,
  at most 2^127), so that |B_ij / s_j| <= 1 before a 16-bit cast.
* ``partition(...)``: Algorithm 1 (CSR -> LOOPS) with the structural-split reading; values
  are the f64 sums of duplicates, rounded once into the compute format.

Parity pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "loops_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle's C file into a shared library (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.oracle_spmm.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i32p, _f64p, _f64p,
                                      ctypes.c_int64, _f64p, ctypes.c_int64]
            L.oracle_spmm_rows.argtypes = [_i64p, _i32p, _f64p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                           _i64p, ctypes.c_int64, _f64p]
            L.oracle_spmm_t.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p, _i32p,
                                        _f64p, _f64p, ctypes.c_int64, _f64p, ctypes.c_int64]
            L.oracle_sddmm.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i32p, _f64p,
                                       ctypes.c_int64, _f64p, ctypes.c_int64, _f64p]
            L.oracle_gemm_dense.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _f64p,
                                            _f64p, _f64p]
            L.oracle_partition_sizes.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int64,
                                                 ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_int64, ctypes.c_int64, _i64p]
            L.oracle_partition_fill.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int64, ctypes.c_int64, _i32p, _i64p, _i32p, _f64p,
                                                _i32p, _i64p, _i32p, _f64p]
            for f in (L.oracle_partition_sizes, L.oracle_partition_fill):
                f.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _csr_arrays(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.vals, dtype=np.float64)
    return rp, ci, v


def spmm(A, B: np.ndarray) -> np.ndarray:
    """C = A.B in float64 (Sec. 2.1 inner-product definition)."""
    L = _load()
    rp, ci, v = _csr_arrays(A)
    B = np.ascontiguousarray(B, dtype=np.float64)
    N = B.shape[1] if B.ndim == 2 else 0
    C = np.empty((A.n_rows, N), dtype=np.float64)
    L.oracle_spmm(A.n_rows, N, _p(rp, _i64p), _p(ci, _i32p), _p(v, _f64p), _p(B, _f64p), N,
                  _p(C, _f64p), N)
    return C


def spmm_threads(A, B: np.ndarray, threads: int) -> np.ndarray:
    """C = A.B by the same row loop as ``spmm``, on ``threads`` host threads: the rows are cut
    into contiguous ranges of about equal nnz and each thread runs ``oracle_spmm`` on its
    range (ctypes releases the GIL for the call). Every row is computed exactly as in
    ``spmm``, so the result is bit-identical; only the wall time differs."""
    from concurrent.futures import ThreadPoolExecutor

    L = _load()
    rp, ci, v = _csr_arrays(A)
    B = np.ascontiguousarray(B, dtype=np.float64)
    N = B.shape[1]
    C = np.empty((A.n_rows, N), dtype=np.float64)
    threads = max(1, int(threads))
    cuts = np.searchsorted(rp, np.linspace(0, rp[-1], threads + 1), side="left")
    cuts[0], cuts[-1] = 0, A.n_rows
    cuts = np.maximum.accumulate(np.minimum(cuts, A.n_rows))
    base_c = C.ctypes.data

    def run(t):
        r0, r1 = int(cuts[t]), int(cuts[t + 1])
        if r1 <= r0:
            return
        rp_t = ctypes.cast(rp.ctypes.data + 8 * r0, _i64p)
        C_t = ctypes.cast(base_c + 8 * r0 * N, _f64p)
        L.oracle_spmm(r1 - r0, N, rp_t, _p(ci, _i32p), _p(v, _f64p), _p(B, _f64p), N, C_t, N)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(threads)))
    return C


def spmm_rows(A, B: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Rows ``rows`` of A.B in float64."""
    L = _load()
    rp, ci, v = _csr_arrays(A)
    B = np.ascontiguousarray(B, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    N = B.shape[1]
    C = np.empty((rows.size, N), dtype=np.float64)
    L.oracle_spmm_rows(_p(rp, _i64p), _p(ci, _i32p), _p(v, _f64p), _p(B, _f64p), N, N,
                       _p(rows, _i64p), rows.size, _p(C, _f64p))
    return C


def spmm_t(A, dC: np.ndarray) -> np.ndarray:
    """dB = A^T . dC in float64, by scattering the rows of A."""
    L = _load()
    rp, ci, v = _csr_arrays(A)
    dC = np.ascontiguousarray(dC, dtype=np.float64)
    N = dC.shape[1]
    dB = np.empty((A.n_cols, N), dtype=np.float64)
    L.oracle_spmm_t(A.n_rows, A.n_cols, N, _p(rp, _i64p), _p(ci, _i32p), _p(v, _f64p),
                    _p(dC, _f64p), N, _p(dB, _f64p), N)
    return dB


def sddmm(A, dC: np.ndarray, B: np.ndarray) -> np.ndarray:
    """dvals[k] = <dC[i_k, :], B[j_k, :]> in A's storage order, float64."""
    L = _load()
    rp, ci, _ = _csr_arrays(A)
    dC = np.ascontiguousarray(dC, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    N = dC.shape[1]
    out = np.empty(A.nnz, dtype=np.float64)
    L.oracle_sddmm(A.n_rows, N, _p(rp, _i64p), _p(ci, _i32p), _p(dC, _f64p), N, _p(B, _f64p), N,
                   _p(out, _f64p))
    return out


def gemm_dense(Ad: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Brute-force triple loop C = Ad . B in float64."""
    L = _load()
    Ad = np.ascontiguousarray(Ad, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = Ad.shape
    N = B.shape[1]
    C = np.empty((M, N), dtype=np.float64)
    L.oracle_gemm_dense(M, K, N, _p(Ad, _f64p), _p(B, _f64p), _p(C, _f64p))
    return C


# --------------------------------------------------------------------------------------------
# Number formats (IEEE 754 binary32/binary16 and bfloat16), round to nearest, ties to even.
# Each format: (stored significand bits p-1, minimum normal exponent, largest finite value).
# --------------------------------------------------------------------------------------------
_FORMATS = {
    "f32": (23, -126, (2.0 - 2.0 ** -23) * 2.0 ** 127),
    "f16": (10, -14, 65504.0),
    "bf16": (7, -126, (2.0 - 2.0 ** -7) * 2.0 ** 127),
}


def round_to(x, fmt: str) -> np.ndarray:
    """Round float64 values to the nearest value of ``fmt`` (ties to even); f64 is identity.
    A value's quantum is 2^(max(e, emin) - m) for its binary exponent e = floor(log2|x|);
    x / quantum is an exact float64 operation (power-of-two scaling), numpy's ``rint``
    rounds it half-to-even, and results above the largest finite value overflow to inf
    (a value at or past the midpoint to the next binade above max rounds up)."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == "f64":
        return x.copy()
    m, emin, fmax = _FORMATS[fmt]
    out = np.array(x, dtype=np.float64, copy=True)
    fin = np.isfinite(x) & (x != 0.0)
    xv = x[fin]
    _, e2 = np.frexp(np.abs(xv))          # |x| = f * 2^e2, f in [0.5, 1) -> floor(log2|x|) = e2 - 1
    e = np.maximum(e2 - 1, emin)
    q = np.ldexp(1.0, (e - m).astype(np.int64))
    r = np.rint(xv / q) * q
    big = np.abs(r) > fmax
    r[big] = np.copysign(np.inf, xv[big])
    out[fin] = r
    return out


def plan_scale(vals, fmt: str) -> float:
    """s_A = 2^(14 - ceil(log2 max|a|)), the largest power of two with max|a| * s_A <= 2^14,
    for the 16-bit formats; 1 for f64/f32 or an all-zero A."""
    if fmt not in ("f16", "bf16"):
        return 1.0
    v = np.abs(np.asarray(vals, dtype=np.float64))
    v = v[np.isfinite(v)]
    if v.size == 0 or v.max() == 0.0:
        return 1.0
    mx = float(v.max())
    f, e2 = np.frexp(mx)                  # mx = f * 2^e2; ceil(log2 mx) = e2 - 1 if f == 0.5 else e2
    c = int(e2) - 1 if f == 0.5 else int(e2)
    return float(np.ldexp(1.0, 14 - c))


def col_scales(B) -> np.ndarray:
    """s_j = 2^ceil(log2 max_i |B_ij|) (1 for an all-zero column), capped at 2^127 (the largest
    power of two of binary32, in which the scales are kept), float64[N]."""
    B = np.asarray(B, dtype=np.float64)
    mx = np.abs(B).max(axis=0) if B.shape[0] else np.zeros(B.shape[1])
    s = np.ones(B.shape[1], dtype=np.float64)
    nz = mx > 0
    f, e2 = np.frexp(mx[nz])
    c = np.minimum(np.where(f == 0.5, e2 - 1, e2), 127)
    s[nz] = np.ldexp(1.0, c.astype(np.int64))
    return s


def scale_round_columns(B, fmt: str):
    """(B16, s): s = col_scales(B), B16 = round_to(B / s, fmt) as float64 values."""
    s = col_scales(B)
    return round_to(np.asarray(B, dtype=np.float64) / s[None, :], fmt), s


def default_block_rows(fmt: str) -> int:
    return 8 if fmt == "f64" else 16


def partition(A, fmt: str = "f64", block_rows: int | None = None, k_pad: int = 1,
              tau: float = 2.0, contiguous: bool = False, r_boundary: int = 0, tile_min: int = 0) -> dict:
    """Algorithm 1 with the structural split (see ``loops_oracle.c``). Returns the canonical
    partition: csr_rows, csr_ptr, csr_col, csr_val, rb_ids, rb_ptr, tile_col, tile_val
    (tile_val shaped [n_tiles, B_r]); values rounded once into ``fmt`` after the plan scale
    s_A (returned as 'scale', values are stored as round(s_A * a)). tile_min > 1 keeps only
    tiles with at least tile_min stored entries in BCSR blocks; the rest go to the CSR part."""
    L = _load()
    br = default_block_rows(fmt) if block_rows is None else int(block_rows)
    rp, ci, v = _csr_arrays(A)
    sz = np.zeros(4, dtype=np.int64)
    L.oracle_partition_sizes(A.n_rows, _p(rp, _i64p), _p(ci, _i32p), br, int(k_pad), float(tau),
                             int(contiguous), int(r_boundary), int(tile_min), _p(sz, _i64p))
    n_csr, nnz_csr, n_rb, n_t = (int(x) for x in sz)
    out = dict(
        csr_rows=np.zeros(n_csr, np.int32), csr_ptr=np.zeros(n_csr + 1, np.int64),
        csr_col=np.zeros(nnz_csr, np.int32), csr_val=np.zeros(nnz_csr, np.float64),
        rb_ids=np.zeros(n_rb, np.int32), rb_ptr=np.zeros(n_rb + 1, np.int64),
        tile_col=np.zeros(n_t, np.int32), tile_val=np.zeros(n_t * br, np.float64))
    L.oracle_partition_fill(A.n_rows, _p(rp, _i64p), _p(ci, _i32p), _p(v, _f64p), br, int(k_pad),
                            float(tau), int(contiguous), int(r_boundary), int(tile_min),
                            _p(out["csr_rows"], _i32p), _p(out["csr_ptr"], _i64p),
                            _p(out["csr_col"], _i32p), _p(out["csr_val"], _f64p),
                            _p(out["rb_ids"], _i32p), _p(out["rb_ptr"], _i64p),
                            _p(out["tile_col"], _i32p), _p(out["tile_val"], _f64p))
    s = plan_scale(A.vals, fmt)
    out["csr_val"] = round_to(out["csr_val"] * s, fmt)
    out["tile_val"] = round_to(out["tile_val"] * s, fmt).reshape(n_t, br)
    out["scale"] = s
    out["block_rows"] = br
    return out


def expand_partition(part: dict, n_rows: int, n_cols: int) -> np.ndarray:
    """Dense matrix represented by a partition (values divided back by the plan scale):
    CSR-part entries plus every BCSR tile value at (rb_id * B_r + r, col)."""
    br = part["block_rows"]
    D = np.zeros((n_rows, n_cols), dtype=np.float64)
    s = part["scale"]
    for x, i in enumerate(part["csr_rows"]):
        for k in range(part["csr_ptr"][x], part["csr_ptr"][x + 1]):
            D[i, part["csr_col"][k]] += part["csr_val"][k] / s
    for x, b in enumerate(part["rb_ids"]):
        for t in range(part["rb_ptr"][x], part["rb_ptr"][x + 1]):
            c = part["tile_col"][t]
            for r in range(br):
                i = int(b) * br + r
                v = part["tile_val"][t, r]
                if c < 0:
                    assert v == 0.0
                    continue
                if i < n_rows:
                    D[i, c] += v / s
                else:
                    assert v == 0.0
    return D


def spmm_partitioned(part: dict, n_rows: int, B: np.ndarray) -> np.ndarray:
    """C computed part by part from a partition (CSR rows by the inner product, BCSR blocks
    by rank-1 tile updates acc += a_tile (B_r x 1) * B[col, :], Algorithm 2), with values
    divided back by the plan scale; a row present in both parts gets both contributions. Rows
    covered by neither part stay NaN, so a coverage gap shows. Used to pin the partition
    invariant."""
    B = np.asarray(B, dtype=np.float64)
    N = B.shape[1]
    br = part["block_rows"]
    s = part["scale"]
    C = np.zeros((n_rows, N))
    covered = np.zeros(n_rows, dtype=bool)
    for x, i in enumerate(part["csr_rows"]):
        acc = np.zeros(N)
        for k in range(part["csr_ptr"][x], part["csr_ptr"][x + 1]):
            acc += (part["csr_val"][k] / s) * B[part["csr_col"][k]]
        C[i] += acc
        covered[i] = True
    for x, b in enumerate(part["rb_ids"]):
        acc = np.zeros((br, N))
        for t in range(part["rb_ptr"][x], part["rb_ptr"][x + 1]):
            c = part["tile_col"][t]
            if c < 0:
                continue
            acc += np.outer(part["tile_val"][t] / s, B[c])
        r0 = int(b) * br
        r1 = min(r0 + br, n_rows)
        C[r0:r1] += acc[: r1 - r0]
        covered[r0:r1] = True
    C[~covered] = np.nan
    return C
