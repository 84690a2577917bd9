"""GB300-native LOOPS hybrid SpMM (arxiv 2511.08158): Python binding of libloops.so.

This module only marshals arguments into the C ABI declared in ``include/loops.h``; every
step of the SpMM runs in the library's CUDA kernels. PyTorch is used for device memory and
streams. If the library is not built, importing works but every call raises -- there is no
CPU fallback.

    plan = Plan(A, N=64, dtype="f64", tau=2.0, want_backward=True)
    C = plan.spmm(B)                      # C = A . B on the current CUDA stream
    dB, dvals = plan.backward(dC, B)      # A^T . dC and SDDMM(dC, B^T) on A's pattern
    C = spmm(plan, vals, B)               # autograd-aware (LoopsSpMM)
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libloops.so")

F64, F32, F16, BF16 = 0, 1, 2, 3
_DT = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16}
_ERR = {0: "LOOPS_OK", 1: "LOOPS_ERR_INVALID_ARG", 2: "LOOPS_ERR_INVALID_CSR", 3: "LOOPS_ERR_UNSUPPORTED",
        4: "LOOPS_ERR_OOM", 5: "LOOPS_ERR_CUDA", 6: "LOOPS_ERR_TIMEOUT", 7: "LOOPS_ERR_STATE"}

# symbols declared in include/loops.h (checked by the tests)
EXPORTED = ["loops_version", "loops_status_str", "loops_last_error", "loops_plan_opts_default",
            "loops_partition_host", "loops_partition_free", "loops_plan", "loops_plan_destroy",
            "loops_plan_info_get", "loops_plan_export", "loops_plan_update_values", "loops_spmm",
            "loops_spmm_scaled", "loops_spmm_host", "loops_spmm_backward", "loops_cast_scaled",
            "loops_plan_check", "loops_plan_set_timing_events", "loops_plan_set_values",
            "loops_csr_spmm_noalloc", "loops_plan_batched", "loops_spmm_batched", "loops_plan_batched_info",
            "loops_spmm_host_async", "loops_spmm_host_flush", "loops_plan_device",
            "loops_plan_batched_device", "loops_test_fail_alloc", "loops_spmm_backward_scaled",
            "loops_test_wait_limit", "loops_spmm_batched_host", "loops_plan_batched_stats",
            "loops_plan_batched_matrix_info", "loops_perf_model_fit", "loops_perf_model_argmax"]


class LoopsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_ERR.get(status, status)}: {msg}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("vals_dtype", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("block_rows", ctypes.c_int32),
                ("contiguous_split", ctypes.c_int32), ("r_boundary", ctypes.c_int64),
                ("want_backward", ctypes.c_int32), ("split_len", ctypes.c_int32),
                ("tile_min", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class _Info(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("block_rows", ctypes.c_int32), ("k_pad", ctypes.c_int32),
                ("has_backward", ctypes.c_int32), ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("N", ctypes.c_int64), ("tau", ctypes.c_double),
                ("scale", ctypes.c_double), ("n_csr_rows", ctypes.c_int64), ("nnz_csr", ctypes.c_int64),
                ("n_row_blocks", ctypes.c_int64), ("n_tiles", ctypes.c_int64), ("nnz_bcsr", ctypes.c_int64),
                ("n_split_rows", ctypes.c_int64), ("n_segments", ctypes.c_int64),
                ("n_subnormal_vals", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("r_boundary", ctypes.c_int64), ("tile_min", ctypes.c_int64), ("tau_source", ctypes.c_int32),
                ("csr_lane_vectors", ctypes.c_int32), ("bcsr_col_tile", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("model_gflops", ctypes.c_double),
                ("model_coef", ctypes.c_double * 5)]


TAU_MODEL = -2.0   # tau value of LOOPS_TAU_MODEL: the performance model (Eq. 2/3) picks the split


def _info_dict(inf) -> dict:
    out = {name: getattr(inf, name) for name, _ in _Info._fields_ if name != "reserved0"}
    out["model_coef"] = list(out["model_coef"])
    return out


def perf_model_fit(x, y, perf):
    """Eq. 2 coefficients a0..a4 by least squares (``loops_perf_model_fit``; host only)."""
    x, y, p = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, perf))
    coef = np.zeros(5)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().loops_perf_model_fit(x.ctypes.data_as(dp), y.ctypes.data_as(dp), p.ctypes.data_as(dp), x.size,
                                       coef.ctypes.data_as(dp)))
    return coef


def perf_model_argmax(coef, x, y):
    """Eq. 3: (index, predicted perf) of the best candidate (``loops_perf_model_argmax``)."""
    c, x, y = (np.ascontiguousarray(v, dtype=np.float64) for v in (coef, x, y))
    dp = ctypes.POINTER(ctypes.c_double)
    best, bp = ctypes.c_int32(), ctypes.c_double()
    _check(load().loops_perf_model_argmax(c.ctypes.data_as(dp), x.ctypes.data_as(dp), y.ctypes.data_as(dp), x.size,
                                          ctypes.byref(best), ctypes.byref(bp)))
    return best.value, bp.value


class _BatchedInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("block_rows", ctypes.c_int32), ("tau", ctypes.c_double),
                ("n_tasks", ctypes.c_int64), ("n_kernels", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("n_split_rows", ctypes.c_int64), ("n_split_blocks", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("nnz_bcsr", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("tau_source", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("model_gflops", ctypes.c_double),
                ("model_measured_gflops", ctypes.c_double), ("timed_best_gflops", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 2)]


class _Part(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("block_rows", ctypes.c_int32),
                ("k_pad", ctypes.c_int32), ("scale", ctypes.c_double), ("n_csr_rows", ctypes.c_int64),
                ("nnz_csr", ctypes.c_int64), ("n_row_blocks", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("csr_rows", ctypes.POINTER(ctypes.c_int32)), ("csr_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("csr_col", ctypes.POINTER(ctypes.c_int32)), ("csr_val", ctypes.POINTER(ctypes.c_double)),
                ("rb_ids", ctypes.POINTER(ctypes.c_int32)), ("rb_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("tile_col", ctypes.POINTER(ctypes.c_int32)), ("tile_val", ctypes.POINTER(ctypes.c_double))]


_lib = None


def library_path() -> str:
    return LIB_PATH


def load():
    """Load libloops.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libloops.so is not built: run paper_2511_08158_gb300.build() "
                           "(or __graft_entry__.build()) first")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.loops_version.restype = i32
    L.loops_status_str.restype = ctypes.c_char_p
    L.loops_status_str.argtypes = [ctypes.c_int]
    L.loops_last_error.restype = ctypes.c_char_p
    L.loops_plan_opts_default.argtypes = [ctypes.POINTER(_Opts)]
    L.loops_plan_opts_default.restype = None
    L.loops_partition_host.argtypes = [ctypes.POINTER(_Csr), ctypes.c_int, ctypes.POINTER(_Opts), ctypes.POINTER(_Part)]
    L.loops_partition_free.argtypes = [ctypes.POINTER(_Part)]
    L.loops_partition_free.restype = None
    L.loops_plan.argtypes = [ctypes.POINTER(_Csr), i64, ctypes.c_int, ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]
    L.loops_test_fail_alloc.argtypes = [i64]
    L.loops_test_fail_alloc.restype = i64
    L.loops_test_wait_limit.argtypes = [i64]
    L.loops_test_wait_limit.restype = i64
    L.loops_plan_device.argtypes = [ctypes.POINTER(_Csr), i64, ctypes.c_int, ctypes.POINTER(_Opts), vp,
                                    ctypes.POINTER(vp)]
    L.loops_plan_destroy.argtypes = [vp]
    L.loops_plan_info_get.argtypes = [vp, ctypes.POINTER(_Info)]
    L.loops_plan_export.argtypes = [vp, ctypes.POINTER(_Part)]
    L.loops_plan_update_values.argtypes = [vp, vp, ctypes.c_int, vp]
    L.loops_spmm.argtypes = [vp, vp, i64, vp, i64, vp]
    L.loops_spmm_scaled.argtypes = [vp, vp, i64, vp, vp, i64, vp]
    L.loops_spmm_host.argtypes = [vp, vp, i64, vp, i64, vp]
    L.loops_spmm_host_async.argtypes = [vp, vp, i64, vp, i64, vp]
    L.loops_spmm_host_flush.argtypes = [vp, vp]
    L.loops_spmm_backward.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, vp]
    L.loops_spmm_backward_scaled.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, i64, vp, vp]
    L.loops_cast_scaled.argtypes = [vp, i64, i64, i64, ctypes.c_int, vp, i64, vp, vp]
    L.loops_plan_check.argtypes = [vp, vp]
    L.loops_plan_set_values.argtypes = [vp, vp, ctypes.c_int, vp]
    L.loops_csr_spmm_noalloc.argtypes = [i64, i64, i64, vp, vp, vp, ctypes.c_int, vp, i64, i64, vp, i64, vp]
    L.loops_plan_batched.argtypes = [ctypes.POINTER(_Csr), ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int,
                                     ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]
    L.loops_plan_batched_device.argtypes = [ctypes.POINTER(_Csr), ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int,
                                     ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]
    L.loops_spmm_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(vp),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(vp), vp]
    L.loops_spmm_batched_host.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(vp),
                                          ctypes.POINTER(ctypes.c_int64), vp]
    dp = ctypes.POINTER(ctypes.c_double)
    L.loops_perf_model_fit.argtypes = [dp, dp, dp, ctypes.c_int32, dp]
    L.loops_perf_model_argmax.argtypes = [dp, dp, dp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), dp]
    L.loops_plan_batched_stats.argtypes = [vp, ctypes.POINTER(_BatchedInfo)]
    L.loops_plan_batched_matrix_info.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(_Info)]
    L.loops_plan_batched_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    L.loops_plan_set_timing_events.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p)]
    for name in EXPORTED:
        fn = getattr(L, name)
        if name not in ("loops_version", "loops_status_str", "loops_last_error", "loops_plan_opts_default",
                        "loops_partition_free", "loops_test_fail_alloc", "loops_test_wait_limit"):
            fn.restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise LoopsError(status, load().loops_last_error().decode())


def _csr_struct(A):
    """Host CSR arrays of A (attributes n_rows, n_cols, row_ptr, col_idx, vals) -> (_Csr, keepalive).
    nnz is the length of col_idx, so the library's validation (row_ptr[n_rows] == nnz) catches
    arrays shorter than row_ptr claims instead of reading past them."""
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.vals)
    if v.dtype == np.float32:
        vd = F32
    else:
        v = np.ascontiguousarray(v, dtype=np.float64)
        vd = F64
    if rp.size != int(A.n_rows) + 1:
        raise ValueError("row_ptr must have n_rows + 1 entries")
    if v.size != ci.size:
        raise ValueError("vals and col_idx must have the same length")
    s = _Csr(int(A.n_rows), int(A.n_cols), int(ci.size), rp.ctypes.data, ci.ctypes.data, v.ctypes.data, vd)
    return s, (rp, ci, v)


def _csr_struct_device(A):
    """A's CSR arrays as CUDA tensors (copied to the device if they are host arrays) ->
    (_Csr with device pointers, keepalive)."""
    torch = _torch()

    def dev(x, dt):
        t = x if isinstance(x, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(x))
        return t.to(device="cuda", dtype=dt).contiguous()

    rp = dev(A.row_ptr, torch.int64)
    ci = dev(A.col_idx, torch.int32)
    v0 = A.vals
    f32 = (v0.dtype == torch.float32) if isinstance(v0, torch.Tensor) else (np.asarray(v0).dtype == np.float32)
    v = dev(v0, torch.float32 if f32 else torch.float64)
    if rp.numel() != int(A.n_rows) + 1:
        raise ValueError("row_ptr must have n_rows + 1 entries")
    if v.numel() != ci.numel():
        raise ValueError("vals and col_idx must have the same length")
    s = _Csr(int(A.n_rows), int(A.n_cols), int(ci.numel()), rp.data_ptr(), ci.data_ptr(), v.data_ptr(),
             F32 if f32 else F64)
    return s, (rp, ci, v)


def _opts(tau=2.0, block_rows=0, contiguous_split=False, r_boundary=0, want_backward=False, split_len=0,
          tile_min=None):
    o = _Opts()
    load().loops_plan_opts_default(ctypes.byref(o))
    if tile_min is not None:
        o.tile_min = int(tile_min)
    o.tau = float(tau)
    o.block_rows = int(block_rows)
    o.contiguous_split = int(bool(contiguous_split))
    o.r_boundary = int(r_boundary)
    o.want_backward = int(bool(want_backward))
    o.split_len = int(split_len)
    return o


def _part_to_dict(p: _Part) -> dict:
    def arr(ptr, n, dt):
        return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True) if n > 0 else np.zeros(0, dt)
    br = int(p.block_rows)
    out = dict(
        csr_rows=arr(p.csr_rows, p.n_csr_rows, np.int32), csr_ptr=arr(p.csr_ptr, p.n_csr_rows + 1, np.int64),
        csr_col=arr(p.csr_col, p.nnz_csr, np.int32), csr_val=arr(p.csr_val, p.nnz_csr, np.float64),
        rb_ids=arr(p.rb_ids, p.n_row_blocks, np.int32), rb_ptr=arr(p.rb_ptr, p.n_row_blocks + 1, np.int64),
        tile_col=arr(p.tile_col, p.n_tiles, np.int32),
        tile_val=arr(p.tile_val, p.n_tiles * br, np.float64).reshape(int(p.n_tiles), br),
        scale=float(p.scale), block_rows=br, k_pad=int(p.k_pad))
    return out


def partition_host(A, dtype: str = "f64", tau: float = 2.0, block_rows: int = 0, contiguous_split: bool = False,
                   r_boundary: int = 0, tile_min: int = 0) -> dict:
    """Host-only LOOPS partition (no GPU), canonical arrays as numpy."""
    L = load()
    cs, keep = _csr_struct(A)
    o = _opts(tau, block_rows, contiguous_split, r_boundary, tile_min=tile_min)
    part = _Part()
    _check(L.loops_partition_host(ctypes.byref(cs), _DT[dtype], ctypes.byref(o), ctypes.byref(part)))
    try:
        return _part_to_dict(part)
    finally:
        L.loops_partition_free(ctypes.byref(part))


def _torch():
    import torch
    return torch


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_TORCH_IN = {F64: "float64", F32: "float32", F16: "float16", BF16: "bfloat16"}
_TORCH_OUT = {F64: "float64", F32: "float32", F16: "float32", BF16: "float32"}


class Plan:
    """A LOOPS plan for C = A . B with B of N columns (``loops_plan``)."""

    def __init__(self, A, N: int, dtype: str = "f64", tau: float = 2.0, block_rows: int = 0,
                 want_backward: bool = False, contiguous_split: bool = False, r_boundary: int = 0,
                 split_len: int = 0, tile_min=None, stream=None, build_on_device: bool = False):
        """build_on_device: run the whole conversion on the GPU (``loops_plan_device``); A's
        arrays may then be CUDA tensors (host arrays are copied to the device first)."""
        L = load()
        self._L = L
        self.dtype = _DT[dtype]
        self.dtype_name = dtype
        self.N = int(N)
        self.n_rows, self.n_cols = int(A.n_rows), int(A.n_cols)
        o = _opts(tau, block_rows, contiguous_split, r_boundary, want_backward, split_len, tile_min)
        h = ctypes.c_void_p()
        s = _stream_handle(stream) if _torch().cuda.is_available() else ctypes.c_void_p(0)
        if build_on_device:
            cs, keep = _csr_struct_device(A)
            self.nnz = int(cs.nnz)
            _check(L.loops_plan_device(ctypes.byref(cs), self.N, self.dtype, ctypes.byref(o), s, ctypes.byref(h)))
        else:
            cs, keep = _csr_struct(A)
            self.nnz = int(cs.nnz)
            _check(L.loops_plan(ctypes.byref(cs), self.N, self.dtype, ctypes.byref(o), s, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.loops_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def info(self) -> dict:
        inf = _Info()
        _check(self._L.loops_plan_info_get(self._h, ctypes.byref(inf)))
        return _info_dict(inf)

    def export(self) -> dict:
        part = _Part()
        _check(self._L.loops_plan_export(self._h, ctypes.byref(part)))
        try:
            return _part_to_dict(part)
        finally:
            self._L.loops_partition_free(ctypes.byref(part))

    def set_timing_events(self, events):
        """events: 4 raw cudaEvent_t handles (ints) recorded around the CSR and BCSR parts of
        each later spmm call, or None to stop."""
        if events is None:
            _check(self._L.loops_plan_set_timing_events(self._h, None))
            return
        arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(int(e)) for e in events])
        _check(self._L.loops_plan_set_timing_events(self._h, arr))

    def check(self, stream=None):
        _check(self._L.loops_plan_check(self._h, _stream_handle(stream)))

    def update_values(self, vals, stream=None):
        v = np.ascontiguousarray(vals)
        vd = F32 if v.dtype == np.float32 else F64
        if vd == F64:
            v = np.ascontiguousarray(v, dtype=np.float64)
        _check(self._L.loops_plan_update_values(self._h, v.ctypes.data, vd, _stream_handle(stream)))

    def set_values(self, vals, stream=None):
        """Refresh A's values from a CUDA tensor (float64/float32, input order, nnz entries)."""
        torch = _torch()
        if not (isinstance(vals, torch.Tensor) and vals.is_cuda and vals.dim() == 1 and vals.numel() == self.nnz):
            raise ValueError("vals must be a 1-D CUDA tensor with nnz entries")
        if vals.dtype not in (torch.float64, torch.float32):
            raise TypeError("vals must be float64 or float32")
        vals = vals.contiguous()
        _check(self._L.loops_plan_set_values(self._h, vals.data_ptr(), F64 if vals.dtype == torch.float64 else F32,
                                             _stream_handle(stream)))

    def out_dtype(self):
        return getattr(_torch(), _TORCH_OUT[self.dtype])

    def in_dtype(self):
        return getattr(_torch(), _TORCH_IN[self.dtype])

    def _check_dense(self, X, rows, name):
        torch = _torch()
        if not (isinstance(X, torch.Tensor) and X.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
        if X.dtype != self.in_dtype():
            raise TypeError(f"{name} must be {self.in_dtype()} for this plan")
        if X.dim() != 2 or X.shape[0] != rows or X.shape[1] != self.N or X.stride(1) != 1:
            raise ValueError(f"{name} must be {rows} x {self.N} with unit column stride")

    def spmm(self, B, C=None, col_scale=None, stream=None):
        """C = A . B (device tensors; C allocated if not given). col_scale: optional f32[N] device
        tensor of per-column scales (16-bit dtypes)."""
        torch = _torch()
        self._check_dense(B, self.n_cols, "B")
        if C is None:
            C = torch.empty((self.n_rows, self.N), dtype=self.out_dtype(), device=B.device)
        cs = 0 if col_scale is None else col_scale.data_ptr()
        _check(self._L.loops_spmm_scaled(self._h, B.data_ptr(), B.stride(0), cs, C.data_ptr(), C.stride(0),
                                         _stream_handle(stream)))
        return C

    def spmm_host(self, B_host, C_host, stream=None):
        """End-to-end C = A . B with host (ideally pinned) CPU tensors; synchronises."""
        _check(self._L.loops_spmm_host(self._h, B_host.data_ptr(), B_host.stride(0), C_host.data_ptr(),
                                       C_host.stride(0), _stream_handle(stream)))
        return C_host

    def spmm_host_async(self, B_host, C_host, stream=None):
        """Pipelined end-to-end C = A . B with pinned host tensors (consecutive calls overlap
        their transfers); C_host is complete after host_flush() and a stream synchronisation."""
        _check(self._L.loops_spmm_host_async(self._h, B_host.data_ptr(), B_host.stride(0), C_host.data_ptr(),
                                             C_host.stride(0), _stream_handle(stream)))
        return C_host

    def host_flush(self, stream=None):
        """Make the stream wait for the last pipelined call's copy-out."""
        _check(self._L.loops_spmm_host_flush(self._h, _stream_handle(stream)))

    def backward(self, dC, B, need_dB=True, need_dvals=True, dc_scale=None, b_scale=None, stream=None):
        """(dB, dvals) = (A^T . dC, <dC[i_k], B[j_k]> per stored entry in input order).
        dc_scale / b_scale: optional f32[N] CUDA tensors of per-column scales of dC and B (16-bit
        plans, e.g. from cast_scaled): the gradients of the true operands dC diag(dc_scale) and
        B diag(b_scale) are returned (``loops_spmm_backward_scaled``)."""
        torch = _torch()
        self._check_dense(dC, self.n_rows, "dC")
        for name, sc in (("dc_scale", dc_scale), ("b_scale", b_scale)):
            if sc is not None and not (isinstance(sc, torch.Tensor) and sc.is_cuda and sc.dtype == torch.float32
                                       and sc.dim() == 1 and sc.numel() == self.N and sc.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of N entries")
        dB = dv = None
        if need_dB:
            dB = torch.empty((self.n_cols, self.N), dtype=self.out_dtype(), device=dC.device)
        if need_dvals:
            self._check_dense(B, self.n_cols, "B")
            dv = torch.empty((self.nnz,), dtype=self.out_dtype(), device=dC.device)
        _check(self._L.loops_spmm_backward_scaled(
            self._h, dC.data_ptr(), dC.stride(0), 0 if dc_scale is None else dc_scale.data_ptr(),
            B.data_ptr() if B is not None else 0, B.stride(0) if B is not None else self.N,
            0 if b_scale is None else b_scale.data_ptr(), dB.data_ptr() if dB is not None else 0,
            dB.stride(0) if dB is not None else self.N, dv.data_ptr() if dv is not None else 0,
            _stream_handle(stream)))
        return dB, dv


class BatchedPlan:
    """Many matrices with their own N behind one persistent, graph-captured launch
    (``loops_plan_batched`` / ``loops_spmm_batched``)."""

    def __init__(self, As, Ns, dtype: str = "f32", tau: float = -1.0, block_rows: int = 0, split_len: int = 0,
                 stream=None, build_on_device: bool = False):
        """build_on_device: convert every matrix on the GPU (``loops_plan_batched_device``);
        the matrices' arrays may then be CUDA tensors (host arrays are copied first)."""
        L = load()
        self._L = L
        self.dtype = _DT[dtype]
        self.count = len(As)
        self.Ns = [int(n) for n in Ns]
        self.shapes = [(int(A.n_rows), int(A.n_cols)) for A in As]
        structs, self._keep = [], []
        for A in As:
            cs, keep = _csr_struct_device(A) if build_on_device else _csr_struct(A)
            structs.append(cs)
            self._keep.append(keep)
        arr = (_Csr * max(1, self.count))(*structs)
        ns = (ctypes.c_int64 * max(1, self.count))(*self.Ns)
        o = _opts(tau, block_rows, False, 0, False, split_len)
        h = ctypes.c_void_p()
        entry = L.loops_plan_batched_device if build_on_device else L.loops_plan_batched
        _check(entry(arr, ns, self.count, self.dtype, ctypes.byref(o), _stream_handle(stream), ctypes.byref(h)))
        self._keep = None  # the plan does not keep the host CSR arrays
        self._h = h

    def info(self) -> dict:
        c, t, tau, br = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32()
        _check(self._L.loops_plan_batched_info(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(tau),
                                               ctypes.byref(br)))
        return {"count": c.value, "n_tasks": t.value, "tau": tau.value, "block_rows": br.value}

    def stats(self) -> dict:
        """Totals of the plan (``loops_plan_batched_stats``)."""
        inf = _BatchedInfo()
        _check(self._L.loops_plan_batched_stats(self._h, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in _BatchedInfo._fields_ if not name.startswith("reserved")}

    def matrix_info(self, m: int) -> dict:
        """The plan info of matrix m (``loops_plan_batched_matrix_info``)."""
        inf = _Info()
        _check(self._L.loops_plan_batched_matrix_info(self._h, int(m), ctypes.byref(inf)))
        return _info_dict(inf)

    def spmm(self, Bs, Cs=None, col_scales=None, stream=None):
        torch = _torch()
        if Cs is None:
            Cs = [torch.empty((r, n), dtype=getattr(torch, _TORCH_OUT[self.dtype]), device=B.device)
                  for (r, _), n, B in zip(self.shapes, self.Ns, Bs)]
        n = max(1, self.count)
        bp = (ctypes.c_void_p * n)(*[B.data_ptr() for B in Bs])
        cp = (ctypes.c_void_p * n)(*[C.data_ptr() for C in Cs])
        lb = (ctypes.c_int64 * n)(*[B.stride(0) for B in Bs])
        lc = (ctypes.c_int64 * n)(*[C.stride(0) for C in Cs])
        sp = None
        if col_scales is not None:
            sp = (ctypes.c_void_p * n)(*[0 if s is None else s.data_ptr() for s in col_scales])
        _check(self._L.loops_spmm_batched(self._h, bp, lb, cp, lc, sp, _stream_handle(stream)))
        return Cs

    def spmm_host(self, Bs_host, Cs_host, stream=None):
        """End-to-end batch with host (ideally pinned) CPU tensors: B_m copied in, the batch run,
        C_m (f32) copied out; synchronises (``loops_spmm_batched_host``)."""
        n = max(1, self.count)
        for (r, c), N, B, C in zip(self.shapes, self.Ns, Bs_host, Cs_host):
            if B.is_cuda or C.is_cuda or B.dim() != 2 or C.dim() != 2 or B.shape != (c, N) or C.shape != (r, N) \
                    or B.stride(1) != 1 or C.stride(1) != 1:
                raise ValueError("host operands must be CPU tensors of n_cols x N and n_rows x N, unit column stride")
        bp = (ctypes.c_void_p * n)(*[B.data_ptr() for B in Bs_host])
        cp = (ctypes.c_void_p * n)(*[C.data_ptr() for C in Cs_host])
        lb = (ctypes.c_int64 * n)(*[B.stride(0) for B in Bs_host])
        lc = (ctypes.c_int64 * n)(*[C.stride(0) for C in Cs_host])
        _check(self._L.loops_spmm_batched_host(self._h, bp, lb, cp, lc, _stream_handle(stream)))
        return Cs_host

    def set_timing_events(self, events):
        """events: 4 raw cudaEvent_t handles recorded around the persistent kernel ([0], [1]) and
        the partial-sum launches ([2], [3]) of every later call, or None to stop."""
        if events is None:
            _check(self._L.loops_plan_set_timing_events(self._h, None))
            return
        arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(int(e)) for e in events])
        _check(self._L.loops_plan_set_timing_events(self._h, arr))

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.loops_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def cast_scaled(X, dtype: str = "f16", stream=None):
    """(Y, s): s_j = 2^ceil(log2 max|X[:, j]|), Y = round(X / s) in f16/bf16 (``loops_cast_scaled``)."""
    torch = _torch()
    L = load()
    if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2 or X.stride(1) != 1:
        raise TypeError("X must be a 2-D float32 CUDA tensor with unit column stride")
    yd = _DT[dtype]
    Y = torch.empty(X.shape, dtype=torch.float16 if yd == F16 else torch.bfloat16, device=X.device)
    s = torch.empty((X.shape[1],), dtype=torch.float32, device=X.device)
    _check(L.loops_cast_scaled(X.data_ptr(), X.shape[0], X.shape[1], X.stride(0), yd, Y.data_ptr(), Y.stride(0),
                               s.data_ptr(), _stream_handle(stream)))
    return Y, s


def csr_spmm_noalloc(row_ptr, col_idx, vals, n_cols, B, C, stream=None):
    """C = A . B from device CSR tensors without any device allocation
    (``loops_csr_spmm_noalloc``). row_ptr: int64 [n_rows + 1]; col_idx: int32 [nnz]; vals: nnz
    values in B's dtype (float64, float32, float16 or bfloat16); B: n_cols x N; C: n_rows x N,
    preallocated, float64 for float64 inputs and float32 for every other input dtype. All on
    one CUDA device, 1-D arrays contiguous, B and C with unit column stride."""
    torch = _torch()
    dts = {torch.float64: F64, torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}
    for name, t in (("row_ptr", row_ptr), ("col_idx", col_idx), ("vals", vals), ("B", B), ("C", C)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
    if B.dtype not in dts:
        raise TypeError("B must be float64, float32, float16 or bfloat16")
    c_dtype = torch.float64 if B.dtype == torch.float64 else torch.float32
    if row_ptr.dtype != torch.int64 or row_ptr.dim() != 1 or not row_ptr.is_contiguous() or row_ptr.numel() < 1:
        raise TypeError("row_ptr must be a contiguous 1-D int64 tensor of n_rows + 1 entries")
    if col_idx.dtype != torch.int32 or col_idx.dim() != 1 or not col_idx.is_contiguous():
        raise TypeError("col_idx must be a contiguous 1-D int32 tensor")
    if vals.dtype != B.dtype or vals.dim() != 1 or not vals.is_contiguous() or vals.numel() != col_idx.numel():
        raise TypeError("vals must be a contiguous 1-D tensor of B's dtype with one value per column index")
    n_rows = row_ptr.numel() - 1
    if B.dim() != 2 or B.shape[0] != int(n_cols) or B.stride(1) != 1:
        raise ValueError("B must be n_cols x N with unit column stride")
    N = B.shape[1]
    if C.dtype != c_dtype or C.dim() != 2 or C.shape[0] != n_rows or C.shape[1] != N or C.stride(1) != 1:
        raise ValueError(f"C must be a {c_dtype} tensor of n_rows x N with unit column stride")
    if not all(t.is_cuda for t in (row_ptr, col_idx, vals, B, C)):
        raise TypeError("all operands must be CUDA tensors")
    if len({t.device for t in (row_ptr, col_idx, vals, B, C)}) != 1:
        raise ValueError("all operands must be on one device")
    _check(load().loops_csr_spmm_noalloc(
        n_rows, int(n_cols), col_idx.numel(), row_ptr.data_ptr(), col_idx.data_ptr(), vals.data_ptr(),
        dts[B.dtype], B.data_ptr(), B.stride(0), N, C.data_ptr(), C.stride(0), _stream_handle(stream)))
    return C


def _autograd_fn():
    torch = _torch()

    class LoopsSpMM(torch.autograd.Function):
        """C = A(vals) . B with the plan's pattern. Backward: dB = A^T . dC (transposed hybrid
        SpMM), dvals = SDDMM(dC, B^T) on A's pattern. The forward refreshes the plan's stored
        values from ``vals`` on the device (plan built with want_backward); ``vals`` is saved
        for the backward, which stores it into the plan again, so another forward on the same
        plan in between (shared weights) does not change this call's gradients, and autograd's
        version check refuses an in-place edit of ``vals`` after the forward. For FP16/BF16
        plans dC (f32) is scaled per column by a power of two before its cast (as the forward
        operands of loops_spmm_scaled are), and the scales are undone on dB and dvals."""

        @staticmethod
        def forward(ctx, vals, B, plan):
            ctx.plan = plan
            ctx.save_for_backward(vals, B)
            plan.set_values(vals.detach())
            return plan.spmm(B.contiguous())

        @staticmethod
        def backward(ctx, dC):
            vals, B = ctx.saved_tensors
            plan = ctx.plan
            plan.set_values(vals.detach())
            dc_scale = None
            if plan.dtype in (F16, BF16):
                dC, dc_scale = cast_scaled(dC.float().contiguous(), plan.dtype_name)
            else:
                dC = dC.to(plan.in_dtype()).contiguous()
            dB, dv = plan.backward(dC, B.contiguous(), need_dB=ctx.needs_input_grad[1],
                                   need_dvals=ctx.needs_input_grad[0], dc_scale=dc_scale)
            if dB is not None:
                dB = dB.to(B.dtype)
            if dv is not None:
                dv = dv.to(vals.dtype)
            return dv, dB, None

    return LoopsSpMM


_FN = None


def spmm(plan: Plan, vals, B):
    """Autograd-aware C = A . B (LoopsSpMM)."""
    global _FN
    if _FN is None:
        _FN = _autograd_fn()
    return _FN.apply(vals, B, plan)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libloops.so for sm_103a (see builder.py)."""
    from .builder import build as _build
    return _build(force=force, verbose=verbose)
