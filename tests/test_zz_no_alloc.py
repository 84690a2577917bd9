"""The allocation-free entry point, loops_csr_spmm_noalloc, against the oracle.

Some callers cannot allocate device memory where they multiply: work recorded into a CUDA
graph under the global capture mode, host callbacks, or services that reserve all memory up
front. They pass their own device CSR arrays to loops_csr_spmm_noalloc, which keeps its
partial sums in one static device array instead of allocating. The GPU test calls it twice in
a row through the C ABI -- the second call finds the first call's partial sums still in that
array -- and checks each result against the oracle on the same rounded inputs, within the
parity tests' tolerance. The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, torch_dtype

torch = pytest.importorskip("torch")

SCRATCH = 16 << 20        # LOOPS_NOALLOC_SCRATCH_BYTES


def _matrix(fmt):
    # short rows, empty rows, and long rows that cross several 128-entry chunks
    A = W.random_csr(300, 280, 0.03, 41, duplicates=True, unsorted=True)
    rows = [A.row_ids(), np.full(280, 17), np.full(280, 200), np.full(150, 299)]
    cols = [A.col_idx.astype(np.int64), np.arange(280), np.arange(280)[::-1], np.arange(150) * 1]
    vals = [A.vals, np.random.default_rng(1).standard_normal(280), np.random.default_rng(2).standard_normal(280),
            np.random.default_rng(3).standard_normal(150)]
    r = np.concatenate(rows)
    keep = (r % 23) != 5                       # leave some rows empty
    A = W.csr_from_coo(300, 280, r[keep], np.concatenate(cols)[keep], np.concatenate(vals)[keep],
                       sort_cols=False)
    # the kernel multiplies the values as stored in the format (no plan scale)
    A.vals = oracle.round_to(A.vals, fmt)
    return A


@pytest.mark.gpu
@pytest.mark.parametrize("fmt", ["f64", "f32", "f16", "bf16"])
def test_noalloc_matches_oracle_on_two_calls(loops_lib, fmt):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lp = loops_lib
    L = lp.load()
    A = _matrix(fmt)
    N = 48
    dt = torch_dtype(torch, fmt)
    out_dt = torch.float64 if fmt == "f64" else torch.float32
    rp = torch.as_tensor(A.row_ptr, dtype=torch.int64).cuda()
    ci = torch.as_tensor(A.col_idx, dtype=torch.int32).cuda()
    va = torch.as_tensor(A.vals).to(dt).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        Bq = oracle.round_to(W.dense_normal(280, N, 100 + call), fmt)
        B = torch.as_tensor(Bq).to(dt).cuda()
        C = torch.full((300, N), float("nan"), dtype=out_dt, device="cuda")
        st = L.loops_csr_spmm_noalloc(300, 280, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                                      lp._DT[fmt], B.data_ptr(), B.stride(0), N, C.data_ptr(), C.stride(0),
                                      ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.loops_last_error()
        torch.cuda.synchronize()
        got = C.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, oracle.spmm(A, Bq)) <= TOL[fmt]


@pytest.mark.gpu
def test_noalloc_rejects_problems_beyond_its_scratch(loops_lib):
    # every buffer is real and as large as the sizes passed claim, so nothing could be read or
    # written out of bounds even if a size check were missing
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = loops_lib.load()
    dev = "cuda"
    # 2 * ceil(nnz / 128) * N * 4 bytes = 64 MiB > 16 MiB
    n_rows, n_cols, nnz, N = 1000, 1000, 1 << 24, 64
    rp = torch.zeros(n_rows + 1, dtype=torch.int64, device=dev)
    rp[-1] = nnz
    ci = torch.zeros(nnz, dtype=torch.int32, device=dev)
    va = torch.zeros(nnz, dtype=torch.float32, device=dev)
    B = torch.zeros((n_cols, N), dtype=torch.float32, device=dev)
    C = torch.zeros((n_rows, N), dtype=torch.float32, device=dev)
    st = L.loops_csr_spmm_noalloc(n_rows, n_cols, nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1,
                                  B.data_ptr(), N, N, C.data_ptr(), N, None)
    assert st == 3
    assert b"scratch" in L.loops_last_error()
    # a problem whose scratch fits exactly but whose N needs more than 65535 column slices
    N = 65536 * 32
    assert 2 * 1 * N * 4 == SCRATCH
    rp = torch.tensor([0, 1], dtype=torch.int64, device=dev)
    ci = torch.zeros(1, dtype=torch.int32, device=dev)
    va = torch.ones(1, dtype=torch.float32, device=dev)
    B = torch.zeros((1, N), dtype=torch.float32, device=dev)
    C = torch.zeros((1, N), dtype=torch.float32, device=dev)
    st = L.loops_csr_spmm_noalloc(1, 1, 1, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1, B.data_ptr(), N, N,
                                  C.data_ptr(), N, None)
    assert st == 3
    assert b"launch shape" in L.loops_last_error()
    torch.cuda.synchronize()


def test_noalloc_size_checks_need_no_device(loops_lib):
    # the size checks come before any device call: on a machine without a GPU they answer
    # LOOPS_ERR_UNSUPPORTED for problems the static array cannot hold, including an N so large
    # that the byte count would wrap around in 64-bit arithmetic
    if torch.cuda.is_available():
        pytest.skip("runs only where no GPU exists (its pointers are placeholders)")
    L = loops_lib.load()
    dummy = ctypes.c_void_p(16)
    for n_rows, nnz, N in ((1000, 1 << 24, 64), (10, 0, 1 << 62), (10, 1000, (1 << 61) + 1),
                           (1, 1, 65536 * 32)):
        st = L.loops_csr_spmm_noalloc(n_rows, 10, nnz, dummy, dummy, dummy, 1, dummy, N, N, dummy, N, None)
        assert st == 3, (n_rows, nnz, N, L.loops_last_error())


def test_noalloc_binding_rejects_bad_operands(loops_lib):
    # argument checks of the Python binding (CPU tensors: each case fails before the device test)
    lp = loops_lib
    rp = torch.tensor([0, 1, 2], dtype=torch.int64)
    ci = torch.tensor([0, 1], dtype=torch.int32)
    v32 = torch.ones(2, dtype=torch.float32)
    B = torch.ones((3, 8), dtype=torch.float32)
    C = torch.empty((2, 8), dtype=torch.float32)
    cases = [
        (rp.int(), ci, v32, B, C),                                   # int32 row_ptr
        (rp, ci.long(), v32, B, C),                                  # int64 col_idx
        (rp, ci, v32.double(), B, C),                                # vals not in B's dtype
        (rp, ci, torch.ones(3, dtype=torch.float32), B, C),          # vals length != nnz
        (rp, ci, v32, torch.ones((4, 8)), C),                        # B rows != n_cols
        (rp, ci, v32, B.t().contiguous().t(), C),                    # B without unit column stride
        (rp, ci, v32, B, torch.empty((3, 8))),                       # C rows != n_rows
        (rp, ci, v32, B, torch.empty((2, 8), dtype=torch.float64)),  # C dtype
        (rp, ci, v32.half(), B.half(), C.half()),                    # F16 needs an f32 C
        (rp, ci, v32, B, C),                                         # host tensors
    ]
    for args in cases:
        with pytest.raises((TypeError, ValueError)):
            lp.csr_spmm_noalloc(args[0], args[1], args[2], 3, args[3], args[4])
