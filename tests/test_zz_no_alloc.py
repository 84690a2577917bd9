"""The allocation-free entry point, loops_csr_spmm_noalloc, against the plan-based loops_spmm.

Some callers cannot allocate device memory where they multiply: work recorded into a CUDA
graph under the global capture mode, host callbacks, or services that reserve all memory up
front. They pass their own device CSR arrays to loops_csr_spmm_noalloc, which keeps its
partial sums in one static device array instead of allocating. This test calls it twice in a
row through the C ABI -- the second call finds the first call's partial sums still in that
array -- and checks each result against loops_spmm within the parity tests' tolerance. The
file name makes pytest collect it last.
"""
import ctypes
import math

import numpy as np
import pytest

import workloads as W
from gpu_util import TOL, rel_l2, torch_dtype

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
    # values representable in the format, so the plan path's power-of-two scale is exact
    A.vals = torch.as_tensor(A.vals).to(torch_dtype(torch, fmt)).double().numpy()
    return A


@pytest.mark.parametrize("fmt", ["f64", "f32", "f16", "bf16"])
def test_noalloc_matches_plan_path_on_two_calls(loops_lib, fmt):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lp = loops_lib
    L = lp.load()
    A = _matrix(fmt)
    N = 48
    dt = torch_dtype(torch, fmt)
    rp = torch.as_tensor(A.row_ptr, dtype=torch.int64).cuda()
    ci = torch.as_tensor(A.col_idx, dtype=torch.int32).cuda()
    va = torch.as_tensor(A.vals).to(dt).cuda()
    plan = lp.Plan(A, N, fmt, tau=math.inf)
    stream = torch.cuda.current_stream()
    for call in range(2):
        B = torch.as_tensor(W.dense_normal(280, N, 100 + call)).to(dt).cuda()
        ref = plan.spmm(B)
        C = torch.full((300, N), float("nan"), dtype=ref.dtype, device="cuda")
        st = L.loops_csr_spmm_noalloc(300, 280, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                                      lp._DT[fmt], B.data_ptr(), B.stride(0), N, C.data_ptr(), C.stride(0),
                                      ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, L.loops_last_error()
        torch.cuda.synchronize()
        got = C.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref.double().cpu().numpy()) <= TOL[fmt]


def test_noalloc_rejects_problems_beyond_its_scratch(loops_lib):
    L = loops_lib.load()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    # 2 * ceil(nnz / 128) * N * 4 bytes > 16 MiB
    st = L.loops_csr_spmm_noalloc(1000, 1000, 1 << 24, dummy, dummy, dummy, 1, dummy, 64, 64, dummy, 64, None)
    assert st == 3
    assert b"scratch" in L.loops_last_error()
