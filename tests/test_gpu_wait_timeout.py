"""Failure detection of the bounded waits, without faulting or hanging the GPU.

The F16/BF16 BCSR kernel waits on shared-memory barriers for its bulk copies of B rows, and
every wait has an iteration bound. A test hook of the library (loops_test_wait_limit) lowers
that bound to zero polls, so each wait gives up at once: the kernel must record the timeout in
the plan's error word (loops_plan_check -> LOOPS_ERR_TIMEOUT), let its copies in flight land,
skip its store, and leave the context usable -- the next call with the default bound is
correct again."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, rounded_inputs, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_bcsr_wait_timeout_is_reported_and_recovers(loops_lib, fmt):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lp = loops_lib
    L = lp.load()
    rng = np.random.default_rng(31)
    A = W.dense_blocks(256, 2, 16, rng)        # every row block holds two dense 16 x 16 blocks
    N = 64
    B = W.dense_normal(256, N, 32)
    A_r, Bq, _, B_eff = rounded_inputs(A, B, fmt, scale_columns=False)
    plan = lp.Plan(A, N, fmt, tau=0.0)
    info = plan.info()
    assert info["n_row_blocks"] == 16 and info["n_csr_rows"] == 0
    Bd = to_device(torch, Bq, fmt)
    C = torch.full((256, N), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    L.loops_test_wait_limit(0)
    try:
        plan.spmm(Bd, C)
    finally:
        L.loops_test_wait_limit(-1)
    torch.cuda.synchronize()
    with pytest.raises(lp.LoopsError) as e:
        plan.check()
    assert e.value.status == 6                  # LOOPS_ERR_TIMEOUT
    assert torch.isnan(C).all()                 # every CTA gave up and skipped its store
    plan.check()                                # the error word was read and cleared
    # the same plan, default bound: correct output, no error
    plan.spmm(Bd, C)
    torch.cuda.synchronize()
    plan.check()
    assert rel_l2(C.double().cpu().numpy(), oracle.spmm(A_r, B_eff)) <= TOL[fmt]
