"""Error paths on the GPU without a GPU fault: every device (and pinned host) allocation of a
plan build is made to fail in turn through the library's test hook (loops_test_fail_alloc),
and each failure must come back as LOOPS_ERR_OOM with everything released -- free device
memory back where it started -- and the library still working. Destroyed handles are refused
without their memory being read."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, rounded_inputs, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OOM = 4
STATE = 7


@pytest.fixture(scope="module")
def lp(loops_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return loops_lib


def _matrix():
    # both parts, a row long enough to be cut into segments, a block cut into units
    A, _ = W.laplacian_blocks(grid=24, n_blocks=10, block=8, seed=3, N=8)
    n = A.n_rows
    rng = np.random.default_rng(4)
    # row 5: 300 distinct extra columns (its row block stays sparse, d < 2, and the row is longer
    # than the split length 128); rows 32-47: 300 entries each over 576 columns (dense, > 256 tiles)
    r = np.concatenate([A.row_ids(), np.full(300, 5), np.repeat(np.arange(32, 48), 300)])
    c = np.concatenate([A.col_idx.astype(np.int64), rng.choice(n, 300, replace=False),
                        rng.integers(0, n, 16 * 300)])
    v = np.concatenate([A.vals, rng.standard_normal(300 + 16 * 300)])
    return W.csr_from_coo(n, n, r, c, v)


def _on_device(A):
    return W.CSR(A.n_rows, A.n_cols, torch.as_tensor(A.row_ptr).cuda(), torch.as_tensor(A.col_idx).cuda(),
                 torch.as_tensor(A.vals).cuda())


def _every_allocation_fails_cleanly(lp, build):
    L = lp.load()
    L.loops_test_fail_alloc(0)
    build().destroy()
    n_alloc = L.loops_test_fail_alloc(0)
    assert n_alloc > 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for k in range(1, n_alloc + 1):
            L.loops_test_fail_alloc(k)
            with pytest.raises(lp.LoopsError) as ei:
                build()
            assert ei.value.status == OOM, (k, str(ei.value))
            L.loops_test_fail_alloc(0)
    finally:
        L.loops_test_fail_alloc(0)
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < (32 << 20)  # nothing left allocated
    return n_alloc


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("backward", [False, True])
def test_plan_build_allocation_failures(lp, device, backward):
    A = _matrix()
    src = _on_device(A) if device else A
    fmt = "bf16"

    def build():
        return lp.Plan(src, 16, fmt, tau=2.0, split_len=128, want_backward=backward, build_on_device=device)

    n_alloc = _every_allocation_fails_cleanly(lp, build)
    print(f"device={device} backward={backward}: {n_alloc} allocations, each failed in turn")
    # the library still works: a fresh plan agrees with the oracle
    plan = build()
    info = plan.info()
    assert info["n_row_blocks"] > 0 and info["n_split_rows"] > 0
    B = W.dense_normal(A.n_cols, 16, 1)
    A_r, Bg, s, B_eff = rounded_inputs(A, B, fmt)
    C = plan.spmm(to_device(torch, Bg, fmt), col_scale=torch.as_tensor(s, dtype=torch.float32).cuda())
    assert rel_l2(C.double().cpu().numpy(), oracle.spmm(A_r, B_eff)) <= TOL[fmt]


@pytest.mark.parametrize("device", [False, True])
def test_batched_plan_allocation_failures(lp, device):
    mats = W.batched_mix(count=5, seed=2, min_rows=200, max_rows=1500)
    As = [_on_device(A) if device else A for A, _ in mats]
    Ns = [N for _, N in mats]

    def build():
        return lp.BatchedPlan(As, Ns, "f32", tau=2.0, build_on_device=device)

    _every_allocation_fails_cleanly(lp, build)
    bp = build()
    Bs = [torch.randn((A.n_cols, N), device="cuda") for A, N in mats]
    for (A, N), B, C in zip(mats, Bs, bp.spmm(Bs)):
        ref = oracle.spmm(W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, oracle.round_to(A.vals, "f32")),
                          B.double().cpu().numpy())
        assert rel_l2(C.double().cpu().numpy(), ref) <= TOL["f32"]


def test_host_pipeline_allocation_failure(lp):
    A = _matrix()
    plan = lp.Plan(A, 16, "f64", tau=math.inf)
    B = torch.as_tensor(W.dense_normal(A.n_cols, 16, 2)).pin_memory()
    C = torch.empty((A.n_rows, 16), dtype=torch.float64).pin_memory()
    L = lp.load()
    L.loops_test_fail_alloc(1)  # the first staging buffer of the pipelined host call
    try:
        with pytest.raises(lp.LoopsError) as ei:
            plan.spmm_host_async(B, C)
    finally:
        L.loops_test_fail_alloc(0)
    assert ei.value.status == OOM
    plan.spmm_host_async(B, C)  # a later call sets the pipeline up and works
    plan.host_flush()
    torch.cuda.current_stream().synchronize()
    assert rel_l2(C.numpy(), oracle.spmm(A, B.numpy())) <= TOL["f64"]


def test_destroyed_handle_is_refused(lp):
    A = _matrix()
    plan = lp.Plan(A, 8, "f64", tau=2.0)
    h = ctypes.c_void_p(plan.handle.value)
    plan.destroy()
    L = lp.load()
    info = lp._Info()
    assert L.loops_plan_info_get(h, ctypes.byref(info)) == STATE
    assert L.loops_plan_destroy(h) == STATE
    assert L.loops_spmm(h, None, 8, None, 8, None) == STATE
    assert b"destroyed" in L.loops_last_error()


def test_fault_alloc_environment_variable(lp):
    # LOOPS_FAULT_ALLOC=k arms the same hook at start-up: the process's first allocation fails
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_2511_08158_gb300 as lp, workloads as W\n"
        "A = W.random_csr(50, 50, 0.1, 1)\n"
        "try:\n"
        "    lp.Plan(A, 8, 'f64', tau=2.0)\n"
        "    print('built')\n"
        "except lp.LoopsError as e:\n"
        "    print('status', e.status)\n"
        "lp.Plan(A, 8, 'f64', tau=2.0)\n"
        "print('second ok')\n" % root)
    env = dict(os.environ, LOOPS_FAULT_ALLOC="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "status 4" in out.stdout and "second ok" in out.stdout, out.stdout
