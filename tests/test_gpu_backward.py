"""GPU backward parity: dB = A^T . dC by the transposed hybrid plan and dvals = SDDMM(dC, B^T)
on A's pattern, against the oracle's own scatter loop and SDDMM; finite differences in FP64 on
a 1,024-node GCN instance; torch.autograd.gradcheck of LoopsSpMM in FP64; device-side value
refresh equal to the host packer bit for bit."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp(loops_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return loops_lib


def _rounded(A, fmt):
    s = oracle.plan_scale(A.vals, fmt)
    return W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, oracle.round_to(A.vals * s, fmt) / s)


@pytest.mark.parametrize("fmt", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("tau", [0.0, 1.5, math.inf])
@pytest.mark.parametrize("N", [16, 40, 64, 128])
def test_backward_matches_oracle(lp, fmt, tau, N):
    A = W.random_csr(190, 230, 0.05, N, duplicates=True, unsorted=True, explicit_zeros=True)
    A_r = _rounded(A, fmt)
    B = oracle.round_to(W.dense_normal(230, N, 1), fmt)
    dC = oracle.round_to(W.dense_normal(190, N, 2), fmt)
    plan = lp.Plan(A, N, fmt, tau=tau, want_backward=True, split_len=16)
    dB, dv = plan.backward(to_device(torch, dC, fmt), to_device(torch, B, fmt))
    torch.cuda.synchronize()
    plan.check()
    assert rel_l2(dB.double().cpu().numpy(), oracle.spmm_t(A_r, dC)) <= TOL[fmt]
    assert rel_l2(dv.double().cpu().numpy(), oracle.sddmm(A_r, dC, B)) <= TOL[fmt]


def test_backward_integers_bit_exact(lp):
    A = W.random_csr(100, 120, 0.08, 5, integer_values=True, duplicates=True)
    B = np.random.default_rng(1).integers(-3, 4, (120, 32)).astype(np.float64)
    dC = np.random.default_rng(2).integers(-3, 4, (100, 32)).astype(np.float64)
    for fmt in ("f64", "f32", "f16", "bf16"):
        plan = lp.Plan(A, 32, fmt, tau=1.0, want_backward=True)
        dB, dv = plan.backward(to_device(torch, dC, fmt), to_device(torch, B, fmt))
        assert np.array_equal(dB.double().cpu().numpy(), oracle.spmm_t(A, dC))
        assert np.array_equal(dv.double().cpu().numpy(), oracle.sddmm(A, dC, B))


def test_set_values_device_matches_host_packer(lp):
    A = W.random_csr(150, 150, 0.06, 9, duplicates=True, unsorted=True)
    for fmt in ("f64", "f32", "f16", "bf16"):
        kpad = {"f64": 4, "f32": 1}.get(fmt, 16)
        br = oracle.default_block_rows(fmt)
        plan = lp.Plan(A, 32, fmt, tau=1.2, want_backward=True, split_len=8)
        new = W.dense_normal(1, A.nnz, 3)[0] * 0.37
        plan.set_values(torch.as_tensor(new).cuda())
        torch.cuda.synchronize()
        ex = plan.export()
        # same structure; values = round(s_A * f64 sum of each slot) with s_A fixed at plan time
        A2 = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, new)
        raw = oracle.partition(A2, "f64", block_rows=br, k_pad=kpad, tau=1.2)
        s_old = oracle.plan_scale(A.vals, fmt)
        assert np.array_equal(ex["tile_col"], raw["tile_col"])
        assert np.array_equal(ex["csr_val"], oracle.round_to(raw["csr_val"] * s_old, fmt))
        assert np.array_equal(ex["tile_val"], oracle.round_to(raw["tile_val"] * s_old, fmt))


def test_update_values_host_then_spmm(lp):
    A = W.random_csr(120, 110, 0.07, 4)
    B = W.dense_normal(110, 24, 5)
    plan = lp.Plan(A, 24, "f64", tau=1.0, want_backward=True)
    new = W.dense_normal(1, A.nnz, 6)[0]
    plan.update_values(new)
    C = plan.spmm(torch.as_tensor(B).cuda()).cpu().numpy()
    A2 = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, new)
    assert rel_l2(C, oracle.spmm(A2, B)) <= TOL["f64"]
    dC = W.dense_normal(120, 24, 7)
    dB, dv = plan.backward(torch.as_tensor(dC).cuda(), torch.as_tensor(B).cuda())
    assert rel_l2(dB.cpu().numpy(), oracle.spmm_t(A2, dC)) <= TOL["f64"]


def test_finite_differences_gcn_1024(lp):
    # GCN layer Y = A X on a 1,024-node R-MAT graph (A + I, symmetric normalisation), FP64;
    # loss L = sum(Wt * Y); central differences with h = 1e-6
    A, X, Wt = W.gcn_graph(scale=10, samples_per_node=16, seed=21, N=32)
    plan = lp.Plan(A, 32, "f64", tau=-1.0, want_backward=True)
    Xd = torch.as_tensor(X).cuda()
    Wd = torch.as_tensor(Wt).cuda()
    vals = torch.as_tensor(A.vals).cuda()

    def loss(v, Xt):
        plan.set_values(v)
        return float((plan.spmm(Xt) * Wd).sum())

    dX, dv = plan.backward(Wd, Xd)
    dX = dX.cpu().numpy()
    dv = dv.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(6):
        j, n = int(rng.integers(0, 1024)), int(rng.integers(0, 32))
        Xp, Xm = Xd.clone(), Xd.clone()
        Xp[j, n] += h
        Xm[j, n] -= h
        fd = (loss(vals, Xp) - loss(vals, Xm)) / (2 * h)
        assert abs(fd - dX[j, n]) <= 1e-6 * max(1.0, abs(dX[j, n]))
    for k in rng.integers(0, A.nnz, 6):
        vp, vm = vals.clone(), vals.clone()
        vp[int(k)] += h
        vm[int(k)] -= h
        fd = (loss(vp, Xd) - loss(vm, Xd)) / (2 * h)
        assert abs(fd - dv[int(k)]) <= 1e-6 * max(1.0, abs(dv[int(k)]))
    # oracle gradient
    assert rel_l2(dX, oracle.spmm_t(A, Wt)) <= 1e-12
    assert rel_l2(dv, oracle.sddmm(A, Wt, X)) <= 1e-12


def test_gradcheck_fp64(lp):
    A = W.random_csr(23, 17, 0.25, 8, duplicates=True)
    plan = lp.Plan(A, 5, "f64", tau=1.0, want_backward=True)
    vals = torch.as_tensor(A.vals).cuda().requires_grad_(True)
    B = torch.as_tensor(W.dense_normal(17, 5, 9)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v, b: lp.spmm(plan, v, b), (vals, B), eps=1e-6, atol=1e-8)


def test_autograd_fp32_matches_oracle(lp):
    A, X, dY = W.gcn_graph(scale=11, samples_per_node=16, seed=5, N=64)
    A32 = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.vals.astype(np.float32))
    plan = lp.Plan(A32, 64, "f32", tau=-1.0, want_backward=True)
    vals = torch.as_tensor(A32.vals).cuda().requires_grad_(True)
    Xt = torch.as_tensor(X.astype(np.float32)).cuda().requires_grad_(True)
    Y = lp.spmm(plan, vals, Xt)
    Y.backward(torch.as_tensor(dY.astype(np.float32)).cuda())
    A_r = _rounded(A32, "f32")
    Xq = X.astype(np.float32).astype(np.float64)
    dYq = dY.astype(np.float32).astype(np.float64)
    assert rel_l2(Y.detach().double().cpu().numpy(), oracle.spmm(A_r, Xq)) <= TOL["f32"]
    assert rel_l2(Xt.grad.double().cpu().numpy(), oracle.spmm_t(A_r, dYq)) <= TOL["f32"]
    assert rel_l2(vals.grad.double().cpu().numpy(), oracle.sddmm(A_r, dYq, Xq)) <= TOL["f32"]


def test_two_forwards_one_backward_use_each_calls_values(lp):
    # weights shared by two calls on one plan: the first call's backward must see its own values
    A = W.random_csr(80, 70, 0.08, 12, duplicates=True)
    plan = lp.Plan(A, 16, "f64", tau=1.0, want_backward=True)
    v1 = torch.as_tensor(A.vals).cuda().requires_grad_(True)
    v2 = torch.as_tensor(W.dense_normal(1, A.nnz, 13)[0]).cuda().requires_grad_(True)
    B = torch.as_tensor(W.dense_normal(70, 16, 14)).cuda().requires_grad_(True)
    dC = W.dense_normal(80, 16, 15)
    Y1 = lp.spmm(plan, v1, B)
    Y2 = lp.spmm(plan, v2, B)
    Y1.backward(torch.as_tensor(dC).cuda())
    assert rel_l2(B.grad.cpu().numpy(), oracle.spmm_t(A, dC)) <= TOL["f64"]
    assert rel_l2(v1.grad.cpu().numpy(), oracle.sddmm(A, dC, B.detach().cpu().numpy())) <= TOL["f64"]
    B.grad = None
    Y2.backward(torch.as_tensor(dC).cuda())
    A2 = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, v2.detach().cpu().numpy())
    assert rel_l2(B.grad.cpu().numpy(), oracle.spmm_t(A2, dC)) <= TOL["f64"]


def test_in_place_edit_of_values_after_forward_is_refused(lp):
    A = W.random_csr(40, 30, 0.1, 16)
    plan = lp.Plan(A, 8, "f64", tau=1.0, want_backward=True)
    v = torch.as_tensor(A.vals).cuda().requires_grad_(True)
    w = v * 1.0                      # a non-leaf the caller could edit in place
    Y = lp.spmm(plan, w, torch.as_tensor(W.dense_normal(30, 8, 17)).cuda())
    with torch.no_grad():
        w.mul_(2.0)
    with pytest.raises(RuntimeError):
        Y.sum().backward()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_half_backward_keeps_small_gradients(lp, fmt):
    # dC of magnitude ~1e-9 lies below the smallest FP16 subnormal (6e-8): cast as it is, it
    # would flush to zero; scaled per column first, dB and dvals keep the 2e-3 bound
    A = W.random_csr(120, 100, 0.06, 18, duplicates=True)
    A_r = _rounded(A, fmt)
    N = 32
    B = oracle.round_to(W.dense_normal(100, N, 19), fmt)
    # binary32 values (the library's cast starts from f32), so both sides round the same numbers
    dC = (W.dense_normal(120, N, 20) * 1e-9).astype(np.float32).astype(np.float64)
    dCq, s = oracle.scale_round_columns(dC, fmt)
    dC_eff = dCq * s[None, :]
    plan = lp.Plan(A, N, fmt, tau=1.0, want_backward=True)
    # through the C ABI with the library's own scaled cast
    dC16, sd = lp.cast_scaled(torch.as_tensor(dC, dtype=torch.float32).cuda(), fmt)
    assert np.array_equal(sd.double().cpu().numpy(), s)
    dB, dv = plan.backward(dC16, to_device(torch, B, fmt), dc_scale=sd)
    torch.cuda.synchronize()
    ref_dB, ref_dv = oracle.spmm_t(A_r, dC_eff), oracle.sddmm(A_r, dC_eff, B)
    assert rel_l2(dB.double().cpu().numpy(), ref_dB) <= TOL[fmt]
    assert rel_l2(dv.double().cpu().numpy(), ref_dv) <= TOL[fmt]
    # against the unrounded problem (information: the inputs' own rounding dominates)
    err_raw = rel_l2(dv.double().cpu().numpy(), oracle.sddmm(A_r, dC, B))
    print(f"{fmt} half backward: dvals rel-L2 vs unrounded dC {err_raw:.2e}")
    assert err_raw <= 1e-2
    # the autograd function scales dC itself
    vals = torch.as_tensor(A.vals).cuda().requires_grad_(True)
    Bt = to_device(torch, B, fmt)
    Y = lp.spmm(plan, vals, Bt)
    Y.backward(torch.as_tensor(dC, dtype=torch.float32).cuda())
    assert rel_l2(vals.grad.double().cpu().numpy(), ref_dv) <= TOL[fmt]
    # scales are refused for plans without a 16-bit dtype
    p32 = lp.Plan(A, N, "f32", tau=1.0, want_backward=True)
    with pytest.raises(lp.LoopsError):
        p32.backward(torch.as_tensor(dC, dtype=torch.float32).cuda(), to_device(torch, B, "f32"), dc_scale=sd)
