"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs, element by element. Tolerances are the stated rel-L2 bounds (f64 1e-12, f32 1e-5,
f16/bf16 2e-3 against the oracle on the same rounded inputs); small-integer inputs must match
bit for bit in every format, and the plan's device arrays must export to exactly the oracle's
partition."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, rounded_inputs, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp(loops_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return loops_lib


FMTS = ["f64", "f32", "f16", "bf16"]


def run_case(lp, A, B, fmt, tau, N=None, ld_pad=0, split_len=0, block_rows=0, scale_columns=True):
    N = B.shape[1]
    A_r, Bg, s, B_eff = rounded_inputs(A, B, fmt, scale_columns)
    plan = lp.Plan(A, N, fmt, tau=tau, split_len=split_len, block_rows=block_rows)
    Bd = to_device(torch, Bg, fmt, ld=N + ld_pad if ld_pad else None)
    cs = torch.as_tensor(s, dtype=torch.float32).cuda() if s is not None else None
    C = plan.spmm(Bd, col_scale=cs)
    torch.cuda.synchronize()
    plan.check()
    ref = oracle.spmm(A_r, B_eff)
    return C.double().cpu().numpy(), ref, plan


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("tau", [0.0, 1.5, math.inf])
@pytest.mark.parametrize("N", [1, 8, 24, 32, 64, 72, 128, 256])
def test_random_matrix(lp, fmt, tau, N):
    A = W.random_csr(203, 157, 0.06, N + 7, duplicates=True, unsorted=True, explicit_zeros=True)
    B = W.dense_normal(157, N, N)
    C, ref, _ = run_case(lp, A, B, fmt, tau)
    assert rel_l2(C, ref) <= TOL[fmt]


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("tau", [0.0, 2.0, math.inf])
def test_small_integers_bit_exact(lp, fmt, tau):
    # every product and partial sum is a small integer: exact in f16/bf16 inputs with f32 or
    # f64 accumulation, whatever the order
    A = W.random_csr(150, 140, 0.1, 3, integer_values=True, duplicates=True, unsorted=True)
    B = np.random.default_rng(4).integers(-4, 5, size=(140, 64)).astype(np.float64)
    C, ref, _ = run_case(lp, A, B, fmt, tau, scale_columns=False)
    assert np.array_equal(C, ref)


@pytest.mark.parametrize("fmt", FMTS)
def test_export_matches_oracle_partition(lp, fmt):
    A = W.random_csr(301, 220, 0.05, 11, duplicates=True, unsorted=True, explicit_zeros=True)
    kpad = {"f64": 4, "f32": 1, "f16": 16, "bf16": 16}[fmt]
    for tau in (0.0, 1.3, math.inf):
        plan = lp.Plan(A, 32, fmt, tau=tau, split_len=4)   # tiny split_len: rows become segments
        ex = plan.export()
        ora = oracle.partition(A, fmt, k_pad=kpad, tau=tau)
        for k in ("csr_rows", "csr_ptr", "csr_col", "rb_ids", "rb_ptr", "tile_col"):
            assert np.array_equal(ex[k], ora[k]), k
        assert np.array_equal(ex["csr_val"].view(np.uint64), ora["csr_val"].view(np.uint64))
        assert np.array_equal(ex["tile_val"].view(np.uint64), ora["tile_val"].view(np.uint64))


@pytest.mark.parametrize("fmt", FMTS)
def test_closed_forms_identity_permutation(lp, fmt):
    n, N = 333, 40
    B = W.dense_normal(n, N, 5)
    perm = np.random.default_rng(1).permutation(n)
    for tau in (0.0, math.inf):
        P = W.csr_from_coo(n, n, np.arange(n), perm, np.ones(n))
        C, ref, _ = run_case(lp, P, B, fmt, tau, scale_columns=False)
        assert np.array_equal(C, ref)        # one product by 1.0 per entry: exact
        I = W.csr_from_coo(n, n, np.arange(n), np.arange(n), np.ones(n))
        C, ref, _ = run_case(lp, I, B, fmt, tau, scale_columns=False)
        assert np.array_equal(C, ref)


@pytest.mark.parametrize("fmt", FMTS)
def test_edge_cases(lp, fmt):
    tol = TOL[fmt]
    # empty rows everywhere but a few; ragged last block; a dense row of length n (split)
    n = 261
    rows = np.concatenate([np.zeros(n, np.int64), [5, 5, 100, 260]])
    cols = np.concatenate([np.arange(n), [3, 3, 7, 260]])
    vals = np.random.default_rng(2).standard_normal(rows.size)
    A = W.csr_from_coo(n, n, rows, cols, vals)
    B = W.dense_normal(n, 48, 9)
    for tau in (0.0, 1.0, math.inf):
        C, ref, plan = run_case(lp, A, B, fmt, tau, split_len=32)
        assert rel_l2(C, ref) <= tol
        assert plan.info()["n_split_rows"] >= (1 if tau == math.inf else 0)
    # padded leading dimensions
    A = W.random_csr(97, 89, 0.1, 8)
    B = W.dense_normal(89, 32, 3)
    C, ref, _ = run_case(lp, A, B, fmt, 1.0, ld_pad=8)
    assert rel_l2(C, ref) <= tol
    # an all-zero matrix and an empty one
    Z = W.csr_from_coo(40, 30, np.zeros(0), np.zeros(0), np.zeros(0))
    C, ref, _ = run_case(lp, Z, W.dense_normal(30, 16, 1), fmt, 2.0)
    assert np.all(C == 0.0)
    E = W.csr_from_coo(0, 30, np.zeros(0), np.zeros(0), np.zeros(0))
    plan = lp.Plan(E, 16, fmt)
    out = plan.spmm(to_device(torch, W.dense_normal(30, 16, 1), fmt if fmt != "f16" else "f16"))
    assert out.shape == (0, 16)


def test_cast_scaled_bit_exact(lp):
    X = W.dense_normal(1000, 72, 4) * np.logspace(-3, 3, 72)[None, :]
    X[:, 5] = 0.0
    X32 = X.astype(np.float32).astype(np.float64)
    for fmt in ("f16", "bf16"):
        Y, s = lp.cast_scaled(torch.as_tensor(X32, dtype=torch.float32).cuda(), fmt)
        ref_y, ref_s = oracle.scale_round_columns(X32, fmt)
        assert np.array_equal(s.double().cpu().numpy(), ref_s)
        assert np.array_equal(Y.double().cpu().numpy(), ref_y)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_error_vs_unrounded_fp64_reported(lp, fmt):
    # information: the error of the 16-bit path against the unrounded f64 problem
    A = W.random_csr(400, 400, 0.03, 12)
    B = W.dense_normal(400, 64, 13)
    C, ref, _ = run_case(lp, A, B, fmt, 1.5)
    err_rounded = rel_l2(C, ref)
    err_exact = rel_l2(C, oracle.spmm(A, B))
    assert err_rounded <= TOL[fmt]
    assert err_exact <= {"f16": 2e-3, "bf16": 1e-2}[fmt]
    print(f"{fmt}: rel-L2 vs oracle(rounded inputs) {err_rounded:.3e}, vs f64 inputs {err_exact:.3e}")


@pytest.mark.parametrize("fmt", FMTS)
def test_autotuned_plan_parity(lp, fmt):
    A, B = W.laplacian_blocks(grid=64, n_blocks=128, block=8, seed=3, N=32)
    C, ref, plan = run_case(lp, A, B, fmt, -1.0)
    assert rel_l2(C, ref) <= TOL[fmt]
    assert plan.info()["tau"] >= 0.0


def test_spmm_host_end_to_end(lp):
    A, B = W.uniform_rows(2000, 10, 32, seed=1)
    plan = lp.Plan(A, 32, "f32", tau=2.0)
    Bh = torch.as_tensor(B.astype(np.float32)).pin_memory()
    Ch = torch.empty((2000, 32), dtype=torch.float32).pin_memory()
    plan.spmm_host(Bh, Ch)
    ref = oracle.spmm(W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, oracle.round_to(A.vals, "f32")),
                      B.astype(np.float32).astype(np.float64))
    assert rel_l2(Ch.double().numpy(), ref) <= TOL["f32"]


def test_contiguous_paper_split(lp):
    A = W.random_csr(300, 300, 0.05, 17)
    B = W.dense_normal(300, 32, 18)
    for rb in (0, 100, 300):
        A_r, Bg, _, B_eff = rounded_inputs(A, B, "f64")
        plan = lp.Plan(A, 32, "f64", contiguous_split=True, r_boundary=rb)
        C = plan.spmm(to_device(torch, Bg, "f64")).cpu().numpy()
        assert rel_l2(C, oracle.spmm(A_r, B_eff)) <= TOL["f64"]


@pytest.mark.parametrize("fmt", FMTS)
def test_blocks_cut_into_units(lp, fmt):
    # a row block whose rows touch ~700 distinct columns: more tiles than one work unit takes,
    # so the block is cut into units whose partial sums are added in order
    n = 1000
    rng = np.random.default_rng(3)
    rows = np.concatenate([np.repeat(np.arange(16, 32), 500), rng.integers(0, n, 3000)])
    cols = np.concatenate([rng.integers(0, 700, 16 * 500), rng.integers(0, n, 3000)])
    A = W.csr_from_coo(n, n, rows, cols, rng.standard_normal(rows.size))
    B = W.dense_normal(n, 40, 4)
    for tau in (0.0, 1.5):
        C, ref, plan = run_case(lp, A, B, fmt, tau)
        assert rel_l2(C, ref) <= TOL[fmt]
        assert plan.info()["n_tiles"] > 256


def test_spmm_host_async_pipeline(lp):
    A, _ = W.uniform_rows(3000, 12, 16, seed=2)
    plan = lp.Plan(A, 16, "f64", tau=2.0)
    Bs = [torch.as_tensor(W.dense_normal(3000, 16, 30 + k)).pin_memory() for k in range(5)]
    Cs = [torch.full((3000, 16), float("nan"), dtype=torch.float64).pin_memory() for _ in range(5)]
    for B, C in zip(Bs, Cs):
        plan.spmm_host_async(B, C)
    plan.host_flush()
    torch.cuda.current_stream().synchronize()
    for B, C in zip(Bs, Cs):
        assert rel_l2(C.numpy(), oracle.spmm(A, B.numpy())) <= TOL["f64"]
    # a flush with no pipelined call before it is a no-op; one C buffer reused by every call
    # ends with the last call's result
    fresh = lp.Plan(A, 16, "f64", tau=2.0)
    fresh.host_flush()
    C1 = torch.full((3000, 16), float("nan"), dtype=torch.float64).pin_memory()
    for B in Bs:
        fresh.spmm_host_async(B, C1)
        fresh.host_flush()
        torch.cuda.current_stream().synchronize()
        assert rel_l2(C1.numpy(), oracle.spmm(A, B.numpy())) <= TOL["f64"]


@pytest.mark.parametrize("fmt", ["f64", "bf16"])
def test_paper_mode_boundary_from_eq1(lp, fmt):
    # contiguous split with r_b derived from Eq. 1 (timed pure-CSR and pure-BCSR throughputs)
    A, B = W.laplacian_blocks(grid=64, n_blocks=128, block=8, seed=5, N=32)
    A_r, Bg, s, B_eff = rounded_inputs(A, B, fmt)
    plan = lp.Plan(A, 32, fmt, contiguous_split=True, r_boundary=-1)
    info = plan.info()
    assert 0 <= info["r_boundary"] <= A.n_rows
    cs = torch.as_tensor(s, dtype=torch.float32).cuda() if s is not None else None
    C = plan.spmm(to_device(torch, Bg, fmt), col_scale=cs).double().cpu().numpy()
    assert rel_l2(C, oracle.spmm(A_r, B_eff)) <= TOL[fmt]
    # the split is the contiguous one at that boundary (rounded up to B_r)
    ex = plan.export()
    ora = oracle.partition(A, fmt, k_pad={"f64": 4}.get(fmt, 16), contiguous=True, r_boundary=info["r_boundary"])
    assert np.array_equal(ex["rb_ids"], ora["rb_ids"]) and np.array_equal(ex["csr_rows"], ora["csr_rows"])


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("tile_min", [2, 3])
def test_tile_level_split(lp, fmt, tile_min):
    # sparse tiles of BCSR blocks move to the CSR part, which adds them after the BCSR part
    kpad = {"f64": 4, "f32": 1, "f16": 16, "bf16": 16}[fmt]
    A, B = W.laplacian_blocks(grid=64, n_blocks=96, block=8, seed=9, N=40)
    R = W.random_csr(301, 220, 0.05, 11, duplicates=True, unsorted=True, explicit_zeros=True)
    for M, Bm in ((A, B), (R, W.dense_normal(220, 40, 3))):
        for tau in (0.0, 1.5):
            C, ref, plan = run_case(lp, M, Bm, fmt, tau, split_len=8)
            assert rel_l2(C, ref) <= TOL[fmt]
            plan2 = lp.Plan(M, 40, fmt, tau=tau, tile_min=tile_min, split_len=8)
            assert plan2.info()["tile_min"] == tile_min
            A_r, Bg, s, B_eff = rounded_inputs(M, Bm, fmt)
            cs = torch.as_tensor(s, dtype=torch.float32).cuda() if s is not None else None
            C2 = plan2.spmm(to_device(torch, Bg, fmt), col_scale=cs).double().cpu().numpy()
            assert rel_l2(C2, ref) <= TOL[fmt]
            ex = plan2.export()
            ora = oracle.partition(M, fmt, k_pad=kpad, tau=tau, tile_min=tile_min)
            for k in ("csr_rows", "csr_ptr", "csr_col", "rb_ids", "rb_ptr", "tile_col"):
                assert np.array_equal(ex[k], ora[k]), k
            assert np.array_equal(ex["tile_val"].view(np.uint64), ora["tile_val"].view(np.uint64))


def test_tile_level_split_integers_bit_exact(lp):
    A = W.random_csr(150, 140, 0.1, 3, integer_values=True, duplicates=True, unsorted=True)
    B = np.random.default_rng(4).integers(-4, 5, size=(140, 64)).astype(np.float64)
    for fmt in FMTS:
        plan = lp.Plan(A, 64, fmt, tau=0.0, tile_min=2)
        C = plan.spmm(to_device(torch, B, fmt)).double().cpu().numpy()
        assert np.array_equal(C, oracle.spmm(A, B))
