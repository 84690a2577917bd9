"""GPU tests of the device-side plan build (loops_plan_device): the conversion of Algorithm 1
run on the GPU must give the host builder's plan bit for bit -- the same canonical partition
(export), the same counts, the same stored values and therefore the same C -- and, through
that, the oracle's partition and product. Cases cover every dtype, split thresholds, the
contiguous Eq. 1 split, the tile-level split, long rows (segments), large blocks (units),
duplicates and unsorted columns, empty rows and matrices, the backward plan and value
refreshes, and invalid input (rejected before any packing kernel runs)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, rounded_inputs, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FMTS = ["f64", "f32", "f16", "bf16"]
COUNT_KEYS = ("n_csr_rows", "nnz_csr", "n_row_blocks", "n_tiles", "nnz_bcsr", "n_split_rows", "n_segments",
              "n_subnormal_vals", "scale", "tau", "tile_min", "block_rows", "k_pad")


@pytest.fixture(scope="module")
def lp(loops_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return loops_lib


def _hub_matrix(seed=3, n=700):
    # rows with long runs (split into segments), dense blocks (> 256 tiles: cut into units),
    # duplicates, unsorted columns and empty rows
    rng = np.random.default_rng(seed)
    rows = np.concatenate([np.repeat(np.arange(16, 32), 420), np.full(2000, 100), rng.integers(0, n, 3000),
                           np.repeat(np.arange(48, 56), 40)])
    cols = np.concatenate([rng.integers(0, 650, 16 * 420), rng.integers(0, n, 2000), rng.integers(0, n, 3000),
                           np.tile(np.arange(200, 240), 8)])
    keep = (rows < 600) | (rows > 640)  # rows 600..640 stay empty
    vals = rng.standard_normal(rows.size)
    vals[::97] = 0.0  # explicit zeros are stored entries
    return W.csr_from_coo(n, n, rows[keep], cols[keep], vals[keep])


def _cases():
    return {
        "random_dup": W.random_csr(300, 260, 0.03, 2, duplicates=True, unsorted=True),
        "hub": _hub_matrix(),
        "laplacian": W.laplacian_blocks(grid=48, n_blocks=60, block=8, seed=2, N=8)[0],
        "rect_tail": W.random_csr(203, 77, 0.08, 4),  # ragged last row block, few columns
    }


def _same_partition(a, b):
    for k in ("csr_rows", "csr_ptr", "csr_col", "rb_ids", "rb_ptr", "tile_col"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    for k in ("csr_val", "tile_val"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=True), k
    assert a["scale"] == b["scale"]


def _same_counts(pa, pb):
    ia, ib = pa.info(), pb.info()
    for k in COUNT_KEYS:
        assert ia[k] == ib[k], (k, ia[k], ib[k])


def _spmm_both(lp, ph, pd, A, fmt, N, seed=0):
    B = W.dense_normal(A.n_cols, N, seed)
    A_r, Bg, s, B_eff = rounded_inputs(A, B, fmt)
    cs = torch.as_tensor(s, dtype=torch.float32).cuda() if s is not None else None
    Bd = to_device(torch, Bg, fmt)
    Ch = ph.spmm(Bd, col_scale=cs).cpu().numpy()
    Cd = pd.spmm(Bd, col_scale=cs).cpu().numpy()
    return Ch, Cd, oracle.spmm(A_r, B_eff)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("tau", [math.inf, 2.0, 1.25, 0.0])
@pytest.mark.parametrize("name", ["random_dup", "hub", "laplacian", "rect_tail"])
def test_device_build_equals_host_build(lp, fmt, tau, name):
    A = _cases()[name]
    N = 24
    ph = lp.Plan(A, N, fmt, tau=tau, split_len=64)
    pd = lp.Plan(A, N, fmt, tau=tau, split_len=64, build_on_device=True)
    _same_partition(ph.export(), pd.export())
    _same_counts(ph, pd)
    Ch, Cd, ref = _spmm_both(lp, ph, pd, A, fmt, N)
    assert np.array_equal(Ch, Cd)
    assert rel_l2(Cd, ref) <= TOL[fmt]


@pytest.mark.parametrize("fmt", FMTS)
def test_device_build_matches_oracle_partition(lp, fmt):
    A = _cases()["laplacian"]
    br = 8 if fmt == "f64" else 16
    kpad = {"f64": 4, "f32": 1, "f16": 16, "bf16": 16}[fmt]
    pd = lp.Plan(A, 16, fmt, tau=2.0, build_on_device=True)
    part = oracle.partition(A, fmt, block_rows=br, k_pad=kpad, tau=2.0)
    ex = pd.export()
    assert list(ex["rb_ids"]) == list(part["rb_ids"]) and list(ex["tile_col"]) == list(part["tile_col"])
    assert np.array_equal(np.asarray(ex["tile_val"]).reshape(-1, br), part["tile_val"])
    assert list(ex["csr_rows"]) == list(part["csr_rows"]) and np.array_equal(ex["csr_val"], part["csr_val"])


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("tile_min", [2, 3])
def test_device_build_tile_level_split(lp, fmt, tile_min):
    for name in ("laplacian", "hub"):
        A = _cases()[name]
        ph = lp.Plan(A, 16, fmt, tau=1.5, tile_min=tile_min)
        pd = lp.Plan(A, 16, fmt, tau=1.5, tile_min=tile_min, build_on_device=True)
        _same_partition(ph.export(), pd.export())
        _same_counts(ph, pd)
        Ch, Cd, ref = _spmm_both(lp, ph, pd, A, fmt, 16, seed=1)
        assert np.array_equal(Ch, Cd)
        assert rel_l2(Cd, ref) <= TOL[fmt]


@pytest.mark.parametrize("fmt", ["f64", "bf16"])
def test_device_build_contiguous_split(lp, fmt):
    A = _cases()["hub"]
    for rb in (0, 37, 300, A.n_rows):
        ph = lp.Plan(A, 16, fmt, contiguous_split=True, r_boundary=rb)
        pd = lp.Plan(A, 16, fmt, contiguous_split=True, r_boundary=rb, build_on_device=True)
        _same_partition(ph.export(), pd.export())
        _same_counts(ph, pd)
    # Eq. 1 boundary derived by timing the device-built pure plans: any boundary is valid
    pd = lp.Plan(A, 16, fmt, contiguous_split=True, r_boundary=-1, build_on_device=True)
    assert 0 <= pd.info()["r_boundary"] <= A.n_rows
    B = W.dense_normal(A.n_cols, 16, 3)
    A_r, Bg, s, B_eff = rounded_inputs(A, B, fmt)
    cs = torch.as_tensor(s, dtype=torch.float32).cuda() if s is not None else None
    C = pd.spmm(to_device(torch, Bg, fmt), col_scale=cs).double().cpu().numpy()
    assert rel_l2(C, oracle.spmm(A_r, B_eff)) <= TOL[fmt]


@pytest.mark.parametrize("fmt", FMTS)
def test_device_build_autotuned(lp, fmt):
    A = _cases()["hub"]
    pd = lp.Plan(A, 32, fmt, tau=-1.0, build_on_device=True)
    B = W.dense_normal(A.n_cols, 32, 5)
    A_r, Bg, s, B_eff = rounded_inputs(A, B, fmt)
    cs = torch.as_tensor(s, dtype=torch.float32).cuda() if s is not None else None
    C = pd.spmm(to_device(torch, Bg, fmt), col_scale=cs).double().cpu().numpy()
    assert rel_l2(C, oracle.spmm(A_r, B_eff)) <= TOL[fmt]
    # the chosen threshold rebuilt on the host gives the same plan
    inf = pd.info()
    ph = lp.Plan(A, 32, fmt, tau=inf["tau"], tile_min=inf["tile_min"])
    _same_partition(ph.export(), pd.export())


def test_device_build_from_cuda_tensors_and_f32_values(lp):
    A = _cases()["random_dup"]
    for vals in (A.vals, A.vals.astype(np.float32)):
        Ad = W.CSR(A.n_rows, A.n_cols, torch.as_tensor(A.row_ptr).cuda(), torch.as_tensor(A.col_idx).cuda(),
                   torch.as_tensor(vals).cuda())
        pd = lp.Plan(Ad, 8, "f32", tau=1.5, build_on_device=True)
        ph = lp.Plan(W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, vals), 8, "f32", tau=1.5)
        _same_partition(ph.export(), pd.export())


@pytest.mark.parametrize("fmt", FMTS)
def test_device_build_edge_cases(lp, fmt):
    cases = [
        W.CSR(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)),       # no rows
        W.CSR(7, 9, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0)),       # no entries
        W.csr_from_coo(1, 3000, np.zeros(2500, np.int64), np.arange(2500), np.ones(2500)),  # one long row
        W.csr_from_coo(19, 1, np.arange(19), np.zeros(19, np.int64), np.arange(19.0) - 9),  # one column
    ]
    for A in cases:
        for tau in (math.inf, 0.0):
            ph = lp.Plan(A, 8, fmt, tau=tau, split_len=100)
            pd = lp.Plan(A, 8, fmt, tau=tau, split_len=100, build_on_device=True)
            _same_partition(ph.export(), pd.export())
            _same_counts(ph, pd)
            if A.n_rows and A.n_cols:
                Ch, Cd, ref = _spmm_both(lp, ph, pd, A, fmt, 8)
                assert np.array_equal(Ch, Cd)
                assert rel_l2(Cd, ref) <= TOL[fmt]


@pytest.mark.parametrize("fmt", ["f64", "f32", "bf16"])
def test_device_build_backward_and_values(lp, fmt):
    A = _cases()["hub"]
    N = 16
    ph = lp.Plan(A, N, fmt, tau=1.5, want_backward=True)
    pd = lp.Plan(A, N, fmt, tau=1.5, want_backward=True, build_on_device=True)
    _same_counts(ph, pd)
    rng = np.random.default_rng(7)
    dC = rng.standard_normal((A.n_rows, N))
    B = rng.standard_normal((A.n_cols, N))
    A_r, Bg, _, B_eff = rounded_inputs(A, B, fmt, scale_columns=False)
    _, dCg, _, dC_eff = rounded_inputs(A, dC, fmt, scale_columns=False)
    outs = []
    for p in (ph, pd):
        dB, dv = p.backward(to_device(torch, dCg, fmt), to_device(torch, Bg, fmt))
        outs.append((dB.cpu().numpy(), dv.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert rel_l2(outs[1][0], oracle.spmm_t(A_r, dC_eff)) <= TOL[fmt]
    assert rel_l2(outs[1][1], oracle.sddmm(A, dC_eff, B_eff)) <= TOL[fmt]
    # value refresh from the device (set_values) and from the host (update_values) agree with
    # a plan built from the new values (a permutation keeps max|a|, so the kept plan scale
    # s_A is also the new plan's)
    v2 = rng.permutation(A.vals)
    A2 = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, v2)
    fresh = lp.Plan(A2, N, fmt, tau=1.5, want_backward=True)
    pd.set_values(torch.as_tensor(v2).cuda())
    torch.cuda.synchronize()
    _same_partition(fresh.export(), pd.export())
    pd2 = lp.Plan(A, N, fmt, tau=1.5, build_on_device=True)  # no backward: device maps all the same
    pd2.update_values(v2)
    _same_partition(fresh.export(), pd2.export())


def test_device_build_rejects_invalid_csr_like_host(lp):
    good = W.random_csr(40, 30, 0.1, 1)
    assert good.row_ptr[9] >= 1
    dec = good.row_ptr.copy()
    dec[10] = dec[9] - 1  # row 9 ends before it starts (reads stay inside the arrays)
    start = good.row_ptr.copy()
    start[0] = 1
    bad = {
        "row_ptr_start": (start, good.col_idx),
        "row_ptr_decreasing": (dec, good.col_idx),
        "col_out_of_range": (good.row_ptr, np.where(np.arange(good.nnz) == 5, 30, good.col_idx).astype(np.int32)),
        "col_negative": (good.row_ptr, np.where(np.arange(good.nnz) == 7, -1, good.col_idx).astype(np.int32)),
    }
    for name, (rp, ci) in bad.items():
        A = W.CSR(40, 30, np.asarray(rp, np.int64), np.asarray(ci, np.int32), good.vals)
        msgs = []
        for dev in (False, True):
            with pytest.raises(lp.LoopsError) as ei:
                lp.Plan(A, 8, "f64", tau=2.0, build_on_device=dev)
            msgs.append(str(ei.value))
        assert msgs[0] == msgs[1], (name, msgs)
    # the context is still usable afterwards
    lp.Plan(good, 8, "f64", tau=2.0, build_on_device=True)


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
@pytest.mark.parametrize("tau", [math.inf, 2.0, 0.0, -1.0])
def test_batched_device_build_equals_host_build(lp, fmt, tau):
    mats = W.batched_mix(count=12, seed=9, min_rows=100, max_rows=4000)
    As = [A for A, _ in mats]
    Ns = [N for _, N in mats]
    bh = lp.BatchedPlan(As, Ns, fmt, tau=tau)
    bd = lp.BatchedPlan(As, Ns, fmt, tau=tau, build_on_device=True)
    dt = torch.float32 if fmt == "f32" else torch.bfloat16
    g = torch.Generator(device="cuda").manual_seed(3)
    Bs = [torch.randn((A.n_cols, N), device="cuda", generator=g).to(dt) for A, N in mats]
    if tau >= 0:  # fixed split: the same sub-plans and task list, so the same outputs bit for bit
        assert bh.info() == bd.info()
        for Ch, Cd in zip(bh.spmm(Bs), bd.spmm(Bs)):
            assert torch.equal(Ch, Cd)
    else:  # autotuned: each may time a different winner; both agree with the oracle
        for (A, N), B, C in zip(mats, Bs, bd.spmm(Bs)):
            s_a = oracle.plan_scale(A.vals, fmt)
            A_r = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, oracle.round_to(A.vals * s_a, fmt) / s_a)
            ref = oracle.spmm(A_r, B.double().cpu().numpy())
            assert rel_l2(C.double().cpu().numpy(), ref) <= TOL[fmt]


def test_batched_device_build_names_the_invalid_matrix(lp):
    mats = W.batched_mix(count=3, seed=9, min_rows=100, max_rows=400)
    As = [A for A, _ in mats]
    bad = As[1]
    ci = bad.col_idx.copy()
    ci[3] = bad.n_cols  # out of range (only compared, never used as an index)
    As[1] = W.CSR(bad.n_rows, bad.n_cols, bad.row_ptr, ci, bad.vals)
    with pytest.raises(lp.LoopsError) as ei:
        lp.BatchedPlan(As, [N for _, N in mats], "f32", tau=2.0, build_on_device=True)
    assert "matrix 1" in str(ei.value) and "column index out of range at entry 3" in str(ei.value)


def _random_case(seed):
    """A seeded random matrix and plan options: uneven shapes, clustered rows (dense column
    runs, so that some row blocks pass every threshold), long rows, empty row blocks,
    duplicates, unsorted columns and explicit zeros."""
    rng = np.random.default_rng(1000 + seed)
    n_rows, n_cols = int(rng.integers(1, 2500)), int(rng.integers(1, 2500))
    A = W.random_csr(n_rows, n_cols, float(rng.choice([0.0005, 0.004, 0.02])), seed,
                     duplicates=bool(rng.integers(0, 2)), unsorted=bool(rng.integers(0, 2)),
                     explicit_zeros=bool(rng.integers(0, 2)))
    r, c, v = [A.row_ids()], [A.col_idx.astype(np.int64)], [A.vals]
    for _ in range(int(rng.integers(0, 4))):  # dense patches and a long row
        r0, c0 = int(rng.integers(0, n_rows)), int(rng.integers(0, n_cols))
        h, w = int(rng.integers(1, 40)), int(rng.integers(1, 300))
        rr, cc = np.meshgrid(np.arange(r0, min(r0 + h, n_rows)), np.arange(c0, min(c0 + w, n_cols)), indexing="ij")
        r.append(rr.ravel()); c.append(cc.ravel()); v.append(rng.standard_normal(rr.size))
    A = W.csr_from_coo(n_rows, n_cols, np.concatenate(r), np.concatenate(c), np.concatenate(v),
                       sort_cols=bool(rng.integers(0, 2)))
    fmt = str(rng.choice(FMTS))
    opts = {"tau": float(rng.choice([0.0, 0.5, 1.0, 1.25, 2.0, 3.0, math.inf])),
            "split_len": int(rng.choice([0, 16, 64])),
            "tile_min": int(rng.choice([0, 0, 2, 3]))}
    if rng.integers(0, 5) == 0:
        opts = {"contiguous_split": True, "r_boundary": int(rng.integers(0, n_rows + 1)),
                "split_len": opts["split_len"]}
    return A, fmt, opts


@pytest.mark.parametrize("seed", range(40))
def test_device_build_random_cases_equal_host_build(lp, seed):
    A, fmt, opts = _random_case(seed)
    N = 8 if fmt in ("f16", "bf16") else 4
    ph = lp.Plan(A, N, fmt, **opts)
    pd = lp.Plan(A, N, fmt, build_on_device=True, **opts)
    _same_partition(ph.export(), pd.export())
    _same_counts(ph, pd)
    if A.nnz:
        Ch, Cd, ref = _spmm_both(lp, ph, pd, A, fmt, N, seed=seed)
        assert np.array_equal(Ch, Cd)
        assert rel_l2(Cd, ref) <= TOL[fmt]
