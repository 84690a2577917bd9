"""GPU parity of the batched path: one persistent, graph-captured launch over many matrices of
uneven size, structure and N, against the oracle per matrix."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL, rel_l2, torch_dtype

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp(loops_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return loops_lib


@pytest.fixture(scope="module")
def small_batch():
    return W.batched_mix(count=18, seed=7, min_rows=100, max_rows=3000)


def _run(lp, mats, fmt, tau, split_len=0, scale_columns=False, seed=0):
    As = [A for A, _ in mats]
    Ns = [N for _, N in mats]
    plan = lp.BatchedPlan(As, Ns, fmt, tau=tau, split_len=split_len)
    Bs, refs, scales = [], [], []
    for m, (A, N) in enumerate(mats):
        B = W.dense_normal(A.n_cols, N, seed * 1000 + m)
        s_a = oracle.plan_scale(A.vals, fmt)
        A_r = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, oracle.round_to(A.vals * s_a, fmt) / s_a)
        if scale_columns:
            Bq, s = oracle.scale_round_columns(B, fmt)
            scales.append(torch.as_tensor(s, dtype=torch.float32).cuda())
            refs.append(oracle.spmm(A_r, Bq * s[None, :]))
        else:
            Bq = oracle.round_to(B, fmt)
            refs.append(oracle.spmm(A_r, Bq))
        Bs.append(torch.as_tensor(Bq).to(torch_dtype(torch, fmt)).cuda())
    Cs = plan.spmm(Bs, col_scales=scales if scale_columns else None)
    torch.cuda.synchronize()
    errs = [rel_l2(C.double().cpu().numpy(), r) for C, r in zip(Cs, refs)]
    return plan, Bs, Cs, refs, errs


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("tau", [math.inf, 2.0, 0.0])
def test_batched_fixed_tau(lp, small_batch, fmt, tau):
    plan, _, _, _, errs = _run(lp, small_batch, fmt, tau)
    assert max(errs) <= TOL[fmt], errs


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_batched_autotuned(lp, small_batch, fmt):
    plan, _, _, _, errs = _run(lp, small_batch, fmt, -1.0)
    assert max(errs) <= TOL[fmt], errs
    inf = plan.info()
    assert inf["count"] == len(small_batch) and inf["n_tasks"] > 0


def test_batched_graph_replay_and_pointer_change(lp, small_batch):
    fmt = "f32"
    plan, Bs, Cs, refs, errs = _run(lp, small_batch, fmt, 2.0)
    assert max(errs) <= TOL[fmt]
    # same pointers: replay only
    for C in Cs:
        C.fill_(float("nan"))
    plan.spmm(Bs, Cs)
    torch.cuda.synchronize()
    assert max(rel_l2(C.double().cpu().numpy(), r) for C, r in zip(Cs, refs)) <= TOL[fmt]
    # new buffers (different pointers, padded leading dimensions): descriptors re-uploaded
    Bs2 = []
    for B in Bs:
        buf = torch.zeros((B.shape[0], B.shape[1] + 4), dtype=B.dtype, device="cuda")
        buf[:, : B.shape[1]] = B
        Bs2.append(buf[:, : B.shape[1]])
    Cs2 = [torch.full((C.shape[0], C.shape[1] + 8), float("nan"), device="cuda")[:, : C.shape[1]] for C in Cs]
    plan.spmm(Bs2, Cs2)
    torch.cuda.synchronize()
    assert max(rel_l2(C.double().cpu().numpy(), r) for C, r in zip(Cs2, refs)) <= TOL[fmt]


def test_batched_timing_events_swapped_between_calls(lp, small_batch):
    """New timing events before every call (as a timed loop does) repoint the captured graph's
    event nodes; every call still computes the product, every event pair measures it, and
    switching the events off and on again works."""
    fmt = "f32"
    plan, Bs, Cs, refs, errs = _run(lp, small_batch, fmt, 2.0)
    assert max(errs) <= TOL[fmt]
    s = torch.cuda.current_stream()
    for rnd in range(2):
        pairs = []
        for k in range(4):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            for e in evs:
                e.record(s)
            torch.cuda.synchronize()
            plan.set_timing_events([e.cuda_event for e in evs])
            for C in Cs:
                C.fill_(float("nan"))
            plan.spmm(Bs, Cs)
            torch.cuda.synchronize()
            assert max(rel_l2(C.double().cpu().numpy(), r) for C, r in zip(Cs, refs)) <= TOL[fmt]
            pairs.append(evs)
        for evs in pairs:
            assert evs[0].elapsed_time(evs[1]) > 0.0
            assert evs[2].elapsed_time(evs[3]) >= 0.0
        plan.set_timing_events(None)
        plan.spmm(Bs, Cs)
        torch.cuda.synchronize()
        assert max(rel_l2(C.double().cpu().numpy(), r) for C, r in zip(Cs, refs)) <= TOL[fmt]


def test_batched_split_rows_and_column_scales(lp):
    mats = W.batched_mix(count=6, seed=9, min_rows=200, max_rows=1500)
    # a long row in every matrix
    out = []
    for A, N in mats:
        n = A.n_rows
        r = np.concatenate([A.row_ids(), np.full(n, n // 2)])
        c = np.concatenate([A.col_idx.astype(np.int64), np.arange(n)])
        v = np.concatenate([A.vals, np.ones(n) * 0.5])
        out.append((W.csr_from_coo(n, n, r, c, v), N))
    for fmt in ("f32", "bf16"):
        _, _, _, _, errs = _run(lp, out, fmt, 1.5, split_len=64)
        assert max(errs) <= TOL[fmt], errs
    _, _, _, _, errs = _run(lp, out, "bf16", 1.5, split_len=64, scale_columns=True)
    assert max(errs) <= TOL["bf16"], errs


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_batched_host_call_pipeline(lp, fmt):
    """The end-to-end call with host buffers (groups of matrices whose copies in, kernels and
    copies out overlap) gives the device call's product for every matrix: pinned and pageable
    host memory, padded host rows, split rows and split blocks in several groups, repeated
    calls and fresh buffers."""
    mats = W.batched_mix(count=21, seed=13, min_rows=100, max_rows=2500)

    def with_long_row(A):
        n = A.n_rows
        r = np.concatenate([A.row_ids(), np.full(n, n // 3)])
        c = np.concatenate([A.col_idx.astype(np.int64), np.arange(n)])
        v = np.concatenate([A.vals, np.ones(n) * 0.25])
        return W.csr_from_coo(n, n, r, c, v)

    out = []
    for k, (A, N) in enumerate(mats):
        if k % 4 == 1:      # sparse rows around a long one: a CSR row split into segments
            A = with_long_row(W.random_csr(3000, 3000, 8 / 3000, 100 + k))
        elif k % 4 == 3:    # dense rows around a long one: a BCSR block cut into units
            A = with_long_row(W.random_csr(300, 300, 0.1, 100 + k))
        out.append((A, N))
    plan, Bs, Cs, refs, errs = _run(lp, out, fmt, 1.5, split_len=64)
    assert max(errs) <= TOL[fmt], errs
    st = plan.stats()
    assert st["n_split_rows"] > 0 and st["n_split_blocks"] > 0, st
    def separate(pinned, pad):
        Bh, Ch, keep = [], [], []
        for B, C in zip(Bs, Cs):
            hb = torch.zeros((B.shape[0], B.shape[1] + pad), dtype=B.dtype, pin_memory=pinned)
            hb[:, : B.shape[1]] = B.cpu()
            Bh.append(hb[:, : B.shape[1]])
            hc = torch.full((C.shape[0], C.shape[1] + pad), 7.0, pin_memory=pinned)
            Ch.append(hc[:, : C.shape[1]])
            keep.append(hc)
        return Bh, Ch, keep

    def arena(pinned):
        # one host buffer for all B and one for all C, operands back to back (runs copied in
        # one piece), except matrix 5, whose C rows are padded and whose B sits after a gap
        eb = Bs[0].element_size()
        nb = sum(B.numel() for B in Bs) + 64
        nc = sum(C.shape[0] * (C.shape[1] + 4) for C in Cs)
        hb = torch.zeros(nb, dtype=Bs[0].dtype, pin_memory=pinned)
        hc = torch.full((nc,), 7.0, pin_memory=pinned)
        Bh, Ch, ob, oc = [], [], 0, 0
        for m, (B, C) in enumerate(zip(Bs, Cs)):
            if m == 5:
                ob += 64 // eb
            v = hb[ob: ob + B.numel()].view(B.shape)
            v.copy_(B.cpu())
            Bh.append(v)
            ob += B.numel()
            w = C.shape[1] + (4 if m == 5 else 0)
            Ch.append(hc[oc: oc + C.shape[0] * w].view(C.shape[0], w)[:, : C.shape[1]])
            oc += C.shape[0] * w
        return Bh, Ch, [hc]

    layouts = [("pinned", separate(True, 0)), ("pageable", separate(False, 0)), ("pinned padded", separate(True, 8)),
               ("pinned arena", arena(True)), ("pageable arena", arena(False))]
    for name, (Bh, Ch, keep) in layouts:
        plan.spmm_host(Bh, Ch)
        for m, (C, hc, r) in enumerate(zip(Cs, Ch, refs)):
            assert torch.equal(hc, C.cpu()), (name, m)     # same kernels, same order: bit for bit
            assert rel_l2(hc.double().numpy(), r) <= TOL[fmt]
        # no byte of the host buffers outside the C operands was written
        written = sum(C.numel() for C in Ch)
        assert sum(int((k == 7.0).sum()) for k in keep) >= sum(k.numel() for k in keep) - written, name
        if name.startswith("pinned padded"):
            assert all(bool((k[:, -8:] == 7.0).all()) for k in keep)
    plan.destroy()


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_batched_degenerate_matrices(lp, fmt):
    """Degenerate members of a batch, beside ordinary ones: an all-zero matrix, one without
    rows, a 1 x 1 matrix, rows empty everywhere but a few with one long (split) row, and a
    ragged rectangular one; the device call and the host call give the oracle's product."""
    n = 261
    rows = np.concatenate([np.zeros(n, np.int64), [5, 5, 100, 260]])
    cols = np.concatenate([np.arange(n), [3, 3, 7, 260]])
    vals = np.random.default_rng(2).standard_normal(rows.size)
    mats = [
        (W.csr_from_coo(40, 30, np.zeros(0), np.zeros(0), np.zeros(0)), 16),
        (W.batched_mix(count=1, seed=3, min_rows=500, max_rows=600)[0][0], 32),
        (W.csr_from_coo(0, 30, np.zeros(0), np.zeros(0), np.zeros(0)), 16),
        (W.csr_from_coo(1, 1, np.zeros(1, np.int64), np.zeros(1, np.int64), np.array([1.5])), 16),
        (W.csr_from_coo(n, n, rows, cols, vals), 48),
        (W.random_csr(97, 89, 0.1, 8), 64),
    ]
    for tau in (0.0, 2.0, math.inf):
        plan, Bs, Cs, refs, errs = _run(lp, mats, fmt, tau, split_len=32)
        assert max(errs) <= TOL[fmt], errs
        assert bool((Cs[0] == 0).all()) and tuple(Cs[2].shape) == (0, 16)
        Bh = [B.cpu().pin_memory() for B in Bs]
        Ch = [torch.full(tuple(C.shape), float("nan")).pin_memory() for C in Cs]
        plan.spmm_host(Bh, Ch)
        for m, (C, hc) in enumerate(zip(Cs, Ch)):
            assert torch.equal(hc, C.cpu()), (tau, m)
        plan.destroy()


def test_batched_rejects_unsupported_n(lp):
    A = W.random_csr(50, 50, 0.1, 1)
    with pytest.raises(lp.LoopsError):
        lp.BatchedPlan([A], [6], "f32", tau=2.0)
    with pytest.raises(lp.LoopsError):
        lp.BatchedPlan([A], [32], "f64", tau=2.0)


def test_batched_rejects_b_beyond_32bit_offsets(lp):
    """The kernels index B with 32-bit element offsets: a leading dimension that puts the last
    row of B at or past 2^31 elements is refused before anything runs."""
    import ctypes
    A = W.random_csr(64, 1 << 16, 0.001, 3)
    plan = lp.BatchedPlan([A], [32], "f32", tau=2.0)
    B = torch.zeros((A.n_cols, 32), device="cuda")
    C = torch.zeros((A.n_rows, 32), device="cuda")
    L = plan._L
    ldb_bad = ((1 << 31) // A.n_cols + 4) // 4 * 4        # 16-byte rows, n_cols x ldb > 2^31
    bp = (ctypes.c_void_p * 1)(B.data_ptr())
    cp = (ctypes.c_void_p * 1)(C.data_ptr())
    lc = (ctypes.c_int64 * 1)(32)
    st = L.loops_spmm_batched(plan._h, bp, (ctypes.c_int64 * 1)(ldb_bad), cp, lc, None, None)
    assert st == 3                                          # LOOPS_ERR_UNSUPPORTED
    assert b"32-bit" in L.loops_last_error()
    st = L.loops_spmm_batched(plan._h, bp, (ctypes.c_int64 * 1)(32), cp, lc, None, None)
    assert st == 0
    torch.cuda.synchronize()
    plan.destroy()


def test_batched_blocks_cut_into_units(lp):
    rng = np.random.default_rng(11)
    mats = []
    for m, N in enumerate((16, 32, 64)):
        n = 800
        rows = np.concatenate([np.repeat(np.arange(32, 48), 400), rng.integers(0, n, 2000)])
        cols = np.concatenate([rng.integers(0, 600, 16 * 400), rng.integers(0, n, 2000)])
        mats.append((W.csr_from_coo(n, n, rows, cols, rng.standard_normal(rows.size)), N))
    for fmt in ("f32", "bf16"):
        _, _, _, _, errs = _run(lp, mats, fmt, 0.0)
        assert max(errs) <= TOL[fmt], errs


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
@pytest.mark.parametrize("tau", [math.inf, 2.0])
def test_batched_n_not_a_power_of_two(lp, fmt, tau):
    # N values whose 16-byte vectors per row are not a power of two: lane groups are rounded
    # up and the lanes past N idle
    mats = W.batched_mix(count=16, seed=11, min_rows=200, max_rows=2500, Ns=(8, 24, 40, 48, 56, 96, 104, 120))
    plan, _, _, _, errs = _run(lp, mats, fmt, tau, seed=3)
    assert max(errs) <= TOL[fmt], errs
