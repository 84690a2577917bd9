"""The performance model (Sec. 3.5, Eq. 2 and Eq. 3, restated for the GPU) choosing the split on
the GPU: plans built in model mode (LOOPS_TAU_MODEL) and the batched autotuner's per-matrix
candidate are checked against the oracle, and their choices are reported."""
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


def _cases():
    yield "block_mix_f32", W.block_mix(n=1 << 13, N=64)[0], 64, "f32"
    yield "block_mix_bf16", W.block_mix(n=1 << 13, N=64)[0], 64, "bf16"
    yield "laplacian_f64", W.laplacian_blocks(grid=64, n_blocks=64, block=8, seed=2, N=32)[0], 32, "f64"
    yield "uniform_f32", W.uniform_rows(3000, 12, 32, seed=5)[0], 32, "f32"


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_model_mode_plan_matches_oracle(lp, case):
    name, A, N, fmt = case
    B = W.dense_normal(A.n_cols, N, 9)
    A_r, Bq, s, B_eff = rounded_inputs(A, B, fmt)
    plan = lp.Plan(A, N, fmt, tau=lp.TAU_MODEL)
    inf = plan.info()
    assert inf["tau_source"] == 2
    assert math.isfinite(inf["model_gflops"]) and inf["model_gflops"] > 0
    sc = None if s is None else torch.as_tensor(s, dtype=torch.float32).cuda()
    C = plan.spmm(to_device(torch, Bq, fmt), col_scale=sc)
    torch.cuda.synchronize()
    assert rel_l2(C.double().cpu().numpy(), oracle.spmm(A_r, B_eff)) <= TOL[fmt]
    timed = lp.Plan(A, N, fmt, tau=-1.0).info()
    print(f"{name}: model tau {inf['tau']} (predicted {inf['model_gflops']:.0f} GFLOP/s), timed tau {timed['tau']}")


def test_model_mode_is_refused_for_device_builds(lp):
    A = W.uniform_rows(500, 8, 16, seed=2)[0]
    with pytest.raises(lp.LoopsError):
        lp.Plan(A, 16, "f32", tau=lp.TAU_MODEL, build_on_device=True)


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_batched_autotuner_reports_its_choice_and_matches_oracle(lp, fmt):
    mats = W.batched_mix(count=24, seed=13, min_rows=300, max_rows=6000)
    As = [A for A, _ in mats]
    Ns = [N for _, N in mats]
    plan = lp.BatchedPlan(As, Ns, fmt, tau=-1.0)
    st = plan.stats()
    assert st["tau_source"] in (1, 2)
    assert st["timed_best_gflops"] > 0
    Bs, refs = [], []
    for m, (A, N) in enumerate(mats):
        A_r, Bq, _, B_eff = rounded_inputs(A, W.dense_normal(A.n_cols, N, 70 + m), fmt, scale_columns=False)
        Bs.append(to_device(torch, Bq, fmt))
        refs.append(oracle.spmm(A_r, B_eff))
    Cs = plan.spmm(Bs)
    torch.cuda.synchronize()
    errs = [rel_l2(C.double().cpu().numpy(), r) for C, r in zip(Cs, refs)]
    assert max(errs) <= TOL[fmt], errs
    # per-matrix shapes: the dense-block matrices (index mod 3 = 2) never put a smaller share of
    # their entries in the BCSR part than the uniform ones (mod 3 = 0)
    infos = [plan.matrix_info(m) for m in range(len(mats))]
    share = [i["nnz_bcsr"] / max(i["nnz"], 1) for i in infos]
    assert min(share[2::3]) >= max(share[0::3])
    print(f"{fmt}: source {st['tau_source']}, tau {st['tau']}, B_r {st['block_rows']}, model predicted "
          f"{st['model_gflops']:.0f}, measured {st['model_measured_gflops']:.0f}, best single-threshold "
          f"{st['timed_best_gflops']:.0f} GFLOP/s; per-matrix tau "
          f"{sorted(set((i['tau'], i['block_rows']) for i in infos))}")


def test_autotuner_gives_different_structures_different_shapes(lp):
    # dense 16 x 16 blocks in half the row blocks: the autotuner splits (finite tau, BCSR blocks);
    # uniform random rows: it keeps the CSR kernel alone (tau = inf, no BCSR block)
    A_mix = W.block_mix(n=1 << 17, N=64)[0]
    A_uni = W.uniform_rows(1 << 17, 16, 64, seed=8)[0]
    for fmt in ("f32", "bf16"):
        mix = lp.Plan(A_mix, 64, fmt, tau=-1.0).info()
        uni = lp.Plan(A_uni, 64, fmt, tau=-1.0).info()
        print(f"{fmt}: block mix tau {mix['tau']} ({mix['n_row_blocks']} BCSR blocks, B_r {mix['block_rows']}, "
              f"CSR vectors per lane {mix['csr_lane_vectors']}, BCSR tile {mix['bcsr_col_tile']}), uniform tau "
              f"{uni['tau']} (CSR vectors per lane {uni['csr_lane_vectors']})")
        assert math.isfinite(mix["tau"]) and mix["n_row_blocks"] > 0
        assert uni["n_row_blocks"] == 0 and (uni["tau"] == math.inf or uni["tau"] > 1.0)
        assert mix["block_rows"] in ((8, 16) if fmt == "f32" else (16,))
        # 0: the built-in rule was kept (no timed alternative was faster)
        assert uni["csr_lane_vectors"] in (0, 1, 2)
        assert mix["bcsr_col_tile"] in ((0,) if fmt == "f32" else (0, 32, 64, 128))
        # the tuned plan is correct
        p = lp.Plan(A_mix, 64, fmt, tau=-1.0)
        B = W.dense_normal(A_mix.n_cols, 64, 3)
        A_r, Bq, s, B_eff = rounded_inputs(A_mix, B, fmt)
        sc = None if s is None else torch.as_tensor(s, dtype=torch.float32).cuda()
        C = p.spmm(to_device(torch, Bq, fmt), col_scale=sc)
        rows = np.arange(0, A_mix.n_rows, 97)
        ref = oracle.spmm_rows(A_r, B_eff, rows)
        assert rel_l2(C[torch.as_tensor(rows).cuda()].double().cpu().numpy(), ref) <= TOL[fmt]
