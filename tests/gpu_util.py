"""Shared helpers of the GPU parity tests: run the library through its Python binding (which
calls the C ABI) and compare with the oracle on the same inputs."""
import numpy as np

import oracle

TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3, "bf16": 2e-3}


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nr = np.linalg.norm(ref)
    if nr == 0.0:
        return 0.0 if np.all(got == 0) else float("inf")
    return float(np.linalg.norm(got - ref) / nr)


def torch_dtype(torch, fmt):
    return {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[fmt]


def rounded_inputs(A, B, fmt, scale_columns=True):
    """Round the operands the way the GPU stores them: A's values after the plan scale, B
    (optionally per-column scaled for 16-bit formats). Returns (A_rounded, B_values_for_gpu,
    col_scale or None, B_effective) with A_rounded/B_effective in float64 exactly equal to the
    values the kernels multiply."""
    import workloads as W
    s_a = oracle.plan_scale(A.vals, fmt)
    a_r = oracle.round_to(A.vals * s_a, fmt) / s_a
    A_r = W.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, a_r)
    if fmt in ("f16", "bf16") and scale_columns:
        B16, s = oracle.scale_round_columns(B, fmt)
        return A_r, B16, s, B16 * s[None, :]
    Bq = oracle.round_to(B, fmt)
    return A_r, Bq, None, Bq


def to_device(torch, X, fmt, ld=None):
    t = torch.as_tensor(np.asarray(X, dtype=np.float64))
    dt = torch_dtype(torch, fmt)
    if ld is not None and ld > X.shape[1]:
        buf = torch.zeros((X.shape[0], ld), dtype=dt, device="cuda")
        buf[:, : X.shape[1]] = t.to(dt).cuda()
        return buf[:, : X.shape[1]]
    return t.to(dt).cuda().contiguous()
