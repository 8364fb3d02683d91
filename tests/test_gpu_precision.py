"""FP32-mixed form: local solves, S~, ILU(0) factors and the preconditioner
application in FP32 with FP32 accumulation; FGMRES vectors, Arnoldi, the
Hessenberg least squares and the true residual in FP64.

Measured against the FP64 oracle on the same inputs: X~ and S~ normwise per
column/row (FP32 rounding amplified by the conditioning of the restricted
blocks), and the outer solve, which must still reach the FP64 stopping rule
||b - A x|| / ||b|| <= 1e-8 with an iteration count close to the FP64 one."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP32, gpu_handle, gpu_results, normwise_cols_fast

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def full_tensor(n, seed=11):
    s = W.Stream(seed)
    Ne = int(np.prod(n))
    m = np.exp(2.0 * s.normal(Ne))
    q = s.normal(4 * Ne).reshape(Ne, 4)
    sysd = W.assemble(*n, W.rotated_K(m, 0.1, q))
    sysd.extra["qmode"] = "nbr"
    return sysd


CASES = {
    "full_tensor_12x10x8": (lambda: full_tensor((12, 10, 8)), "nbr"),
    "c3_small": (lambda: W.config3(32, 24, 8), "thresh"),
    "c5_small": (lambda: W.config5(12), "crow"),
}


@pytest.mark.parametrize("case", list(CASES))
def test_fp32_mixed_against_fp64_oracle(case):
    torch = _torch()
    make, mode = CASES[case]
    sysd = make()
    ref = O.edfa_pipeline(sysd, mode=mode, solve=True)
    h = gpu_handle(sysd, mode=mode, precision=1)
    g = gpu_results(h)
    assert np.array_equal(g["qidx"], ref["qidx"])
    ex = normwise_cols_fast(g["xval"].astype(np.float64), ref["xval"], ref["qptr"])
    es = normwise_cols_fast(g["s_val"].astype(np.float64), ref["S"].val, ref["S"].rowptr)
    assert np.array_equal(g["s_col"], ref["S"].col)
    print(f"\n{case}: FP32 X~ normwise error {ex:.2e}, S~ normwise error {es:.2e}")
    assert ex <= TOL_FP32 and es <= TOL_FP32
    x, info = h.solve(torch.as_tensor(sysd.b, device="cuda"), restart=50, rtol=1e-8, maxit=3000)
    res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    print(f"{case}: FP32-mixed iterations {info.iterations} (FP64 oracle {ref['iters']}), true residual {res:.2e}")
    assert info.converged and res <= 1.05e-8
    assert info.iterations <= ref["iters"] * 1.25 + 2
    h.close()
