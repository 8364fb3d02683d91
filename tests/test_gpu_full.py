"""Parity at the benchmark size, in the benchmark's launch configuration:
the 64^3 full-tensor workload with own + neighbour-face sets (262,144 local
systems, 1,060,864 unknowns).  Sets and S~ pattern bit-exact, X~ and S~
within 1e-10 normwise, FGMRES(50) to 1e-8 within one iteration of the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP64, gpu_handle, gpu_results, normwise_cols_fast

pytestmark = pytest.mark.gpu


def test_config2_full_size_parity():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sysd = W.config2()
    h = gpu_handle(sysd, mode="nbr")
    g = gpu_results(h)
    qptr, qidx = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    assert np.array_equal(g["qptr"], qptr) and np.array_equal(g["qidx"], qidx)
    s = np.diff(qptr)
    assert s.max() == 36 and s.min() == 18
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx)
    assert normwise_cols_fast(g["xval"], x, qptr) <= TOL_FP64
    S = O.schur(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x)
    assert np.array_equal(g["s_rowptr"], S.rowptr) and np.array_equal(g["s_col"], S.col)
    assert normwise_cols_fast(g["s_val"], S.val, S.rowptr) <= TOL_FP64
    P = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=S)
    ref = O.fgmres(P, sysd.b, 50, 1e-8, 2000)
    xg, info = h.solve(torch.as_tensor(sysd.b, device="cuda"), restart=50, rtol=1e-8, maxit=2000)
    assert info.converged and abs(info.iterations - ref["iters"]) <= 1, (info.iterations, ref["iters"])
    res = np.linalg.norm(sysd.full_scipy() @ xg.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert res <= 1.05e-8
    h.close()
