"""The 128x128x64 channelised workload at full size (1,048,576 local systems,
4,227,072 unknowns, thresh-0.05 sets): sets and S~ pattern bit-exact and X~,
S~ within 1e-10 against the oracle; FP64 and FP32-mixed FGMRES(50) to 1e-8,
FP64 iteration count within 2 of the oracle's (golden file written by
tests/golden/make_c3_fgmres.py from the oracle; the inputs are regenerated
on each host, so a count off by rounding is allowed one extra iteration)."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP64, gpu_handle, gpu_results, normwise_cols_fast

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c3_oracle_fgmres.txt")


def golden_iterations():
    for line in open(GOLDEN):
        if line.startswith("iterations"):
            return int(line.split()[1])
    raise RuntimeError("no iteration count in golden file")


def test_config3_full_size():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sysd = W.config3()
    h = gpu_handle(sysd, mode="thresh", thresh=0.05)
    g = gpu_results(h)
    qptr, qidx = O.qsets("thresh", sysd.A, sysd.B, sysd.C, 0.05)
    assert np.array_equal(g["qptr"], qptr) and np.array_equal(g["qidx"], qidx)
    s = np.diff(qptr)
    assert s.min() >= 5 and s.max() <= 12
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx)
    assert normwise_cols_fast(g["xval"], x, qptr) <= TOL_FP64
    S = O.schur(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x)
    assert np.array_equal(g["s_rowptr"], S.rowptr) and np.array_equal(g["s_col"], S.col)
    assert normwise_cols_fast(g["s_val"], S.val, S.rowptr) <= TOL_FP64
    b = torch.as_tensor(sysd.b, device="cuda")
    xg, info = h.solve(b, restart=50, rtol=1e-8, maxit=3000)
    res = np.linalg.norm(sysd.full_scipy() @ xg.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert info.converged and res <= 1.05e-8
    assert abs(info.iterations - golden_iterations()) <= 2, (info.iterations, golden_iterations())
    h.close()
    h32 = gpu_handle(sysd, mode="thresh", thresh=0.05, precision=1)
    x32, info32 = h32.solve(b, restart=50, rtol=1e-8, maxit=3000)
    res32 = np.linalg.norm(sysd.full_scipy() @ x32.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert info32.converged and res32 <= 1.05e-8
    assert info32.iterations <= info.iterations * 1.25 + 2
    h32.close()
