"""Failure detection without a GPU fault: a bounded device wait that can never
be satisfied runs out, the call reports EDFA_ERR_TIMEOUT, and the CUDA context
stays usable (a normal EDFA build and solve on the same device afterwards
matches the oracle)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_handle

pytestmark = pytest.mark.gpu

EDFA_ERR_TIMEOUT = 6


def test_lost_dependency_times_out_then_solve_succeeds():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_13916_gb300 as P
    for _ in range(2):
        rc, detail, ms = P.selftest_wait_timeout()
        assert rc == EDFA_ERR_TIMEOUT, rc
        assert detail == 1          # the row whose dependency was never computed
        assert 0.0 < ms < 30000.0   # the poll budget ends the wait, in bounded time
    sysd = W.brick(6, seed=3, sigma=1.0)
    ref = O.edfa_pipeline(sysd, mode="nbr", rtol=1e-8)
    h = gpu_handle(sysd, mode="nbr")
    x, info = h.solve(torch.as_tensor(sysd.b, device="cuda"), restart=50, rtol=1e-8, maxit=500)
    assert info.converged and abs(info.iterations - ref["iters"]) <= 1
    res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert res <= 1.05e-8
    h.close()
