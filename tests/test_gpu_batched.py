"""Batched form: many independent systems of uneven size held block-diagonally
in one handle (one launch per setup kernel over all systems) and solved by one
FGMRES per system in lock step, with the restart cycle replayed as a CUDA
graph.  Checked per system against the oracle: sets bit-exact, X~/S~ within
1e-10 (FP64) / 1e-5 (FP32), every system converged to 1e-8 on its own
residual, iteration counts within 1 of the oracle's own per-system FGMRES
(FP64) and close to it (FP32-mixed)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP32, TOL_FP64, gpu_handle, gpu_results, normwise_cols_fast

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def batch(nsys=9, lo=5, hi=12, seed=7):
    s = W.Stream(seed)
    sizes = (lo + np.floor((hi - lo + 1) * s.uniform(nsys))).astype(int)
    systems = [W.config4_system(100 + i, int(n)) for i, n in enumerate(sizes)]
    big, fo, co = W.concat(systems)
    return systems, big, fo, co


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_setup_and_solve(precision):
    torch = _torch()
    systems, big, fo, co = batch()
    ref = O.edfa_pipeline(big, mode="nbr", solve=False)
    h = gpu_handle(big, mode="nbr", precision=precision)
    g = gpu_results(h)
    assert np.array_equal(g["qptr"], ref["qptr"]) and np.array_equal(g["qidx"], ref["qidx"])
    assert np.array_equal(g["s_col"], ref["S"].col)
    tol = TOL_FP64 if precision == 0 else TOL_FP32
    assert normwise_cols_fast(g["xval"].astype(np.float64), ref["xval"], ref["qptr"]) <= tol
    assert normwise_cols_fast(g["s_val"].astype(np.float64), ref["S"].val, ref["S"].rowptr) <= tol
    b = torch.as_tensor(big.b, device="cuda")
    x, it, tr, cycles, rc = h.solve_batched(fo, co, b, restart=50, rtol=1e-8, maxit=2000)
    assert rc == 0
    xh = x.cpu().numpy()
    for i, s in enumerate(systems):
        xi = W.sub_vector(xh, systems, fo, co, i)
        res = np.linalg.norm(s.full_scipy() @ xi - s.b) / np.linalg.norm(s.b)
        assert res <= 1.05e-8 and tr[i] <= 1e-8, (i, res, tr[i])
        r = O.edfa_pipeline(s, mode="nbr", solve=True)
        if precision == 0:
            assert abs(int(it[i]) - r["iters"]) <= 1, (i, it[i], r["iters"])
        else:
            assert int(it[i]) <= r["iters"] * 1.25 + 2, (i, it[i], r["iters"])
    h.close()


def test_batched_equals_single_solves_and_repeat():
    # the batched solve of each system matches the single-system GPU solve, and a
    # second call on the same handle (workspace reuse, fresh graph) repeats it
    torch = _torch()
    systems, big, fo, co = batch(nsys=5, lo=6, hi=9, seed=11)
    h = gpu_handle(big, mode="nbr")
    b = torch.as_tensor(big.b, device="cuda")
    x1, it1, tr1, _, rc1 = h.solve_batched(fo, co, b)
    x2, it2, tr2, _, rc2 = h.solve_batched(fo, co, b)
    assert rc1 == 0 and rc2 == 0 and np.array_equal(it1, it2)
    assert np.abs(x1.cpu().numpy() - x2.cpu().numpy()).max() <= 1e-12 * np.abs(x1.cpu().numpy()).max()
    for i, s in enumerate(systems):
        hs = gpu_handle(s, mode="nbr")
        xs, info = hs.solve(torch.as_tensor(s.b, device="cuda"))
        assert abs(info.iterations - int(it1[i])) <= 1
        xi = W.sub_vector(x1.cpu().numpy(), systems, fo, co, i)
        assert np.abs(xi - xs.cpu().numpy()).max() <= 1e-6 * np.abs(xs.cpu().numpy()).max()
        hs.close()
    h.close()
