"""Pre- and post-filtration of S~ (Sec. 3 implementation details, Algorithms 1
and 2): CUDA path vs the oracle on the same seeded inputs, through the C ABI.

Bar: the filtered S~ pattern bit-exact (both sides decide |v| < tau ||row||_2 in
FP64), S~ values within 1e-10 normwise per row, one application within 1e-9,
FGMRES(50) to 1e-8 within one iteration of the oracle.  Post-filtration of S~
is a Stage-2 step: a new D through edfa_setup changes the pattern of S~ and its
ILU(0) plans, checked against the oracle on the new D.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP64, normwise_cols_fast

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
    return W.assemble(*n, W.rotated_K(m, 0.1, q))


CASES = {
    "brick6_paper": (lambda: W.brick(6, seed=3, sigma=1.0), "nbr"),
    "ragged_full_7x5x3": (lambda: full_tensor((7, 5, 3)), "nbr"),
    "c3_small": (lambda: W.config3(24, 20, 6), "thresh"),
}


def _handle(sysd, mode, form, filt, tau, precision=0, sweep_mode=0):
    import paper_2009_13916_gb300 as P
    A, B, C, D = P.system_to_device(sysd)
    return P.Edfa(A, B, C, D, sysd.Nf, sysd.Ne, qmode=mode, thresh=sysd.extra.get("thresh", 0.05),
                  schur_form=form, precision=precision, filtration=filt, tau_filt=tau, sweep_mode=sweep_mode)


def _check_s(h, S):
    g = h.tensors()
    assert np.array_equal(g["s_rowptr"].cpu().numpy(), S.rowptr)
    assert np.array_equal(g["s_col"].cpu().numpy(), S.col)
    es = normwise_cols_fast(g["s_val"].cpu().numpy(), S.val, S.rowptr)
    assert es <= TOL_FP64, f"S~ error {es:.3e}"


@pytest.mark.parametrize("filt", ["pre", "post_h", "post_s"])
@pytest.mark.parametrize("case,form,tau", [("ragged_full_7x5x3", 0, 1e-3), ("ragged_full_7x5x3", 1, 1e-2),
                                           ("brick6_paper", 0, 1e-2), ("c3_small", 0, 1e-3)])
def test_filtered_schur_apply_and_fgmres(filt, case, form, tau):
    torch = _torch()
    make, mode = CASES[case]
    sysd = make()
    ref = O.edfa_pipeline(sysd, mode=mode, form=form, filt=filt, tau=tau)
    S0 = O.edfa_pipeline(sysd, mode=mode, form=form, solve=False)["S"]
    assert ref["S"].nnz < S0.nnz  # the tolerance does drop entries here
    h = _handle(sysd, mode, form, filt, tau)
    _check_s(h, ref["S"])
    assert h.stats().s_nnz == ref["S"].nnz
    r = W.Stream(78).normal(sysd.n)
    z_ref = ref["prec"].apply(r)
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max()
    x, info = h.solve(torch.as_tensor(sysd.b, device="cuda"), restart=50, rtol=1e-8, maxit=2000)
    assert info.converged and abs(info.iterations - ref["iters"]) <= 1, (info.iterations, ref["iters"])
    res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert res <= 1.05e-8
    h.close()


@pytest.mark.parametrize("filt", ["post_s", "post_h"])
@pytest.mark.parametrize("sweep_mode", [0, 1])
def test_stage2_new_D_with_filtration(filt, sweep_mode):
    # post-filtration of S~ re-derives the pattern from the new D (Stage 2);
    # post-filtration of H~ keeps the Stage-1 pattern
    torch = _torch()
    sysd = full_tensor((7, 5, 3))
    tau = 2e-3
    h = _handle(sysd, "nbr", 0, filt, tau, sweep_mode=sweep_mode)
    q = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, *q)
    for scale in (3.0, 0.2, 1.0):
        D2 = sysd.D.to_scipy().tocsr().copy()
        D2.setdiag(D2.diagonal() * scale)
        D2.sort_indices()
        Dt = (torch.as_tensor(D2.indptr, dtype=torch.int64, device="cuda"),
              torch.as_tensor(D2.indices, dtype=torch.int32, device="cuda"),
              torch.as_tensor(D2.data, dtype=torch.float64, device="cuda"))
        h.setup(Dt)
        Dm = O.Mat(D2.shape[0], D2.shape[1], D2.indptr.astype(np.int64), D2.indices.astype(np.int32), D2.data)
        S, _ = O.schur_filtered(0, sysd.A, sysd.C, Dm, *q, x, None, filt, tau)
        _check_s(h, S)
        P = O.Prec(sysd.A, sysd.B, sysd.C, Dm, S=S)
        r = W.Stream(79).normal(sysd.n)
        z_ref = P.apply(r)
        z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
        assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max(), scale
    h.close()


@pytest.mark.parametrize("filt", ["pre", "post_h", "post_s"])
def test_fp32_mixed_with_filtration(filt):
    # FP32 local solves, S~ and application (decisions taken on FP32 values),
    # FP64 Krylov: reaches 1e-8 within a few iterations of the FP64 path
    torch = _torch()
    sysd = full_tensor((12, 10, 8), seed=5)
    b = torch.as_tensor(sysd.b, device="cuda")
    its = []
    for prec in (0, 1):
        h = _handle(sysd, "nbr", 0, filt, 1e-3, precision=prec)
        x, info = h.solve(b, restart=50, rtol=1e-8, maxit=2000)
        assert info.converged
        res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
        assert res <= 1.05e-8
        its.append(info.iterations)
        h.close()
    assert abs(its[1] - its[0]) <= 2, its


def test_filtration_option_validation():
    _torch()
    import paper_2009_13916_gb300 as P
    sysd = W.brick(3, seed=2)
    for filt, tau in ((4, 1e-3), (-1, 1e-3), (1, -1.0), (2, float("nan"))):
        with pytest.raises(P.EdfaError) as e:
            _handle(sysd, "own", 0, filt, tau)
        assert e.value.code == 1
