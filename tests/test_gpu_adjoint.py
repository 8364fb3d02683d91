"""Adjoint (differentiable solve) parity: the hand-written EDFA adjoint on the
GPU against central finite differences of GPU forward solves and against the
oracle's FP64 adjoint gradient.  Loss L = sum of squared cell pressures at
seeded observation cells; gradient with respect to per-cell log-conductivity.

Tolerances: relative error <= 1e-4 per cell against central differences
(step 1e-5) and <= 1e-8 normwise against the oracle's adjoint (both adjoint
solves at rtol 1e-13).  The central difference (L(theta + h e) - L(theta - h e))
/ 2h is evaluated without cancellation: the perturbed solutions are
u(theta +- h e) = u0 + delta+-, with delta+- from an EDFA-preconditioned GPU
solve of A(theta +- h e) delta = b(theta +- h e) - A(theta +- h e) u0 (defect
correction from the base solution u0, rtol 1e-13 relative to that small
right-hand side), and L+ - L- = sum over the observation cells of
(delta+ - delta-)(u+ + u-).  Subtracting two losses of size ~10 solved to
1e-13 would leave noise of ~1e-8 L / h, several per cent of the smallest
sampled gradients."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from helpers import gpu_handle, gpu_results

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def oracle_state_and_adjoint(sysd, obs, rtol=1e-13):
    """u, lambda and the gradient from the oracle alone (EDFA-preconditioned
    FGMRES on the system and on its transpose, C-row sets)."""
    A, B, C, D = sysd.A, sysd.B, sysd.C, sysd.D
    q = O.qsets("crow", A, B, C)
    x, _ = O.local_solves(A, B, C, *q)
    S = O.schur(0, A, C, D, *q, x)
    P = O.Prec(A, B, C, D, S=S)
    r = O.fgmres(P, sysd.f_phys, 50, rtol, 5000)
    u = r["x"]
    dLdu = np.zeros(sysd.n)
    dLdu[sysd.Nf + obs] = 2 * u[sysd.Nf + obs]
    Bt = O.Mat.of(C.to_scipy().T.tocsr())
    Ct = O.Mat.of(B.to_scipy().T.tocsr())
    Dt = O.Mat.of(D.to_scipy().T.tocsr())
    xt, _ = O.local_solves(A, Bt, Ct, *q)
    St = O.schur(0, A, Ct, Dt, *q, xt)
    Pt = O.Prec(A, Bt, Ct, Dt, S=St)
    ra = O.fgmres(Pt, dLdu, 50, rtol, 5000)
    lam = ra["x"]
    g = O.adjoint_grad(sysd, u, lam, np.log(sysd.K[:, 0]))
    return u, lam, g


def gpu_grad(sysd, obs, rtol=1e-13):
    torch = _torch()
    from paper_2009_13916_gb300.adjoint import edfa_solve_diff
    assemble = W.device_assembler(sysd)
    theta = torch.tensor(np.log(sysd.K[:, 0]), dtype=torch.float64, device="cuda", requires_grad=True)
    u = edfa_solve_diff(theta, assemble, qmode="crow", rtol=rtol)
    obs_t = torch.as_tensor(sysd.Nf + obs, device="cuda")
    L = (u[obs_t] ** 2).sum()
    L.backward()
    return u.detach().cpu().numpy(), theta.grad.cpu().numpy(), float(L.item())


def fd_gradient(sysd, obs, cells, h=1e-5, rtol=1e-13):
    """Central differences of L at `cells` from GPU forward solves (defect
    correction from the base solution, see the module docstring)."""
    torch = _torch()
    import paper_2009_13916_gb300 as P
    assemble = W.device_assembler(sysd)
    theta = np.log(sysd.K[:, 0])

    def solve(d, rhs):
        hd = P.Edfa(d["A"], d["B"], d["C"], d["D"], d["Nf"], d["Ne"], qmode="crow")
        x, info = hd.solve(rhs, restart=50, rtol=rtol, maxit=5000)
        assert info.converged, info.true_rel
        return hd, x

    d0 = assemble(torch.as_tensor(theta))
    h0, u0 = solve(d0, d0["b"])
    h0.close()
    o = torch.as_tensor(sysd.Nf + obs, device="cuda")
    out = []
    for e in cells:
        dl = []
        for sgn in (1.0, -1.0):
            t = theta.copy()
            t[e] += sgn * h
            d = assemble(torch.as_tensor(t))
            hd = P.Edfa(d["A"], d["B"], d["C"], d["D"], d["Nf"], d["Ne"], qmode="crow")
            r = d["b"] - hd.matvec(u0)
            delta, info = hd.solve(r, restart=50, rtol=rtol, maxit=5000)
            assert info.converged, info.true_rel
            hd.close()
            dl.append(delta)
        up, um = u0 + dl[0], u0 + dl[1]
        out.append(float(((dl[0][o] - dl[1][o]) * (up[o] + um[o])).sum().item()) / (2 * h))
    return np.array(out)


def small_case():
    sysd = W.config5(9, nobs=12, nfd=6)
    return sysd, sysd.extra["obs"], sysd.extra["fd_cells"]


def test_adjoint_gradient_matches_oracle_adjoint():
    sysd, obs, _ = small_case()
    u_g, g_g, _ = gpu_grad(sysd, obs)
    u_o, lam_o, g_o = oracle_state_and_adjoint(sysd, obs)
    assert np.abs(u_g - u_o).max() <= 1e-10 * np.abs(u_o).max()
    err = np.abs(g_g - g_o).max() / np.abs(g_o).max()
    assert err <= 1e-8, err


def test_adjoint_gradient_matches_central_differences():
    sysd, obs, fd = small_case()
    _, g, _ = gpu_grad(sysd, obs)
    fdv = fd_gradient(sysd, obs, fd)
    rel = np.abs(g[fd] - fdv) / np.abs(fdv)
    assert rel.max() <= 1e-4, (rel, g[fd], fdv)


def test_transposed_two_sided_schur_is_transpose():
    torch = _torch()
    sysd, _, _ = small_case()
    h = gpu_handle(sysd, mode="crow", form=1)
    adj = h.adjoint()
    S = gpu_results(h)
    St = gpu_results(adj)
    M = sp.csr_matrix((S["s_val"], S["s_col"], S["s_rowptr"]), shape=(sysd.Ne, sysd.Ne))
    Mt = sp.csr_matrix((St["s_val"], St["s_col"], St["s_rowptr"]), shape=(sysd.Ne, sysd.Ne))
    d = abs(M.T - Mt)
    assert d.max() <= 1e-12 * abs(M).max()
    assert np.array_equal(St["qidx"], S["qidx"])
    adj.close()
    h.close()


def test_adjoint_config5_full():
    # 48^3, 64 observation cells: oracle adjoint (normwise 1e-8) and central
    # differences at the 20 seeded cells (relative 1e-4 per cell)
    sysd = W.config5()
    obs, fd = sysd.extra["obs"], sysd.extra["fd_cells"]
    u_g, g_g, _ = gpu_grad(sysd, obs)
    u_o, lam_o, g_o = oracle_state_and_adjoint(sysd, obs)
    err = np.abs(g_g - g_o).max() / np.abs(g_o).max()
    assert err <= 1e-8, err
    # central differences at the 20 seeded cells, per cell
    fdv = fd_gradient(sysd, obs, fd)
    rel = np.abs(g_g[fd] - fdv) / np.abs(fdv)
    assert rel.max() <= 1e-4, (rel, g_g[fd], fdv)
