"""Differentiable EDFA-preconditioned solve (torch.autograd.Function).

forward:  theta = log k (one value per cell) -> u with A(theta) u = b(theta),
          solved by FGMRES preconditioned with EDFA (edfa_build + edfa_solve).
backward: dL/du -> adjoint solve A^T lambda = dL/du with EDFA rebuilt on the
          transposed system (edfa_build_adjoint: same restriction sets, the
          right-hand-side roles swapped) -> dL/dtheta through the elemental
          RT0 matrices (edfa_grad_logk).

The system is produced by a caller-supplied `assemble(theta)` that returns a
dict with the device CSR triples A, B, C, D, the device right-hand side b,
Nf, Ne and the grid description cell_faces, face_cells, face_dir, face_pbar,
W (device tensors, see edfa_grad_logk in include/edfa.h).
"""
from __future__ import annotations

import torch

from . import Edfa, grad_logk


class EDFASolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, assemble, opts):
        opts = dict(opts or {})
        rtol = opts.pop("rtol", 1e-12)
        adj_rtol = opts.pop("adj_rtol", rtol)
        restart = opts.pop("restart", 50)
        maxit = opts.pop("maxit", 5000)
        sysd = assemble(theta.detach())
        h = Edfa(sysd["A"], sysd["B"], sysd["C"], sysd["D"], sysd["Nf"], sysd["Ne"], **opts)
        u, info = h.solve(sysd["b"], restart=restart, rtol=rtol, maxit=maxit)
        if not info.converged:
            raise RuntimeError(f"forward solve did not converge: {info.true_rel:.3e}")
        ctx.h = h
        ctx.sysd = sysd
        ctx.solve_args = (restart, adj_rtol, maxit)
        ctx.save_for_backward(u)
        ctx.forward_info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        h, sysd = ctx.h, ctx.sysd
        restart, rtol, maxit = ctx.solve_args
        adj = h.adjoint()
        lam, info = adj.solve(grad_u.contiguous(), restart=restart, rtol=rtol, maxit=maxit)
        if not info.converged:
            raise RuntimeError(f"adjoint solve did not converge: {info.true_rel:.3e}")
        g = grad_logk(sysd, u, lam, sysd["Nf"], sysd["Ne"])
        ctx.adjoint_info = info
        adj.close()
        return g, None, None


def edfa_solve_diff(theta, assemble, **opts):
    """u(theta) with gradients flowing back to theta through the EDFA adjoint."""
    return EDFASolve.apply(theta, assemble, opts)
