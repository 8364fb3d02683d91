"""Transient sequence with Stage-2-only reuse (the paper's two-stage set-up, Sec. 3
implementation details, Algorithms 1 and 2): between implicit-Euler steps only D and the cell
right-hand side change (Sec. 4, Eq. delta_t_dyn time-step rule), so the handle keeps Stage 1
and every step calls edfa_setup with the new D.  Each step is checked against the oracle run
on that step's system (FGMRES within one iteration, true residual <= 1e-8), and the reused
handle must give exactly what a fresh build with the same D gives (with and without
post-filtration of S~, whose pattern changes with D)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("filt", ["none", "post_s"])
def test_transient_stage2_reuse(filt):
    torch = _torch()
    import paper_2009_13916_gb300 as P
    sysd = W.brick(8, seed=3, sigma=1.0)
    tr = W.Transient(sysd, dt_mult=2.0, dp_target=0.05, dt_max=10.0)
    A, B, C, D = P.system_to_device(sysd)
    kw = dict(qmode="nbr", filtration=filt, tau_filt=1e-3)
    h = P.Edfa(A, B, C, D, sysd.Nf, sysd.Ne, **kw)
    p = np.zeros(sysd.Ne)
    dt = sysd.dt
    dts = []
    for step in range(5):
        Dn = tr.D(dt)
        Dd = (D[0], D[1], torch.as_tensor(Dn.val, device="cuda"))
        if step > 0:
            h.setup(Dd)
        b = tr.rhs(dt, p)
        x, info = h.solve(torch.as_tensor(b, device="cuda"), restart=50, rtol=1e-8, maxit=2000)
        sn = dataclasses.replace(sysd, D=Dn, b=b)
        ref = O.edfa_pipeline(sn, mode="nbr", filt=filt, tau=1e-3)
        assert info.converged and abs(info.iterations - ref["iters"]) <= 1, (step, info.iterations, ref["iters"])
        xh = x.cpu().numpy()
        res = np.linalg.norm(sn.full_scipy() @ xh - b) / np.linalg.norm(b)
        assert res <= 1.05e-8, (step, res)
        if step == 3:
            hf = P.Edfa(A, B, C, Dd, sysd.Nf, sysd.Ne, **kw)
            xf, infof = hf.solve(torch.as_tensor(b, device="cuda"), restart=50, rtol=1e-8, maxit=2000)
            assert infof.iterations == info.iterations
            assert np.array_equal(xf.cpu().numpy(), xh)
            hf.close()
        pn = xh[sysd.Nf:]
        dt = tr.next_dt(dt, float(np.max(pn - p)))
        dts.append(dt)
        p = pn
    assert len(set(dts)) > 1  # the step size did change along the sequence
    h.close()
