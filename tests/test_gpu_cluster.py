"""The single-cluster S~ sweeps against the oracle and against the sync-free
sweeps, including the degenerate shapes of its data layout: fewer rows than
CTAs, levels longer than the in-block sort handles, both block variants and
both precisions, and a new D through edfa_setup (re-packed values)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_handle

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _apply(h, r):
    torch = _torch()
    return h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _check(sysd, mode, variant=0, precision=0, sweep_mode=0):
    """cluster sweeps (dataflow: sweep_mode 0, one barrier per level: 2) vs the
    oracle's application and vs the sync-free sweeps"""
    _torch()
    ref = O.edfa_pipeline(sysd, mode=mode, variant=variant, solve=False)
    r = W.Stream(5).normal(sysd.n)
    z_ref = ref["prec"].apply(r)
    import paper_2009_13916_gb300 as P
    A, B, C, D = P.system_to_device(sysd)
    h_cl = P.Edfa(A, B, C, D, sysd.Nf, sysd.Ne, qmode=mode, thresh=sysd.extra.get("thresh", 0.05),
                  variant=variant, precision=precision, sweep_mode=sweep_mode)
    assert h_cl.stats().s_cluster == 1
    z_cl = _apply(h_cl, r)
    # a second handle with the all-SM sweeps only
    h_sf = P.Edfa(A, B, C, D, sysd.Nf, sysd.Ne, qmode=mode, thresh=sysd.extra.get("thresh", 0.05),
                  variant=variant, precision=precision, sweep_mode=1)
    assert h_sf.stats().s_cluster == 0
    z_sf = _apply(h_sf, r)
    tol = 1e-9 if precision == 0 else 2e-4
    assert _rel(z_cl, z_ref) <= tol
    # same arithmetic per row, only the order of the partial sums differs
    assert _rel(z_cl, z_sf) <= (1e-13 if precision == 0 else 1e-5)
    h_cl.close()
    h_sf.close()


@pytest.mark.parametrize("sweep_mode", [0, 2])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_cluster_sweep_matches_oracle_and_syncfree(variant, precision, sweep_mode):
    s = W.Stream(11)
    n = (12, 10, 9)
    Ne = int(np.prod(n))
    m = np.exp(2.0 * s.normal(Ne))
    q = s.normal(4 * Ne).reshape(Ne, 4)
    sysd = W.assemble(*n, W.rotated_K(m, 0.1, q))
    _check(sysd, "nbr", variant=variant, precision=precision, sweep_mode=sweep_mode)


@pytest.mark.parametrize("sweep_mode", [0, 2])
def test_cluster_sweep_fewer_rows_than_ctas(sweep_mode):
    # 8 cells: half of the 16 CTAs own no row at all
    _check(W.brick(2, seed=4), "nbr", sweep_mode=sweep_mode)


@pytest.mark.parametrize("sweep_mode", [0, 2])
def test_cluster_sweep_levels_longer_than_sort_block(sweep_mode):
    # 8300 independent 2x2x2 bricks: the first forward level holds > 8192 rows
    sysd, _, _ = W.concat([W.brick(2, seed=1 + k % 7) for k in range(8300)])
    _check(sysd, "own", sweep_mode=sweep_mode)


@pytest.mark.parametrize("precision", [0, 1])
def test_cluster_sweep_long_rows_overflow(precision):
    # given sets: own faces + 20 faces drawn anywhere in the grid, so that S~
    # rows couple far more than the 32 dependencies a dataflow record holds inline
    torch = _torch()
    import paper_2009_13916_gb300 as P
    sysd = W.brick(7, seed=5, sigma=1.0)
    st = W.Stream(3)
    own = [set(sysd.B.to_scipy().tocsc()[:, m].indices) for m in range(sysd.Ne)]
    qptr, qidx = [0], []
    for m in range(sysd.Ne):
        extra = (st.uniform(40) * sysd.Nf).astype(np.int64)
        q = sorted(own[m] | set(int(f) for f in extra[:20]))
        qidx += q
        qptr.append(len(qidx))
    qptr, qidx = np.asarray(qptr, np.int64), np.asarray(qidx, np.int32)
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx)
    S = O.schur(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x)
    rows = np.repeat(np.arange(sysd.Ne), np.diff(S.rowptr))
    assert np.bincount(rows[S.col < rows]).max() > 40
    prec = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=S)
    r = W.Stream(5).normal(sysd.n)
    z_ref = prec.apply(r)
    A, B, C, D = P.system_to_device(sysd)
    qs = (torch.as_tensor(qptr, device="cuda"), torch.as_tensor(qidx, device="cuda"))
    zs = []
    for mode in (0, 2, 1):
        h = P.Edfa(A, B, C, D, sysd.Nf, sysd.Ne, qsets=qs, precision=precision, sweep_mode=mode)
        assert h.stats().s_cluster == (mode != 1)
        zs.append(_apply(h, r))
        h.close()
    tol = 1e-9 if precision == 0 else 2e-4
    for z in zs:
        assert _rel(z, z_ref) <= tol
    assert _rel(zs[0], zs[2]) <= (1e-13 if precision == 0 else 1e-5)


def test_cluster_sweep_after_new_D():
    torch = _torch()
    import paper_2009_13916_gb300 as P
    sysd = W.brick(6, seed=3, sigma=1.0)
    h = gpu_handle(sysd, mode="nbr")
    assert h.stats().s_cluster == 1
    # new storage term (diagonal of D): Stage 2 refactors S~ and re-packs the chunk values
    D2 = sysd.D.to_scipy().tocsr().copy()
    D2.setdiag(D2.diagonal() * 3.0)
    D2.sort_indices()
    Dt = (torch.as_tensor(D2.indptr, dtype=torch.int64, device="cuda"),
          torch.as_tensor(D2.indices, dtype=torch.int32, device="cuda"),
          torch.as_tensor(D2.data, dtype=torch.float64, device="cuda"))
    h.setup(Dt)
    q = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, *q)
    S = O.schur(0, sysd.A, sysd.C, D2, *q, x)
    prec = O.Prec(sysd.A, sysd.B, sysd.C, D2, S=S)
    r = W.Stream(9).normal(sysd.n)
    assert _rel(_apply(h, r), prec.apply(r)) <= 1e-9
    h.close()
