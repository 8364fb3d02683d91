"""The 128x128x64 channelised workload at full size (1,048,576 local systems,
4,227,072 unknowns, thresh-0.05 sets): sets and S~ pattern bit-exact and X~,
S~ within 1e-10 against the oracle; FP64 and FP32-mixed FGMRES(50) to 1e-8,
FP64 iteration count within 1 of the oracle's.  The oracle's count is stored
in tests/golden/c3_oracle_fgmres.txt (written by make_c3_fgmres.py from the
oracle) together with the digest of the inputs it belongs to; the generator
uses no host math library, so the inputs are the same on every host, and if
the digest ever differs the oracle's FGMRES is run here instead."""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import TOL_FP64, gpu_handle, gpu_results, normwise_cols_fast

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c3_oracle_fgmres.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        if not line.startswith("#") and line.strip():
            k, v = line.split(None, 1)
            vals[k] = v.strip()
    return vals


def oracle_iterations(sysd):
    """The oracle's FGMRES(50) count on these inputs: the stored one when the
    input digest matches, else computed now (several minutes of CPU time)."""
    g = golden()
    if g.get("inputs_sha256") == W.digest(sysd):
        return int(g["iterations"])
    r = O.edfa_pipeline(sysd, mode="thresh", restart=50, rtol=1e-8, maxit=3000)
    return int(r["iters"])


def check_first_cycle(h, suffix, sysd):
    """Residual estimates of the first restart cycle against the oracle's
    (stored beside its counts): the GPU iteration is the oracle's up to
    rounding, so the two agree closely before rounding differences compound."""
    g = golden()
    key = "cycle1" + suffix
    if g.get("inputs_sha256") != W.digest(sysd) or key not in g:
        return
    ref = np.array([float(v) for v in g[key].split()])
    hist = np.asarray(h.history())[1: 1 + len(ref)]
    assert len(hist) == len(ref)
    assert np.allclose(hist, ref, rtol=1e-6, atol=0), np.abs(hist / ref - 1).max()


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
    it_orc = oracle_iterations(sysd)
    assert abs(info.iterations - it_orc) <= 1, (info.iterations, it_orc)
    check_first_cycle(h, "", sysd)
    h.close()
    h32 = gpu_handle(sysd, mode="thresh", thresh=0.05, precision=1)
    x32, info32 = h32.solve(b, restart=50, rtol=1e-8, maxit=3000)
    res32 = np.linalg.norm(sysd.full_scipy() @ x32.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert info32.converged and res32 <= 1.05e-8
    assert info32.iterations <= info.iterations * 1.25 + 2
    h32.close()


def test_inputs_identical_on_this_host():
    """Runs with the GPU tests so that it runs on the GPU host (aarch64): the
    generated inputs equal, bit for bit, those recorded on the x86-64 host."""
    from test_workloads import DIGEST_C1, DIGEST_C2_8, DIGEST_C3_SMALL
    assert W.digest(W.config1()) == DIGEST_C1
    assert W.digest(W.config2(8)) == DIGEST_C2_8
    assert W.digest(W.config3(16, 12, 6)) == DIGEST_C3_SMALL


@pytest.mark.parametrize("s_block", [1, 4])
def test_config3_full_size_multicolour_ordering(s_block):
    """The same workload with multicolour orderings of both inner factors
    (ordering 2; with the point colouring of S~ and with the block colouring
    in blocks of 4 rows, the benchmark's configuration): colourings and orderings
    bit-exact, ordered factor patterns bit-exact and values within 1e-10 of
    the oracle's ILU(0) of the ordered matrices, one application within 1e-9,
    FGMRES converged to 1e-8 with the first cycle's residual estimates within
    1e-6 of the oracle's and the count within 0.5% of the oracle's with the same
    orderings (stored beside the natural one); FP32-mixed converges too.
    The library runs this FGMRES in the ordered numbering, the oracle in the
    natural one: FGMRES is invariant under a symmetric permutation of the
    system in exact arithmetic (inner products and norms are unchanged), but
    the dot products are summed in another order, and over the 17 restart
    cycles of this solve the rounding moves the count by a few iterations."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sysd = W.config3()
    h = gpu_handle(sysd, mode="thresh", thresh=0.05, ordering=2, s_block=s_block)
    f = h.factors()
    qptr, qidx = O.qsets("thresh", sysd.A, sysd.B, sysd.C, 0.05)
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx)
    S = O.schur(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x)
    _, aperm, nca = O.colour_order(sysd.A)
    _, sperm, ncs = O.colour_order(S, s_block)
    assert np.array_equal(f["a_perm"].cpu().numpy(), aperm) and f["a_ncolours"] == nca
    assert np.array_equal(f["s_perm"].cpu().numpy(), sperm) and f["s_ncolours"] == ncs
    Pc = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=S, aperm=aperm, sperm=sperm)
    for key, which in (("fa", "a"), ("fs", "s")):
        pat, lu = Pc.ordered_factor(which)
        assert np.array_equal(f[key + "_rowptr"].cpu().numpy(), pat.rowptr)
        assert np.array_equal(f[key + "_col"].cpu().numpy(), pat.col)
        assert normwise_cols_fast(f[key + "_lu"].cpu().numpy(), lu, pat.rowptr) <= TOL_FP64
    r = W.Stream(77).normal(sysd.n)
    z_ref = Pc.apply(r)
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max()
    b = torch.as_tensor(sysd.b, device="cuda")
    xg, info = h.solve(b, restart=50, rtol=1e-8, maxit=3000)
    res = np.linalg.norm(sysd.full_scipy() @ xg.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert info.converged and res <= 1.05e-8
    g = golden()
    suffix = "_ordering2" + ("" if s_block == 1 else f"_block{s_block}")
    if g.get("inputs_sha256") == W.digest(sysd) and "iterations" + suffix in g:
        it_orc = int(g["iterations" + suffix])
    else:
        it_orc = O.fgmres(Pc, sysd.b, 50, 1e-8, 3000)["iters"]
    assert abs(info.iterations - it_orc) <= max(1, 0.005 * it_orc), (info.iterations, it_orc)
    check_first_cycle(h, suffix, sysd)
    h.close()
    h32 = gpu_handle(sysd, mode="thresh", thresh=0.05, precision=1, ordering=2, s_block=s_block)
    x32, info32 = h32.solve(b, restart=50, rtol=1e-8, maxit=3000)
    res32 = np.linalg.norm(sysd.full_scipy() @ x32.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert info32.converged and res32 <= 1.05e-8
    assert info32.iterations <= info.iterations * 1.25 + 2
    h32.close()
