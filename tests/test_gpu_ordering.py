"""Multicolour orderings of the inner ILU(0) factorisations (edfa_options
.ordering; 1 = S~, 2 = A~ and S~; edfa_options.s_block: block multicolour
ordering of S~) on the GPU against the oracle with the same orderings: colourings and orderings bit-exact, the ordered factor patterns
bit-exact, the factor values within 1e-10 (normwise per row), one application
of the preconditioner within 1e-9 and FGMRES within one iteration of the
oracle, converged at 1e-8.  The paper leaves the inner preconditioners and
their ordering open (Sec. 3, inner preconditioners); the natural order stays
the default."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_handle, normwise_cols_fast

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
    "full": (lambda: full_tensor((12, 10, 8)), "nbr"),
    "c3_small": (lambda: W.config3(24, 20, 6), "thresh"),
    "c3_ragged": (lambda: W.config3(13, 11, 5), "thresh"),  # 715 cells: a short last block
    "dome8": (lambda: W.dome(8), "nbr"),
    "c5_small": (lambda: W.config5(10), "crow"),
}


def factor_check(g, key, perm_key, ref_perm, ref_pat, ref_lu, n):
    if ref_perm is not None:
        assert np.array_equal(g[perm_key].cpu().numpy(), ref_perm)
    assert np.array_equal(g[key + "_rowptr"].cpu().numpy(), ref_pat.rowptr)
    assert np.array_equal(g[key + "_col"].cpu().numpy(), ref_pat.col)
    err = normwise_cols_fast(g[key + "_lu"].cpu().numpy().astype(np.float64), ref_lu, ref_pat.rowptr)
    assert err <= 1e-10, (key, err)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("ordering", [1, 2])
@pytest.mark.parametrize("variant", [0, 1])
def test_ordered_factors_apply_and_fgmres(case, ordering, variant):
    torch = _torch()
    make, mode = CASES[case]
    sysd = make()
    ref = O.edfa_pipeline(sysd, mode=mode, variant=variant, ordering=ordering, solve=True)
    h = gpu_handle(sysd, mode=mode, variant=variant, ordering=ordering)
    g = h.factors()
    P = ref["prec"]
    pat_s, lu_s = P.ordered_factor("s")
    factor_check(g, "fs", "s_perm", ref["sperm"], pat_s, lu_s, sysd.Ne)
    assert g["s_ncolours"] == O.colour_order(ref["S"])[2]
    if ordering == 2:
        pat_a, lu_a = P.ordered_factor("a")
        factor_check(g, "fa", "a_perm", ref["aperm"], pat_a, lu_a, sysd.Nf)
        assert g["a_ncolours"] == O.colour_order(sysd.A)[2]
    else:
        assert g["a_perm"] is None
    st = h.stats()
    assert st.levels_s <= g["s_ncolours"]
    if ordering == 2:
        assert st.levels_a <= g["a_ncolours"]
    r = W.Stream(77).normal(sysd.n)
    z_ref = P.apply(r)
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    err = np.abs(z - z_ref).max() / np.abs(z_ref).max()
    assert err <= 1e-9, f"apply error {err:.3e}"
    x, info = h.solve(torch.as_tensor(sysd.b, device="cuda"), restart=50, rtol=1e-8, maxit=2000)
    assert info.converged and abs(info.iterations - ref["iters"]) <= 1, (info.iterations, ref["iters"])
    res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert res <= 1.05e-8
    h.close()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("s_block", [3, 4, 8, 16])
def test_block_ordered_factors_apply_and_fgmres(case, s_block):
    """Block multicolour ordering of S~ (blocks of s_block consecutive rows
    coloured as units; A~ point-coloured): colours, ordering, factors,
    application and FGMRES against the oracle with the same orderings; FP32-mixed
    converges."""
    torch = _torch()
    make, mode = CASES[case]
    sysd = make()
    ref = O.edfa_pipeline(sysd, mode=mode, ordering=2, s_block=s_block, solve=True)
    h = gpu_handle(sysd, mode=mode, ordering=2, s_block=s_block)
    g = h.factors()
    P = ref["prec"]
    pat_s, lu_s = P.ordered_factor("s")
    factor_check(g, "fs", "s_perm", ref["sperm"], pat_s, lu_s, sysd.Ne)
    assert g["s_ncolours"] == O.colour_order(ref["S"], s_block)[2]
    pat_a, lu_a = P.ordered_factor("a")
    factor_check(g, "fa", "a_perm", ref["aperm"], pat_a, lu_a, sysd.Nf)
    r = W.Stream(78).normal(sysd.n)
    z_ref = P.apply(r)
    z = h.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    err = np.abs(z - z_ref).max() / np.abs(z_ref).max()
    assert err <= 1e-9, f"apply error {err:.3e}"
    b = torch.as_tensor(sysd.b, device="cuda")
    x, info = h.solve(b, restart=50, rtol=1e-8, maxit=2000)
    assert info.converged and abs(info.iterations - ref["iters"]) <= 1, (info.iterations, ref["iters"])
    res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert res <= 1.05e-8
    h.close()
    h32 = gpu_handle(sysd, mode=mode, ordering=2, s_block=s_block, precision=1)
    x32, info32 = h32.solve(b, restart=50, rtol=1e-8, maxit=2000)
    res32 = np.linalg.norm(sysd.full_scipy() @ x32.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
    assert info32.converged and res32 <= 1.05e-8
    h32.close()


@pytest.mark.parametrize("ordering", [1, 2])
def test_ordered_fp32_mixed_converges(ordering):
    torch = _torch()
    for case in ("full", "c3_small"):
        make, mode = CASES[case]
        sysd = make()
        ref = O.edfa_pipeline(sysd, mode=mode, ordering=ordering, solve=True)
        h = gpu_handle(sysd, mode=mode, precision=1, ordering=ordering)
        g = h.factors()
        assert np.array_equal(g["s_perm"].cpu().numpy(), ref["sperm"])
        x, info = h.solve(torch.as_tensor(sysd.b, device="cuda"), restart=50, rtol=1e-8, maxit=2000)
        res = np.linalg.norm(sysd.full_scipy() @ x.cpu().numpy() - sysd.b) / np.linalg.norm(sysd.b)
        assert info.converged and res <= 1.05e-8
        assert info.iterations <= ref["iters"] * 1.25 + 2, (info.iterations, ref["iters"])
        h.close()


def test_ordered_setup_reuse_and_post_filtration():
    # Stage 2 with new D values on an ordered handle equals a fresh build bit for
    # bit; with post-filtration of S~ the colouring follows the new pattern
    torch = _torch()
    import paper_2009_13916_gb300 as P
    sysd = full_tensor((10, 9, 8), seed=5)
    tr = W.Transient(sysd)
    A, B, C, D = P.system_to_device(sysd)
    for filt in ("none", "post_s"):
        kw = dict(qmode="nbr", ordering=2, filtration=filt, tau_filt=1e-3)
        h = P.Edfa(A, B, C, D, sysd.Nf, sysd.Ne, **kw)
        Dn = (D[0], D[1], torch.as_tensor(tr.D_values(0.37), device="cuda"))
        h.setup(Dn)
        h2 = P.Edfa(A, B, C, Dn, sysd.Nf, sysd.Ne, **kw)
        f1, f2 = h.factors(), h2.factors()
        for k in ("s_perm", "fs_rowptr", "fs_col", "fs_lu", "a_perm", "fa_lu"):
            assert torch.equal(f1[k], f2[k]), (filt, k)
        r = torch.as_tensor(W.Stream(9).normal(sysd.n), device="cuda")
        assert torch.equal(h.apply(r), h2.apply(r))
        # against the oracle on the new system
        s2 = W.System(**{**sysd.__dict__, "D": tr.D(0.37)})
        ref = O.edfa_pipeline(s2, mode="nbr", ordering=2, filt=filt, tau=1e-3, solve=False)
        assert np.array_equal(f1["s_perm"].cpu().numpy(), ref["sperm"])
        z_ref = ref["prec"].apply(r.cpu().numpy())
        z = h.apply(r).cpu().numpy()
        assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max()
        h.close()
        h2.close()
