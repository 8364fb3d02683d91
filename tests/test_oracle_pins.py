"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong index set) fails it:
  * restriction sets against the grid topology, computed here independently
  * X~ = A^{-1} B, G~ = -C A^{-1} and S~ = S when Q^(m) covers every face
    (Eq. dec_fac, Eq. schur_compl, dense brute force)
  * Galerkin orthogonality and energy minimality of the restricted solve
    (Proposition min_energy)
  * own-face solves with diagonal K: three independent 2x2 systems (Cramer)
  * ILU(0) = exact LU when the pattern has no fill (tridiagonal / dense)
  * exact blocks => FGMRES converges in 1 iteration (Eq. inv_A_fac), <= 2 with
    the block upper-triangular variant; identity preconditioner => the dense solution
  * the dynamic technique adds exactly the largest prolonged-residual entries
    (Eq. prol_res), recomputed here with dense algebra
  * the two-sided S~ built on the transposed system is S~^T (F/G role swap)
  * adjoint gradient against central finite differences of dense solves
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W


def full_tensor(n=(3, 3, 2), seed=11, **kw):
    s = W.Stream(seed)
    Ne = int(np.prod(n))
    m = np.exp(s.normal(Ne))
    q = s.normal(4 * Ne).reshape(Ne, 4)
    return W.assemble(*n, W.rotated_K(m, 0.1, q), **kw)


def iso(n=(3, 3, 2), seed=5, sigma=1.0, **kw):
    Ne = int(np.prod(n))
    return W.assemble(*n, W.iso_K(np.exp(sigma * W.Stream(seed).normal(Ne))), **kw)


def all_faces_q(sysd):
    Ne, Nf = sysd.Ne, sysd.Nf
    qptr = np.arange(Ne + 1, dtype=np.int64) * Nf
    qidx = np.tile(np.arange(Nf, dtype=np.int32), Ne)
    return qptr, qidx


def sets_of(qptr, qidx):
    return [list(qidx[qptr[m]:qptr[m + 1]]) for m in range(len(qptr) - 1)]


# ------------------------------------------------------------ restriction sets
def topo_sets(sysd, mode):
    """Restriction sets from the grid topology (cell -> faces, face -> cells)."""
    out = []
    live = ~sysd.face_dir  # prescribed faces carry no B entry
    for m in range(sysd.Ne):
        own = {f for f in sysd.cell_faces[m] if live[f]}
        if mode == "own":
            out.append(sorted(own))
        elif mode == "nbr":
            q = set(own)
            for f in own:
                for e2 in sysd.face_cells[f]:
                    if e2 >= 0 and e2 != m:
                        q |= {g for g in sysd.cell_faces[e2] if live[g]}
            out.append(sorted(q))
    return out


@pytest.mark.parametrize("mode", ["own", "nbr"])
def test_static_sets_match_topology(mode):
    sysd = full_tensor((4, 3, 3))
    qptr, qidx = O.qsets(mode, sysd.A, sysd.B, sysd.C)
    assert sets_of(qptr, qidx) == topo_sets(sysd, mode)


def test_nbr_sizes_interior():
    sysd = iso((5, 5, 5))
    qptr, _ = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    s = np.diff(qptr)
    centre = 2 + 5 * (2 + 5 * 2)
    assert s[centre] == 36  # 6 own + 6 neighbours x 5 far faces


def test_crow_and_thresh_sets():
    sysd = iso((4, 4, 3))
    qptr, qidx = O.qsets("crow", sysd.A, sysd.B, sysd.C)
    Cd = sysd.C.dense()
    assert sets_of(qptr, qidx) == [list(np.nonzero(Cd[m])[0]) for m in range(sysd.Ne)]
    Ad = sysd.A.dense()
    own = topo_sets(sysd, "own")
    for thr in (0.0, 0.05, 0.4, 10.0):
        qptr, qidx = O.qsets("thresh", sysd.A, sysd.B, sysd.C, thr)
        ref = []
        for m in range(sysd.Ne):
            q = set(own[m])
            for i in own[m]:
                q |= {j for j in np.nonzero(Ad[i])[0] if abs(Ad[i, j]) >= thr * abs(Ad[i, i])}
            ref.append(sorted(q))
        assert sets_of(qptr, qidx) == ref
    qptr, qidx = O.qsets("thresh", sysd.A, sysd.B, sysd.C, 10.0)
    assert sets_of(qptr, qidx) == own


def test_static_pattern_a_reading_is_the_axis_extension():
    """Static pattern A (Sec. 4, Fig. static_patterns; the figure is missing):
    read as the A-couplings of the own faces (qmode thresh, tau = 0).  With a
    diagonal K every elemental matrix couples a face only to the opposite face
    of its cell, so this adds, for every face-neighbour, the neighbour's face
    opposite the shared one: the straight extension along the principal axes
    that the text describes (flux along the principal conductivity axes), six
    new faces for an interior cell."""
    sysd = iso((5, 5, 4))
    qptr, qidx = O.qsets("thresh", sysd.A, sysd.B, sysd.C, 0.0)
    live = ~sysd.face_dir
    cf, fc = np.asarray(sysd.cell_faces), np.asarray(sysd.face_cells)
    ref = []
    for m in range(sysd.Ne):
        q = {f for f in cf[m] if live[f]}
        for k in range(6):  # local faces x-, x+, y-, y+, z-, z+
            f = cf[m][k]
            for e2 in fc[f]:
                if e2 >= 0 and e2 != m and live[f] and live[cf[e2][k]]:
                    q.add(int(cf[e2][k]))
        ref.append(sorted(q))
    assert sets_of(qptr, qidx) == ref
    centre = 2 + 5 * (2 + 5 * 1)
    assert len(ref[centre]) == 12
    # pattern E (all directions) reads as every face of the face-neighbours
    qptr_e, _ = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    assert np.diff(qptr_e)[centre] == 36


# ------------------------------------------------------------ local solves
@pytest.mark.parametrize("maker", [full_tensor, iso])
def test_all_faces_restriction_is_exact(maker):
    sysd = maker()
    Ad, Bd, Cd, Dd = (M.dense() for M in (sysd.A, sysd.B, sysd.C, sysd.D))
    qptr, qidx = all_faces_q(sysd)
    x, g = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx, True, True)
    X = x.reshape(sysd.Ne, sysd.Nf).T  # column m
    G = g.reshape(sysd.Ne, sysd.Nf)    # row m
    Xref = np.linalg.solve(Ad, Bd)
    Gref = -Cd @ np.linalg.inv(Ad)
    np.testing.assert_allclose(X, Xref, atol=1e-10 * np.abs(Xref).max())
    np.testing.assert_allclose(G, Gref, atol=1e-10 * np.abs(Gref).max())
    Sref = Dd - Cd @ Xref
    for form in (0, 1):
        S = O.schur(form, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g).to_scipy().toarray()
        np.testing.assert_allclose(S, Sref, atol=1e-10 * np.abs(Sref).max())


def test_galerkin_orthogonality_and_energy_minimality():
    # Proposition (min_energy): R (b - A R^T x) = 0 and x minimises ||A^{-1}b - R^T x||_{-A}
    sysd = full_tensor((3, 3, 3))
    Ad, Bd = sysd.A.dense(), sysd.B.dense()
    qptr, qidx = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx)
    rng = np.random.default_rng(1)
    Mspd = -Ad
    for m in range(sysd.Ne):
        q = qidx[qptr[m]:qptr[m + 1]]
        xt = np.zeros(sysd.Nf)
        xt[q] = x[qptr[m]:qptr[m + 1]]
        r = Bd[:, m] - Ad @ xt
        assert np.abs(r[q]).max() <= 1e-12 * max(np.abs(r).max(), np.abs(Bd[:, m]).max())
        ex = np.linalg.solve(Ad, Bd[:, m])
        e0 = ex - xt
        base = e0 @ Mspd @ e0
        for _ in range(3):
            d = np.zeros(sysd.Nf)
            d[q] = rng.normal(size=q.size) * 1e-3 * np.abs(xt).max()
            e1 = e0 - d
            assert e1 @ Mspd @ e1 > base


def test_own_faces_diagonal_K_closed_form():
    # isotropic K, own faces: A^(m) splits into three 2x2 axis blocks
    sysd = W.config1()
    Ad = sysd.A.to_scipy().tolil()
    Bd = sysd.B.to_scipy().tocsc()
    qptr, qidx = O.qsets("own", sysd.A, sysd.B, sysd.C)
    x, _ = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx)
    for m in range(0, sysd.Ne, 7):
        faces = list(sysd.cell_faces[m])
        for a in range(3):
            f0, f1 = faces[2 * a], faces[2 * a + 1]
            live = [f for f in (f0, f1) if not sysd.face_dir[f]]
            if len(live) == 2:
                a11, a12, a22 = Ad[f0, f0], Ad[f0, f1], Ad[f1, f1]
                b1, b2 = Bd[f0, m], Bd[f1, m]
                det = a11 * a22 - a12 * a12
                ref = {f0: (b1 * a22 - a12 * b2) / det, f1: (a11 * b2 - a12 * b1) / det}
            else:
                f = live[0]
                ref = {f: Bd[f, m] / Ad[f, f]}
            q = list(qidx[qptr[m]:qptr[m + 1]])
            for f, v in ref.items():
                assert x[qptr[m] + q.index(f)] == pytest.approx(v, rel=1e-12)


# ------------------------------------------------------------ ILU(0)
def dense_ilu0(M):
    """Textbook ILU(0) on a dense array restricted to M's pattern (IKJ)."""
    A = M.copy()
    P = M != 0
    n = A.shape[0]
    for i in range(1, n):
        for k in range(i):
            if not P[i, k]:
                continue
            A[i, k] /= A[k, k]
            for j in range(k + 1, n):
                if P[i, j]:
                    A[i, j] -= A[i, k] * A[k, j]
    return A


def test_ilu0_exact_when_no_fill():
    n = 30
    rng = np.random.default_rng(2)
    T = sp.diags([rng.uniform(-1, 0, n - 1), rng.uniform(3, 4, n), rng.uniform(-1, 0, n - 1)],
                 [-1, 0, 1], format="csr")
    lu = O.ilu0(T)
    r = rng.normal(size=n)
    np.testing.assert_allclose(O.ilu0_solve(T, lu, r), np.linalg.solve(T.toarray(), r), rtol=1e-12)
    Dn = rng.normal(size=(12, 12)) + 12 * np.eye(12)
    Dm = O.Mat.of(sp.csr_matrix(Dn))
    lu = O.ilu0(Dm)
    np.testing.assert_allclose(O.ilu0_solve(Dm, lu, r[:12]), np.linalg.solve(Dn, r[:12]), rtol=1e-11)


def test_ilu0_matches_textbook_on_sparse_pattern():
    sysd = full_tensor((3, 2, 2))
    M = sysd.A.to_scipy()
    lu = O.ilu0(sysd.A)
    ref = dense_ilu0(M.toarray())
    got = sp.csr_matrix((lu, sysd.A.col, sysd.A.rowptr), shape=M.shape).toarray()
    mask = M.toarray() != 0
    np.testing.assert_allclose(got[mask], ref[mask], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------ apply + FGMRES
def dense_mat(a):
    """CSR with every entry stored: ILU(0) on it is the exact LU factorisation."""
    n = a.shape[0]
    return O.Mat(n, a.shape[1], np.arange(n + 1) * a.shape[1], np.tile(np.arange(a.shape[1]), n), a.ravel())


@pytest.mark.parametrize("maker", [full_tensor, iso])
def test_exact_blocks_converge_in_one_iteration(maker):
    sysd = maker()
    Ad, Bd, Cd, Dd = (M.dense() for M in (sysd.A, sysd.B, sysd.C, sysd.D))
    S = Dd - Cd @ np.linalg.solve(Ad, Bd)
    b = W.Stream(3).normal(sysd.n)
    P = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=dense_mat(S), Ma=dense_mat(Ad), variant=0)
    r = O.fgmres(P, b, 50, 1e-10, 20)
    assert r["converged"] and r["iters"] == 1
    P2 = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=dense_mat(S), Ma=dense_mat(Ad), variant=1)
    r2 = O.fgmres(P2, b, 50, 1e-10, 20)
    assert r2["converged"] and r2["iters"] <= 2
    xd = np.linalg.solve(sysd.full_scipy().toarray(), b)
    np.testing.assert_allclose(r["x"], xd, atol=1e-8 * np.abs(xd).max())


def test_apply_matches_block_ldu_inverse():
    # Eq. (EDFA_prec) with exact blocks equals the inverse of the block system (Eq. inv_A_fac)
    sysd = full_tensor((2, 2, 2))
    Ad, Bd, Cd, Dd = (M.dense() for M in (sysd.A, sysd.B, sysd.C, sysd.D))
    S = Dd - Cd @ np.linalg.solve(Ad, Bd)
    P = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=dense_mat(S), Ma=dense_mat(Ad))
    Minv = np.linalg.inv(sysd.full_scipy().toarray())
    for k in range(3):
        r = W.Stream(10 + k).normal(sysd.n)
        np.testing.assert_allclose(P.apply(r), Minv @ r, atol=1e-9 * np.abs(Minv @ r).max())


def test_identity_preconditioner_is_gmres():
    sysd = iso((3, 2, 2))
    b = W.Stream(4).normal(sysd.n)
    P = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, identity=True)
    r = O.fgmres(P, b, 200, 1e-11, 400)
    assert r["converged"]
    xd = np.linalg.solve(sysd.full_scipy().toarray(), b)
    np.testing.assert_allclose(r["x"], xd, atol=1e-8 * np.abs(xd).max())
    assert np.all(np.diff(r["hist"]) <= 1e-14)  # GMRES residual is non-increasing within a cycle


def test_edfa_pipeline_converges_and_bigger_sets_help():
    # qualitative behaviour of Sec. 4: a larger restriction set gives fewer iterations
    sysd = full_tensor((6, 6, 6))
    it = {}
    for mode in ("own", "nbr"):
        r = O.edfa_pipeline(sysd, mode=mode, rtol=1e-8, maxit=600)
        assert r["converged"] and r["true_rel"] <= 1e-8
        it[mode] = r["iters"]
    assert it["nbr"] < it["own"]


# ------------------------------------------------------------ dynamic technique
def test_dynamic_first_step_adds_largest_residual_entries():
    sysd = full_tensor((3, 3, 3), seed=21)
    Ad, Cd = sysd.A.dense(), sysd.C.dense()
    for n_add in (1, 3):
        qptr, qidx = O.qsets_dynamic(sysd.A, sysd.C, n_add, n_add, 1)
        for m in range(sysd.Ne):
            q0 = list(np.nonzero(Cd[m])[0])
            M = -Ad[np.ix_(q0, q0)]
            g = np.linalg.solve(M, Cd[m, q0])
            r = Cd[m].copy()
            r += Ad[:, q0] @ g  # prolonged residual, Eq. (prol_res)
            cand = [j for j in range(sysd.Nf) if j not in q0 and np.any(Ad[j, q0] != 0)]
            picked = []
            for _ in range(n_add):
                left = [j for j in cand if j not in picked]
                if not left:
                    break
                rmax = max(abs(r[j]) for j in left)
                picked.append(min(j for j in left if abs(r[j]) >= rmax * (1 - 1e-12)))
            ref = sorted(q0 + picked)
            assert list(qidx[qptr[m]:qptr[m + 1]]) == ref
    qptr0, qidx0 = O.qsets_dynamic(sysd.A, sysd.C, 2, 0, 5)
    qptr1, qidx1 = O.qsets("crow", sysd.A, sysd.B, sysd.C)
    assert np.array_equal(qptr0, qptr1) and np.array_equal(qidx0, qidx1)


def test_dynamic_growth_bounds():
    sysd = full_tensor((3, 3, 2), seed=22)
    base, _ = O.qsets("crow", sysd.A, sysd.B, sysd.C)
    for n_add, n_ent, it_max in ((2, 6, 10), (4, 6, 1), (1, 5, 3)):
        qptr, qidx = O.qsets_dynamic(sysd.A, sysd.C, n_add, n_ent, it_max)
        grown = np.diff(qptr) - np.diff(base)
        assert grown.max() <= min(n_ent, n_add * it_max)
        assert grown.min() >= 0


# ------------------------------------------------------------ transpose / adjoint
def test_two_sided_schur_of_transposed_system_is_transpose():
    # On [A C^T; B^T D^T] the roles of F~ and G~ swap; with the same Q^(m) the
    # two-sided S~ is the transpose of the original one.
    sysd = full_tensor((3, 3, 2))
    qptr, qidx = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    x, g = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx, True, True)
    S = O.schur(1, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g).to_scipy().toarray()
    Bt = O.Mat.of(sysd.C.to_scipy().T.tocsr())
    Ct = O.Mat.of(sysd.B.to_scipy().T.tocsr())
    Dt = O.Mat.of(sysd.D.to_scipy().T.tocsr())
    xt, gt = O.local_solves(sysd.A, Bt, Ct, qptr, qidx, True, True)
    St = O.schur(1, sysd.A, Ct, Dt, qptr, qidx, xt, gt).to_scipy().toarray()
    np.testing.assert_allclose(St, S.T, atol=1e-12 * np.abs(S).max())


def test_adjoint_gradient_matches_finite_differences():
    n = (4, 3, 3)
    Ne = int(np.prod(n))
    logk = W.Stream(31).normal(Ne)
    obs = np.array([1, 7, 20, 33])

    def solve(lk):
        s = W.assemble(*n, W.iso_K(np.exp(lk)))
        M = s.full_scipy().toarray()
        return s, M, np.linalg.solve(M, s.f_phys)

    def loss(lk):
        s, _, u = solve(lk)
        return np.sum(u[s.Nf + obs] ** 2)

    s, M, u = solve(logk)
    dLdu = np.zeros(s.n)
    dLdu[s.Nf + obs] = 2 * u[s.Nf + obs]
    lam = np.linalg.solve(M.T, dLdu)
    g = O.adjoint_grad(s, u, lam, logk)
    h = 1e-6
    for e in (0, 5, 17, 35):
        lp, lm = logk.copy(), logk.copy()
        lp[e] += h
        lm[e] -= h
        fd = (loss(lp) - loss(lm)) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=1e-6, abs=1e-12)


# ------------------------------------------------------------ filtration
# Pre- and post-filtration (Sec. 3, implementation details; Algorithms 1 and
# 2): drop entries below tau times the Euclidean norm of their row (column of
# X~, row of G~, H~ or S~), the diagonal of H~ and S~ always kept.
def _pattern(M):
    return {(i, int(j)) for i in range(M.nrows) for j in M.col[M.rowptr[i]:M.rowptr[i + 1]]}


def _filter_dense_rows(M, struct, tau, keep_diag):
    """Zero the entries of dense M (structural mask struct) that the paper's
    rule discards; returns (values, mask)."""
    out = M.copy()
    mask = struct.copy()
    for i in range(M.shape[0]):
        lim = tau * np.sqrt(np.sum(M[i][struct[i]] ** 2))
        drop = struct[i] & (np.abs(M[i]) < lim)
        if keep_diag:
            drop[i] = False
        # no entry may sit at the threshold up to rounding, or the decision is fragile
        near = struct[i] & (np.abs(np.abs(M[i]) - lim) <= 1e-9 * max(lim, 1e-300))
        assert not near.any()
        out[i][drop] = 0.0
        mask[i][drop] = False
    return out, mask


@pytest.mark.parametrize("filt", ["pre", "post_h", "post_s"])
@pytest.mark.parametrize("form", [0, 1])
def test_filtration_zero_tolerance_is_unfiltered(filt, form):
    sysd = full_tensor()
    qptr, qidx = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    x, g = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx, True, True)
    S0 = O.schur(form, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g)
    S1, _ = O.schur_filtered(form, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g, filt, 0.0)
    assert np.array_equal(S0.rowptr, S1.rowptr) and np.array_equal(S0.col, S1.col)
    assert np.array_equal(S0.val, S1.val)


@pytest.mark.parametrize("tau", [1e-3, 3e-2])
def test_filtration_against_dense_definitions(tau):
    # Q^(m) = all faces: X~ = A^{-1} B exactly, so every filtered S~ has a dense
    # definition computed here from numpy solves
    sysd = full_tensor(n=(3, 2, 2), seed=21)
    Ad, Cd, Dd = (M.dense() for M in (sysd.A, sysd.C, sysd.D))
    Bd = sysd.B.dense()
    qptr, qidx = all_faces_q(sysd)
    x, g = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx, True, False)
    X = np.linalg.solve(Ad, Bd)
    Cs, Ds = Cd != 0, Dd != 0
    eye = np.eye(sysd.Ne, dtype=bool)
    # pre-filtration of the columns of X~ (no diagonal for an N_f x N_e block)
    Xf, Xm = _filter_dense_rows(X.T, np.ones_like(X.T, dtype=bool), tau, keep_diag=False)
    Xf, Xm = Xf.T, Xm.T
    H = Cd @ Xf
    Hs = (Cs.astype(int) @ Xm.astype(int)) > 0
    ref = {"pre": (Dd - H, Hs | Ds | eye)}
    # post-filtration of the rows of H~ = C X~
    H = Cd @ X
    Hs = (Cs.astype(int) @ np.ones_like(X, dtype=int)) > 0
    Hf, Hm = _filter_dense_rows(H, Hs, tau, keep_diag=True)
    ref["post_h"] = (Dd - Hf, Hm | Ds | eye)
    # post-filtration of the rows of S~ = D - H~
    S = Dd - H
    Sf, Sm = _filter_dense_rows(S, Hs | Ds | eye, tau, keep_diag=True)
    ref["post_s"] = (Sf, Sm)
    for filt, (Sref, Mref) in ref.items():
        Sg, _ = O.schur_filtered(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x, None, filt, tau)
        assert _pattern(Sg) == {(int(i), int(j)) for i, j in zip(*np.nonzero(Mref))}, filt
        np.testing.assert_allclose(Sg.to_scipy().toarray(), Sref, atol=1e-10 * np.abs(Sref).max())


def test_filtration_limits_and_monotonicity():
    sysd = full_tensor(n=(4, 3, 3), seed=8)
    qptr, qidx = O.qsets("nbr", sysd.A, sysd.B, sysd.C)
    x, g = O.local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx, True, True)
    S0 = O.schur(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g).to_scipy().toarray()
    Dd = sysd.D.dense()
    H0 = Dd - S0
    big = 1e30
    # tau -> infinity: post_s keeps the diagonal of S~ only
    Sg, _ = O.schur_filtered(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g, "post_s", big)
    assert np.array_equal(Sg.to_scipy().toarray(), np.diag(np.diag(S0)))
    # post_h keeps only the diagonal of H~: S~ = D - diag(H~) on pattern(D) u diagonal
    Sg, _ = O.schur_filtered(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g, "post_h", big)
    ref = Dd - np.diag(np.diag(H0))
    np.testing.assert_allclose(Sg.to_scipy().toarray(), ref, atol=1e-13 * np.abs(ref).max())
    assert _pattern(Sg) == {(int(i), int(j)) for i, j in zip(*np.nonzero((Dd != 0) | np.eye(sysd.Ne, dtype=bool)))}
    # pre-filtration that drops every entry of X~: S~ = D
    Sg, _ = O.schur_filtered(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g, "pre", big)
    assert np.array_equal(Sg.to_scipy().toarray(), Dd)
    # patterns shrink as tau grows
    for filt in ("pre", "post_h", "post_s"):
        prev = None
        for tau in (0.0, 1e-4, 1e-3, 1e-2, 1e-1):
            Sg, _ = O.schur_filtered(0, sysd.A, sysd.C, sysd.D, qptr, qidx, x, g, filt, tau)
            pat = _pattern(Sg)
            if prev is not None:
                assert pat <= prev, (filt, tau)
            prev = pat


# ------------------------------------------------------------ Bi-CGStab (Sec. 4)
def _bicgstab_textbook(Mv, Pinv, b, rtol, maxit):
    """Independent dense restatement of right-preconditioned Bi-CGStab (van der Vorst
    1992) for the pins below (no restarts); returns x, iterations and the history of
    ||r_k|| / ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    rh = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_old = alpha = omega = 1.0
    nb = np.linalg.norm(b)
    hist = [1.0]
    for it in range(1, maxit + 1):
        rho = rh @ r
        beta = rho / rho_old * alpha / omega
        p = r + beta * (p - omega * v)
        ph = Pinv(p)
        v = Mv(ph)
        alpha = rho / (rh @ v)
        s = r - alpha * v
        if np.linalg.norm(s) <= rtol * nb:
            hist.append(np.linalg.norm(s) / nb)
            return x + alpha * ph, it, np.array(hist)
        sh = Pinv(s)
        t = Mv(sh)
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / nb)
        if np.linalg.norm(r) <= rtol * nb:
            return x, it, np.array(hist)
    return x, maxit, np.array(hist)


@pytest.mark.parametrize("maker", [full_tensor, iso])
def test_bicgstab_exact_blocks_one_iteration(maker):
    # with the exact block LDU (Eq. inv_A_fac) the preconditioned operator is the
    # identity: p^ = A^{-1} r0, v = r0, alpha = 1, s = 0 -> one iteration
    sysd = maker()
    Ad, Bd, Cd, Dd = (M.dense() for M in (sysd.A, sysd.B, sysd.C, sysd.D))
    S = Dd - Cd @ np.linalg.solve(Ad, Bd)
    b = W.Stream(3).normal(sysd.n)
    P = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=dense_mat(S), Ma=dense_mat(Ad))
    r = O.bicgstab(P, b, 1e-10, 20)
    assert r["converged"] and r["iters"] == 1
    xd = np.linalg.solve(sysd.full_scipy().toarray(), b)
    np.testing.assert_allclose(r["x"], xd, atol=1e-8 * np.abs(xd).max())


def test_bicgstab_matches_dense_restatement_and_solution():
    # identity and EDFA preconditioners: the oracle's iterates follow the dense
    # restatement (same iteration count) and reach the dense solution
    sysd = iso((3, 3, 2))
    full = sysd.full_scipy().toarray()
    b = W.Stream(6).normal(sysd.n)
    xd = np.linalg.solve(full, b)
    P_id = O.Prec(sysd.A, sysd.B, sysd.C, sysd.D, identity=True)
    ref = O.edfa_pipeline(sysd, mode="nbr", solve=False)
    for P, exact_count in ((P_id, False), (ref["prec"], True)):
        r = O.bicgstab(P, b, 1e-11, 1000)
        xt, itt, ht = _bicgstab_textbook(lambda z: full @ z, P.apply, b, 1e-11, 1000)
        assert r["converged"]
        # the first iterates agree with the restatement (rounding then lets the erratic
        # unpreconditioned trajectories drift apart, so only the EDFA count is compared)
        k = min(8 if exact_count else 5, len(ht), len(r["hist"]))
        np.testing.assert_allclose(r["hist"][:k], ht[:k], rtol=1e-6)
        if exact_count:
            assert abs(r["iters"] - itt) <= 1, (r["iters"], itt)
        np.testing.assert_allclose(r["x"], xd, atol=1e-8 * np.abs(xd).max())
        assert r["true_rel"] <= 1e-11


def test_bicgstab_edfa_workload_converges():
    sysd = W.brick(6, seed=3)
    ref = O.edfa_pipeline(sysd, mode="nbr", solve=False)
    r = O.bicgstab(ref["prec"], sysd.b, 1e-8, 2000)
    assert r["converged"] and r["true_rel"] <= 1e-8
    res = np.linalg.norm(sysd.full_scipy() @ r["x"] - sysd.b) / np.linalg.norm(sysd.b)
    assert res <= 1.05e-8


def test_local_solves_do_not_depend_on_thread_count():
    """The per-cell loop may run on several threads (the paper's parallel loop
    over cells); every cell's arithmetic is unchanged, so X~ and G~ are equal
    bit for bit."""
    s = W.config2(10)
    q = O.qsets("nbr", s.A, s.B, s.C)
    x1, g1 = O.local_solves(s.A, s.B, s.C, *q, want_g=True)
    try:
        O.set_threads(4)
        x4, g4 = O.local_solves(s.A, s.B, s.C, *q, want_g=True)
    finally:
        O.set_threads(1)
    assert np.array_equal(x1, x4) and np.array_equal(g1, g4)


# ------------------------------------------------ multicolour ordering
_M64 = (1 << 64) - 1


def _splitmix_finaliser(v):
    """SplitMix64 finaliser of v + 1 (Steele, Lea & Flood 2014), retyped here
    from its published definition in Python integers."""
    z = ((v + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _ordering_cases():
    s = W.config2(7)
    q = O.qsets("nbr", s.A, s.B, s.C)
    x, _ = O.local_solves(s.A, s.B, s.C, *q)
    S = O.schur(0, s.A, s.C, s.D, *q, x)
    c3 = W.config3(12, 10, 6)
    q3 = O.qsets("thresh", c3.A, c3.B, c3.C, 0.05)
    x3, _ = O.local_solves(c3.A, c3.B, c3.C, *q3)
    S3 = O.schur(0, c3.A, c3.C, c3.D, *q3, x3)
    return [("A full-tensor", s.A.to_scipy()), ("S~ full-tensor", S.to_scipy()),
            ("A channelised", c3.A.to_scipy()), ("S~ channelised", S3.to_scipy())]


def test_multicolour_ordering_is_the_jones_plassmann_colouring():
    """Every vertex of the graph of M + M^T has the smallest colour that none of
    its higher-priority neighbours has (the fixed point of Jones & Plassmann's
    parallel colouring), which makes the colouring proper; the ordering sorts
    rows by (colour, index)."""
    import scipy.sparse as sp
    for name, M in _ordering_cases():
        colour, perm, nc = O.colour_order(M)
        G = ((abs(M) + abs(M.T)) != 0).astype(np.int8).tocsr()
        n = M.shape[0]
        pri = [_splitmix_finaliser(v) for v in range(n)]
        for v in range(n):
            nb = [u for u in G.indices[G.indptr[v]:G.indptr[v + 1]] if u != v]
            assert all(colour[u] != colour[v] for u in nb), (name, v)
            higher = {int(colour[u]) for u in nb if pri[u] > pri[v]}
            mex = 0
            while mex in higher:
                mex += 1
            assert colour[v] == mex, (name, v)
        assert nc == colour.max() + 1
        assert np.array_equal(perm, np.lexsort((np.arange(n), colour)))
        # no edge inside a colour: the lower triangle of P M P^T has at most
        # nc dependency levels (longest chain of strictly decreasing columns)
        Pm = sp.csr_matrix(M)[perm][:, perm].tocsr()
        L = sp.tril(Pm, -1).tocsr()
        lev = np.zeros(n, int)
        for i in range(n):
            js = L.indices[L.indptr[i]:L.indptr[i + 1]]
            lev[i] = lev[js].max() + 1 if len(js) else 0
        assert lev.max() + 1 <= nc


@pytest.mark.parametrize("block", [2, 3, 8])
def test_block_multicolour_ordering(block):
    """Blocks of `block` consecutive rows coloured as units: every block has the
    smallest colour none of its higher-priority neighbouring blocks has (the
    block graph and the greedy rule restated here with scipy), row r of block B
    has colour c(B) * block + r - B * block, and rows are sorted by (colour,
    index).  The rows of one colour are then independent, and the ILU(0) of
    this ordering equals (to rounding) the ILU(0) of the ordering by (block
    colour, block, position): the two orders agree on every coupled pair."""
    import scipy.sparse as sp
    for name, M in _ordering_cases():
        n = M.shape[0]
        colour, perm, nc = O.colour_order(M, block)
        nb = (n + block - 1) // block
        blk = np.arange(n) // block
        Pm = sp.csr_matrix((np.ones(n), (blk, np.arange(n))), shape=(nb, n))
        G = ((abs(M) + abs(M.T)) != 0).astype(np.int8)
        Q = (Pm @ G @ Pm.T).tocsr()
        pri = [_splitmix_finaliser(B) for B in range(nb)]
        bcol = np.full(nb, -1)
        for B in sorted(range(nb), key=lambda x: -pri[x]):
            used = {int(bcol[U]) for U in Q.indices[Q.indptr[B]:Q.indptr[B + 1]] if U != B and bcol[U] >= 0}
            c = 0
            while c in used:
                c += 1
            bcol[B] = c
        ref = bcol[blk] * block + np.arange(n) % block
        assert np.array_equal(colour, ref), name
        assert nc == colour.max() + 1
        assert np.array_equal(perm, np.lexsort((np.arange(n), colour)))
        Gc = G.tocsr()
        rows = np.repeat(np.arange(n), np.diff(Gc.indptr))
        off = rows != Gc.indices
        assert not np.any(colour[rows[off]] == colour[Gc.indices[off]]), name
        # the same preconditioner as the (block colour, block, position) order
        p1 = np.lexsort((np.arange(n), blk, bcol[blk])).astype(np.int32)
        M1 = O.permute(M, p1)
        M2 = O.permute(M, perm)
        lu1 = sp.csr_matrix((O.ilu0(M1), M1.col, M1.rowptr), shape=(n, n))
        lu2 = sp.csr_matrix((O.ilu0(M2), M2.col, M2.rowptr), shape=(n, n))
        back = np.empty(n, np.int64)
        back[p1] = np.arange(n)
        to1 = back[perm]  # position in order 1 of the k-th row of order 2
        lu2_in1 = sp.csr_matrix(lu2)[np.argsort(to1)][:, np.argsort(to1)].toarray()
        d1 = lu1.toarray()
        assert np.abs(d1 - lu2_in1).max() <= 1e-12 * np.abs(d1).max(), name


def test_permute_matches_scipy_fancy_indexing():
    for name, M in _ordering_cases():
        _, perm, _ = O.colour_order(M)
        Pm = O.permute(M, perm)
        ref = M.tocsr()[perm][:, perm].tocsr()
        ref.sort_indices()
        assert np.array_equal(Pm.rowptr, ref.indptr) and np.array_equal(Pm.col, ref.indices), name
        assert np.array_equal(Pm.val, ref.data), name


def test_ordered_apply_is_the_natural_apply_of_the_permuted_system():
    """With orderings P_a (faces) and P_s (cells), the preconditioner applied to
    r equals the natural-order preconditioner of the permuted system
    [P_a A P_a^T, P_a B P_s^T; P_s C P_a^T, P_s D P_s^T] (blocks permuted by
    scipy) applied to the permuted r, permuted back."""
    s = W.config2(7)
    q = O.qsets("nbr", s.A, s.B, s.C)
    x, _ = O.local_solves(s.A, s.B, s.C, *q)
    S = O.schur(0, s.A, s.C, s.D, *q, x)
    _, pa, _ = O.colour_order(s.A)
    _, ps, _ = O.colour_order(S)
    r = W.Stream(77).normal(s.n)
    for variant in (0, 1):
        z = O.Prec(s.A, s.B, s.C, s.D, S=S, variant=variant, aperm=pa, sperm=ps).apply(r)
        A, B, C_, D, Ss = (M.to_scipy().tocsr() for M in (s.A, s.B, s.C, s.D, S))
        Pq = O.Prec(A[pa][:, pa], B[pa][:, ps], C_[ps][:, pa], D[ps][:, ps], S=Ss[ps][:, ps], variant=variant)
        zq = Pq.apply(np.concatenate([r[:s.Nf][pa], r[s.Nf:][ps]]))
        zr = np.empty_like(zq)
        zr[pa] = zq[:s.Nf]
        zr[s.Nf + ps] = zq[s.Nf:]
        assert np.abs(z - zr).max() <= 1e-12 * np.abs(zr).max(), variant


def test_fgmres_on_the_permuted_system_is_the_same_iteration():
    """FGMRES with the ordered preconditioner on the natural system and FGMRES on
    the permuted system (blocks and right-hand side permuted, the natural-order
    preconditioner of the permuted blocks) take the same iterations: inner
    products and norms are permutation invariant, so the residual estimates
    agree to rounding and the solutions are permutations of each other."""
    s = W.config3(16, 12, 6)
    q = O.qsets("thresh", s.A, s.B, s.C, 0.05)
    x, _ = O.local_solves(s.A, s.B, s.C, *q)
    S = O.schur(0, s.A, s.C, s.D, *q, x)
    _, pa, _ = O.colour_order(s.A)
    _, ps, _ = O.colour_order(S, 4)
    r1 = O.fgmres(O.Prec(s.A, s.B, s.C, s.D, S=S, aperm=pa, sperm=ps), s.b, 50, 1e-8, 2000)
    A, B, C_, D, Ss = (M.to_scipy().tocsr() for M in (s.A, s.B, s.C, s.D, S))
    Pq = O.Prec(A[pa][:, pa], B[pa][:, ps], C_[ps][:, pa], D[ps][:, ps], S=Ss[ps][:, ps])
    bq = np.concatenate([s.b[:s.Nf][pa], s.b[s.Nf:][ps]])
    r2 = O.fgmres(Pq, bq, 50, 1e-8, 2000)
    assert r1["converged"] and r2["converged"]
    assert abs(r1["iters"] - r2["iters"]) <= 1
    k = min(len(r1["hist"]), len(r2["hist"]), 51)
    assert np.allclose(r1["hist"][:k], r2["hist"][:k], rtol=1e-8, atol=0)
    xb = np.empty_like(r2["x"])
    xb[pa] = r2["x"][:s.Nf]
    xb[s.Nf + ps] = r2["x"][s.Nf:]
    assert np.linalg.norm(xb - r1["x"]) <= 1e-6 * np.linalg.norm(r1["x"])


def test_ordered_preconditioner_fgmres_converges():
    for sysd, mode in ((W.config2(10), "nbr"), (W.config3(16, 12, 6), "thresh")):
        for ordering in (1, 2):
            r = O.edfa_pipeline(sysd, mode=mode, ordering=ordering)
            assert r["converged"] and r["true_rel"] <= 1e-8, (mode, ordering, r["true_rel"])


def test_config1_own_face_sets_give_a_schur_approximation_with_negative_spectrum():
    """Workload 1 (weak-form cell rows with upwind face mobilities) stalls with
    own-face sets under either reading of "C = -(upwind mobility) B^T":
    C_Ej = -lambda_j B_jE (the one the generator uses) or the flux-weighted
    C_Ej = -sum_{f in F_E} lambda_f W^E_fj (same D).  With Q^(m) = the cell's
    own faces, S~ = D - C X~ has eigenvalues with negative real part in both,
    so the block preconditioner is indefinite (FGMRES(50) does not reach 1e-8);
    the exact Schur complement of the flux-weighted form has none, and
    neighbour-face sets converge for both."""
    import scipy.sparse as sp
    s = W.config1()
    st = W.Stream(1)
    Ne, nx = 1000, 10
    W.wexp(st.normal(Ne))
    lam = W.wexp(0.5 * st.normal(Ne))
    tmp = W.assemble(nx, nx, nx, W.iso_K(np.ones(Ne)))
    lam_f = W._face_upwind_mobility(nx, nx, nx, lam, st.uniform(tmp.Nf), tmp.face_cells)
    assert np.allclose(lam, s.extra["lam_cell"])
    Wm, cf = s.W.reshape(Ne, 6, 6), s.cell_faces
    rows, cols, vals = [], [], []
    for e in range(Ne):
        for j in range(6):
            if not s.face_dir[cf[e, j]]:
                rows.append(e)
                cols.append(cf[e, j])
                vals.append(-sum(lam_f[cf[e, l]] * Wm[e, l, j] for l in range(6)))
    Cw = sp.csr_matrix((vals, (rows, cols)), shape=(Ne, s.Nf))
    Cw.sort_indices()
    A, B, D = (M.to_scipy().toarray() for M in (s.A, s.B, s.D))
    for C in (s.C.to_scipy(), Cw):
        s2 = W.System(**{**s.__dict__, "C": W.CSR(Ne, s.Nf, C.indptr.astype(np.int64),
                                                  C.indices.astype(np.int32), C.data)})
        r = O.edfa_pipeline(s2, mode="own", solve=False)
        ev = np.linalg.eigvals(r["S"].to_scipy().toarray())
        assert (ev.real < 0).sum() >= 10
        assert O.edfa_pipeline(s2, mode="nbr", maxit=1000)["converged"]
    S_exact = D - Cw.toarray() @ np.linalg.solve(A, B)
    assert np.linalg.eigvals(S_exact).real.min() > 0
