"""EDFA oracle: plain FP64 CPU implementation of the preconditioner hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package; the product path
never does.  The arithmetic lives in ``oracle.c`` (plain loops, built on first
use with gcc); this file only marshals numpy arrays.  It shares no code with
the CUDA library.

Paper: Nardean, Ferronato, Abushaikha, arXiv 2009.13916.
  * restriction sets: Sec. 3 (Eq. r_r^m, static and dynamic techniques, Algorithm 1)
  * restricted local solves: Eq. syst_MRHS_res, Eq. syst_MRHS_res-F
  * approximate Schur complement: Eq. sparse_S
  * preconditioner application: Eq. EDFA_prec, Remark 1
  * outer Krylov stopping rule: Sec. 4 (||r_k||/||r_0|| <= tau, x0 = 0)
  * outer Krylov methods: flexible GMRES(m) and Bi-CGStab (the paper's, Sec. 4)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")

QMODES = {"own": 0, "nbr": 1, "crow": 2, "thresh": 3}


def build(force: bool = False) -> str:
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_SO))
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fvisibility=hidden",
                           "-ffp-contract=off", "-fopenmp", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _CSR(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class _Prec(C.Structure):
    _fields_ = [("A", _CSR), ("B", _CSR), ("C", _CSR), ("D", _CSR), ("Ma", _CSR),
                ("lua", C.c_void_p), ("Ms", _CSR), ("lus", C.c_void_p),
                ("variant", C.c_int), ("identity", C.c_int),
                ("aperm", C.c_void_p), ("sperm", C.c_void_p), ("own_a", _CSR), ("own_s", _CSR)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        L.orc_free_csr.argtypes = [P(_CSR)]
        L.orc_qsets.argtypes = [C.c_int, C.c_double, P(_CSR), P(_CSR), P(_CSR),
                                P(C.c_void_p), P(C.c_void_p)]
        L.orc_qsets_dynamic.argtypes = [P(_CSR), P(_CSR), C.c_int, C.c_int, C.c_int,
                                        P(C.c_void_p), P(C.c_void_p)]
        L.orc_local_solves.argtypes = [P(_CSR), P(_CSR), P(_CSR), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, P(C.c_int32)]
        L.orc_schur.argtypes = [C.c_int, P(_CSR), P(_CSR), P(_CSR), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, P(_CSR)]
        L.orc_filter_vectors.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                         P(C.c_void_p), P(C.c_void_p), P(C.c_void_p)]
        L.orc_filter_rows.argtypes = [P(_CSR), C.c_double, P(_CSR)]
        L.orc_htilde.argtypes = [C.c_int, P(_CSR), P(_CSR), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, P(_CSR)]
        L.orc_d_minus_h.argtypes = [P(_CSR), P(_CSR), P(_CSR)]
        L.orc_ilu0.argtypes = [P(_CSR), C.c_void_p, P(C.c_int32)]
        L.orc_ilu0_solve.argtypes = [P(_CSR), C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_ilu0_solve.restype = None
        L.orc_apply.argtypes = [P(_Prec), C.c_void_p, C.c_void_p]
        L.orc_apply.restype = None
        L.orc_fgmres.argtypes = [P(_Prec), C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                                 P(C.c_int), C.c_void_p, P(C.c_double)]
        L.orc_bicgstab.argtypes = [P(_Prec), C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                   P(C.c_int), C.c_void_p, P(C.c_double)]
        L.orc_prec_setup.argtypes = [P(_Prec), P(_CSR), P(_CSR), P(_CSR), P(_CSR), P(_CSR),
                                     P(_CSR), C.c_int, C.c_int, P(C.c_int32)]
        L.orc_prec_setup_ordered.argtypes = [P(_Prec), P(_CSR), P(_CSR), P(_CSR), P(_CSR), P(_CSR),
                                             P(_CSR), C.c_int, C.c_int, C.c_void_p, C.c_void_p, P(C.c_int32)]
        L.orc_colour_order.argtypes = [P(_CSR), C.c_void_p, C.c_void_p, P(C.c_int32)]
        L.orc_block_colour_order.argtypes = [P(_CSR), C.c_int32, C.c_void_p, C.c_void_p, P(C.c_int32)]
        L.orc_permute.argtypes = [P(_CSR), C.c_void_p, P(_CSR)]
        L.orc_prec_free.argtypes = [P(_Prec)]
        L.orc_prec_free.restype = None
        L.orc_prec_sizeof.restype = C.c_int
        L.orc_adjoint_grad.argtypes = [C.c_int32, C.c_int32] + [C.c_void_p] * 9
        for name in ("orc_qsets", "orc_qsets_dynamic", "orc_local_solves", "orc_schur",
                     "orc_ilu0", "orc_fgmres", "orc_prec_setup", "orc_adjoint_grad",
                     "orc_prec_setup_ordered", "orc_colour_order", "orc_block_colour_order", "orc_permute"):
            getattr(L, name).restype = C.c_int
        assert L.orc_prec_sizeof() == C.sizeof(_Prec)
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads of the per-cell local-solve loop (1 by default; results do not
    depend on it)."""
    lib().orc_set_threads(int(n))


def _ptr(a):
    return a.ctypes.data if a is not None else None


class Mat:
    """CSR view held alive together with its ctypes descriptor."""

    def __init__(self, nrows, ncols, rowptr, col, val):
        self.nrows, self.ncols = int(nrows), int(ncols)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.c = _CSR(self.nrows, self.ncols, int(self.rowptr[-1]), _ptr(self.rowptr),
                      _ptr(self.col), _ptr(self.val))

    @classmethod
    def of(cls, M):
        if isinstance(M, Mat):
            return M
        if hasattr(M, "rowptr"):
            return cls(M.nrows, M.ncols, M.rowptr, M.col, M.val)
        M = M.tocsr()
        M.sort_indices()
        return cls(M.shape[0], M.shape[1], M.indptr, M.indices, M.data)

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.nrows, self.ncols))


def _take_int(p, n, dtype):
    ct = C.c_int64 if dtype == np.int64 else C.c_int32
    if n == 0:
        out = np.zeros(0, dtype)
    else:
        out = np.ctypeslib.as_array(C.cast(p, C.POINTER(ct)), shape=(n,)).copy()
    lib().orc_free(p)
    return out


def qsets(mode, A, B, C_, thresh=0.05):
    """Static restriction sets (own / nbr / crow / thresh).  Returns (qptr, qidx)."""
    A, B, C_ = Mat.of(A), Mat.of(B), Mat.of(C_)
    pq, pi = C.c_void_p(), C.c_void_p()
    rc = lib().orc_qsets(QMODES[mode], float(thresh), C.byref(A.c), C.byref(B.c), C.byref(C_.c),
                         C.byref(pq), C.byref(pi))
    if rc:
        raise RuntimeError(f"orc_qsets failed ({rc})")
    Ne = B.ncols
    qptr = _take_int(pq, Ne + 1, np.int64)
    qidx = _take_int(pi, int(qptr[-1]), np.int32)
    return qptr, qidx


def qsets_dynamic(A, C_, n_add, n_ent, it_max):
    """Dynamic restriction sets grown by the prolonged residual (Algorithm 1)."""
    A, C_ = Mat.of(A), Mat.of(C_)
    pq, pi = C.c_void_p(), C.c_void_p()
    rc = lib().orc_qsets_dynamic(C.byref(A.c), C.byref(C_.c), int(n_add), int(n_ent), int(it_max),
                                 C.byref(pq), C.byref(pi))
    if rc:
        raise RuntimeError(f"orc_qsets_dynamic failed ({rc})")
    qptr = _take_int(pq, C_.nrows + 1, np.int64)
    qidx = _take_int(pi, int(qptr[-1]), np.int32)
    return qptr, qidx


def local_solves(A, B, C_, qptr, qidx, want_x=True, want_g=False):
    """X~ (column m on Q^(m)) and G~ (row m on Q^(m)) from the restricted solves."""
    A, B, C_ = Mat.of(A), Mat.of(B), Mat.of(C_)
    qptr = np.ascontiguousarray(qptr, np.int64)
    qidx = np.ascontiguousarray(qidx, np.int32)
    n = int(qptr[-1])
    x = np.zeros(n) if want_x else None
    g = np.zeros(n) if want_g else None
    bad = C.c_int32(-1)
    rc = lib().orc_local_solves(C.byref(A.c), C.byref(B.c), C.byref(C_.c), _ptr(qptr), _ptr(qidx),
                                _ptr(x), _ptr(g), C.byref(bad))
    if rc:
        raise RuntimeError(f"orc_local_solves failed ({rc}) at cell {bad.value}")
    return x, g


def schur(form, A, C_, D, qptr, qidx, xval, gval=None) -> Mat:
    """S~ = D - C X~ (form 0) or S~ = D - G~ A F~ (form 1)."""
    A, C_, D = Mat.of(A), Mat.of(C_), Mat.of(D)
    qptr = np.ascontiguousarray(qptr, np.int64)
    qidx = np.ascontiguousarray(qidx, np.int32)
    xval = np.ascontiguousarray(xval, np.float64)
    gval = None if gval is None else np.ascontiguousarray(gval, np.float64)
    out = _CSR()
    rc = lib().orc_schur(int(form), C.byref(A.c), C.byref(C_.c), C.byref(D.c), _ptr(qptr), _ptr(qidx),
                         _ptr(xval), _ptr(gval), C.byref(out))
    if rc:
        raise RuntimeError(f"orc_schur failed ({rc})")
    n, ncols, nnz = out.nrows, out.ncols, out.nnz
    rp = np.ctypeslib.as_array(C.cast(out.rowptr, C.POINTER(C.c_int64)), shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(C.cast(out.col, C.POINTER(C.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(C.cast(out.val, C.POINTER(C.c_double)), shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free_csr(C.byref(out))
    return Mat(n, ncols, rp, col, val)


def _take_csr(out) -> Mat:
    n, ncols, nnz = out.nrows, out.ncols, out.nnz
    rp = np.ctypeslib.as_array(C.cast(out.rowptr, C.POINTER(C.c_int64)), shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(C.cast(out.col, C.POINTER(C.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(C.cast(out.val, C.POINTER(C.c_double)), shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free_csr(C.byref(out))
    return Mat(n, ncols, rp, col, val)


def filter_vectors(ptr, idx, val, tau):
    """Pre-filtration (Algorithm 1): drop entries of each segment (column of
    X~ or row of G~) with |v| < tau * ||segment||_2."""
    ptr = np.ascontiguousarray(ptr, np.int64)
    idx = np.ascontiguousarray(idx, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    nseg = len(ptr) - 1
    op, oi, ov = C.c_void_p(), C.c_void_p(), C.c_void_p()
    rc = lib().orc_filter_vectors(nseg, _ptr(ptr), _ptr(idx), _ptr(val), float(tau),
                                  C.byref(op), C.byref(oi), C.byref(ov))
    if rc:
        raise RuntimeError("orc_filter_vectors failed")
    optr = _take_int(op, nseg + 1, np.int64)
    n = int(optr[-1])
    oidx = _take_int(oi, n, np.int32)
    oval = np.ctypeslib.as_array(C.cast(ov, C.POINTER(C.c_double)), shape=(max(n, 1),))[:n].copy()
    lib().orc_free(ov)
    return optr, oidx, oval


def filter_rows(M, tau) -> Mat:
    """Post-filtration (Algorithms 1 and 2): drop off-diagonal entries with
    |m_ij| < tau * ||row i||_2."""
    M = Mat.of(M)
    out = _CSR()
    if lib().orc_filter_rows(C.byref(M.c), float(tau), C.byref(out)):
        raise RuntimeError("orc_filter_rows failed")
    return _take_csr(out)


def htilde(form, A, C_, Ne, xptr, xidx, xval, gptr=None, gidx=None, gval=None) -> Mat:
    """H~ = C X~ (form 0) or G~ A F~ (form 1) on its structural pattern."""
    A, C_ = Mat.of(A), Mat.of(C_)
    xptr = np.ascontiguousarray(xptr, np.int64)
    xidx = np.ascontiguousarray(xidx, np.int32)
    xval = np.ascontiguousarray(xval, np.float64)
    if gval is not None:
        gptr = np.ascontiguousarray(gptr, np.int64)
        gidx = np.ascontiguousarray(gidx, np.int32)
        gval = np.ascontiguousarray(gval, np.float64)
    out = _CSR()
    rc = lib().orc_htilde(int(form), C.byref(A.c), C.byref(C_.c), int(Ne), _ptr(xptr), _ptr(xidx), _ptr(xval),
                          _ptr(gptr), _ptr(gidx), _ptr(gval), C.byref(out))
    if rc:
        raise RuntimeError("orc_htilde failed")
    return _take_csr(out)


def d_minus_h(D, H) -> Mat:
    """S~ = D - H~ on pattern(H~) u pattern(D) u diagonal (Algorithm 2)."""
    D, H = Mat.of(D), Mat.of(H)
    out = _CSR()
    if lib().orc_d_minus_h(C.byref(D.c), C.byref(H.c), C.byref(out)):
        raise RuntimeError("orc_d_minus_h failed")
    return _take_csr(out)


FILTERS = {"none": 0, "pre": 1, "post_h": 2, "post_s": 3}


def schur_filtered(form, A, C_, D, qptr, qidx, xval, gval=None, filt="none", tau=0.0):
    """S~ with one of the paper's filtrations (Sec. 3, Algorithms 1 and 2):
    'pre' filters every X~ column (and G~ row) before H~ is formed, 'post_h'
    filters the rows of H~ (Stage 1), 'post_s' the rows of S~ (Stage 2).
    Returns (S~, H~ after filtration)."""
    Ne = D.nrows
    xptr, xidx, xv = qptr, qidx, xval
    gptr, gidx, gv = (qptr, qidx, gval) if form == 1 else (None, None, None)
    if filt == "pre":
        xptr, xidx, xv = filter_vectors(qptr, qidx, xval, tau)
        if form == 1:
            gptr, gidx, gv = filter_vectors(qptr, qidx, gval, tau)
    H = htilde(form, A, C_, Ne, xptr, xidx, xv, gptr, gidx, gv)
    if filt == "post_h":
        H = filter_rows(H, tau)
    S = d_minus_h(D, H)
    if filt == "post_s":
        S = filter_rows(S, tau)
    return S, H


def ilu0(M):
    M = Mat.of(M)
    lu = np.empty(M.nnz)
    bad = C.c_int32(-1)
    rc = lib().orc_ilu0(C.byref(M.c), _ptr(lu), C.byref(bad))
    if rc:
        raise RuntimeError(f"orc_ilu0 failed ({rc}) at row {bad.value}")
    return lu


def ilu0_solve(M, lu, r):
    M = Mat.of(M)
    r = np.ascontiguousarray(r, np.float64)
    z = np.empty_like(r)
    lib().orc_ilu0_solve(C.byref(M.c), _ptr(lu), _ptr(r), _ptr(z))
    return z


class Prec:
    """Preconditioner record: the system blocks, ILU(0) of Ma (for A~^{-1}) and of S~."""

    def __init__(self, A, B, C_, D, S=None, Ma=None, variant=0, identity=False, aperm=None, sperm=None):
        self.A, self.B, self.C, self.D = Mat.of(A), Mat.of(B), Mat.of(C_), Mat.of(D)
        self.Ma = self.A if Ma is None else Mat.of(Ma)
        self.S = None if S is None else Mat.of(S)
        self.aperm = None if aperm is None else np.ascontiguousarray(aperm, dtype=np.int32)
        self.sperm = None if sperm is None else np.ascontiguousarray(sperm, dtype=np.int32)
        self.p = _Prec()
        bad = C.c_int32(-1)
        Sc = self.S.c if self.S is not None else _CSR()
        rc = lib().orc_prec_setup_ordered(C.byref(self.p), C.byref(self.A.c), C.byref(self.B.c),
                                          C.byref(self.C.c), C.byref(self.D.c), C.byref(self.Ma.c),
                                          C.byref(Sc), int(variant), 1 if identity else 0,
                                          _ptr(self.aperm), _ptr(self.sperm), C.byref(bad))
        if rc:
            raise RuntimeError(f"orc_prec_setup failed ({rc}) at row {bad.value}")
        self._owned = not identity

    def __del__(self):
        try:
            if self._owned:
                lib().orc_prec_free(C.byref(self.p))
        except Exception:
            pass

    @property
    def n(self):
        return self.A.nrows + self.D.nrows

    def apply(self, r):
        r = np.ascontiguousarray(r, np.float64)
        z = np.empty_like(r)
        lib().orc_apply(C.byref(self.p), _ptr(r), _ptr(z))
        return z

    def lua(self):
        return np.ctypeslib.as_array(C.cast(self.p.lua, C.POINTER(C.c_double)), shape=(self.Ma.nnz,)).copy()

    def ordered_factor(self, which="s"):
        """(pattern, ILU(0) values) of the factorised matrix (ordered when an
        ordering was given): which = "a" (A~) or "s" (S~)."""
        M = self.p.Ma if which == "a" else self.p.Ms
        lu = self.p.lua if which == "a" else self.p.lus
        nnz = int(M.nnz)
        g = lambda ptr, n, t: np.ctypeslib.as_array(C.cast(ptr, C.POINTER(t)), shape=(n,)).copy()
        pat = Mat(M.nrows, M.ncols, g(M.rowptr, M.nrows + 1, C.c_int64), g(M.col, nnz, C.c_int32),
                  g(M.val, nnz, C.c_double))
        return pat, g(lu, nnz, C.c_double)

    def lus(self):
        return np.ctypeslib.as_array(C.cast(self.p.lus, C.POINTER(C.c_double)), shape=(self.S.nnz,)).copy()


def colour_order(M, block=1):
    """Multicolour ordering of the graph of M + M^T (the oracle's colouring):
    returns (colour per row, perm with rows sorted by (colour, index), number
    of colours).  block > 1: the block multicolour ordering, blocks of `block`
    consecutive rows coloured as units, row r of block B taking the colour
    c(B) * block + (r - B * block)."""
    M = Mat.of(M)
    colour = np.empty(M.nrows, np.int32)
    perm = np.empty(M.nrows, np.int32)
    nc = C.c_int32(0)
    rc = lib().orc_block_colour_order(C.byref(M.c), int(block), _ptr(colour), _ptr(perm), C.byref(nc))
    if rc:
        raise RuntimeError("orc_block_colour_order failed")
    return colour, perm, int(nc.value)


def permute(M, perm) -> Mat:
    """P M P^T (row k = row perm[k] of M, columns renamed and sorted)."""
    M = Mat.of(M)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    out = _CSR()
    rc = lib().orc_permute(C.byref(M.c), _ptr(perm), C.byref(out))
    if rc:
        raise RuntimeError("orc_permute failed")
    return _take_csr(out)


def fgmres(prec: Prec, b, restart=50, rtol=1e-8, maxit=2000):
    """Right-preconditioned FGMRES(restart), x0 = 0.  Returns dict with x,
    iterations, converged flag, residual-estimate history and true residual."""
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    hist = np.zeros(maxit + 1)
    it = C.c_int(0)
    tr = C.c_double(np.nan)
    rc = lib().orc_fgmres(C.byref(prec.p), _ptr(b), _ptr(x), int(restart), float(rtol), int(maxit),
                          C.byref(it), _ptr(hist), C.byref(tr))
    if rc < 0:
        raise RuntimeError(f"orc_fgmres failed ({rc})")
    return dict(x=x, iters=it.value, converged=(rc == 0), hist=hist[: it.value + 1],
                true_rel=tr.value)


def bicgstab(prec: Prec, b, rtol=1e-8, maxit=2000):
    """Right-preconditioned Bi-CGStab, x0 = 0 (the paper's outer solver, Sec. 4).
    Returns dict with x, iterations (two preconditioner applications each),
    converged flag, residual history and true residual."""
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    hist = np.zeros(maxit + 1)
    it = C.c_int(0)
    tr = C.c_double(np.nan)
    rc = lib().orc_bicgstab(C.byref(prec.p), _ptr(b), _ptr(x), float(rtol), int(maxit), C.byref(it),
                            _ptr(hist), C.byref(tr))
    if rc < 0:
        raise RuntimeError(f"orc_bicgstab failed ({rc})")
    return dict(x=x, iters=it.value, converged=(rc == 0), hist=hist[: it.value + 1], true_rel=tr.value)


def adjoint_grad(sysd, u, lam, logk):
    """dL/dlog k_E for isotropic K (rows of Appendix A differentiated by dual numbers)."""
    k = np.exp(logk)
    W1 = np.ascontiguousarray(sysd.W / k[:, None, None], np.float64).reshape(-1)
    cf = np.ascontiguousarray(sysd.cell_faces, np.int32)
    fc = np.ascontiguousarray(sysd.face_cells, np.int32)
    fd = np.ascontiguousarray(sysd.face_dir, np.int8)
    pb = np.ascontiguousarray(sysd.face_pbar, np.float64)
    lg = np.ascontiguousarray(logk, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    lam = np.ascontiguousarray(lam, np.float64)
    g = np.zeros(sysd.Ne)
    rc = lib().orc_adjoint_grad(sysd.Nf, sysd.Ne, _ptr(cf), _ptr(fc), _ptr(fd), _ptr(pb), _ptr(W1),
                                _ptr(lg), _ptr(u), _ptr(lam), _ptr(g))
    if rc:
        raise RuntimeError("orc_adjoint_grad failed")
    return g


def qsets_for(sysd, mode=None, thresh=None, dyn=None):
    mode = mode or sysd.extra.get("qmode", "own")
    if mode == "dynamic":
        n_add, n_ent, it_max = dyn
        return qsets_dynamic(sysd.A, sysd.C, n_add, n_ent, it_max)
    return qsets(mode, sysd.A, sysd.B, sysd.C,
                 thresh if thresh is not None else sysd.extra.get("thresh", 0.05))


def edfa_pipeline(sysd, mode=None, form=0, variant=0, restart=50, rtol=1e-8, maxit=2000, b=None,
                  dyn=None, solve=True, filt="none", tau=0.0, ordering=0, s_block=1):
    """The whole hot path on the CPU: Q sets, local solves, S~ (optionally
    filtered), ILU(0)s (ordering 0: natural; 1: multicolour ordering of S~;
    2: multicolour orderings of A and S~; s_block > 1: the block multicolour
    ordering of S~ with blocks of s_block consecutive rows), FGMRES."""
    qptr, qidx = qsets_for(sysd, mode, dyn=dyn)
    xval, gval = local_solves(sysd.A, sysd.B, sysd.C, qptr, qidx, True, form == 1)
    if filt == "none":
        S = schur(form, sysd.A, sysd.C, sysd.D, qptr, qidx, xval, gval)
    else:
        S, _ = schur_filtered(form, sysd.A, sysd.C, sysd.D, qptr, qidx, xval, gval, filt, tau)
    aperm = colour_order(sysd.A)[1] if ordering == 2 else None
    sperm = colour_order(S, s_block)[1] if ordering >= 1 else None
    P = Prec(sysd.A, sysd.B, sysd.C, sysd.D, S=S, variant=variant, aperm=aperm, sperm=sperm)
    out = dict(qptr=qptr, qidx=qidx, xval=xval, gval=gval, S=S, prec=P, aperm=aperm, sperm=sperm)
    if solve:
        out.update(fgmres(P, sysd.b if b is None else b, restart, rtol, maxit))
    return out
