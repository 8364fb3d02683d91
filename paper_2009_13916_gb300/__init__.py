"""GB300 (sm_103a) EDFA preconditioner: thin Python binding of libedfa.so.

The functions here only marshal arguments (torch CUDA tensors -> raw device
pointers, streams) into the C ABI declared in include/edfa.h; every step of
the preconditioner and the Krylov solve runs in the library's CUDA kernels.
There is no CPU fallback: if the library cannot be loaded, importing the
binding raises.

Block system (Sec. 2.3 of arXiv 2009.13916): [A B; C D] [pi; p] = [f_pi; f_p]
with A = A_pipi (faces), B = A_pip, C = A_ppi, D = A_pp (cells).
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

__all__ = ["EdfaError", "Csr", "Options", "SolveInfo", "Stats", "Edfa", "lib", "csr", "QMODES",
           "edfa_build", "edfa_setup", "edfa_apply", "edfa_matvec", "edfa_solve", "edfa_free"]

QMODES = {"own": 0, "nbr": 1, "crow": 2, "thresh": 3, "dynamic": 4, "given": 5}
FILTERS = {"none": 0, "pre": 1, "post_h": 2, "post_s": 3}

EDFA_OK = 0
EDFA_ERR_NOT_CONVERGED = 5


class EdfaError(RuntimeError):
    def __init__(self, code, where, detail=-1):
        self.code = code
        self.detail = detail
        msg = lib().edfa_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code}, detail {detail})")


class Csr(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("qmode", C.c_int32), ("thresh", C.c_double), ("n_add", C.c_int32),
                ("n_ent", C.c_int32), ("it_max", C.c_int32), ("qptr", C.c_void_p),
                ("qidx", C.c_void_p), ("schur_form", C.c_int32), ("variant", C.c_int32),
                ("precision", C.c_int32), ("warps_per_block", C.c_int32),
                ("sweep_warps_per_sm", C.c_int32), ("sweep_mode", C.c_int32),
                ("filtration", C.c_int32), ("tau_filt", C.c_double), ("ordering", C.c_int32),
                ("s_block", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("restarts", C.c_int32),
                ("est_rel", C.c_double), ("true_rel", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("ms_qsets", C.c_float), ("ms_local", C.c_float), ("ms_schur", C.c_float),
                ("ms_ilu_a", C.c_float), ("ms_stage2", C.c_float), ("ms_solve", C.c_float),
                ("n_local", C.c_int64), ("q_total", C.c_int64), ("q_max", C.c_int32),
                ("s_nnz", C.c_int64), ("levels_a", C.c_int32), ("levels_s", C.c_int32),
                ("sweep_ms", C.c_double * 5), ("sweep_n", C.c_int64 * 5),
                ("tuned_lanes", C.c_int32), ("tuned_warps", C.c_int32), ("tuned_schur_warps", C.c_int32),
                ("s_cluster", C.c_int32), ("s_cluster_bytes", C.c_int64),
                ("ms_s_values", C.c_float), ("ms_s_plan", C.c_float), ("ms_s_factor", C.c_float),
                ("ms_s_cluster", C.c_float), ("kry_ms", C.c_double * 3), ("kry_n", C.c_int64 * 3),
                ("kry_vecs", C.c_int64)]


class View(C.Structure):
    _fields_ = [("Nf", C.c_int32), ("Ne", C.c_int32), ("qptr", C.c_void_p), ("qidx", C.c_void_p),
                ("xval", C.c_void_p), ("gval", C.c_void_p), ("xval_f32", C.c_void_p),
                ("s_nnz", C.c_int64), ("s_rowptr", C.c_void_p), ("s_col", C.c_void_p),
                ("s_val", C.c_void_p), ("s_val_f32", C.c_void_p),
                ("a_ncolours", C.c_int32), ("s_ncolours", C.c_int32), ("a_perm", C.c_void_p),
                ("s_perm", C.c_void_p), ("fa_nnz", C.c_int64), ("fs_nnz", C.c_int64),
                ("fa_rowptr", C.c_void_p), ("fa_col", C.c_void_p), ("fa_lu", C.c_void_p),
                ("fa_lu_f32", C.c_void_p), ("fs_rowptr", C.c_void_p), ("fs_col", C.c_void_p),
                ("fs_lu", C.c_void_p), ("fs_lu_f32", C.c_void_p)]


_lib = None
EXPORTS = ("edfa_default_options", "edfa_build", "edfa_setup", "edfa_apply", "edfa_matvec",
           "edfa_solve", "edfa_history", "edfa_get_view", "edfa_get_stats", "edfa_set_profiling",
           "edfa_set_profiling_mask", "edfa_launch_count", "edfa_qsets_noalloc", "edfa_build_adjoint", "edfa_grad_logk",
           "edfa_solve_batched", "edfa_solve_bicgstab", "edfa_selftest_wait_timeout", "edfa_probe_fma_rate",
           "edfa_free", "edfa_strerror",
           "edfa_last_error_detail")


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libedfa.so (building it in-tree first if needed)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libedfa.so not found at {path}; run paper_2009_13916_gb300._build.build()")
        L = C.CDLL(path)
        P = C.POINTER
        vp = C.c_void_p
        L.edfa_default_options.argtypes = [P(Options)]
        L.edfa_default_options.restype = None
        L.edfa_build.argtypes = [P(vp), P(Csr), P(Csr), P(Csr), P(Csr), P(Options), vp]
        L.edfa_setup.argtypes = [vp, P(Csr), vp]
        L.edfa_apply.argtypes = [vp, vp, vp, vp]
        L.edfa_matvec.argtypes = [vp, vp, vp, vp]
        L.edfa_solve.argtypes = [vp, vp, vp, C.c_int32, C.c_double, C.c_int32, P(SolveInfo), vp]
        L.edfa_history.argtypes = [vp, P(C.c_double), C.c_int32]
        L.edfa_history.restype = C.c_int32
        L.edfa_get_view.argtypes = [vp, P(View)]
        L.edfa_get_stats.argtypes = [vp, P(Stats)]
        L.edfa_free.argtypes = [vp]
        L.edfa_set_profiling.argtypes = [vp, C.c_int32]
        L.edfa_set_profiling.restype = C.c_int
        L.edfa_set_profiling_mask.argtypes = [vp, C.c_uint32]
        L.edfa_set_profiling_mask.restype = C.c_int
        L.edfa_qsets_noalloc.argtypes = [P(Csr), P(Csr), P(Csr), C.c_int32, C.c_double, vp, vp, C.c_int64,
                                         P(C.c_int64), vp]
        L.edfa_qsets_noalloc.restype = C.c_int
        L.edfa_probe_fma_rate.argtypes = [C.c_int32, P(C.c_double), vp]
        L.edfa_probe_fma_rate.restype = C.c_int
        L.edfa_selftest_wait_timeout.argtypes = [P(C.c_float), vp]
        L.edfa_selftest_wait_timeout.restype = C.c_int
        L.edfa_build_adjoint.argtypes = [P(vp), vp, vp]
        L.edfa_build_adjoint.restype = C.c_int
        L.edfa_grad_logk.argtypes = [C.c_int32, C.c_int32] + [vp] * 8 + [vp]
        L.edfa_grad_logk.restype = C.c_int
        L.edfa_solve_batched.argtypes = [vp, C.c_int32, vp, vp, vp, vp, C.c_int32, C.c_double, C.c_int32,
                                         vp, vp, vp, vp]
        L.edfa_solve_batched.restype = C.c_int
        L.edfa_solve_bicgstab.argtypes = [vp, vp, vp, C.c_double, C.c_int32, P(SolveInfo), vp]
        L.edfa_solve_bicgstab.restype = C.c_int
        L.edfa_launch_count.argtypes = []
        L.edfa_launch_count.restype = C.c_int64
        L.edfa_strerror.argtypes = [C.c_int]
        L.edfa_strerror.restype = C.c_char_p
        L.edfa_last_error_detail.restype = C.c_int64
        for n in ("edfa_build", "edfa_setup", "edfa_apply", "edfa_matvec", "edfa_solve",
                  "edfa_get_view", "edfa_get_stats", "edfa_free"):
            getattr(L, n).restype = C.c_int
        _lib = L
    return _lib


# ---------------------------------------------------------------- raw ABI
def edfa_build(A: Csr, B: Csr, C_: Csr, D: Csr, opt: Options, stream: int = 0):
    h = C.c_void_p()
    rc = lib().edfa_build(C.byref(h), C.byref(A), C.byref(B), C.byref(C_), C.byref(D), C.byref(opt),
                          C.c_void_p(stream))
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_build", lib().edfa_last_error_detail())
    return h


def edfa_setup(h, D: Csr, stream: int = 0):
    rc = lib().edfa_setup(h, C.byref(D), C.c_void_p(stream))
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_setup", lib().edfa_last_error_detail())


def edfa_apply(h, r_ptr: int, z_ptr: int, stream: int = 0):
    rc = lib().edfa_apply(h, C.c_void_p(r_ptr), C.c_void_p(z_ptr), C.c_void_p(stream))
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_apply", lib().edfa_last_error_detail())


def edfa_matvec(h, x_ptr: int, y_ptr: int, stream: int = 0):
    rc = lib().edfa_matvec(h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), C.c_void_p(stream))
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_matvec", lib().edfa_last_error_detail())


def edfa_solve(h, b_ptr: int, x_ptr: int, restart: int, rtol: float, maxit: int, stream: int = 0,
               raise_on_nonconv: bool = False) -> SolveInfo:
    info = SolveInfo()
    rc = lib().edfa_solve(h, C.c_void_p(b_ptr), C.c_void_p(x_ptr), int(restart), float(rtol), int(maxit),
                          C.byref(info), C.c_void_p(stream))
    if rc != EDFA_OK and not (rc == EDFA_ERR_NOT_CONVERGED and not raise_on_nonconv):
        raise EdfaError(rc, "edfa_solve", lib().edfa_last_error_detail())
    return info


def qsets_noalloc(A, B, C_, Nf: int, Ne: int, qmode="nbr", thresh=0.05, qptr=None, qidx=None,
                  stream=None):
    """Restriction sets through edfa_qsets_noalloc (no device allocation inside
    the library; the caller provides qptr [Ne+1] int64 and qidx int32).
    Returns (rc, qtot)."""
    tot = C.c_int64(0)
    mode = QMODES[qmode] if isinstance(qmode, str) else int(qmode)
    rc = lib().edfa_qsets_noalloc(C.byref(csr(*A, Nf)), C.byref(csr(*B, Ne)), C.byref(csr(*C_, Nf)), mode,
                                  float(thresh), qptr.data_ptr(), qidx.data_ptr() if qidx is not None else None,
                                  qidx.numel() if qidx is not None else 0, C.byref(tot), _stream(stream))
    return rc, tot.value


def grad_logk(geom, u, lam, Nf: int, Ne: int, stream=None):
    """edfa_grad_logk on device tensors; geom = dict(cell_faces int32 [Ne,6],
    face_cells int32 [Nf,2], face_dir int8 [Nf], face_pbar f64 [Nf], W f64 [Ne,6,6])."""
    import torch
    g = torch.empty(Ne, dtype=torch.float64, device=u.device)
    rc = lib().edfa_grad_logk(int(Nf), int(Ne), geom["cell_faces"].data_ptr(), geom["face_cells"].data_ptr(),
                              geom["face_dir"].data_ptr(), geom["face_pbar"].data_ptr(), geom["W"].data_ptr(),
                              u.data_ptr(), lam.data_ptr(), g.data_ptr(), C.c_void_p(_stream(stream)))
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_grad_logk")
    return g


def selftest_wait_timeout(stream=None):
    """edfa_selftest_wait_timeout: returns (rc, detail, kernel ms)."""
    ms = C.c_float(0)
    rc = lib().edfa_selftest_wait_timeout(C.byref(ms), C.c_void_p(_stream(stream)))
    return rc, int(lib().edfa_last_error_detail()), float(ms.value)


def probe_fma_rate(precision: int = 0, stream=None) -> float:
    """edfa_probe_fma_rate: FMA per second of the device (0 = FP64, 1 = FP32)."""
    r = C.c_double(0)
    rc = lib().edfa_probe_fma_rate(int(precision), C.byref(r), C.c_void_p(_stream(stream)))
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_probe_fma_rate")
    return float(r.value)


def launch_count() -> int:
    return int(lib().edfa_launch_count())


def edfa_free(h):
    rc = lib().edfa_free(h)
    if rc != EDFA_OK:
        raise EdfaError(rc, "edfa_free")


# ---------------------------------------------------------------- torch helpers
def csr(rowptr, col, val, ncols: int) -> Csr:
    """Csr descriptor over CUDA tensors (rowptr int64, col int32, val float64)."""
    import torch
    for t, dt in ((rowptr, torch.int64), (col, torch.int32), (val, torch.float64)):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError("csr expects contiguous CUDA tensors rowptr:int64, col:int32, val:float64")
    return Csr(rowptr.numel() - 1, int(ncols), col.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Edfa:
    """Owning wrapper around one EDFA handle built on CUDA tensors.

    A, B, C, D are (rowptr int64, col int32, val float64) triples of CUDA
    tensors; the wrapper keeps them alive as the handle requires.
    """

    def __init__(self, A, B, C_, D, Nf: int, Ne: int, qmode="own", thresh=0.05, n_add=1, n_ent=4,
                 it_max=100, qsets=None, schur_form=0, variant=0, precision=0, warps_per_block=0,
                 sweep_warps_per_sm=0, sweep_mode=0, filtration="none", tau_filt=0.0, ordering=0, s_block=0, stream=None):
        self._keep = [A, B, C_, D]
        self.Nf, self.Ne = int(Nf), int(Ne)
        opt = Options()
        lib().edfa_default_options(C.byref(opt))
        opt.qmode = QMODES[qmode] if isinstance(qmode, str) else int(qmode)
        opt.thresh = float(thresh)
        opt.n_add, opt.n_ent, opt.it_max = int(n_add), int(n_ent), int(it_max)
        if qsets is not None:
            qp, qi = qsets
            self._keep += [qp, qi]
            opt.qptr, opt.qidx = qp.data_ptr(), qi.data_ptr()
            opt.qmode = QMODES["given"]
        opt.schur_form, opt.variant = int(schur_form), int(variant)
        opt.precision = int(precision)
        opt.warps_per_block = int(warps_per_block)
        opt.sweep_warps_per_sm = int(sweep_warps_per_sm)
        opt.sweep_mode = int(sweep_mode)
        opt.filtration = FILTERS[filtration] if isinstance(filtration, str) else int(filtration)
        opt.tau_filt = float(tau_filt)
        opt.ordering = int(ordering)
        opt.s_block = int(s_block)
        self.opt = opt
        self._D = D
        self.h = edfa_build(csr(*A, self.Nf), csr(*B, self.Ne), csr(*C_, self.Nf), csr(*D, self.Ne), opt,
                            _stream(stream))

    @property
    def n(self):
        return self.Nf + self.Ne

    def setup(self, D, stream=None):
        self._D = D
        self._keep[3] = D
        edfa_setup(self.h, csr(*D, self.Ne), _stream(stream))

    def apply(self, r, z=None, stream=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        edfa_apply(self.h, r.data_ptr(), z.data_ptr(), _stream(stream))
        return z

    def matvec(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        edfa_matvec(self.h, x.data_ptr(), y.data_ptr(), _stream(stream))
        return y

    def solve(self, b, x=None, restart=50, rtol=1e-8, maxit=2000, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(b)
        info = edfa_solve(self.h, b.data_ptr(), x.data_ptr(), restart, rtol, maxit, _stream(stream))
        return x, info

    def solve_bicgstab(self, b, x=None, rtol=1e-8, maxit=2000, stream=None):
        """Bi-CGStab with this preconditioner (edfa_solve_bicgstab)."""
        import torch
        if x is None:
            x = torch.empty_like(b)
        info = SolveInfo()
        rc = lib().edfa_solve_bicgstab(self.h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), float(rtol),
                                       int(maxit), C.byref(info), C.c_void_p(_stream(stream)))
        if rc not in (EDFA_OK, EDFA_ERR_NOT_CONVERGED):
            raise EdfaError(rc, "edfa_solve_bicgstab", lib().edfa_last_error_detail())
        return x, info

    def history(self):
        import numpy as np
        buf = (C.c_double * 100000)()
        n = lib().edfa_history(self.h, buf, 100000)
        return np.array(buf[:n])

    def solve_batched(self, face_off, cell_off, b, x=None, restart=50, rtol=1e-8, maxit=2000, stream=None):
        """One FGMRES per block-diagonal subsystem (edfa_solve_batched).
        Returns (x, iterations[nsys], true_rel[nsys], cycles, rc)."""
        import numpy as np
        import torch
        fo = np.ascontiguousarray(face_off, dtype=np.int64)
        co = np.ascontiguousarray(cell_off, dtype=np.int64)
        nsys = len(fo) - 1
        if x is None:
            x = torch.empty_like(b)
        it = np.zeros(nsys, dtype=np.int32)
        tr = np.zeros(nsys, dtype=np.float64)
        cyc = C.c_int32(0)
        rc = lib().edfa_solve_batched(self.h, nsys, fo.ctypes.data, co.ctypes.data, b.data_ptr(), x.data_ptr(),
                                      int(restart), float(rtol), int(maxit), it.ctypes.data, tr.ctypes.data,
                                      C.byref(cyc), C.c_void_p(_stream(stream)))
        if rc not in (EDFA_OK, EDFA_ERR_NOT_CONVERGED):
            raise EdfaError(rc, "edfa_solve_batched", lib().edfa_last_error_detail())
        return x, it, tr, cyc.value, rc

    def adjoint(self, stream=None) -> "Edfa":
        """Handle for the transposed system [A C^T; B^T D^T] (edfa_build_adjoint)."""
        h = C.c_void_p()
        rc = lib().edfa_build_adjoint(C.byref(h), self.h, C.c_void_p(_stream(stream)))
        if rc != EDFA_OK:
            raise EdfaError(rc, "edfa_build_adjoint", lib().edfa_last_error_detail())
        adj = Edfa.__new__(Edfa)
        adj._keep = [self]
        adj.Nf, adj.Ne = self.Nf, self.Ne
        adj.opt = self.opt
        adj._D = None
        adj.h = h
        return adj

    def set_profiling(self, on: bool, kinds=None):
        """Per-launch event timing: all timed kinds (on=True), none, or the
        given kinds (indices 0-7 as in edfa_set_profiling_mask)."""
        if kinds is None:
            lib().edfa_set_profiling(self.h, 1 if on else 0)
        else:
            mask = 0
            for k in kinds:
                mask |= 1 << int(k)
            rc = lib().edfa_set_profiling_mask(self.h, mask if on else 0)
            if rc != 0:
                raise ValueError(f"edfa_set_profiling_mask: {rc}")

    def stats(self) -> Stats:
        st = Stats()
        lib().edfa_get_stats(self.h, C.byref(st))
        return st

    def view(self) -> View:
        v = View()
        lib().edfa_get_view(self.h, C.byref(v))
        return v

    def tensors(self):
        """Copies of the restriction sets, X~ (and G~) and S~ as torch tensors."""
        import torch
        v = self.view()
        st = self.stats()
        dev = torch.device("cuda", torch.cuda.current_device())

        class _Dev:
            # a borrowed device buffer of the handle, exposed for a copy
            def __init__(self, ptr, n, typestr):
                self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                                 "version": 3, "strides": None}

        codes = {torch.int64: "<i8", torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}

        def wrap(ptr, n, dtype):
            if not ptr or n == 0:
                return None
            return torch.as_tensor(_Dev(ptr, int(n), codes[dtype]), device=dev).clone()

        torch.cuda.synchronize()
        out = dict(qptr=wrap(v.qptr, self.Ne + 1, torch.int64))
        qtot = int(out["qptr"][-1].item())
        out["qidx"] = wrap(v.qidx, qtot, torch.int32)
        out["xval"] = wrap(v.xval, qtot, torch.float64) if v.xval else wrap(v.xval_f32, qtot, torch.float32)
        out["gval"] = wrap(v.gval, qtot, torch.float64)
        out["s_rowptr"] = wrap(v.s_rowptr, self.Ne + 1, torch.int64)
        out["s_col"] = wrap(v.s_col, st.s_nnz, torch.int32)
        out["s_val"] = wrap(v.s_val, st.s_nnz, torch.float64) if v.s_val else wrap(v.s_val_f32, st.s_nnz,
                                                                                     torch.float32)
        return out

    def factors(self):
        """Copies of the orderings and of the ILU(0) factors as computed (of the
        ordered matrices when an ordering is on)."""
        import torch
        v = self.view()
        dev = torch.device("cuda", torch.cuda.current_device())

        class _Dev:
            def __init__(self, ptr, n, typestr):
                self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                                 "version": 3, "strides": None}

        def wrap(ptr, n, ts):
            if not ptr or n == 0:
                return None
            return torch.as_tensor(_Dev(ptr, int(n), ts), device=dev).clone()

        torch.cuda.synchronize()
        out = dict(a_ncolours=int(v.a_ncolours), s_ncolours=int(v.s_ncolours),
                   a_perm=wrap(v.a_perm, self.Nf, "<i4"), s_perm=wrap(v.s_perm, self.Ne, "<i4"))
        for k, n, nnz in (("fa", self.Nf, v.fa_nnz), ("fs", self.Ne, v.fs_nnz)):
            out[k + "_rowptr"] = wrap(getattr(v, k + "_rowptr"), n + 1, "<i8")
            out[k + "_col"] = wrap(getattr(v, k + "_col"), nnz, "<i4")
            lu = getattr(v, k + "_lu")
            out[k + "_lu"] = wrap(lu, nnz, "<f8") if lu else wrap(getattr(v, k + "_lu_f32"), nnz, "<f4")
        return out

    def close(self):
        if getattr(self, "h", None):
            edfa_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def system_to_device(sysd, device="cuda"):
    """CSR blocks of a generated system (numpy) as CUDA tensor triples."""
    import torch

    def t(M):
        return (torch.as_tensor(M.rowptr, dtype=torch.int64, device=device),
                torch.as_tensor(M.col, dtype=torch.int32, device=device),
                torch.as_tensor(M.val, dtype=torch.float64, device=device))

    return t(sysd.A), t(sysd.B), t(sysd.C), t(sysd.D)
