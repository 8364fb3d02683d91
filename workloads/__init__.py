"""Seeded synthetic workloads for the EDFA hot path.

The five workloads stand in for the paper's SPE10 test cases (Sec. 4,
Table 1), whose data is not available: brick grids of cubic cells with the
MHFE(RT0)-FV block system [A B; C D] of Sec. 2.3 (A = A_pipi faces x faces,
B = A_pip, C = A_ppi, D = A_pp).  All random numbers come from one SplitMix64
stream per workload (Box-Muller normals), so a workload is a pure function of
its index.

This module produces inputs only; it holds none of the preconditioner's
arithmetic.  The assembly itself lives in ``gen.c`` (built on first use).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "_build", "libwl.so")


def build(force: bool = False) -> str:
    """Compile gen.c into workloads/_build/libwl.so (plain gcc, -O2)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(_SO))
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fvisibility=hidden",
                           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _CSR(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double))]


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("dt", C.c_double), ("stor", C.c_double),
                ("fv_kind", C.c_int32), ("dirichlet", C.c_int32),
                ("p_left", C.c_double), ("p_right", C.c_double),
                ("K", C.POINTER(C.c_double)), ("lam_face", C.POINTER(C.c_double)),
                ("xyz", C.POINTER(C.c_double))]


class _System(C.Structure):
    _fields_ = [("Nf", C.c_int32), ("Ne", C.c_int32),
                ("A", _CSR), ("B", _CSR), ("C", _CSR), ("D", _CSR),
                ("f", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
                ("cell_faces", C.POINTER(C.c_int32)), ("face_cells", C.POINTER(C.c_int32)),
                ("face_dir", C.POINTER(C.c_int8)), ("face_pbar", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.wl_splitmix64.restype = C.c_uint64
        L.wl_splitmix64.argtypes = [C.POINTER(C.c_uint64)]
        L.wl_uniform.restype = C.c_double
        L.wl_uniform.argtypes = [C.POINTER(C.c_uint64)]
        L.wl_normal.restype = C.c_double
        L.wl_normal.argtypes = [C.POINTER(C.c_uint64)]
        for fn in (L.wl_fill_uniform, L.wl_fill_normal):
            fn.restype = None
            fn.argtypes = [C.POINTER(C.c_uint64), C.c_int64, C.POINTER(C.c_double)]
        L.wl_assemble.restype = C.c_int
        L.wl_assemble.argtypes = [C.POINTER(_Problem), C.POINTER(_System)]
        L.wl_free_system.restype = None
        L.wl_free_system.argtypes = [C.POINTER(_System)]
        L.wl_elem_W.restype = C.c_int
        L.wl_elem_W.argtypes = [C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double,
                                C.POINTER(C.c_double)]
        L.wl_vmath.restype = None
        L.wl_vmath.argtypes = [C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.wl_elem_B.restype = None
        L.wl_elem_B.argtypes = [C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double,
                                C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vmath(f: int, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib().wl_vmath(int(f), int(x.size), _dp(x), _dp(out))
    return out


# exp, log and sin of the generator (gen.c): IEEE arithmetic only, so that a seed
# gives the same inputs bit for bit on every host (host math libraries differ in
# the last bit between machines)
def wexp(x) -> np.ndarray:
    return _vmath(0, x)


def wlog(x) -> np.ndarray:
    return _vmath(1, x)


def wsin(x) -> np.ndarray:
    return _vmath(2, x)


LN10 = 2.302585092994046


class Stream:
    """SplitMix64 stream with Box-Muller normals (the generator in gen.c)."""

    def __init__(self, seed: int):
        self.state = C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def uniform(self, n: int) -> np.ndarray:
        out = np.empty(int(n), dtype=np.float64)
        lib().wl_fill_uniform(C.byref(self.state), int(n), _dp(out))
        return out

    def normal(self, n: int) -> np.ndarray:
        out = np.empty(int(n), dtype=np.float64)
        lib().wl_fill_normal(C.byref(self.state), int(n), _dp(out))
        return out


@dataclass
class CSR:
    nrows: int
    ncols: int
    rowptr: np.ndarray  # int64 [nrows+1]
    col: np.ndarray     # int32 [nnz], ascending within a row
    val: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.nrows, self.ncols))

    def dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


@dataclass
class System:
    """One block system [A B; C D] u = b with its grid description."""
    name: str
    nx: int
    ny: int
    nz: int
    h: tuple
    Nf: int
    Ne: int
    A: CSR
    B: CSR
    C: CSR
    D: CSR
    b: np.ndarray            # [Nf+Ne] right-hand side used by the workload
    f_phys: np.ndarray       # [Nf+Ne] right-hand side from the prescribed pressures
    K: np.ndarray            # [Ne,6]
    W: np.ndarray            # [Ne,6,6] elemental B^{E,-1}
    cell_faces: np.ndarray   # [Ne,6]
    face_cells: np.ndarray   # [Nf,2]
    face_dir: np.ndarray     # [Nf] bool
    face_pbar: np.ndarray    # [Nf]
    dt: float
    stor: float
    fv_kind: int
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.Nf + self.Ne

    def full_scipy(self):
        import scipy.sparse as sp
        return sp.bmat([[self.A.to_scipy(), self.B.to_scipy()],
                        [self.C.to_scipy(), self.D.to_scipy()]], format="csr")


def _csr_from(c: _CSR) -> CSR:
    n, nnz = c.nrows, c.nnz
    rp = np.ctypeslib.as_array(c.rowptr, shape=(n + 1,)).copy()
    if nnz:
        col = np.ctypeslib.as_array(c.col, shape=(nnz,)).copy()
        val = np.ctypeslib.as_array(c.val, shape=(nnz,)).copy()
    else:
        col = np.zeros(0, np.int32)
        val = np.zeros(0, np.float64)
    return CSR(c.nrows, c.ncols, rp, col, val)


def assemble(nx, ny, nz, K, *, h=None, dt=0.1, stor=1e-2, fv_kind=0, lam_face=None,
             dirichlet=True, p_left=1.0, p_right=0.0, name="custom", b=None, xyz=None) -> System:
    """Assemble the MHFE-FV block system for a structured grid with per-cell K[Ne,6]:
    brick cells h[0] x h[1] x h[2], or general hexahedra with node coordinates
    xyz[(nx+1)(ny+1)(nz+1), 3] (node (i,j,k) lexicographic, i fastest)."""
    if h is None:
        h = (1.0 / nx, 1.0 / nx, 1.0 / nx)
    Ne = nx * ny * nz
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(Ne, 6)
    P = _Problem(nx, ny, nz, h[0], h[1], h[2], dt, stor, fv_kind, 1 if dirichlet else 0,
                 p_left, p_right, _dp(K), None, None)
    if xyz is not None:
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape((nx + 1) * (ny + 1) * (nz + 1), 3)
        P.xyz = _dp(xyz)
    if fv_kind == 1:
        lam_face = np.ascontiguousarray(lam_face, dtype=np.float64)
        P.lam_face = _dp(lam_face)
    S = _System()
    rc = lib().wl_assemble(C.byref(P), C.byref(S))
    if rc != 0:
        raise RuntimeError(f"wl_assemble failed ({rc})")
    try:
        Nf, Ne = S.Nf, S.Ne
        sysd = System(
            name=name, nx=nx, ny=ny, nz=nz, h=tuple(h), Nf=Nf, Ne=Ne,
            A=_csr_from(S.A), B=_csr_from(S.B), C=_csr_from(S.C), D=_csr_from(S.D),
            b=None, f_phys=np.ctypeslib.as_array(S.f, shape=(Nf + Ne,)).copy(), K=K.copy(),
            W=np.ctypeslib.as_array(S.W, shape=(Ne * 36,)).copy().reshape(Ne, 6, 6),
            cell_faces=np.ctypeslib.as_array(S.cell_faces, shape=(Ne * 6,)).copy().reshape(Ne, 6),
            face_cells=np.ctypeslib.as_array(S.face_cells, shape=(Nf * 2,)).copy().reshape(Nf, 2),
            face_dir=np.ctypeslib.as_array(S.face_dir, shape=(Nf,)).copy().astype(bool),
            face_pbar=np.ctypeslib.as_array(S.face_pbar, shape=(Nf,)).copy(),
            dt=dt, stor=stor, fv_kind=fv_kind)
    finally:
        lib().wl_free_system(C.byref(S))
    sysd.b = sysd.f_phys.copy() if b is None else np.ascontiguousarray(b, dtype=np.float64)
    return sysd


def elem_W(K6, h):
    K6 = np.ascontiguousarray(K6, dtype=np.float64)
    out = np.empty(36)
    if lib().wl_elem_W(_dp(K6), h[0], h[1], h[2], _dp(out)) != 0:
        raise ValueError("elemental matrix not SPD")
    return out.reshape(6, 6)


def elem_B(K6, h):
    K6 = np.ascontiguousarray(K6, dtype=np.float64)
    out = np.empty(36)
    lib().wl_elem_B(_dp(K6), h[0], h[1], h[2], _dp(out))
    return out.reshape(6, 6)


def elem_B_hex(K6, X):
    """B^E of a general hexahedron with nodes X[8,3] (Piola-mapped RT0, Gauss
    quadrature) and its volume."""
    K6 = np.ascontiguousarray(K6, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(24)
    out = np.empty(36)
    vol = C.c_double(0.0)
    if lib().wl_elem_B_hex(_dp(K6), _dp(X), _dp(out), C.byref(vol)) != 0:
        raise ValueError("inverted cell")
    return out.reshape(6, 6), vol.value


def grid_nodes(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0):
    """Node coordinates of a uniform brick grid, [(nx+1)(ny+1)(nz+1), 3]."""
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return np.stack([i.ravel() * lx / nx, j.ravel() * ly / ny, k.ravel() * lz / nz], axis=1).astype(np.float64)


def dome_nodes(nx, ny, nz, height=0.25, wobble=0.02):
    """A dome-shaped layered grid on the unit cube: every layer is lifted by a smooth
    bump height * (1 - z) * (1 - r^2) (r the distance from the centre of the x-y square,
    scaled to 1 at the corners), and the lateral node positions get a smooth wobble, so
    that cells are general (non-parallelepiped) hexahedra.  The x = 0 and x = 1 planes
    stay planar (the prescribed-pressure boundaries)."""
    X = grid_nodes(nx, ny, nz)
    x, y, z = X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy()
    r2 = ((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.5
    zn = z + height * (1.0 - z) * (1.0 - r2)  # the layers lifted into a dome
    yn = y + wobble * wsin(2 * np.pi * x) * wsin(np.pi * y) * wsin(np.pi * z + 0.3)
    return np.stack([x, yn, zn], axis=1)


def dome(n: int = 12, seed: int = 7, sigma: float = 1.0, name=None) -> System:
    """Dome-shaped structured grid of general hexahedra (a stand-in for the paper's
    dome grids, whose data are not available): n x n x n cells, isotropic lognormal K,
    prescribed pressures on x = 0 and x = 1, own + neighbour-face sets."""
    s = Stream(7000 + seed)
    Ne = n ** 3
    K = iso_K(wexp(sigma * s.normal(Ne)))
    sysd = assemble(n, n, n, K, xyz=dome_nodes(n, n, n), name=name or f"dome {n}^3")
    sysd.extra.update(qmode="nbr")
    return sysd


def iso_K(k: np.ndarray) -> np.ndarray:
    K = np.zeros((k.size, 6))
    K[:, 0] = K[:, 1] = K[:, 2] = k
    return K


def _quat_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrices [n,3,3] from (unnormalised) quaternions [n,4]."""
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def rotated_K(m: np.ndarray, aniso: float, q: np.ndarray) -> np.ndarray:
    """K = R diag(m, m, m*aniso) R^T per cell, stored as xx yy zz xy xz yz."""
    R = _quat_rot(q)
    d = np.stack([m, m, m * aniso], axis=1)
    # sum over j written out in a fixed order (no library contraction whose
    # summation order could depend on the host's vector unit)
    Kf = np.empty_like(R)
    for i in range(3):
        for k in range(3):
            Kf[:, i, k] = ((R[:, i, 0] * d[:, 0]) * R[:, k, 0] + (R[:, i, 1] * d[:, 1]) * R[:, k, 1]) \
                + (R[:, i, 2] * d[:, 2]) * R[:, k, 2]
    Kf = 0.5 * (Kf + np.transpose(Kf, (0, 2, 1)))
    return np.stack([Kf[:, 0, 0], Kf[:, 1, 1], Kf[:, 2, 2], Kf[:, 0, 1], Kf[:, 0, 2], Kf[:, 1, 2]], axis=1)


def _face_upwind_mobility(nx, ny, nz, lam_cell, signs_u, face_cells):
    """Face mobility lam_f = lam of the upwind cell; the upwind side of an
    interior face is chosen by a seeded random flux sign, a boundary face
    takes its only cell."""
    m, p = face_cells[:, 0], face_cells[:, 1]
    pick_plus = signs_u >= 0.5
    up = np.where(m < 0, p, np.where(p < 0, m, np.where(pick_plus, p, m)))
    return lam_cell[up]


# ---------------------------------------------------------------- workloads
def brick(nx, ny=None, nz=None, *, seed=1, sigma=1.0, kind="paper", rhs="phys", name=None,
          dt=0.1, stor=1e-2) -> System:
    """Small seeded isotropic-K brick system (tiny-grid pins and parity cases).

    kind="paper": strong inter-element flux cell rows (Appendix A);
    kind="upwind": C = -B^T diag(lam_upwind), D = diag(sum lam B) + Omega c/dt.
    rhs="phys": prescribed-pressure right-hand side; "random": N(0,1) entries.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    s = Stream(seed)
    Ne = nx * ny * nz
    k = wexp(sigma * s.normal(Ne))
    K = iso_K(k)
    kw = {}
    if kind == "upwind":
        lam = wexp(0.5 * s.normal(Ne))
        tmp = assemble(nx, ny, nz, K, dt=dt, stor=stor)  # for the face-cell map only
        signs = s.uniform(tmp.Nf)
        kw = dict(fv_kind=1, lam_face=_face_upwind_mobility(nx, ny, nz, lam, signs, tmp.face_cells))
    sysd = assemble(nx, ny, nz, K, dt=dt, stor=stor, name=name or f"brick{nx}x{ny}x{nz}", **kw)
    if rhs == "random":
        sysd.b = s.normal(sysd.n)
    return sysd


def config1() -> System:
    """10^3 unit-brick grid, isotropic K = exp(N(0,1)), upwind-mobility C,
    dt = 0.1, c = 1e-2, prescribed p = 1 / 0 on x = 0 / 1, random RHS, Q = own faces."""
    s = Stream(1)
    nx = 10
    Ne = nx ** 3
    K = iso_K(wexp(s.normal(Ne)))
    lam = wexp(0.5 * s.normal(Ne))
    tmp = assemble(nx, nx, nx, K)
    signs = s.uniform(tmp.Nf)
    lam_f = _face_upwind_mobility(nx, nx, nx, lam, signs, tmp.face_cells)
    sysd = assemble(nx, nx, nx, K, fv_kind=1, lam_face=lam_f, name="C1 10^3 upwind-mobility")
    sysd.b = s.normal(sysd.n)
    sysd.extra.update(qmode="own", lam_cell=lam)
    return sysd


def config2(n: int = 64) -> System:
    """n^3 grid (64^3 by default), full-tensor K = R diag(m,m,m/10) R^T with
    m = exp(2 N(0,1)) and R a random rotation per cell; strong-flux FV;
    prescribed-pressure RHS; Q = own faces + faces of face-neighbours."""
    s = Stream(2)
    Ne = n ** 3
    m = wexp(2.0 * s.normal(Ne))
    q = s.normal(4 * Ne).reshape(Ne, 4)
    K = rotated_K(m, 0.1, q)
    sysd = assemble(n, n, n, K, name=f"C2 {n}^3 full-tensor")
    sysd.extra.update(qmode="nbr")
    return sysd


def channel_K(nx, ny, nz, h, s: Stream) -> np.ndarray:
    """Layered channelised diagonal K: background log10 Kh ~ U(-6,-3) per cell,
    three sinusoidal channels per layer with log10 Kh ~ U(-1,0) inside,
    Kv = 0.1 Kh."""
    Ne = nx * ny * nz
    lg = -6.0 + 3.0 * s.uniform(Ne)
    lg_ch = -1.0 + s.uniform(Ne)
    ix = np.arange(nx)
    iy = np.arange(ny)
    xc = (ix + 0.5) * h[0]
    yc = (iy + 0.5) * h[1]
    X, Y = np.meshgrid(xc, yc, indexing="xy")  # [ny, nx]
    lg = lg.reshape(nz, ny, nx)
    lg_ch = lg_ch.reshape(nz, ny, nx)
    for iz in range(nz):
        p = s.uniform(15).reshape(3, 5)
        inside = np.zeros((ny, nx), bool)
        for c in range(3):
            y0 = 0.1 + 0.8 * p[c, 0]
            a = 0.05 + 0.15 * p[c, 1]
            fr = 0.5 + 1.5 * p[c, 2]
            ph = 2 * np.pi * p[c, 3]
            hw = 0.02 + 0.03 * p[c, 4]
            inside |= np.abs(Y - (y0 + a * wsin(2 * np.pi * fr * X + ph))) < hw
        lg[iz][inside] = lg_ch[iz][inside]
    kh = wexp(LN10 * lg.reshape(Ne))
    K = np.zeros((Ne, 6))
    K[:, 0] = kh
    K[:, 1] = kh
    K[:, 2] = 0.1 * kh
    return K


def config3(nx: int = 128, ny: int = 128, nz: int = 64) -> System:
    """128x128x64 layered channelised grid (cells 1/128), diagonal K with
    6 orders of magnitude and Kv = 0.1 Kh; strong-flux FV; prescribed-pressure
    RHS; Q = own faces + strong A-connections |a_ij| >= 0.05 |a_ii|."""
    s = Stream(3)
    h = (1.0 / nx,) * 3
    K = channel_K(nx, ny, nz, h, s)
    sysd = assemble(nx, ny, nz, K, h=h, name=f"C3 {nx}x{ny}x{nz} channelised")
    sysd.extra.update(qmode="thresh", thresh=0.05)
    return sysd


def config4_sizes(nsys: int = 256) -> np.ndarray:
    s = Stream((4 << 32))
    return (16 + np.floor(33 * s.uniform(nsys))).astype(np.int64)


def config4_system(i: int, n: int) -> System:
    """System i of the batched workload: n^3 grid, isotropic K = exp(1.5 N(0,1)),
    strong-flux FV, random N(0,1) RHS, Q = own + neighbour faces."""
    s = Stream((4 << 32) + 1 + i)
    Ne = n ** 3
    K = iso_K(wexp(1.5 * s.normal(Ne)))
    sysd = assemble(n, n, n, K, name=f"C4[{i}] {n}^3")
    sysd.b = s.normal(sysd.n)
    sysd.extra.update(qmode="nbr")
    return sysd


def config4(nsys: int = 256, limit=None):
    sizes = config4_sizes(nsys)
    idx = range(nsys) if limit is None else range(min(limit, nsys))
    return [config4_system(i, int(sizes[i])) for i in idx]


def config5(n: int = 48, nobs: int = 64, nfd: int = 20) -> System:
    """n^3 grid (48^3), isotropic K = exp(N(0,1)), strong-flux FV,
    prescribed-pressure RHS, Q = pattern of row m of C; loss = sum of squared
    cell pressures at 64 seeded observation cells; 20 seeded cells for
    finite-difference checks."""
    s = Stream(5)
    Ne = n ** 3
    logk = s.normal(Ne)
    k = wexp(logk)
    K = iso_K(k)
    sysd = assemble(n, n, n, K, name=f"C5 {n}^3 adjoint")
    perm = np.arange(Ne)
    u = s.uniform(nobs)
    for j in range(nobs):  # partial Fisher-Yates: observation cells without replacement
        r = j + int(u[j] * (Ne - j))
        perm[j], perm[r] = perm[r], perm[j]
    obs = np.sort(perm[:nobs]).astype(np.int64)
    u = s.uniform(nfd)
    perm = np.arange(Ne)
    for j in range(nfd):
        r = j + int(u[j] * (Ne - j))
        perm[j], perm[r] = perm[r], perm[j]
    fd = np.sort(perm[:nfd]).astype(np.int64)
    sysd.extra.update(qmode="crow", obs=obs, fd_cells=fd, logk=logk)
    return sysd


def config5_reassemble(sysd: System, logk: np.ndarray) -> System:
    """Re-assemble workload 5 with a modified per-cell log-conductivity."""
    out = assemble(sysd.nx, sysd.ny, sysd.nz, iso_K(wexp(logk)), h=sysd.h, dt=sysd.dt,
                   stor=sysd.stor, name=sysd.name + " (perturbed)")
    out.extra.update(sysd.extra)
    out.extra["logk"] = logk.copy()
    return out


def device_assembler(template: System, device="cuda"):
    """Callable theta -> device system for the differentiable solve: re-assembles
    the isotropic strong-flux system of `template`'s grid with k = exp(theta)
    (host generator) and returns CUDA tensors (CSR triples, b, grid arrays)."""
    import torch

    def t(M):
        return (torch.as_tensor(M.rowptr, dtype=torch.int64, device=device),
                torch.as_tensor(M.col, dtype=torch.int32, device=device),
                torch.as_tensor(M.val, dtype=torch.float64, device=device))

    def assemble_theta(theta):
        lk = theta.detach().double().cpu().numpy()
        s = assemble(template.nx, template.ny, template.nz, iso_K(wexp(lk)), h=template.h, dt=template.dt,
                     stor=template.stor, name=template.name + " (theta)")
        return dict(
            A=t(s.A), B=t(s.B), C=t(s.C), D=t(s.D), Nf=s.Nf, Ne=s.Ne,
            b=torch.as_tensor(s.f_phys, dtype=torch.float64, device=device),
            cell_faces=torch.as_tensor(s.cell_faces, dtype=torch.int32, device=device).contiguous(),
            face_cells=torch.as_tensor(s.face_cells, dtype=torch.int32, device=device).contiguous(),
            face_dir=torch.as_tensor(s.face_dir.astype(np.int8), device=device).contiguous(),
            face_pbar=torch.as_tensor(s.face_pbar, dtype=torch.float64, device=device),
            W=torch.as_tensor(s.W, dtype=torch.float64, device=device).contiguous(),
            host=s)

    return assemble_theta


def digest(sysd: System) -> str:
    """SHA-256 (hex, first 16 digits) of a system's CSR blocks and right-hand
    side: identifies the exact inputs a stored expected value belongs to."""
    import hashlib
    h = hashlib.sha256()
    for M in (sysd.A, sysd.B, sysd.C, sysd.D):
        for a, dt in ((M.rowptr, "<i8"), (M.col, "<i4"), (M.val, "<f8")):
            h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    h.update(np.ascontiguousarray(sysd.b, dtype="<f8").tobytes())
    return h.hexdigest()[:16]


def concat(systems, name="batch"):
    """Block-diagonal concatenation of independent systems: faces of all systems
    first (system by system), then cells.  Returns (System, face_off, cell_off)."""
    Nf = sum(s.Nf for s in systems)
    Ne = sum(s.Ne for s in systems)
    fo = np.zeros(len(systems) + 1, np.int64)
    co = np.zeros(len(systems) + 1, np.int64)
    for i, s in enumerate(systems):
        fo[i + 1] = fo[i] + s.Nf
        co[i + 1] = co[i] + s.Ne

    def cat(get, roff, coff, nrows, ncols):
        rps, cols, vals = [np.zeros(1, np.int64)], [], []
        base = 0
        for i, s in enumerate(systems):
            M = get(s)
            rps.append(M.rowptr[1:] + base)
            cols.append(M.col.astype(np.int64) + coff[i])
            vals.append(M.val)
            base += M.nnz
        return CSR(nrows, ncols, np.concatenate(rps), np.concatenate(cols).astype(np.int32), np.concatenate(vals))

    A = cat(lambda s: s.A, fo, fo, Nf, Nf)
    B = cat(lambda s: s.B, fo, co, Nf, Ne)
    Cm = cat(lambda s: s.C, co, fo, Ne, Nf)
    D = cat(lambda s: s.D, co, co, Ne, Ne)
    b = np.concatenate([np.concatenate([s.b[: s.Nf] for s in systems]),
                        np.concatenate([s.b[s.Nf:] for s in systems])])
    f = np.concatenate([np.concatenate([s.f_phys[: s.Nf] for s in systems]),
                        np.concatenate([s.f_phys[s.Nf:] for s in systems])])
    big = System(name=name, nx=0, ny=0, nz=0, h=(0, 0, 0), Nf=Nf, Ne=Ne, A=A, B=B, C=Cm, D=D, b=b, f_phys=f,
                 K=np.concatenate([s.K for s in systems]), W=np.concatenate([s.W for s in systems]),
                 cell_faces=np.concatenate([s.cell_faces + fo[i] for i, s in enumerate(systems)]),
                 face_cells=np.concatenate([np.where(s.face_cells >= 0, s.face_cells + co[i], -1)
                                            for i, s in enumerate(systems)]),
                 face_dir=np.concatenate([s.face_dir for s in systems]),
                 face_pbar=np.concatenate([s.face_pbar for s in systems]),
                 dt=systems[0].dt, stor=systems[0].stor, fv_kind=systems[0].fv_kind)
    big.extra.update(qmode=systems[0].extra.get("qmode", "nbr"))
    return big, fo, co


def sub_vector(v, sysd_list, fo, co, i):
    """Unknowns of system i (faces then cells) out of a concatenated vector."""
    Nf = int(fo[-1])
    return np.concatenate([v[fo[i]:fo[i + 1]], v[Nf + co[i]:Nf + co[i + 1]]])


class Transient:
    """Implicit-Euler time stepping of the single-phase compressible MHFE-FV model on an
    assembled system: between steps only the accumulation term of D (Omega c / dt on the
    diagonal) and the cell right-hand side (Omega c / dt) p_n change, so a preconditioner
    keeps its Stage 1 and redoes Stage 2 only.  The step size follows the adaptive rule of
    Sec. 4 (Eq. delta_t_dyn): dt_{n+1} = min(dt_n min(dt_mult, dp_T / dp_max), dt_max)."""

    def __init__(self, sysd: System, dt_mult=2.0, dp_target=0.05, dt_max=10.0):
        self.s = sysd
        self.dt_mult, self.dp_target, self.dt_max = dt_mult, dp_target, dt_max
        self.acc = float(np.prod(sysd.h)) * sysd.stor  # Omega c, per cell (brick cells)
        D = sysd.D
        rows = np.repeat(np.arange(D.nrows), np.diff(D.rowptr))
        self.diag_pos = np.nonzero(D.col == rows)[0]
        assert len(self.diag_pos) == D.nrows
        self.d_base = D.val.copy()
        self.d_base[self.diag_pos] -= self.acc / sysd.dt

    def D_values(self, dt: float) -> np.ndarray:
        v = self.d_base.copy()
        v[self.diag_pos] += self.acc / dt
        return v

    def D(self, dt: float) -> CSR:
        D = self.s.D
        return CSR(D.nrows, D.ncols, D.rowptr, D.col, self.D_values(dt))

    def rhs(self, dt: float, p_cells: np.ndarray) -> np.ndarray:
        b = self.s.f_phys.copy()
        b[self.s.Nf:] += self.acc / dt * p_cells
        return b

    def next_dt(self, dt: float, dp_max: float) -> float:
        f = self.dt_mult if dp_max <= 0 else min(self.dt_mult, self.dp_target / dp_max)
        return min(dt * f, self.dt_max)
