/*
 * Seeded synthetic workloads for the EDFA hot path: brick grids, conductivity
 * fields and the MHFE(RT0)-FV block system [A B; C D] of the model problem
 * (Sec. 2.2-2.3, Eq. (B_ij), Eq. (fluxes_MHFEM_3), Eq. (discr_bal_FV_2),
 * Eq. (fluxes_MHFEM_STRONG), Eq. (cont_fluxes), Appendix A).
 *
 * This module only PRODUCES inputs.  It holds none of the preconditioner's
 * arithmetic (no restriction sets, local solves, Schur complement,
 * incomplete factorisation or Krylov iteration); both the CPU oracle and the
 * CUDA library consume what it writes.
 *
 * Notation: A = A_pipi (faces x faces), B = A_pip (faces x cells),
 * C = A_ppi (cells x faces), D = A_pp (cells x cells).  W^E = (B^E)^{-1} is
 * the inverse elemental matrix of cell E, L_i^E = sum_j W^E_ij.
 *
 * Grid numbering: cells lexicographic (ix fastest).  Faces: all x-faces,
 * then all y-faces, then all z-faces, each lexicographic with the face
 * coordinate fastest.  Local face order in a cell: x-, x+, y-, y+, z-, z+.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WL_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ RNG */
/* SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014): state += golden gamma, then a
 * two-multiply xor-shift finaliser. */
WL_EXPORT uint64_t wl_splitmix64(uint64_t* s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform on [0,1) with 53 random bits */
WL_EXPORT double wl_uniform(uint64_t* s)
{
    return (double)(wl_splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------------
 * exp, log, sin and cos of the generator, written with IEEE +, -, *, / and
 * exact scalings by powers of two only.  Host math libraries differ in the
 * last bit between machines (x86-64 and aarch64 builds of the same library
 * included), which made the generated matrices, and with them iteration
 * counts, depend on the host; with these a seed gives the same bits on every
 * IEEE-754 host (the library is compiled with floating-point contraction off).
 * Accuracy is a few ulp, which is all a synthetic input needs.
 *
 * exp:  x = k ln2 + r with |r| <= ln2/2, ln2 split as LN2_HI + LN2_LO where
 *       LN2_HI has 32 significant bits (k LN2_HI is exact); e^r by its Taylor
 *       polynomial of degree 16 in Horner form; times 2^k.
 * log:  x = m 2^e with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(s) with
 *       s = (m - 1)/(m + 1), |s| <= 0.172, odd series to s^25; plus e ln2.
 * sin, cos: x = k pi/2 + r with |r| <= pi/4, pi/2 split in three parts of 33,
 *       33 and 53 significant bits (Cody-Waite reduction, exact products for
 *       |k| < 2^20); Taylor polynomials of sin r (to r^21) and cos r (to
 *       r^22); the quadrant k mod 4 picks the sign and the function.
 * The split constants are pi/2 and ln 2 computed to 60 digits and cut after
 * the stated numbers of bits.
 * --------------------------------------------------------------------- */
static const double WL_LN2_HI = 0.6931471803691238;
static const double WL_LN2_LO = 1.9082149292705877e-10;
static const double WL_INV_LN2 = 1.4426950408889634;
static const double WL_PIO2_1 = 1.5707963267341256;
static const double WL_PIO2_2 = 6.077100506303966e-11;
static const double WL_PIO2_3 = 2.0222662487959506e-21;
static const double WL_TWO_OVER_PI = 0.6366197723675814;

WL_EXPORT double wl_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return HUGE_VAL;
    if (x < -745.0) return 0.0;
    double k = floor(x * WL_INV_LN2 + 0.5);
    double r = (x - k * WL_LN2_HI) - k * WL_LN2_LO;
    double p = 1.0;
    for (int n = 16; n >= 1; --n) p = 1.0 + p * r / (double)n;
    return ldexp(p, (int)k);
}

WL_EXPORT double wl_log(double x)
{
    if (!(x > 0.0)) return x == 0.0 ? -HUGE_VAL : (x - x) / (x - x);
    if (x == HUGE_VAL) return x;
    int e = 0;
    double m = frexp(x, &e); /* m in [1/2, 1) */
    if (m < 0.7071067811865476) { m *= 2.0; e -= 1; }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double t = 1.0 / 25.0;
    for (int k = 23; k >= 1; k -= 2) t = 1.0 / (double)k + s2 * t;
    return (2.0 * s * t + (double)e * WL_LN2_LO) + (double)e * WL_LN2_HI;
}

static double wl_sin_poly(double r)
{
    double r2 = r * r, t = 1.0;
    for (int n = 21; n >= 3; n -= 2) t = 1.0 - t * r2 / ((double)n * (double)(n - 1));
    return r * t;
}

static double wl_cos_poly(double r)
{
    double r2 = r * r, t = 1.0;
    for (int n = 22; n >= 2; n -= 2) t = 1.0 - t * r2 / ((double)n * (double)(n - 1));
    return t;
}

/* quadrant q = k mod 4 and reduced argument r of x */
static double wl_reduce(double x, int* q)
{
    double k = floor(x * WL_TWO_OVER_PI + 0.5);
    double r = ((x - k * WL_PIO2_1) - k * WL_PIO2_2) - k * WL_PIO2_3;
    long long kk = (long long)k;
    *q = (int)(((kk % 4) + 4) % 4);
    return r;
}

WL_EXPORT double wl_sin(double x)
{
    int q;
    double r = wl_reduce(x, &q);
    switch (q) {
    case 0: return wl_sin_poly(r);
    case 1: return wl_cos_poly(r);
    case 2: return -wl_sin_poly(r);
    default: return -wl_cos_poly(r);
    }
}

WL_EXPORT double wl_cos(double x)
{
    int q;
    double r = wl_reduce(x, &q);
    switch (q) {
    case 0: return wl_cos_poly(r);
    case 1: return -wl_sin_poly(r);
    case 2: return -wl_cos_poly(r);
    default: return wl_sin_poly(r);
    }
}

/* elementwise forms for the Python side: out[i] = f(in[i]), f = 0 exp, 1 log,
 * 2 sin, 3 cos */
WL_EXPORT void wl_vmath(int f, int64_t n, const double* in, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        double x = in[i];
        out[i] = f == 0 ? wl_exp(x) : f == 1 ? wl_log(x) : f == 2 ? wl_sin(x) : wl_cos(x);
    }
}

/* standard normal by the Box-Muller transform (cosine branch only) */
WL_EXPORT double wl_normal(uint64_t* s)
{
    double u1 = 1.0 - wl_uniform(s); /* (0,1] */
    double u2 = wl_uniform(s);
    return sqrt(-2.0 * wl_log(u1)) * wl_cos(6.283185307179586 * u2);
}

WL_EXPORT void wl_fill_uniform(uint64_t* s, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = wl_uniform(s);
}

WL_EXPORT void wl_fill_normal(uint64_t* s, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = wl_normal(s);
}

/* --------------------------------------------------------------- types */
typedef struct {
    int32_t nx, ny, nz;
    double hx, hy, hz;
    double dt, stor;     /* backward-Euler step and storage coefficient c */
    int32_t fv_kind;     /* 0: strong inter-element flux (Appendix A)
                            1: upwind-mobility cell rows C = -B^T diag(lam) */
    int32_t dirichlet;   /* 1: prescribed pressure on the x=0 and x=1 faces */
    double p_left, p_right;
    const double* K;     /* [Ne*6] Kxx Kyy Kzz Kxy Kxz Kyz per cell */
    const double* lam_face; /* [Nf] face mobility (fv_kind 1 only) */
    const double* xyz;   /* optional [(nx+1)(ny+1)(nz+1)*3] node coordinates (node (i,j,k)
                            lexicographic, i fastest): general hexahedra with trilinear
                            maps; NULL = brick cells hx x hy x hz */
} wl_problem;

typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;
    int64_t* rowptr;
    int32_t* col;
    double* val;
} wl_csr;

typedef struct {
    int32_t Nf, Ne;
    wl_csr A, B, C, D;
    double* f;          /* [Nf+Ne] right-hand side from the prescribed pressures */
    double* W;          /* [Ne*36] W^E row-major, local face order */
    int32_t* cell_faces;/* [Ne*6] */
    int32_t* face_cells;/* [Nf*2] minus-side, plus-side cell (-1 = none) */
    int8_t* face_dir;   /* [Nf] 1 = prescribed pressure face */
    double* face_pbar;  /* [Nf] prescribed pressure (0 elsewhere) */
} wl_system;

/* ------------------------------------------------------------ topology */
static inline int64_t nfx(const wl_problem* P) { return (int64_t)(P->nx + 1) * P->ny * P->nz; }
static inline int64_t nfy(const wl_problem* P) { return (int64_t)P->nx * (P->ny + 1) * P->nz; }
static inline int64_t nfz(const wl_problem* P) { return (int64_t)P->nx * P->ny * (P->nz + 1); }

static inline int32_t xface(const wl_problem* P, int fx, int iy, int iz)
{ return (int32_t)(fx + (int64_t)(P->nx + 1) * (iy + (int64_t)P->ny * iz)); }
static inline int32_t yface(const wl_problem* P, int ix, int fy, int iz)
{ return (int32_t)(nfx(P) + ix + (int64_t)P->nx * (fy + (int64_t)(P->ny + 1) * iz)); }
static inline int32_t zface(const wl_problem* P, int ix, int iy, int fz)
{ return (int32_t)(nfx(P) + nfy(P) + ix + (int64_t)P->nx * (iy + (int64_t)P->ny * fz)); }

/* ------------------------------------------------- elemental matrices */
/* B^E_ij = gamma * int eta_i^T K^{-1} eta_j over a brick (Eq. B_ij), gamma = 1,
 * with the RT0 fields eta = s*phi/(h_a*A_a) e_a, phi = distance to the
 * opposite face, s = +1 on the + face and -1 on the - face. */
static void elem_B(const double K6[6], double hx, double hy, double hz, double Bm[36])
{
    double kxx = K6[0], kyy = K6[1], kzz = K6[2], kxy = K6[3], kxz = K6[4], kyz = K6[5];
    /* M = K^{-1} by cofactors */
    double c00 = kyy * kzz - kyz * kyz;
    double c01 = -(kxy * kzz - kyz * kxz);
    double c02 = kxy * kyz - kyy * kxz;
    double c11 = kxx * kzz - kxz * kxz;
    double c12 = -(kxx * kyz - kxy * kxz);
    double c22 = kxx * kyy - kxy * kxy;
    double det = kxx * c00 + kxy * c01 + kxz * c02;
    double M[3][3] = {{c00 / det, c01 / det, c02 / det},
                      {c01 / det, c11 / det, c12 / det},
                      {c02 / det, c12 / det, c22 / det}};
    double h[3] = {hx, hy, hz};
    double Ar[3] = {hy * hz, hx * hz, hx * hy};
    double V = hx * hy * hz;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            int a = i / 2, b = j / 2;
            double si = (i & 1) ? 1.0 : -1.0, sj = (j & 1) ? 1.0 : -1.0;
            double v;
            if (a == b) {
                if (i == j) v = M[a][a] * h[a] / (3.0 * Ar[a]);
                else v = -M[a][a] * h[a] / (6.0 * Ar[a]);
            } else {
                v = si * sj * M[a][b] * V / (4.0 * Ar[a] * Ar[b]);
            }
            Bm[i * 6 + j] = v;
        }
}

/* W = B^{-1} through a 6x6 Cholesky factorisation, then symmetrised so that
 * the assembled face block is exactly symmetric. Returns 0 on success. */
static int spd_inverse6(const double Bm[36], double Wm[36])
{
    double L[36];
    memset(L, 0, sizeof L);
    for (int j = 0; j < 6; ++j) {
        double d = Bm[j * 6 + j];
        for (int k = 0; k < j; ++k) d -= L[j * 6 + k] * L[j * 6 + k];
        if (!(d > 0.0)) return -1;
        L[j * 6 + j] = sqrt(d);
        for (int i = j + 1; i < 6; ++i) {
            double v = Bm[i * 6 + j];
            for (int k = 0; k < j; ++k) v -= L[i * 6 + k] * L[j * 6 + k];
            L[i * 6 + j] = v / L[j * 6 + j];
        }
    }
    for (int c = 0; c < 6; ++c) {
        double y[6], x[6];
        for (int i = 0; i < 6; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[i * 6 + k] * y[k];
            y[i] = v / L[i * 6 + i];
        }
        for (int i = 5; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < 6; ++k) v -= L[k * 6 + i] * x[k];
            x[i] = v / L[i * 6 + i];
        }
        for (int i = 0; i < 6; ++i) Wm[i * 6 + c] = x[i];
    }
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            double s = 0.5 * (Wm[i * 6 + j] + Wm[j * 6 + i]);
            Wm[i * 6 + j] = s;
            Wm[j * 6 + i] = s;
        }
    return 0;
}

/* General hexahedron (Sec. 2.2, Eq. B_ij with the Piola transformation of the
 * RT0 fields): cell = image of the unit cube by the trilinear map F through its
 * 8 nodes X[8][3] (node a = (a&1, (a>>1)&1, (a>>2)&1) in reference coordinates).
 * Reference fields with unit outward flux through their face (local order
 * x-, x+, y-, y+, z-, z+): w_{x-} = (x^-1, 0, 0), w_{x+} = (x^, 0, 0), and
 * cyclic; physical fields w = DF w^ / J (flux preserving), so
 *     B_ij = int_cube (DF w^_i)^T K^{-1} (DF w^_j) / J  dx^,
 * by 3 x 3 x 3 Gauss-Legendre quadrature; vol = int_cube J dx^. */
static void hex_jac(const double X[24], double u, double v, double w, double DF[9])
{
    /* DF[r*3+c] = d x_r / d xhat_c */
    memset(DF, 0, 9 * sizeof(double));
    for (int a = 0; a < 8; ++a) {
        const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
        const double fu = ia ? u : 1.0 - u, fv = ja ? v : 1.0 - v, fw = ka ? w : 1.0 - w;
        const double du = ia ? 1.0 : -1.0, dv = ja ? 1.0 : -1.0, dw = ka ? 1.0 : -1.0;
        const double g[3] = {du * fv * fw, fu * dv * fw, fu * fv * dw};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) DF[r * 3 + c] += X[3 * a + r] * g[c];
    }
}

static int elem_B_hex(const double K6[6], const double X[24], double Bm[36], double* vol)
{
    const double kxx = K6[0], kyy = K6[1], kzz = K6[2], kxy = K6[3], kxz = K6[4], kyz = K6[5];
    const double c00 = kyy * kzz - kyz * kyz, c01 = -(kxy * kzz - kyz * kxz), c02 = kxy * kyz - kyy * kxz;
    const double c11 = kxx * kzz - kxz * kxz, c12 = -(kxx * kyz - kxy * kxz), c22 = kxx * kyy - kxy * kxy;
    const double det = kxx * c00 + kxy * c01 + kxz * c02;
    const double M[9] = {c00 / det, c01 / det, c02 / det, c01 / det, c11 / det, c12 / det,
                         c02 / det, c12 / det, c22 / det};
    /* 3-point Gauss-Legendre on [0,1] */
    const double gx[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    memset(Bm, 0, 36 * sizeof(double));
    double V = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                const double u = gx[a], v = gx[b], w = gx[c], wt = gw[a] * gw[b] * gw[c];
                double DF[9];
                hex_jac(X, u, v, w, DF);
                const double J = DF[0] * (DF[4] * DF[8] - DF[5] * DF[7]) - DF[1] * (DF[3] * DF[8] - DF[5] * DF[6]) +
                                 DF[2] * (DF[3] * DF[7] - DF[4] * DF[6]);
                if (!(J > 0.0)) return -1;
                V += wt * J;
                /* DF w^_l for the six fields: column a of DF times the scalar */
                const double sc[6] = {u - 1.0, u, v - 1.0, v, w - 1.0, w};
                double Y[6][3];
                for (int l = 0; l < 6; ++l)
                    for (int r = 0; r < 3; ++r) Y[l][r] = DF[r * 3 + l / 2] * sc[l];
                for (int i = 0; i < 6; ++i) {
                    double MY[3];
                    for (int r = 0; r < 3; ++r) MY[r] = M[r * 3] * Y[i][0] + M[r * 3 + 1] * Y[i][1] + M[r * 3 + 2] * Y[i][2];
                    for (int j = 0; j < 6; ++j)
                        Bm[i * 6 + j] += wt / J * (MY[0] * Y[j][0] + MY[1] * Y[j][1] + MY[2] * Y[j][2]);
                }
            }
    *vol = V;
    return 0;
}

WL_EXPORT int wl_elem_B_hex(const double K6[6], const double X[24], double Bm[36], double* vol)
{
    return elem_B_hex(K6, X, Bm, vol);
}

/* the 8 nodes of cell (ix, iy, iz) of a structured hexahedral grid */
static void cell_nodes(const wl_problem* P, int ix, int iy, int iz, double X[24])
{
    for (int a = 0; a < 8; ++a) {
        const int i = ix + (a & 1), j = iy + ((a >> 1) & 1), k = iz + ((a >> 2) & 1);
        const int64_t nd = i + (int64_t)(P->nx + 1) * (j + (int64_t)(P->ny + 1) * k);
        for (int r = 0; r < 3; ++r) X[3 * a + r] = P->xyz[3 * nd + r];
    }
}

WL_EXPORT int wl_elem_W(const double K6[6], double hx, double hy, double hz, double Wm[36])
{
    double Bm[36];
    elem_B(K6, hx, hy, hz, Bm);
    return spd_inverse6(Bm, Wm);
}

WL_EXPORT void wl_elem_B(const double K6[6], double hx, double hy, double hz, double Bm[36])
{
    elem_B(K6, hx, hy, hz, Bm);
}

/* ------------------------------------------------------------ triplets */
typedef struct {
    int64_t n, cap;
    int32_t* r;
    int32_t* c;
    double* v;
} trip;

static int trip_push(trip* t, int32_t r, int32_t c, double v)
{
    if (t->n == t->cap) {
        int64_t nc = t->cap ? 2 * t->cap : 1024;
        int32_t* nr = (int32_t*)realloc(t->r, nc * sizeof(int32_t));
        if (!nr) return -1;
        t->r = nr;
        int32_t* ncc = (int32_t*)realloc(t->c, nc * sizeof(int32_t));
        if (!ncc) return -1;
        t->c = ncc;
        double* nv = (double*)realloc(t->v, nc * sizeof(double));
        if (!nv) return -1;
        t->v = nv;
        t->cap = nc;
    }
    t->r[t->n] = r;
    t->c[t->n] = c;
    t->v[t->n] = v;
    t->n++;
    return 0;
}

static void trip_free(trip* t) { free(t->r); free(t->c); free(t->v); memset(t, 0, sizeof *t); }

/* Triplets -> CSR with ascending columns and duplicates summed in push order
 * (stable counting sort by row, then insertion sort by column within a row). */
static int trip_to_csr(const trip* t, int32_t nrows, int32_t ncols, wl_csr* M)
{
    M->nrows = nrows;
    M->ncols = ncols;
    int64_t* cnt = (int64_t*)calloc((size_t)nrows + 1, sizeof(int64_t));
    int32_t* cc = (int32_t*)malloc((size_t)(t->n ? t->n : 1) * sizeof(int32_t));
    double* vv = (double*)malloc((size_t)(t->n ? t->n : 1) * sizeof(double));
    if (!cnt || !cc || !vv) { free(cnt); free(cc); free(vv); return -1; }
    for (int64_t k = 0; k < t->n; ++k) cnt[t->r[k] + 1]++;
    for (int32_t i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
    int64_t* pos = (int64_t*)malloc((size_t)(nrows ? nrows : 1) * sizeof(int64_t));
    if (!pos) { free(cnt); free(cc); free(vv); return -1; }
    memcpy(pos, cnt, (size_t)nrows * sizeof(int64_t));
    for (int64_t k = 0; k < t->n; ++k) {
        int64_t p = pos[t->r[k]]++;
        cc[p] = t->c[k];
        vv[p] = t->v[k];
    }
    free(pos);
    /* sort within rows (stable insertion sort), merge duplicates */
    int64_t* rp = (int64_t*)malloc(((size_t)nrows + 1) * sizeof(int64_t));
    if (!rp) { free(cnt); free(cc); free(vv); return -1; }
    int64_t out = 0;
    rp[0] = 0;
    for (int32_t i = 0; i < nrows; ++i) {
        int64_t b = cnt[i], e = cnt[i + 1];
        for (int64_t p = b + 1; p < e; ++p) {
            int32_t kc = cc[p];
            double kv = vv[p];
            int64_t q = p - 1;
            while (q >= b && cc[q] > kc) { cc[q + 1] = cc[q]; vv[q + 1] = vv[q]; --q; }
            cc[q + 1] = kc;
            vv[q + 1] = kv;
        }
        for (int64_t p = b; p < e; ++p) {
            if (out > rp[i] && cc[out - 1] == cc[p]) vv[out - 1] += vv[p];
            else { cc[out] = cc[p]; vv[out] = vv[p]; out++; }
        }
        rp[i + 1] = out;
    }
    free(cnt);
    M->rowptr = rp;
    M->col = cc;
    M->val = vv;
    M->nnz = out;
    return 0;
}

/* keep entries for which keep(row, col, val) is true; compacts in place */
typedef int (*keep_fn)(const void* ctx, int32_t r, int32_t c, double v);

static void csr_filter(wl_csr* M, keep_fn keep, const void* ctx)
{
    int64_t out = 0, b = 0;
    for (int32_t i = 0; i < M->nrows; ++i) {
        int64_t e = M->rowptr[i + 1];
        for (int64_t p = b; p < e; ++p)
            if (keep(ctx, i, M->col[p], M->val[p])) {
                M->col[out] = M->col[p];
                M->val[out] = M->val[p];
                out++;
            }
        b = e;
        M->rowptr[i + 1] = out;
    }
    M->nnz = out;
}

typedef struct { const int8_t* dir; int mode; } keep_ctx;

/* mode 0: face block A: drop couplings of prescribed faces (keep their
 *         diagonal), drop exact zeros off the diagonal
 * mode 1: B: drop rows of prescribed faces and exact zeros
 * mode 2: C: drop columns of prescribed faces and exact zeros
 * mode 3: D: drop exact zeros off the diagonal */
static int keep_entry(const void* vctx, int32_t r, int32_t c, double v)
{
    const keep_ctx* k = (const keep_ctx*)vctx;
    switch (k->mode) {
    case 0:
        if (r == c) return 1;
        if (k->dir[r] || k->dir[c]) return 0;
        return v != 0.0;
    case 1:
        if (k->dir[r]) return 0;
        return v != 0.0;
    case 2:
        if (k->dir[c]) return 0;
        return v != 0.0;
    default:
        if (r == c) return 1;
        return v != 0.0;
    }
}

WL_EXPORT void wl_free_system(wl_system* S)
{
    wl_csr* m[4] = {&S->A, &S->B, &S->C, &S->D};
    for (int k = 0; k < 4; ++k) {
        free(m[k]->rowptr);
        free(m[k]->col);
        free(m[k]->val);
    }
    free(S->f);
    free(S->W);
    free(S->cell_faces);
    free(S->face_cells);
    free(S->face_dir);
    free(S->face_pbar);
    memset(S, 0, sizeof *S);
}

/* ------------------------------------------------------------ assembly */
WL_EXPORT int wl_assemble(const wl_problem* P, wl_system* S)
{
    memset(S, 0, sizeof *S);
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const int64_t Ne64 = (int64_t)nx * ny * nz;
    const int64_t Nf64 = nfx(P) + nfy(P) + nfz(P);
    if (nx < 1 || ny < 1 || nz < 1 || Nf64 >= INT32_MAX) return -1;
    const int32_t Ne = (int32_t)Ne64, Nf = (int32_t)Nf64;
    S->Ne = Ne;
    S->Nf = Nf;
    S->W = (double*)malloc((size_t)Ne * 36 * sizeof(double));
    S->cell_faces = (int32_t*)malloc((size_t)Ne * 6 * sizeof(int32_t));
    S->face_cells = (int32_t*)malloc((size_t)Nf * 2 * sizeof(int32_t));
    S->face_dir = (int8_t*)calloc((size_t)Nf, 1);
    S->face_pbar = (double*)calloc((size_t)Nf, sizeof(double));
    S->f = (double*)calloc((size_t)Nf + Ne, sizeof(double));
    if (!S->W || !S->cell_faces || !S->face_cells || !S->face_dir || !S->face_pbar || !S->f) {
        wl_free_system(S);
        return -2;
    }
    for (int64_t i = 0; i < 2 * (int64_t)Nf; ++i) S->face_cells[i] = -1;
    double* vol = (double*)malloc((size_t)Ne * sizeof(double));  /* cell volumes Omega_E */
    if (!vol) { wl_free_system(S); return -2; }

    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int32_t e = ix + nx * (iy + ny * iz);
                int32_t* cf = S->cell_faces + (int64_t)e * 6;
                cf[0] = xface(P, ix, iy, iz);
                cf[1] = xface(P, ix + 1, iy, iz);
                cf[2] = yface(P, ix, iy, iz);
                cf[3] = yface(P, ix, iy + 1, iz);
                cf[4] = zface(P, ix, iy, iz);
                cf[5] = zface(P, ix, iy, iz + 1);
                for (int l = 0; l < 6; ++l) {
                    /* a cell is the plus-side cell of its minus faces */
                    int side = (l & 1) ? 0 : 1;
                    S->face_cells[2 * (int64_t)cf[l] + side] = e;
                }
                if (P->xyz) {
                    double X[24], Bm[36];
                    cell_nodes(P, ix, iy, iz, X);
                    if (elem_B_hex(P->K + 6 * (int64_t)e, X, Bm, vol + e) ||
                        spd_inverse6(Bm, S->W + 36 * (int64_t)e)) {
                        free(vol);
                        wl_free_system(S);
                        return -3;
                    }
                } else {
                    vol[e] = P->hx * P->hy * P->hz;
                    if (wl_elem_W(P->K + 6 * (int64_t)e, P->hx, P->hy, P->hz, S->W + 36 * (int64_t)e)) {
                        free(vol);
                        wl_free_system(S);
                        return -3;
                    }
                }
            }
    if (P->dirichlet)
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy) {
                int32_t f0 = xface(P, 0, iy, iz), f1 = xface(P, nx, iy, iz);
                S->face_dir[f0] = 1;
                S->face_pbar[f0] = P->p_left;
                S->face_dir[f1] = 1;
                S->face_pbar[f1] = P->p_right;
            }

    trip tA = {0}, tB = {0}, tC = {0}, tD = {0};
    int err = 0;
    /* face rows: q_i^E + q_i^E' = 0 with q^E = W^E (p^E 1 - pi^E)
       (Eq. fluxes_MHFEM_3, Eq. cont_fluxes); no-flow faces keep only q_i^E */
    for (int32_t i = 0; i < Nf && !err; ++i)
        for (int side = 0; side < 2; ++side) {
            int32_t e = S->face_cells[2 * (int64_t)i + side];
            if (e < 0) continue;
            const int32_t* cf = S->cell_faces + (int64_t)e * 6;
            const double* W = S->W + 36 * (int64_t)e;
            int li = 0;
            while (cf[li] != i) ++li;
            double L = 0.0;
            for (int j = 0; j < 6; ++j) {
                err |= trip_push(&tA, i, cf[j], -W[li * 6 + j]);
                L += W[li * 6 + j];
            }
            err |= trip_push(&tB, i, e, L);
        }
    /* cell rows */
    for (int32_t e = 0; e < Ne && !err; ++e) {
        const double acc = vol[e] * P->stor / P->dt;
        const int32_t* cf = S->cell_faces + (int64_t)e * 6;
        const double* W = S->W + 36 * (int64_t)e;
        double Lrow[6];
        for (int l = 0; l < 6; ++l) {
            double s = 0.0;
            for (int j = 0; j < 6; ++j) s += W[l * 6 + j];
            Lrow[l] = s;
        }
        err |= trip_push(&tD, e, e, acc);
        if (P->fv_kind == 1) {
            /* C = -B^T diag(lam_face), D = diag(sum_f lam_f B_fE) + acc */
            for (int l = 0; l < 6; ++l) {
                double lam = P->lam_face[cf[l]];
                err |= trip_push(&tC, e, cf[l], -lam * Lrow[l]);
                err |= trip_push(&tD, e, e, lam * Lrow[l]);
            }
            continue;
        }
        for (int l = 0; l < 6; ++l) {
            int32_t i = cf[l];
            int side = (l & 1) ? 0 : 1; /* this cell's slot on face i */
            int32_t e2 = S->face_cells[2 * (int64_t)i + (1 - side)];
            if (e2 >= 0) {
                /* strong inter-element flux (Eq. fluxes_MHFEM_STRONG):
                   q = w Lambda^E - (1-w) Lambda^E', w = W'_ii / (W_ii + W'_ii) */
                const int32_t* cf2 = S->cell_faces + (int64_t)e2 * 6;
                const double* W2 = S->W + 36 * (int64_t)e2;
                int l2 = 0;
                while (cf2[l2] != i) ++l2;
                double L2 = 0.0;
                for (int j = 0; j < 6; ++j) L2 += W2[l2 * 6 + j];
                double w = W2[l2 * 6 + l2] / (W[l * 6 + l] + W2[l2 * 6 + l2]);
                double wc = W[l * 6 + l] / (W[l * 6 + l] + W2[l2 * 6 + l2]);
                err |= trip_push(&tD, e, e, w * Lrow[l]);
                for (int j = 0; j < 6; ++j)
                    if (j != l) err |= trip_push(&tC, e, cf[j], -w * W[l * 6 + j]);
                err |= trip_push(&tD, e, e2, -wc * L2);
                for (int j = 0; j < 6; ++j)
                    if (j != l2) err |= trip_push(&tC, e, cf2[j], wc * W2[l2 * 6 + j]);
            } else if (S->face_dir[i]) {
                /* prescribed-pressure face: q_i = sum_j W_ij (p^E - pi_j), pi_i = pbar */
                err |= trip_push(&tD, e, e, Lrow[l]);
                for (int j = 0; j < 6; ++j) err |= trip_push(&tC, e, cf[j], -W[l * 6 + j]);
            }
            /* no-flow face: q_i = 0 */
        }
    }
    free(vol);
    if (err) { trip_free(&tA); trip_free(&tB); trip_free(&tC); trip_free(&tD); wl_free_system(S); return -2; }
    err |= trip_to_csr(&tA, Nf, Nf, &S->A);
    err |= trip_to_csr(&tB, Nf, Ne, &S->B);
    err |= trip_to_csr(&tC, Ne, Nf, &S->C);
    err |= trip_to_csr(&tD, Ne, Ne, &S->D);
    trip_free(&tA); trip_free(&tB); trip_free(&tC); trip_free(&tD);
    if (err) { wl_free_system(S); return -2; }

    /* move the prescribed face pressures to the right-hand side (symmetric
       elimination: the face keeps its unknown, row i reads A_ii pi_i = A_ii pbar) */
    double* fpi = S->f;
    double* fp = S->f + Nf;
    for (int32_t r = 0; r < Nf; ++r)
        for (int64_t p = S->A.rowptr[r]; p < S->A.rowptr[r + 1]; ++p) {
            int32_t c = S->A.col[p];
            if (c == r) { if (S->face_dir[r]) fpi[r] = S->A.val[p] * S->face_pbar[r]; }
            else if (S->face_dir[c] && !S->face_dir[r]) fpi[r] -= S->A.val[p] * S->face_pbar[c];
        }
    for (int32_t r = 0; r < Ne; ++r)
        for (int64_t p = S->C.rowptr[r]; p < S->C.rowptr[r + 1]; ++p) {
            int32_t c = S->C.col[p];
            if (S->face_dir[c]) fp[r] -= S->C.val[p] * S->face_pbar[c];
        }
    keep_ctx k0 = {S->face_dir, 0}, k1 = {S->face_dir, 1}, k2 = {S->face_dir, 2}, k3 = {S->face_dir, 3};
    csr_filter(&S->A, keep_entry, &k0);
    csr_filter(&S->B, keep_entry, &k1);
    csr_filter(&S->C, keep_entry, &k2);
    csr_filter(&S->D, keep_entry, &k3);
    return 0;
}
