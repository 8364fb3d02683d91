/*
 * EDFA oracle: a plain, slow, FP64 CPU implementation of the preconditioner
 * hot path of Nardean, Ferronato & Abushaikha, "A novel block non-symmetric
 * preconditioner for mixed-hybrid finite-element-based flow simulations"
 * (arXiv 2009.13916).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code with the CUDA library.
 *
 * Block notation: A = A_pipi (N_f x N_f), B = A_pip, C = A_ppi, D = A_pp.
 * Every routine is the plain definition written out with loops, in the order
 * the paper states it; no blocking, fusion or reordering.
 *
 *   restriction sets .......... Sec. 3, Eq. (r_r^m), static/dynamic techniques,
 *                               Algorithm 1 (dynamic branch)
 *   restricted local solves ... Eq. (syst_MRHS_res), Eq. (syst_MRHS_res-F)
 *   approximate Schur ......... Eq. (sparse_S): S~ = D - G~ A F~ (two-sided)
 *                               and S~ = D - C X~ with X~ = -F~ (one-sided)
 *   inner factorisations ...... ILU(0), natural ordering (Saad, Alg. 10.4)
 *   preconditioner ............ Eq. (EDFA_prec), Remark 1
 *   outer Krylov .............. right-preconditioned flexible GMRES(m),
 *                               modified Gram-Schmidt, Givens rotations,
 *                               x0 = 0, stop at ||b - Ax|| / ||b|| <= tol
 *                               (stopping rule of Sec. 4)
 *   adjoint gradient .......... dL/dlog k_E = lambda^T (db/dtheta - dA/dtheta u)
 *                               with the row formulas of Appendix A
 *                               differentiated by forward-mode dual numbers
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
} orc_csr;

/* owned CSR returned to the caller; release with orc_free_csr */
typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;
    int64_t* rowptr;
    int32_t* col;
    double* val;
} orc_ocsr;

ORC_EXPORT void orc_free(void* p) { free(p); }

ORC_EXPORT void orc_free_csr(orc_ocsr* M)
{
    free(M->rowptr);
    free(M->col);
    free(M->val);
    memset(M, 0, sizeof *M);
}

/* ------------------------------------------------------------ helpers */
static double csr_get(const orc_csr* M, int32_t r, int32_t c, int* found)
{
    for (int64_t p = M->rowptr[r]; p < M->rowptr[r + 1]; ++p)
        if (M->col[p] == c) { if (found) *found = 1; return M->val[p]; }
    if (found) *found = 0;
    return 0.0;
}

/* transpose pattern+values (plain two-pass counting) */
static int csr_transpose(const orc_csr* M, orc_ocsr* T)
{
    T->nrows = M->ncols;
    T->ncols = M->nrows;
    T->nnz = M->rowptr[M->nrows];
    T->rowptr = (int64_t*)calloc((size_t)T->nrows + 1, sizeof(int64_t));
    T->col = (int32_t*)malloc((size_t)(T->nnz ? T->nnz : 1) * sizeof(int32_t));
    T->val = (double*)malloc((size_t)(T->nnz ? T->nnz : 1) * sizeof(double));
    if (!T->rowptr || !T->col || !T->val) return -1;
    for (int64_t p = 0; p < T->nnz; ++p) T->rowptr[M->col[p] + 1]++;
    for (int32_t i = 0; i < T->nrows; ++i) T->rowptr[i + 1] += T->rowptr[i];
    int64_t* pos = (int64_t*)malloc((size_t)(T->nrows ? T->nrows : 1) * sizeof(int64_t));
    if (!pos) return -1;
    memcpy(pos, T->rowptr, (size_t)T->nrows * sizeof(int64_t));
    for (int32_t r = 0; r < M->nrows; ++r)
        for (int64_t p = M->rowptr[r]; p < M->rowptr[r + 1]; ++p) {
            int64_t q = pos[M->col[p]]++;
            T->col[q] = r;
            T->val[q] = M->val[p];
        }
    free(pos);
    return 0;
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* sort ascending and remove duplicates; returns new length */
static int64_t sort_unique(int32_t* v, int64_t n)
{
    if (n <= 1) return n;
    qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
    int64_t o = 1;
    for (int64_t i = 1; i < n; ++i)
        if (v[i] != v[o - 1]) v[o++] = v[i];
    return o;
}

/* growable int list */
typedef struct { int64_t n, cap; int32_t* v; } ilist;
static int il_push(ilist* l, int32_t x)
{
    if (l->n == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 256;
        int32_t* nv = (int32_t*)realloc(l->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return -1;
        l->v = nv;
        l->cap = nc;
    }
    l->v[l->n++] = x;
    return 0;
}

/* ------------------------------------------------- restriction sets */
/* Static restriction sets Q^(m), ascending and duplicate free.
 *   mode 0 OWN    : F_m, the faces of cell m = stored rows of column m of B
 *   mode 1 NBR    : F_m and the faces of every cell sharing a face with m
 *                   (the overlapping-patch static technique of Sec. 3)
 *   mode 2 CROW   : stored columns of row m of C (the base pattern Q_{A_ppi})
 *   mode 3 THRESH : F_m and every j with A_ij stored, i in F_m, and
 *                   |A_ij| >= thresh * |A_ii|
 * Outputs are malloc'd; release with orc_free. */
ORC_EXPORT int orc_qsets(int mode, double thresh, const orc_csr* A, const orc_csr* B,
                         const orc_csr* C, int64_t** qptr_out, int32_t** qidx_out)
{
    const int32_t Ne = B->ncols;
    orc_ocsr Bt = {0};
    if (csr_transpose(B, &Bt)) return -1;
    int64_t* qptr = (int64_t*)malloc(((size_t)Ne + 1) * sizeof(int64_t));
    ilist out = {0};
    if (!qptr) return -1;
    qptr[0] = 0;
    for (int32_t m = 0; m < Ne; ++m) {
        ilist cand = {0};
        if (mode == 2) {
            for (int64_t p = C->rowptr[m]; p < C->rowptr[m + 1]; ++p) il_push(&cand, C->col[p]);
        } else {
            for (int64_t p = Bt.rowptr[m]; p < Bt.rowptr[m + 1]; ++p) {
                int32_t f = Bt.col[p];
                il_push(&cand, f);
                if (mode == 1) {
                    /* cells on face f */
                    for (int64_t q = B->rowptr[f]; q < B->rowptr[f + 1]; ++q) {
                        int32_t e2 = B->col[q];
                        if (e2 == m) continue;
                        for (int64_t t = Bt.rowptr[e2]; t < Bt.rowptr[e2 + 1]; ++t) il_push(&cand, Bt.col[t]);
                    }
                } else if (mode == 3) {
                    double aii = fabs(csr_get(A, f, f, NULL));
                    for (int64_t q = A->rowptr[f]; q < A->rowptr[f + 1]; ++q)
                        if (fabs(A->val[q]) >= thresh * aii) il_push(&cand, A->col[q]);
                }
            }
        }
        int64_t n = sort_unique(cand.v, cand.n);
        for (int64_t i = 0; i < n; ++i) il_push(&out, cand.v[i]);
        qptr[m + 1] = out.n;
        free(cand.v);
    }
    orc_free_csr(&Bt);
    *qptr_out = qptr;
    *qidx_out = out.v ? out.v : (int32_t*)malloc(sizeof(int32_t));
    return 0;
}

/* ------------------------------------------------- local dense solves */
/* Gather A^(m) = R A R^T for the ascending set q[0..s) (absent entries 0). */
static void gather_local(const orc_csr* A, const int32_t* q, int s, double* M)
{
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) M[i * s + j] = csr_get(A, q[i], q[j], NULL);
}

/* In-place LU factorisation without pivoting (Doolittle), M = L U with unit L. */
static int lu_nopivot(double* M, int s)
{
    for (int k = 0; k < s; ++k) {
        double piv = M[k * s + k];
        if (!(piv != 0.0) || !isfinite(piv)) return -1;
        for (int i = k + 1; i < s; ++i) {
            M[i * s + k] /= piv;
            double lik = M[i * s + k];
            for (int j = k + 1; j < s; ++j) M[i * s + j] -= lik * M[k * s + j];
        }
    }
    return 0;
}

static void lu_solve(const double* M, int s, double* x)
{
    for (int i = 0; i < s; ++i)
        for (int k = 0; k < i; ++k) x[i] -= M[i * s + k] * x[k];
    for (int i = s - 1; i >= 0; --i) {
        for (int k = i + 1; k < s; ++k) x[i] -= M[i * s + k] * x[k];
        x[i] /= M[i * s + i];
    }
}

/* Restricted solves for every cell m (Eq. syst_MRHS_res and syst_MRHS_res-F):
 *   -A^(m) g~ = R c_m^T      (c_m = row m of C)     -> gval: row m of G~ on Q^(m)
 *   -A^(m) f~ = R b_m        (b_m = column m of B)  -> xval: X~ = -F~ on Q^(m)
 * -A^(m) is factorised by LU without pivoting (it is SPD).  Either output may
 * be NULL.  A zero or non-finite pivot returns -2 with the cell in *bad. */
/* Thread count of the per-cell loop below (1 by default).  The local systems
 * are independent (Sec. 3, Remark 5) and the paper solves them under a
 * parallel loop over cells; with n > 1 the loop runs on n OpenMP threads.
 * Every cell's arithmetic is the same whatever n is, so the results are too. */
static int g_threads = 1;
ORC_EXPORT void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

ORC_EXPORT int orc_local_solves(const orc_csr* A, const orc_csr* B, const orc_csr* C,
                                const int64_t* qptr, const int32_t* qidx,
                                double* xval, double* gval, int32_t* bad)
{
    const int32_t Ne = B->ncols;
    int smax = 0;
    for (int32_t m = 0; m < Ne; ++m)
        if (qptr[m + 1] - qptr[m] > smax) smax = (int)(qptr[m + 1] - qptr[m]);
    int rc = 0;
    int32_t first_bad = -1;
#pragma omp parallel num_threads(g_threads)
    {
        double* M = (double*)malloc((size_t)(smax ? smax : 1) * (smax ? smax : 1) * sizeof(double));
        double* x = (double*)malloc((size_t)(smax ? smax : 1) * sizeof(double));
        if (!M || !x) {
#pragma omp critical
            rc = -1;
        }
#pragma omp for schedule(dynamic, 256)
        for (int32_t m = 0; m < Ne; ++m) {
            const int32_t* q = qidx + qptr[m];
            int s = (int)(qptr[m + 1] - qptr[m]);
            if (s == 0 || !M || !x) continue;
            gather_local(A, q, s, M);
            for (int i = 0; i < s * s; ++i) M[i] = -M[i];
            if (lu_nopivot(M, s)) {
#pragma omp critical
                if (first_bad < 0 || m < first_bad) first_bad = m;
                continue;
            }
            if (xval) {
                for (int i = 0; i < s; ++i) x[i] = csr_get(B, q[i], m, NULL);
                lu_solve(M, s, x);              /* x = f~ */
                for (int i = 0; i < s; ++i) xval[qptr[m] + i] = -x[i];
            }
            if (gval) {
                for (int i = 0; i < s; ++i) x[i] = csr_get(C, m, q[i], NULL);
                lu_solve(M, s, x);              /* x = g~ */
                for (int i = 0; i < s; ++i) gval[qptr[m] + i] = x[i];
            }
        }
        free(M);
        free(x);
    }
    if (rc) return rc;
    if (first_bad >= 0) {
        if (bad) *bad = first_bad;
        return -2;
    }
    return 0;
}

/* Dynamic technique (Sec. 3 and Algorithm 1, dynamic branch), one cell m:
 * start from Q_(0) = the stored columns of row m of C, solve for g~, form the
 * prolonged residual r = c_m^T + A R^T g~ (Eq. prol_res), then repeatedly add
 * at most n = min(n_add, n_ent - n_prog) new indices j (j not in Q, A_jq
 * stored for some q in Q) with the largest |r_j| (values within a relative
 * 1e-12 of the largest count as tied; ties: smaller j first),
 * re-solve and recompute r, while n_prog < n_ent and k < it_max.  The loop
 * also ends when no candidate index exists. */
/* relative width of a tie between prolonged-residual magnitudes */
#define DYN_TIE 1e-12

static int dyn_one(const orc_csr* A, const orc_csr* C, int32_t m, int n_add, int n_ent,
                   int it_max, ilist* Q)
{
    Q->n = 0;
    for (int64_t p = C->rowptr[m]; p < C->rowptr[m + 1]; ++p) il_push(Q, C->col[p]);
    int n_prog = 0, k = 0;
    int cap = (int)Q->n + n_ent;
    double* M = (double*)malloc((size_t)cap * cap * sizeof(double));
    double* g = (double*)malloc((size_t)cap * sizeof(double));
    if (!M || !g) { free(M); free(g); return -1; }
    for (;;) {
        int s = (int)Q->n;
        gather_local(A, Q->v, s, M);
        for (int i = 0; i < s * s; ++i) M[i] = -M[i];
        if (lu_nopivot(M, s)) { free(M); free(g); return -2; }
        for (int i = 0; i < s; ++i) g[i] = csr_get(C, m, Q->v[i], NULL);
        lu_solve(M, s, g);
        if (!(n_prog < n_ent && k < it_max)) break;
        /* candidates: j not in Q with a stored A_jq, q in Q; r_j = sum_q A_jq g_q
           (c_j = 0 there because Q_(0) holds every stored column of row m) */
        ilist cj = {0};
        for (int i = 0; i < s; ++i) {
            int32_t qq = Q->v[i];
            for (int64_t p = A->rowptr[qq]; p < A->rowptr[qq + 1]; ++p) il_push(&cj, A->col[p]);
        }
        int64_t nc = sort_unique(cj.v, cj.n);
        int64_t w = 0;
        for (int64_t t = 0; t < nc; ++t) {
            int32_t j = cj.v[t];
            int inq = 0;
            for (int i = 0; i < s; ++i) if (Q->v[i] == j) { inq = 1; break; }
            if (!inq) cj.v[w++] = j;
        }
        nc = w;
        if (nc == 0) { free(cj.v); break; }
        double* rv = (double*)malloc((size_t)nc * sizeof(double));
        for (int64_t t = 0; t < nc; ++t) {
            int32_t j = cj.v[t];
            double r = csr_get(C, m, j, NULL);
            for (int i = 0; i < s; ++i) r += csr_get(A, j, Q->v[i], NULL) * g[i];
            rv[t] = fabs(r);
        }
        k += 1;
        int n = n_add < (n_ent - n_prog) ? n_add : (n_ent - n_prog);
        int added = 0;
        while (added < n) {
            /* largest remaining |r_j|; every candidate within a relative
               DYN_TIE of it counts as tied, and the smallest j among the tied
               wins (candidates are ascending in j) */
            double rmax = -1.0;
            for (int64_t t = 0; t < nc; ++t)
                if (rv[t] >= 0 && rv[t] > rmax) rmax = rv[t];
            if (rmax < 0) break;
            int64_t best = -1;
            for (int64_t t = 0; t < nc; ++t)
                if (rv[t] >= 0 && rv[t] >= rmax * (1.0 - DYN_TIE)) { best = t; break; }
            il_push(Q, cj.v[best]);
            rv[best] = -1.0;
            added++;
        }
        free(rv);
        free(cj.v);
        n_prog += added;
        sort_unique(Q->v, Q->n);
    }
    free(M);
    free(g);
    return 0;
}

ORC_EXPORT int orc_qsets_dynamic(const orc_csr* A, const orc_csr* C, int n_add, int n_ent,
                                 int it_max, int64_t** qptr_out, int32_t** qidx_out)
{
    const int32_t Ne = C->nrows;
    int64_t* qptr = (int64_t*)malloc(((size_t)Ne + 1) * sizeof(int64_t));
    ilist out = {0}, Q = {0};
    if (!qptr) return -1;
    qptr[0] = 0;
    for (int32_t m = 0; m < Ne; ++m) {
        int rc = dyn_one(A, C, m, n_add, n_ent, it_max, &Q);
        if (rc) { free(qptr); free(out.v); free(Q.v); return rc; }
        for (int64_t i = 0; i < Q.n; ++i) il_push(&out, Q.v[i]);
        qptr[m + 1] = out.n;
    }
    free(Q.v);
    *qptr_out = qptr;
    *qidx_out = out.v ? out.v : (int32_t*)malloc(sizeof(int32_t));
    return 0;
}

/* ------------------------------------------------- Schur complement */
/* S~ = D - H~ (Eq. sparse_S).
 *   form 0: H~ = C X~, X~ stored column-wise (column m on Q^(m), values xval)
 *   form 1: H~ = G~ A F~ with F~ = -X~ and G~ stored row-wise on Q^(m) (gval)
 * The pattern of S~ is the union of the pattern of D, the diagonal and every
 * position reached by a product term (kept even when values cancel).
 * Columns ascending.  Result malloc'd (orc_free_csr). */
ORC_EXPORT int orc_schur(int form, const orc_csr* A, const orc_csr* C, const orc_csr* D,
                         const int64_t* qptr, const int32_t* qidx, const double* xval,
                         const double* gval, orc_ocsr* S)
{
    const int32_t Ne = D->nrows;
    const int32_t Nf = C->ncols;
    /* row-wise copy of X~ (N_f x N_e) : for each face f, list of (m, X~[f,m]) */
    int64_t tot = qptr[Ne];
    int64_t* xr_ptr = (int64_t*)calloc((size_t)Nf + 1, sizeof(int64_t));
    int32_t* xr_col = (int32_t*)malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    double* xr_val = (double*)malloc((size_t)(tot ? tot : 1) * sizeof(double));
    if (!xr_ptr || !xr_col || !xr_val) return -1;
    for (int64_t p = 0; p < tot; ++p) xr_ptr[qidx[p] + 1]++;
    for (int32_t f = 0; f < Nf; ++f) xr_ptr[f + 1] += xr_ptr[f];
    int64_t* pos = (int64_t*)malloc(((size_t)Nf + 1) * sizeof(int64_t));
    memcpy(pos, xr_ptr, ((size_t)Nf + 1) * sizeof(int64_t));
    for (int32_t m = 0; m < Ne; ++m)
        for (int64_t p = qptr[m]; p < qptr[m + 1]; ++p) {
            int64_t t = pos[qidx[p]]++;
            xr_col[t] = m;
            xr_val[t] = xval[p];
        }
    free(pos);
    /* dense accumulator per row */
    double* acc = (double*)calloc((size_t)Ne, sizeof(double));
    char* mark = (char*)calloc((size_t)Ne, 1);
    double* af = (double*)calloc((size_t)Nf, sizeof(double)); /* form 1: row of G~ A */
    char* markf = (char*)calloc((size_t)Nf, 1);
    ilist cols = {0}, fcols = {0};
    S->nrows = Ne;
    S->ncols = Ne;
    S->rowptr = (int64_t*)malloc(((size_t)Ne + 1) * sizeof(int64_t));
    ilist scol = {0};
    int64_t vcap = 1024, vn = 0;
    double* sval = (double*)malloc((size_t)vcap * sizeof(double));
    if (!acc || !mark || !af || !markf || !S->rowptr || !sval) return -1;
    S->rowptr[0] = 0;
    for (int32_t E = 0; E < Ne; ++E) {
        cols.n = 0;
        /* H~ row E */
        if (form == 0) {
            for (int64_t p = C->rowptr[E]; p < C->rowptr[E + 1]; ++p) {
                int32_t f = C->col[p];
                double cv = C->val[p];
                for (int64_t t = xr_ptr[f]; t < xr_ptr[f + 1]; ++t) {
                    int32_t m = xr_col[t];
                    if (!mark[m]) { mark[m] = 1; il_push(&cols, m); }
                    acc[m] += cv * xr_val[t];
                }
            }
        } else {
            /* t = G~[E,:] A   (row vector over faces) */
            fcols.n = 0;
            for (int64_t p = qptr[E]; p < qptr[E + 1]; ++p) {
                int32_t f = qidx[p];
                double gv = gval[p];
                for (int64_t q = A->rowptr[f]; q < A->rowptr[f + 1]; ++q) {
                    int32_t g = A->col[q];
                    if (!markf[g]) { markf[g] = 1; il_push(&fcols, g); }
                    af[g] += gv * A->val[q];
                }
            }
            /* H~[E,m] = t F~[:,m] = -t X~[:,m] */
            for (int64_t i = 0; i < fcols.n; ++i) {
                int32_t g = fcols.v[i];
                double tv = af[g];
                for (int64_t t = xr_ptr[g]; t < xr_ptr[g + 1]; ++t) {
                    int32_t m = xr_col[t];
                    if (!mark[m]) { mark[m] = 1; il_push(&cols, m); }
                    acc[m] += tv * (-xr_val[t]);
                }
                af[g] = 0.0;
                markf[g] = 0;
            }
        }
        /* S~ = D - H~ */
        for (int i = 0; i < (int)cols.n; ++i) acc[cols.v[i]] = -acc[cols.v[i]];
        for (int64_t p = D->rowptr[E]; p < D->rowptr[E + 1]; ++p) {
            int32_t m = D->col[p];
            if (!mark[m]) { mark[m] = 1; il_push(&cols, m); }
            acc[m] += D->val[p];
        }
        if (!mark[E]) { mark[E] = 1; il_push(&cols, E); }
        int64_t n = sort_unique(cols.v, cols.n);
        for (int64_t i = 0; i < n; ++i) {
            int32_t m = cols.v[i];
            il_push(&scol, m);
            if (vn == vcap) { vcap *= 2; sval = (double*)realloc(sval, (size_t)vcap * sizeof(double)); }
            sval[vn++] = acc[m];
            acc[m] = 0.0;
            mark[m] = 0;
        }
        S->rowptr[E + 1] = scol.n;
    }
    S->nnz = scol.n;
    S->col = scol.v ? scol.v : (int32_t*)malloc(sizeof(int32_t));
    S->val = sval;
    free(acc); free(mark); free(af); free(markf); free(cols.v); free(fcols.v);
    free(xr_ptr); free(xr_col); free(xr_val);
    return 0;
}

/* ------------------------------------------------------- filtration */
/* Pre- and post-filtration (Sec. 3, implementation details; Algorithm 1 and
 * Algorithm 2): an entry is discarded when its absolute value is smaller than
 * tau times the Euclidean norm of the vector it belongs to; diagonal entries
 * of a square matrix are always kept.  A kept entry satisfies
 * |v| >= tau * ||row||_2 (so tau = 0 keeps everything).  The norm is summed
 * over the stored entries in storage order. */

/* Pre-filtration of the local solution vectors: segment m (entries
 * ptr[m]..ptr[m+1] of idx/val, e.g. column m of X~ on Q^(m) or row m of G~)
 * loses every entry with |v| < tau ||segment m||_2.  Output malloc'd. */
ORC_EXPORT int orc_filter_vectors(int32_t nseg, const int64_t* ptr, const int32_t* idx, const double* val,
                                  double tau, int64_t** optr, int32_t** oidx, double** oval)
{
    int64_t tot = ptr[nseg];
    int64_t* op = (int64_t*)malloc(((size_t)nseg + 1) * sizeof(int64_t));
    int32_t* oi = (int32_t*)malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    double* ov = (double*)malloc((size_t)(tot ? tot : 1) * sizeof(double));
    if (!op || !oi || !ov) { free(op); free(oi); free(ov); return -1; }
    int64_t n = 0;
    op[0] = 0;
    for (int32_t m = 0; m < nseg; ++m) {
        double ss = 0.0;
        for (int64_t p = ptr[m]; p < ptr[m + 1]; ++p) ss += val[p] * val[p];
        double lim = tau * sqrt(ss);
        for (int64_t p = ptr[m]; p < ptr[m + 1]; ++p)
            if (!(fabs(val[p]) < lim)) { oi[n] = idx[p]; ov[n] = val[p]; ++n; }
        op[m + 1] = n;
    }
    *optr = op;
    *oidx = oi;
    *oval = ov;
    return 0;
}

/* Post-filtration of the rows of a square CSR matrix (H~ or S~): entry
 * (i, j), j != i, is discarded when |m_ij| < tau ||row i||_2. */
ORC_EXPORT int orc_filter_rows(const orc_csr* M, double tau, orc_ocsr* out)
{
    const int32_t n = M->nrows;
    int64_t tot = M->rowptr[n];
    out->nrows = n;
    out->ncols = M->ncols;
    out->rowptr = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    out->col = (int32_t*)malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    out->val = (double*)malloc((size_t)(tot ? tot : 1) * sizeof(double));
    if (!out->rowptr || !out->col || !out->val) return -1;
    int64_t k = 0;
    out->rowptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        double ss = 0.0;
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) ss += M->val[p] * M->val[p];
        double lim = tau * sqrt(ss);
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p)
            if (M->col[p] == i || !(fabs(M->val[p]) < lim)) {
                out->col[k] = M->col[p];
                out->val[k] = M->val[p];
                ++k;
            }
        out->rowptr[i + 1] = k;
    }
    out->nnz = k;
    return 0;
}

/* H~ alone, on its structural product pattern (Eq. sparse_S):
 *   form 0: H~ = C X~, X~ column m stored on (xptr, xidx, xval)
 *   form 1: H~ = G~ A F~ = -(G~ A) X~, G~ row m stored on (gptr, gidx, gval)
 * X~ and G~ may carry different patterns (after pre-filtration). */
ORC_EXPORT int orc_htilde(int form, const orc_csr* A, const orc_csr* C, int32_t Ne,
                          const int64_t* xptr, const int32_t* xidx, const double* xval,
                          const int64_t* gptr, const int32_t* gidx, const double* gval, orc_ocsr* H)
{
    const int32_t Nf = C->ncols;
    int64_t tot = xptr[Ne];
    int64_t* xr_ptr = (int64_t*)calloc((size_t)Nf + 1, sizeof(int64_t));
    int32_t* xr_col = (int32_t*)malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
    double* xr_val = (double*)malloc((size_t)(tot ? tot : 1) * sizeof(double));
    int64_t* pos = (int64_t*)malloc(((size_t)Nf + 1) * sizeof(int64_t));
    double* acc = (double*)calloc((size_t)Ne, sizeof(double));
    char* mark = (char*)calloc((size_t)Ne, 1);
    double* af = (double*)calloc((size_t)Nf, sizeof(double));
    char* markf = (char*)calloc((size_t)Nf, 1);
    if (!xr_ptr || !xr_col || !xr_val || !pos || !acc || !mark || !af || !markf) return -1;
    /* row-wise copy of X~: for each face f, (m, X~[f,m]) with m ascending */
    for (int64_t p = 0; p < tot; ++p) xr_ptr[xidx[p] + 1]++;
    for (int32_t f = 0; f < Nf; ++f) xr_ptr[f + 1] += xr_ptr[f];
    memcpy(pos, xr_ptr, ((size_t)Nf + 1) * sizeof(int64_t));
    for (int32_t m = 0; m < Ne; ++m)
        for (int64_t p = xptr[m]; p < xptr[m + 1]; ++p) {
            int64_t t = pos[xidx[p]]++;
            xr_col[t] = m;
            xr_val[t] = xval[p];
        }
    ilist cols = {0}, fcols = {0}, hcol = {0};
    int64_t vcap = 1024, vn = 0;
    double* hval = (double*)malloc((size_t)vcap * sizeof(double));
    H->nrows = Ne;
    H->ncols = Ne;
    H->rowptr = (int64_t*)malloc(((size_t)Ne + 1) * sizeof(int64_t));
    if (!hval || !H->rowptr) return -1;
    H->rowptr[0] = 0;
    for (int32_t E = 0; E < Ne; ++E) {
        cols.n = 0;
        if (form == 0) {
            for (int64_t p = C->rowptr[E]; p < C->rowptr[E + 1]; ++p) {
                int32_t f = C->col[p];
                double cv = C->val[p];
                for (int64_t t = xr_ptr[f]; t < xr_ptr[f + 1]; ++t) {
                    int32_t m = xr_col[t];
                    if (!mark[m]) { mark[m] = 1; il_push(&cols, m); }
                    acc[m] += cv * xr_val[t];
                }
            }
        } else {
            fcols.n = 0;
            for (int64_t p = gptr[E]; p < gptr[E + 1]; ++p) {
                int32_t f = gidx[p];
                double gv = gval[p];
                for (int64_t q = A->rowptr[f]; q < A->rowptr[f + 1]; ++q) {
                    int32_t g = A->col[q];
                    if (!markf[g]) { markf[g] = 1; il_push(&fcols, g); }
                    af[g] += gv * A->val[q];
                }
            }
            for (int64_t i = 0; i < fcols.n; ++i) {
                int32_t g = fcols.v[i];
                double tv = af[g];
                for (int64_t t = xr_ptr[g]; t < xr_ptr[g + 1]; ++t) {
                    int32_t m = xr_col[t];
                    if (!mark[m]) { mark[m] = 1; il_push(&cols, m); }
                    acc[m] += tv * (-xr_val[t]);
                }
                af[g] = 0.0;
                markf[g] = 0;
            }
        }
        int64_t n = sort_unique(cols.v, cols.n);
        for (int64_t i = 0; i < n; ++i) {
            int32_t m = cols.v[i];
            il_push(&hcol, m);
            if (vn == vcap) { vcap *= 2; hval = (double*)realloc(hval, (size_t)vcap * sizeof(double)); }
            hval[vn++] = acc[m];
            acc[m] = 0.0;
            mark[m] = 0;
        }
        H->rowptr[E + 1] = hcol.n;
    }
    H->nnz = hcol.n;
    H->col = hcol.v ? hcol.v : (int32_t*)malloc(sizeof(int32_t));
    H->val = hval;
    free(xr_ptr); free(xr_col); free(xr_val); free(pos); free(acc); free(mark); free(af); free(markf);
    free(cols.v); free(fcols.v);
    return 0;
}

/* S~ = D - H~ on pattern(H~) u pattern(D) u diagonal (Eq. sparse_S,
 * Algorithm 2), columns ascending; each value is (-h) + d. */
ORC_EXPORT int orc_d_minus_h(const orc_csr* D, const orc_csr* H, orc_ocsr* S)
{
    const int32_t Ne = D->nrows;
    double* acc = (double*)calloc((size_t)(Ne ? Ne : 1), sizeof(double));
    char* mark = (char*)calloc((size_t)(Ne ? Ne : 1), 1);
    ilist cols = {0}, scol = {0};
    int64_t vcap = 1024, vn = 0;
    double* sval = (double*)malloc((size_t)vcap * sizeof(double));
    S->nrows = Ne;
    S->ncols = Ne;
    S->rowptr = (int64_t*)malloc(((size_t)Ne + 1) * sizeof(int64_t));
    if (!acc || !mark || !sval || !S->rowptr) return -1;
    S->rowptr[0] = 0;
    for (int32_t E = 0; E < Ne; ++E) {
        cols.n = 0;
        for (int64_t p = H->rowptr[E]; p < H->rowptr[E + 1]; ++p) {
            int32_t m = H->col[p];
            mark[m] = 1;
            il_push(&cols, m);
            acc[m] = -H->val[p];
        }
        for (int64_t p = D->rowptr[E]; p < D->rowptr[E + 1]; ++p) {
            int32_t m = D->col[p];
            if (!mark[m]) { mark[m] = 1; il_push(&cols, m); }
            acc[m] += D->val[p];
        }
        if (!mark[E]) { mark[E] = 1; il_push(&cols, E); }
        int64_t n = sort_unique(cols.v, cols.n);
        for (int64_t i = 0; i < n; ++i) {
            int32_t m = cols.v[i];
            il_push(&scol, m);
            if (vn == vcap) { vcap *= 2; sval = (double*)realloc(sval, (size_t)vcap * sizeof(double)); }
            sval[vn++] = acc[m];
            acc[m] = 0.0;
            mark[m] = 0;
        }
        S->rowptr[E + 1] = scol.n;
    }
    S->nnz = scol.n;
    S->col = scol.v ? scol.v : (int32_t*)malloc(sizeof(int32_t));
    S->val = sval;
    free(acc); free(mark); free(cols.v);
    return 0;
}

/* ------------------------------------------------------------ ILU(0) */
/* ILU(0) in the natural ordering (Saad, "Iterative Methods for Sparse Linear
 * Systems", Alg. 10.4, IKJ variant): L (unit lower) and U share the pattern
 * of M; lu receives the factor values in M's storage order. */
ORC_EXPORT int orc_ilu0(const orc_csr* M, double* lu, int32_t* bad)
{
    const int32_t n = M->nrows;
    memcpy(lu, M->val, (size_t)M->rowptr[n] * sizeof(double));
    int64_t* diag = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!diag) return -1;
    for (int32_t i = 0; i < n; ++i) {
        diag[i] = -1;
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p)
            if (M->col[p] == i) diag[i] = p;
        if (diag[i] < 0) { if (bad) *bad = i; free(diag); return -2; }
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) {
            int32_t k = M->col[p];
            if (k >= i) break;
            double ukk = lu[diag[k]];
            if (!(ukk != 0.0)) { if (bad) *bad = k; free(diag); return -2; }
            lu[p] /= ukk;
            double lik = lu[p];
            /* a_ij -= l_ik u_kj for j > k present in both rows i and k */
            for (int64_t q = p + 1; q < M->rowptr[i + 1]; ++q) {
                int32_t j = M->col[q];
                for (int64_t t = diag[k] + 1; t < M->rowptr[k + 1]; ++t)
                    if (M->col[t] == j) { lu[q] -= lik * lu[t]; break; }
            }
        }
        if (!(lu[diag[i]] != 0.0) || !isfinite(lu[diag[i]])) { if (bad) *bad = i; free(diag); return -2; }
    }
    free(diag);
    return 0;
}

/* z = U^{-1} L^{-1} r with the factors of orc_ilu0 */
ORC_EXPORT void orc_ilu0_solve(const orc_csr* M, const double* lu, const double* r, double* z)
{
    const int32_t n = M->nrows;
    for (int32_t i = 0; i < n; ++i) {
        double v = r[i];
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) {
            if (M->col[p] >= i) break;
            v -= lu[p] * z[M->col[p]];
        }
        z[i] = v;
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double v = z[i], d = 0.0;
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) {
            int32_t c = M->col[p];
            if (c == i) d = lu[p];
            else if (c > i) v -= lu[p] * z[c];
        }
        z[i] = v / d;
    }
}

/* y = M x (or y += M x when accumulate) */
static void spmv(const orc_csr* M, const double* x, double* y, int accumulate)
{
    for (int32_t i = 0; i < M->nrows; ++i) {
        double v = accumulate ? y[i] : 0.0;
        for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) v += M->val[p] * x[M->col[p]];
        y[i] = v;
    }
}

/* -------------------------------------------------- preconditioner */
typedef struct {
    orc_csr A, B, C, D;      /* system blocks */
    orc_csr Ma;              /* matrix whose ILU(0) stands for A~^{-1} */
    const double* lua;
    orc_csr Ms;              /* S~ pattern */
    const double* lus;       /* ILU(0) factor values of S~ */
    int variant;             /* 0: full block LDU (Eq. EDFA_prec); 1: upper block triangular */
    int identity;            /* 1: no preconditioning */
    /* optional orderings of the inner factorisations (NULL: natural order):
     * with aperm the factorised matrix is P_a Ma P_a^T, with sperm P_s S~ P_s^T,
     * row k of the ordered matrix being row perm[k] of the original */
    const int32_t* aperm;
    const int32_t* sperm;
    orc_ocsr own_a, own_s;   /* the ordered copies, owned by the record */
} orc_prec;

/* z = P^{-1} r, Eq. (EDFA_prec) applied right to left:
 *   y   = A~^{-1} r_pi
 *   t   = r_p - C y
 *   z_p = S~^{-1} t
 *   z_pi = A~^{-1} (r_pi - B z_p)
 * (the second application uses linearity: y - A~^{-1} B z_p).  The triangular
 * factors use the exact B and C (Remark 1).  variant 1: z_p = S~^{-1} r_p,
 * z_pi = A~^{-1}(r_pi - B z_p). */
/* z = M~^{-1} r with the ILU(0) factors of the (possibly reordered) matrix:
 * with an ordering, r is gathered into the ordered numbering, solved there and
 * z scattered back (z[perm[k]] = solution[k]). */
static void inner_solve(const orc_csr* M, const double* lu, const int32_t* perm, const double* r, double* z)
{
    if (!perm) {
        orc_ilu0_solve(M, lu, r, z);
        return;
    }
    const int32_t n = M->nrows;
    double* w = (double*)malloc((size_t)(n ? n : 1) * 2 * sizeof(double));
    for (int32_t k = 0; k < n; ++k) w[k] = r[perm[k]];
    orc_ilu0_solve(M, lu, w, w + n);
    for (int32_t k = 0; k < n; ++k) z[perm[k]] = w[n + k];
    free(w);
}

ORC_EXPORT void orc_apply(const orc_prec* P, const double* r, double* z)
{
    const int32_t Nf = P->A.nrows, Ne = P->D.nrows;
    if (P->identity) { memcpy(z, r, ((size_t)Nf + Ne) * sizeof(double)); return; }
    double* y = (double*)malloc((size_t)Nf * sizeof(double));
    double* t = (double*)malloc((size_t)(Nf > Ne ? Nf : Ne) * sizeof(double));
    const double* rpi = r;
    const double* rp = r + Nf;
    double* zpi = z;
    double* zp = z + Nf;
    if (P->variant == 0) {
        inner_solve(&P->Ma, P->lua, P->aperm, rpi, y);
        for (int32_t e = 0; e < Ne; ++e) t[e] = rp[e];
        for (int32_t e = 0; e < Ne; ++e) {
            double v = 0.0;
            for (int64_t p = P->C.rowptr[e]; p < P->C.rowptr[e + 1]; ++p) v += P->C.val[p] * y[P->C.col[p]];
            t[e] -= v;
        }
        inner_solve(&P->Ms, P->lus, P->sperm, t, zp);
    } else {
        inner_solve(&P->Ms, P->lus, P->sperm, rp, zp);
    }
    for (int32_t f = 0; f < Nf; ++f) {
        double v = 0.0;
        for (int64_t p = P->B.rowptr[f]; p < P->B.rowptr[f + 1]; ++p) v += P->B.val[p] * zp[P->B.col[p]];
        t[f] = rpi[f] - v;
    }
    inner_solve(&P->Ma, P->lua, P->aperm, t, zpi);
    free(y);
    free(t);
}

/* y = [A B; C D] x */
static void block_mv(const orc_prec* P, const double* x, double* y)
{
    const int32_t Nf = P->A.nrows;
    spmv(&P->A, x, y, 0);
    spmv(&P->B, x + Nf, y, 1);
    spmv(&P->C, x, y + Nf, 0);
    spmv(&P->D, x + Nf, y + Nf, 1);
}

static double dot(const double* a, const double* b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Right-preconditioned flexible GMRES(m) (Saad, Alg. 9.6) with modified
 * Gram-Schmidt and Givens rotations, x0 = 0.  Stops when the estimated
 * residual |g_{j+1}| <= rtol ||b||; the true residual ||b - A x|| is then
 * computed and the outer loop restarts while it exceeds rtol ||b||.
 * iters = total inner iterations; hist (optional, length maxit+1) receives
 * the estimated relative residual after each inner iteration (hist[0] = 1).
 * Returns 0 converged, 1 not converged within maxit, <0 error. */
ORC_EXPORT int orc_fgmres(const orc_prec* P, const double* b, double* x, int m, double rtol,
                          int maxit, int* iters, double* hist, double* true_rel)
{
    const int64_t n = (int64_t)P->A.nrows + P->D.nrows;
    double* V = (double*)malloc((size_t)(m + 1) * n * sizeof(double));
    double* Z = (double*)malloc((size_t)m * n * sizeof(double));
    double* w = (double*)malloc((size_t)n * sizeof(double));
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)malloc((size_t)m * sizeof(double));
    double* sn = (double*)malloc((size_t)m * sizeof(double));
    double* g = (double*)malloc((size_t)(m + 1) * sizeof(double));
    double* y = (double*)malloc((size_t)m * sizeof(double));
    if (!V || !Z || !w || !H || !cs || !sn || !g || !y) return -1;
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    const double bnorm = sqrt(dot(b, b, n));
    int it = 0, status = 1;
    if (hist) hist[0] = 1.0;
    if (bnorm == 0.0) { *iters = 0; if (true_rel) *true_rel = 0.0; status = 0; goto done; }
    /* r0 = b */
    for (int64_t i = 0; i < n; ++i) w[i] = b[i];
    double beta = bnorm;
    while (it < maxit) {
        for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int j, jlast = -1;
        for (j = 0; j < m && it < maxit; ++j) {
            double* vj = V + (int64_t)j * n;
            double* zj = Z + (int64_t)j * n;
            orc_apply(P, vj, zj);
            block_mv(P, zj, w);
            for (int i = 0; i <= j; ++i) {
                double* vi = V + (int64_t)i * n;
                double hij = dot(w, vi, n);
                H[i * m + j] = hij;
                for (int64_t k = 0; k < n; ++k) w[k] -= hij * vi[k];
            }
            double hn = sqrt(dot(w, w, n));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (int64_t k = 0; k < n; ++k) V[(int64_t)(j + 1) * n + k] = w[k] / hn;
            for (int i = 0; i < j; ++i) {
                double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[j * m + j], c = H[(j + 1) * m + j];
            double den = sqrt(a * a + c * c);
            cs[j] = a / den;
            sn[j] = c / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            it++;
            jlast = j;
            double est = fabs(g[j + 1]) / bnorm;
            if (hist) hist[it] = est;
            if (est <= rtol || hn == 0.0) break;
        }
        int k = jlast + 1;
        for (int i = k - 1; i >= 0; --i) {
            double v = g[i];
            for (int l = i + 1; l < k; ++l) v -= H[i * m + l] * y[l];
            y[i] = v / H[i * m + i];
        }
        for (int i = 0; i < k; ++i) {
            const double* zi = Z + (int64_t)i * n;
            for (int64_t t = 0; t < n; ++t) x[t] += y[i] * zi[t];
        }
        block_mv(P, x, w);
        for (int64_t t = 0; t < n; ++t) w[t] = b[t] - w[t];
        beta = sqrt(dot(w, w, n));
        if (true_rel) *true_rel = beta / bnorm;
        if (beta / bnorm <= rtol) { status = 0; break; }
    }
    *iters = it;
done:
    free(V); free(Z); free(w); free(H); free(cs); free(sn); free(g); free(y);
    return status;
}

/* ---------------------------------------------- preconditioner setup */
/* Assemble the preconditioner record: ILU(0) of Ma (stands for A~^{-1}) and
 * of S~.  Factor arrays are malloc'd and released with orc_prec_free. */
/* Right-preconditioned Bi-CGStab (van der Vorst 1992), the outer solver of the
 * paper's experiments (Sec. 4), x0 = 0, stopping rule ||r_k|| / ||r_0|| <= rtol
 * with r_0 = b.  One iteration applies the preconditioner twice.  When the
 * recursive residual meets the tolerance the true residual b - A x is formed; if
 * it does not meet it too, or on a breakdown (rho = 0, (r^, v) = 0, omega = 0),
 * the method restarts from the true residual.  Returns 0 converged, 1 not
 * converged within maxit iterations. */
ORC_EXPORT int orc_bicgstab(const orc_prec* P, const double* b, double* x, double rtol, int maxit, int* iters,
                            double* hist, double* true_rel)
{
    const int64_t n = (int64_t)P->A.nrows + P->D.nrows;
    double* r = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* rh = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* p = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* v = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* ph = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* sv = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* sh = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* t = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    if (!r || !rh || !p || !v || !ph || !sv || !sh || !t) return -1;
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    const double bnorm = sqrt(dot(b, b, n));
    int it = 0, status = 1;
    if (hist) hist[0] = 1.0;
    if (true_rel) *true_rel = 0.0;
    if (bnorm == 0.0) { *iters = 0; status = 0; goto done; }
    for (int64_t i = 0; i < n; ++i) r[i] = b[i];
    for (;;) {
        /* (re)start from the residual r */
        for (int64_t i = 0; i < n; ++i) { rh[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        int restart = 0;
        while (it < maxit) {
            const double rho = dot(rh, r, n);
            if (rho == 0.0) { restart = 1; break; }
            const double beta = (rho / rho_old) * (alpha / omega);
            for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            orc_apply(P, p, ph);
            block_mv(P, ph, v);
            const double rv = dot(rh, v, n);
            if (rv == 0.0) { restart = 1; break; }
            alpha = rho / rv;
            for (int64_t i = 0; i < n; ++i) sv[i] = r[i] - alpha * v[i];
            it++;
            const double snorm = sqrt(dot(sv, sv, n));
            if (snorm / bnorm <= rtol) {
                for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
                for (int64_t i = 0; i < n; ++i) r[i] = sv[i];
                if (hist) hist[it] = snorm / bnorm;
                break;
            }
            orc_apply(P, sv, sh);
            block_mv(P, sh, t);
            const double tt = dot(t, t, n);
            omega = tt != 0.0 ? dot(t, sv, n) / tt : 0.0;
            for (int64_t i = 0; i < n; ++i) x[i] += alpha * ph[i] + omega * sh[i];
            for (int64_t i = 0; i < n; ++i) r[i] = sv[i] - omega * t[i];
            rho_old = rho;
            const double rn = sqrt(dot(r, r, n));
            if (hist) hist[it] = rn / bnorm;
            if (rn / bnorm <= rtol) break;
            if (omega == 0.0) { restart = 1; break; }
        }
        /* true residual */
        block_mv(P, x, t);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
        const double tr = sqrt(dot(r, r, n)) / bnorm;
        if (true_rel) *true_rel = tr;
        if (tr <= rtol) { status = 0; break; }
        if (it >= maxit) break;
        (void)restart;
    }
    *iters = it;
done:
    free(r); free(rh); free(p); free(v); free(ph); free(sv); free(sh); free(t);
    return status;
}

ORC_EXPORT int orc_permute(const orc_csr* M, const int32_t* perm, orc_ocsr* out);

static orc_csr as_csr(const orc_ocsr* M)
{
    orc_csr c = {M->nrows, M->ncols, M->nnz, M->rowptr, M->col, M->val};
    return c;
}

/* Preconditioner record; aperm / sperm (may be NULL) order the inner ILU(0)
 * factorisations of Ma and S~ (the record keeps the pointers: they must stay
 * valid while it is used). */
ORC_EXPORT int orc_prec_setup_ordered(orc_prec* P, const orc_csr* A, const orc_csr* B, const orc_csr* C,
                                      const orc_csr* D, const orc_csr* Ma, const orc_csr* S, int variant,
                                      int identity, const int32_t* aperm, const int32_t* sperm, int32_t* bad)
{
    memset(P, 0, sizeof *P);
    P->A = *A; P->B = *B; P->C = *C; P->D = *D;
    P->variant = variant;
    P->identity = identity;
    if (identity) return 0;
    P->Ma = *Ma;
    P->Ms = *S;
    if (aperm) {
        if (orc_permute(Ma, aperm, &P->own_a)) return -1;
        P->Ma = as_csr(&P->own_a);
        P->aperm = aperm;
    }
    if (sperm) {
        if (orc_permute(S, sperm, &P->own_s)) return -1;
        P->Ms = as_csr(&P->own_s);
        P->sperm = sperm;
    }
    double* la = (double*)malloc((size_t)(P->Ma.nnz ? P->Ma.nnz : 1) * sizeof(double));
    double* ls = (double*)malloc((size_t)(P->Ms.nnz ? P->Ms.nnz : 1) * sizeof(double));
    if (!la || !ls) return -1;
    int rc = orc_ilu0(&P->Ma, la, bad);
    if (rc) { free(la); free(ls); return rc; }
    rc = orc_ilu0(&P->Ms, ls, bad);
    if (rc) { free(la); free(ls); return rc - 10; }
    P->lua = la;
    P->lus = ls;
    return 0;
}

ORC_EXPORT int orc_prec_setup(orc_prec* P, const orc_csr* A, const orc_csr* B, const orc_csr* C,
                              const orc_csr* D, const orc_csr* Ma, const orc_csr* S, int variant,
                              int identity, int32_t* bad)
{
    return orc_prec_setup_ordered(P, A, B, C, D, Ma, S, variant, identity, NULL, NULL, bad);
}

ORC_EXPORT void orc_prec_free(orc_prec* P)
{
    free((void*)P->lua);
    free((void*)P->lus);
    P->lua = P->lus = NULL;
    if (P->aperm) orc_free_csr(&P->own_a);
    if (P->sperm) orc_free_csr(&P->own_s);
    P->aperm = P->sperm = NULL;
}

/* ------------------------------------------------- multicolour ordering
 * An optional ordering of the inner ILU(0) factorisations.  The paper leaves
 * the inner preconditioners and their ordering open (Sec. 3, inner
 * preconditioners; Sec. 4 uses incomplete factorisations with partial
 * fill-in); in the natural order the triangular solves of ILU(0) form long
 * dependency chains, while after a multicolour ordering the rows of one colour
 * depend only on rows of earlier colours.
 *
 * Graph: vertices = rows of M, an edge {i, j} (i != j) wherever M_ij or M_ji
 * is stored.  Priority of vertex v: the SplitMix64 finaliser (Steele, Lea &
 * Flood 2014) of v + 1, a bijection on 64-bit integers, so no two vertices
 * tie.  Colouring (Jones & Plassmann 1993): every vertex takes the smallest
 * colour not used by its neighbours of higher priority; computed here by
 * visiting the vertices in decreasing priority and giving each the smallest
 * colour its already coloured neighbours do not use, which is the same
 * colouring.  Ordering: rows sorted by (colour, row index). */
static uint64_t orc_priority(int32_t v)
{
    uint64_t z = ((uint64_t)v + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t pri; int32_t v; } orc_pv;

static int cmp_pri_desc(const void* a, const void* b)
{
    const orc_pv* x = (const orc_pv*)a;
    const orc_pv* y = (const orc_pv*)b;
    return x->pri < y->pri ? 1 : (x->pri > y->pri ? -1 : 0);
}

/* Block multicolour ordering (an opt-in variant of the above): the rows are
 * grouped into blocks of b consecutive rows (the last block may be shorter),
 * block B holding rows B b .. B b + b - 1.  Graph: vertices = blocks, an edge
 * between blocks B != B' wherever M or M^T couples a row of B with a row of
 * B'.  The blocks are coloured like the rows above (SplitMix64 priority of
 * B + 1, every block takes the smallest colour not used by its neighbours of
 * higher priority).  Inside a block the rows keep their order: row r of block
 * B gets the colour c(B) b + (r - B b), so the rows of one colour are
 * independent (blocks of one block colour are not coupled, and the rows of
 * one block have distinct positions), and rows sorted by (colour, row index)
 * list, for every block colour, position after position.  The ILU(0) of this
 * ordering equals that of the ordering by (block colour, block, position):
 * the two orders agree on every pair of coupled rows.  b = 1 is the ordering
 * above. */
ORC_EXPORT int orc_block_colour_order(const orc_csr* M, int32_t b, int32_t* colour, int32_t* perm, int32_t* ncolours)
{
    const int32_t n = M->nrows;
    if (b < 1) return -1;
    const int32_t nb = n > 0 ? (int32_t)(((int64_t)n + b - 1) / b) : 0;
    orc_ocsr T = {0};
    if (csr_transpose(M, &T)) { orc_free_csr(&T); return -1; }
    orc_pv* order = (orc_pv*)malloc((size_t)(nb ? nb : 1) * sizeof(orc_pv));
    int32_t* bcol = (int32_t*)malloc((size_t)(nb ? nb : 1) * sizeof(int32_t));
    int32_t* stamp = (int32_t*)malloc((size_t)(nb + 2) * sizeof(int32_t));
    if (!order || !bcol || !stamp) { free(order); free(bcol); free(stamp); orc_free_csr(&T); return -1; }
    for (int32_t B = 0; B < nb; ++B) { order[B].pri = orc_priority(B); order[B].v = B; bcol[B] = -1; }
    qsort(order, (size_t)nb, sizeof(orc_pv), cmp_pri_desc);
    for (int32_t c = 0; c < nb + 2; ++c) stamp[c] = -1;
    for (int32_t k = 0; k < nb; ++k) {
        const int32_t B = order[k].v;
        const int32_t r1 = (int32_t)((int64_t)B * b + b < n ? (int64_t)B * b + b : n);
        /* colours of the neighbouring blocks coloured so far (those of higher priority) */
        for (int32_t v = B * b; v < r1; ++v) {
            for (int64_t p = M->rowptr[v]; p < M->rowptr[v + 1]; ++p) {
                const int32_t U = M->col[p] / b;
                if (U != B && bcol[U] >= 0) stamp[bcol[U]] = B;
            }
            for (int64_t p = T.rowptr[v]; p < T.rowptr[v + 1]; ++p) {
                const int32_t U = T.col[p] / b;
                if (U != B && bcol[U] >= 0) stamp[bcol[U]] = B;
            }
        }
        int32_t c = 0;
        while (stamp[c] == B) ++c;
        bcol[B] = c;
    }
    int32_t ncol = 0;
    for (int32_t v = 0; v < n; ++v) {
        colour[v] = bcol[v / b] * b + v % b;
        if (colour[v] + 1 > ncol) ncol = colour[v] + 1;
    }
    /* rows sorted by (colour, index): counting sort, stable in the index */
    int64_t* start = (int64_t*)calloc((size_t)ncol + 1, sizeof(int64_t));
    if (!start) { free(order); free(bcol); free(stamp); orc_free_csr(&T); return -1; }
    for (int32_t v = 0; v < n; ++v) start[colour[v] + 1]++;
    for (int32_t c = 0; c < ncol; ++c) start[c + 1] += start[c];
    for (int32_t v = 0; v < n; ++v) perm[start[colour[v]]++] = v;
    *ncolours = ncol;
    free(start);
    free(order);
    free(bcol);
    free(stamp);
    orc_free_csr(&T);
    return 0;
}

ORC_EXPORT int orc_colour_order(const orc_csr* M, int32_t* colour, int32_t* perm, int32_t* ncolours)
{
    return orc_block_colour_order(M, 1, colour, perm, ncolours);
}

/* P M P^T: row k is row perm[k] of M with every column j renamed to its
 * position in perm, the columns of each row sorted ascending. */
ORC_EXPORT int orc_permute(const orc_csr* M, const int32_t* perm, orc_ocsr* out)
{
    const int32_t n = M->nrows;
    const int64_t nnz = M->rowptr[n];
    int32_t* iperm = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    out->nrows = n;
    out->ncols = n;
    out->nnz = nnz;
    out->rowptr = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    out->col = (int32_t*)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
    out->val = (double*)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
    if (!iperm || !out->rowptr || !out->col || !out->val) { free(iperm); return -1; }
    for (int32_t k = 0; k < n; ++k) iperm[perm[k]] = k;
    out->rowptr[0] = 0;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t r = perm[k];
        int64_t q = out->rowptr[k];
        for (int64_t p = M->rowptr[r]; p < M->rowptr[r + 1]; ++p, ++q) {
            /* insertion into the sorted row */
            int32_t c = iperm[M->col[p]];
            double v = M->val[p];
            int64_t j = q;
            while (j > out->rowptr[k] && out->col[j - 1] > c) {
                out->col[j] = out->col[j - 1];
                out->val[j] = out->val[j - 1];
                --j;
            }
            out->col[j] = c;
            out->val[j] = v;
        }
        out->rowptr[k + 1] = q;
    }
    free(iperm);
    return 0;
}

ORC_EXPORT int orc_prec_sizeof(void) { return (int)sizeof(orc_prec); }

/* ------------------------------------------------------------ adjoint */
/* Forward-mode dual number: value and derivative with respect to one
 * log-conductivity theta_E. */
typedef struct { double v, d; } dual;
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.d + b.d}; return r; }
static dual dsub(dual a, dual b) { dual r = {a.v - b.v, a.d - b.d}; return r; }
static dual ddiv(dual a, dual b)
{
    dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
    return r;
}
static dual dconst(double v) { dual r = {v, 0.0}; return r; }

/* Gradient of L(u(theta)) with A(theta) u = b(theta) and isotropic cell
 * conductivities k_E = exp(theta_E) on a brick grid (strong-flux cell rows of
 * Appendix A, prescribed-pressure faces eliminated symmetrically):
 *     dL/dtheta_E = lambda^T (db/dtheta_E - dA/dtheta_E u),  A^T lambda = dL/du.
 * With the face pressures of prescribed faces set to their values pbar in u,
 * this equals -sum over non-prescribed rows r of lambda_r (d(A_full u)/dtheta_E)_r
 * where A_full is the assembled matrix before elimination.  Each row that
 * depends on k_E is rebuilt with dual numbers, seeded on theta_E:
 *   face rows i in F_E (Eq. cont_fluxes):  sum over cells E' of i of
 *        q_i^{E'} = sum_j W^{E'}_ij (p^{E'} - pi_j)
 *   cell rows E and its face neighbours (Eq. discr_bal_FV_2 with
 *        Eq. fluxes_MHFEM_STRONG): sum_i q_i^{E,E'}.
 * W^E = k_E W1^E where W1^E is the inverse elemental matrix for k = 1
 * (passed in, [Ne*36]).  u, lambda: [Nf+Ne].  grad: [Ne]. */
static dual cell_W(const double* W1, const double* logk, int32_t e, int32_t seed, int i, int j)
{
    double k = exp(logk[e]);
    dual kk = {k, e == seed ? k : 0.0};
    return dmul(kk, dconst(W1[36 * (int64_t)e + i * 6 + j]));
}

/* residual row of the un-eliminated system, with pi of prescribed faces = pbar */
static dual face_row(int32_t i, const int32_t* cf, const int32_t* fc, const double* W1,
                     const double* logk, const double* u, int32_t Nf, int32_t seed)
{
    dual acc = dconst(0.0);
    for (int side = 0; side < 2; ++side) {
        int32_t e = fc[2 * (int64_t)i + side];
        if (e < 0) continue;
        int li = 0;
        while (cf[6 * (int64_t)e + li] != i) ++li;
        for (int j = 0; j < 6; ++j) {
            dual w = cell_W(W1, logk, e, seed, li, j);
            acc = dadd(acc, dmul(w, dconst(u[Nf + e] - u[cf[6 * (int64_t)e + j]])));
        }
    }
    return acc;
}

static dual cell_row(int32_t e, const int32_t* cf, const int32_t* fc, const int8_t* fdir,
                     const double* W1, const double* logk, const double* u, int32_t Nf,
                     int32_t seed)
{
    dual acc = dconst(0.0);
    const double pe = u[Nf + e];
    for (int l = 0; l < 6; ++l) {
        int32_t i = cf[6 * (int64_t)e + l];
        int side = (l & 1) ? 0 : 1;
        int32_t e2 = fc[2 * (int64_t)i + (1 - side)];
        /* Lambda^E_i */
        dual LE = dconst(0.0), sE = dconst(0.0);
        for (int j = 0; j < 6; ++j) {
            dual w = cell_W(W1, logk, e, seed, l, j);
            LE = dadd(LE, w);
            if (j != l) sE = dadd(sE, dmul(w, dconst(u[cf[6 * (int64_t)e + j]])));
        }
        dual lamE = dsub(dmul(LE, dconst(pe)), sE);
        if (e2 >= 0) {
            int l2 = 0;
            while (cf[6 * (int64_t)e2 + l2] != i) ++l2;
            dual L2 = dconst(0.0), s2 = dconst(0.0);
            for (int j = 0; j < 6; ++j) {
                dual w = cell_W(W1, logk, e2, seed, l2, j);
                L2 = dadd(L2, w);
                if (j != l2) s2 = dadd(s2, dmul(w, dconst(u[cf[6 * (int64_t)e2 + j]])));
            }
            dual lamE2 = dsub(dmul(L2, dconst(u[Nf + e2])), s2);
            dual bE = cell_W(W1, logk, e, seed, l, l);
            dual bE2 = cell_W(W1, logk, e2, seed, l2, l2);
            dual den = dadd(bE, bE2);
            dual w = ddiv(bE2, den);
            dual wc = ddiv(bE, den);
            acc = dadd(acc, dsub(dmul(w, lamE), dmul(wc, lamE2)));
        } else if (fdir[i]) {
            dual wii = cell_W(W1, logk, e, seed, l, l);
            acc = dadd(acc, dsub(lamE, dmul(wii, dconst(u[i]))));
        }
    }
    return acc;
}

ORC_EXPORT int orc_adjoint_grad(int32_t Nf, int32_t Ne, const int32_t* cell_faces,
                                const int32_t* face_cells, const int8_t* face_dir,
                                const double* face_pbar, const double* W1, const double* logk,
                                const double* u_in, const double* lam, double* grad)
{
    double* u = (double*)malloc(((size_t)Nf + Ne) * sizeof(double));
    if (!u) return -1;
    memcpy(u, u_in, ((size_t)Nf + Ne) * sizeof(double));
    for (int32_t i = 0; i < Nf; ++i)
        if (face_dir[i]) u[i] = face_pbar[i];
    for (int32_t e = 0; e < Ne; ++e) {
        double g = 0.0;
        /* face rows of the faces of e */
        for (int l = 0; l < 6; ++l) {
            int32_t i = cell_faces[6 * (int64_t)e + l];
            if (face_dir[i]) continue;
            dual r = face_row(i, cell_faces, face_cells, W1, logk, u, Nf, e);
            g -= lam[i] * r.d;
        }
        /* cell row e and the rows of its face neighbours */
        dual r = cell_row(e, cell_faces, face_cells, face_dir, W1, logk, u, Nf, e);
        g -= lam[Nf + e] * r.d;
        for (int l = 0; l < 6; ++l) {
            int32_t i = cell_faces[6 * (int64_t)e + l];
            int side = (l & 1) ? 0 : 1;
            int32_t e2 = face_cells[2 * (int64_t)i + (1 - side)];
            if (e2 < 0) continue;
            dual r2 = cell_row(e2, cell_faces, face_cells, face_dir, W1, logk, u, Nf, e);
            g -= lam[Nf + e2] * r2.d;
        }
        grad[e] = g;
    }
    free(u);
    return 0;
}
