// Restricted local solves of the EDFA setup (Sec. 3):
//   -A^(m) f~ = R a_pip^(m)    (Eq. syst_MRHS_res-F)  ->  X~[Q,m] = -f~ = (A^(m))^{-1} B[Q,m]
//   -A^(m) g~ = R a_ppi^(m)T   (Eq. syst_MRHS_res)    ->  G~[m,Q] = g~ = -(A^(m))^{-1} C[m,Q]^T
// with A^(m) = R A R^T the principal submatrix of A on Q^(m) (Eq. r_r^m).
//
// GB300 design.  FP64 runs at ~1/64 of the FP32 rate on this part, so the
// kernel is built to keep every FP64 lane busy rather than to save bytes:
//  * a group of LPC lanes owns one cell (32/LPC cells per warp, persistent
//    grid-stride loop over cells, a multiple of the SM count in blocks);
//  * A^(m) is gathered from the CSR rows straight into shared memory as a
//    packed lower triangle (A is symmetric), the row entries are located in
//    Q^(m) by binary search;
//  * A^(m) is negative definite, so the symmetric LU without pivoting
//    A^(m) = L D L^T (U = D L^T) needs half the flops of a general LU; every
//    elimination step updates the trailing triangle element-parallel across
//    the group's lanes (integer index decode is free next to FP64), with the
//    forward elimination of the right-hand sides fused into the same pass;
//  * a zero, positive or non-finite pivot raises EDFA_ERR_BREAKDOWN with the
//    cell index;
//  * results are written coalesced, in the order of Q^(m).
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace edfa {

template <class T>
struct LocalArgs {
    int32_t Ne;
    int pitch;
    const int64_t* qptr;
    const int32_t* qidx;
    Csr<T> A, B, C;
    T* xval;
    T* gval;
    DevErr* err;
};

__device__ __forceinline__ int tri_row(int t)
{
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    return i;
}

template <class T>
__device__ __forceinline__ bool bad_pivot(T d)
{
    return !(d < T(0)) || !isfinite((double)d);
}

template <class T, int NRHS, int LPC>
__global__ void __launch_bounds__(256) k_local(LocalArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = 32 / LPC;
    const int nw = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / LPC, gl = lane % LPC;
    const int P = a.pitch;
    const int tri = P * (P + 1) / 2;
    // odd strides (in elements) between the cells' records: the groups of a
    // warp (every lane, with one lane per cell) then address different banks
    const int per_cell = (tri + (NRHS + 2) * P) | 1;
    const int qstride = P | 1;
    const int slot = wid * G + g;
    T* M = (T*)smem_raw + (size_t)slot * per_cell;
    T* rhs = M + tri;
    T* lc = rhs + NRHS * P;
    T* dv = lc + P;
    int* q = (int*)((T*)smem_raw + (size_t)nw * G * per_cell) + (size_t)slot * qstride;
    const unsigned gmask = (LPC == 32) ? 0xffffffffu : (((1u << LPC) - 1u) << (g * LPC));
    const long long ngroups = (long long)gridDim.x * nw * G;

    for (long long m = ((long long)blockIdx.x * nw + wid) * G + g; m < a.Ne; m += ngroups) {
        const int64_t qb = a.qptr[m];
        const int s = (int)(a.qptr[m + 1] - qb);
        for (int i = gl; i < s; i += LPC) q[i] = a.qidx[qb + i];
        for (int t = gl; t < s * (s + 1) / 2; t += LPC) M[t] = T(0);
        __syncwarp(gmask);
        // gather the lower triangle of A^(m) and the right-hand sides
        for (int i = gl; i < s; i += LPC) {
            const int f = q[i];
            const int64_t rb = a.A.rowptr[f], re = a.A.rowptr[f + 1];
            for (int64_t p = rb; p < re; ++p) {
                const int c = a.A.col[p];
                if (c > f) break;
                int lo = 0, hi = i;
                while (lo <= hi) {
                    int mid = (lo + hi) >> 1;
                    int qm = q[mid];
                    if (qm == c) { M[i * (i + 1) / 2 + mid] = a.A.val[p]; break; }
                    if (qm < c) lo = mid + 1; else hi = mid - 1;
                }
            }
            T bv = T(0);
            for (int64_t p = a.B.rowptr[f]; p < a.B.rowptr[f + 1]; ++p)
                if (a.B.col[p] == m) bv = a.B.val[p];
            rhs[i] = bv;
            if (NRHS == 2) {
                T cv = T(0);
                int64_t lo = a.C.rowptr[m], hi = a.C.rowptr[m + 1] - 1;
                while (lo <= hi) {
                    int64_t mid = (lo + hi) >> 1;
                    int cm = a.C.col[mid];
                    if (cm == f) { cv = a.C.val[mid]; break; }
                    if (cm < f) lo = mid + 1; else hi = mid - 1;
                }
                rhs[P + i] = cv;
            }
        }
        __syncwarp(gmask);
        // A^(m) = L D L^T with right-hand-side forward elimination
        bool ok = true;
        for (int k = 0; k < s; ++k) {
            const T d = M[k * (k + 1) / 2 + k];
            if (bad_pivot(d)) { ok = false; break; }
            const T inv = rcp_rn(d);
            if (gl == 0) dv[k] = inv;
            const int n = s - k - 1;
            for (int t = gl; t < n; t += LPC) {
                const int i = k + 1 + t;
                lc[i] = M[i * (i + 1) / 2 + k] * inv;
            }
            __syncwarp(gmask);
            const int ntri = n * (n + 1) / 2;
            const int tot = ntri + NRHS * n;
            for (int t = gl; t < tot; t += LPC) {
                if (t < ntri) {
                    const int ii = tri_row(t);
                    const int jj = t - ii * (ii + 1) / 2;
                    const int i = k + 1 + ii, j = k + 1 + jj;
                    M[i * (i + 1) / 2 + j] -= lc[i] * M[j * (j + 1) / 2 + k];
                } else {
                    const int r = t - ntri;
                    const int rr = r / n;
                    const int i = k + 1 + (r - rr * n);
                    rhs[rr * P + i] -= lc[i] * rhs[rr * P + k];
                }
            }
            __syncwarp(gmask);
            for (int t = gl; t < n; t += LPC) {
                const int i = k + 1 + t;
                M[i * (i + 1) / 2 + k] = lc[i];
            }
            __syncwarp(gmask);
        }
        if (!ok) {
            if (gl == 0) raise_err(a.err, EDFA_ERR_BREAKDOWN, m);
            __syncwarp(gmask);
            continue;
        }
        // D^{-1}, then L^T x = z by columns
        for (int t = gl; t < NRHS * s; t += LPC) {
            const int rr = t / s;
            const int i = t - rr * s;
            rhs[rr * P + i] *= dv[i];
        }
        __syncwarp(gmask);
        for (int k = s - 1; k >= 1; --k) {
            for (int t = gl; t < NRHS * k; t += LPC) {
                const int rr = t / k;
                const int j = t - rr * k;
                rhs[rr * P + j] -= M[k * (k + 1) / 2 + j] * rhs[rr * P + k];
            }
            __syncwarp(gmask);
        }
        for (int i = gl; i < s; i += LPC) {
            a.xval[qb + i] = rhs[i];
            if (NRHS == 2) a.gval[qb + i] = -rhs[P + i];
        }
        __syncwarp(gmask);
    }
}

template <class T, int NRHS, int LPC>
static int launch_local_t(edfa_handle_s* h, const LocalArgs<T>& a, int warps, cudaStream_t s)
{
    constexpr int G = 32 / LPC;
    const int P = a.pitch;
    const size_t per_cell = (size_t)((P * (P + 1) / 2 + (NRHS + 2) * P) | 1) * sizeof(T) + (size_t)(P | 1) * sizeof(int);
    size_t smem = per_cell * G * warps;
    while (warps > 1 && smem > 220 * 1024) { --warps; smem = per_cell * G * warps; }
    if (smem > 220 * 1024) return EDFA_ERR_BOUNDS;
    auto fn = k_local<T, NRHS, LPC>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return EDFA_ERR_CUDA;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, warps * 32, smem);
    if (per < 1) per = 1;
    long long cells_per_block = (long long)warps * G;
    long long need = (a.Ne + cells_per_block - 1) / cells_per_block;
    long long grid = (long long)per * h->nsm;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    (edfa::count_launch(), fn<<<(unsigned)grid, warps * 32, smem, s>>>(a));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// Autotuner: lanes per local system (LPC) and warps per block are chosen by
// timing the candidates on a prefix sample of the cells (up to 131,072 cells,
// the faster of two launches; results for those cells are overwritten by the
// full launch); the choice is cached per (precision, right-hand sides,
// set-size pitch).
struct TuneKey {
    int tsize, nrhs, pitch;
    bool operator==(const TuneKey& o) const { return tsize == o.tsize && nrhs == o.nrhs && pitch == o.pitch; }
};
struct TuneVal {
    int lpc, warps;
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune;

template <class T, int NRHS>
static int launch_local_cfg(edfa_handle_s* h, const LocalArgs<T>& a, int lpc, int warps, cudaStream_t s)
{
    if (lpc == 1) return launch_local_t<T, NRHS, 1>(h, a, warps, s);
    if (lpc == 2) return launch_local_t<T, NRHS, 2>(h, a, warps, s);
    if (lpc == 4) return launch_local_t<T, NRHS, 4>(h, a, warps, s);
    if (lpc == 8) return launch_local_t<T, NRHS, 8>(h, a, warps, s);
    if (lpc == 16) return launch_local_t<T, NRHS, 16>(h, a, warps, s);
    return launch_local_t<T, NRHS, 32>(h, a, warps, s);
}

template <class T, int NRHS>
static int launch_local_n(edfa_handle_s* h, const LocalArgs<T>& a, cudaStream_t s)
{
    int lpc = a.pitch <= 40 ? 8 : (a.pitch <= 72 ? 16 : 32);
    int warps = 8;
    if (h->opt.warps_per_block > 0) {
        warps = h->opt.warps_per_block;
    } else if (a.Ne >= 32768) {
        const TuneKey key{(int)sizeof(T), NRHS, a.pitch};
        bool found = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            for (auto& kv : g_tune)
                if (kv.first == key) { lpc = kv.second.lpc; warps = kv.second.warps; found = true; }
        }
        if (!found) {
            LocalArgs<T> sample = a;
            // enough cells to fill the GPU in every candidate shape (a
            // sample that leaves SMs idle favours the shapes with more
            // cells per block than their full-size launch deserves)
            sample.Ne = a.Ne < 131072 ? a.Ne : 131072;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best = 1e30f;
            // small sets (pitch <= 16) also try fewer lanes per cell, down to
            // one cell per lane: every FP64 instruction then carries more
            // cells, at the price of shared memory per warp
            const int lpcs[6] = {8, 16, 32, 4, 2, 1};
            const int nl = a.pitch <= 16 ? 6 : 3;
            const int wps[2] = {4, 8};
            for (int li = 0; li < nl; ++li)
                for (int wi = 0; wi < 2; ++wi) {
                    const int c = lpcs[li], w = wps[wi];
                    if (launch_local_cfg<T, NRHS>(h, sample, c, w, s)) { cudaGetLastError(); continue; }
                    float ms = 1e30f;
                    for (int rep = 0; rep < 2; ++rep) {  // the faster of two timed launches
                        cudaEventRecord(e0, s);
                        launch_local_cfg<T, NRHS>(h, sample, c, w, s);
                        cudaEventRecord(e1, s);
                        cudaEventSynchronize(e1);
                        float m = 0;
                        cudaEventElapsedTime(&m, e0, e1);
                        if (m < ms) ms = m;
                    }
                    if (ms < best) { best = ms; lpc = c; warps = w; }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune.push_back({key, TuneVal{lpc, warps}});
        }
    }
    h->stats.tuned_lanes = lpc;
    h->stats.tuned_warps = warps;
    return launch_local_cfg<T, NRHS>(h, a, lpc, warps, s);
}

int run_local_solves(edfa_handle_s* h, cudaStream_t s)
{
    const bool two = h->opt.schur_form == 1;
    const int P = h->qmax > 0 ? h->qmax : 1;
    int rc;
    if (h->opt.precision == 1) {
        rc = dalloc_t(h, &h->xval32, (size_t)(h->qtot > 0 ? h->qtot : 1));
        if (!rc && two) rc = dalloc_t(h, &h->gval32, (size_t)(h->qtot > 0 ? h->qtot : 1));
        if (rc) return rc;
        LocalArgs<float> a{};
        a.Ne = h->Ne;
        a.pitch = P;
        a.qptr = h->qptr;
        a.qidx = h->qidx;
        a.A = Csr<float>{h->A.nrows, h->A.ncols, h->A.nnz, h->A.rowptr, h->A.col, h->a32};
        a.B = Csr<float>{h->B.nrows, h->B.ncols, h->B.nnz, h->B.rowptr, h->B.col, h->b32};
        a.C = Csr<float>{h->C.nrows, h->C.ncols, h->C.nnz, h->C.rowptr, h->C.col, h->c32};
        a.xval = h->xval32;
        a.gval = h->gval32;
        a.err = h->err;
        return two ? launch_local_n<float, 2>(h, a, s) : launch_local_n<float, 1>(h, a, s);
    }
    rc = dalloc_t(h, &h->xval, (size_t)(h->qtot > 0 ? h->qtot : 1));
    if (!rc && two) rc = dalloc_t(h, &h->gval, (size_t)(h->qtot > 0 ? h->qtot : 1));
    if (rc) return rc;
    LocalArgs<double> a{};
    a.Ne = h->Ne;
    a.pitch = P;
    a.qptr = h->qptr;
    a.qidx = h->qidx;
    a.A = csr_of(h->A);
    a.B = csr_of(h->B);
    a.C = csr_of(h->C);
    a.xval = h->xval;
    a.gval = h->gval;
    a.err = h->err;
    return two ? launch_local_n<double, 2>(h, a, s) : launch_local_n<double, 1>(h, a, s);
}

}  // namespace edfa
