// Dynamic restriction sets (Sec. 3, dynamic technique; Algorithm 1, dynamic
// branch).  Per cell m, starting from Q_(0) = the stored columns of row m of
// C (the base pattern Q_{A_ppi}):
//   solve  -A^(m) g~ = R c_m^T            (Eq. syst_MRHS_res)
//   r    = c_m^T + A R^T g~               (Eq. prol_res, the prolonged residual)
//   add at most n = min(n_add, n_ent - n_prog) indices j outside Q with the
//   largest |r_j| (values within a relative 1e-12 of the largest are ties,
//   broken by the smaller j), re-solve, repeat while n_prog < n_ent and
//   the sweep count k < it_max; the loop also ends when no candidate exists.
// Candidates are the j outside Q with a stored A_jq for some q in Q (elsewhere
// r_j = 0, and c_j = 0 outside Q because Q contains the pattern of c_m).
// r_j is summed over the stored entries of row j of A that fall in Q, in
// ascending column order.
//
// One warp per cell; A^(m) is factorised as L D L^T in a packed triangle in
// shared memory, as in the local-solve kernel.  The final sets are written to a
// padded buffer, then compacted into the CSR-like qptr/qidx.
#include <climits>

#include "internal.cuh"

namespace edfa {

constexpr int kDynWarps = 4;
constexpr int kDynCand = 256;  // candidate capacity per sweep

struct DynArgs {
    int32_t Ne;
    int cap;  // max set size (|Q_(0)| max + n_ent)
    int n_add, n_ent, it_max;
    Csr<double> A, C;
    int32_t* qpad;  // [Ne * cap]
    int64_t* cnt;   // [Ne]
    int* qmax;
    DevErr* err;
};

__device__ __forceinline__ int dyn_tri_row(int t)
{
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    return i;
}

__device__ __forceinline__ int dyn_find(const int* q, int s, int key)
{
    int lo = 0, hi = s - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = q[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// relative width of a tie between prolonged-residual magnitudes
constexpr double kDynTie = 1e-12;

__global__ void __launch_bounds__(kDynWarps * 32) k_qsets_dynamic(DynArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = a.cap;
    const int tri = P * (P + 1) / 2;
    // per-warp layout: M[tri] y[P] lc[P] dv[P] rv[kDynCand] (doubles), q[P] cand[kDynCand] tab[kDynCand] (ints)
    const size_t dbl_per_warp = (size_t)tri + 3 * P + kDynCand;
    double* M = (double*)dsm_raw + (size_t)wid * dbl_per_warp;
    double* y = M + tri;
    double* lc = y + P;
    double* dv = lc + P;
    double* rv = dv + P;
    int* ibase = (int*)((double*)dsm_raw + (size_t)kDynWarps * dbl_per_warp) + (size_t)wid * (P + 2 * kDynCand);
    int* q = ibase;
    int* cand = q + P;
    int* tab = cand + kDynCand;

    for (int64_t m = (int64_t)blockIdx.x * kDynWarps + wid; m < a.Ne; m += (int64_t)gridDim.x * kDynWarps) {
        const int64_t cb = a.C.rowptr[m], ce = a.C.rowptr[m + 1];
        int s = (int)(ce - cb);
        bool fail = s > P;
        if (fail) {
            if (lane == 0) raise_err(a.err, EDFA_ERR_BOUNDS, m);
            s = 0;
        }
        for (int i = lane; i < s; i += 32) q[i] = a.C.col[cb + i];
        __syncwarp();
        int n_prog = 0, k = 0;
        for (;;) {
            // gather the lower triangle of A^(m) and the right-hand side c_Q
            for (int t = lane; t < s * (s + 1) / 2; t += 32) M[t] = 0.0;
            __syncwarp();
            for (int i = lane; i < s; i += 32) {
                const int f = q[i];
                for (int64_t p = a.A.rowptr[f]; p < a.A.rowptr[f + 1]; ++p) {
                    const int c = a.A.col[p];
                    if (c > f) break;
                    int j = dyn_find(q, i + 1, c);
                    if (j >= 0) M[i * (i + 1) / 2 + j] = a.A.val[p];
                }
                // c_Q (binary search in row m of C)
                double cv = 0.0;
                int64_t lo = cb, hi = ce - 1;
                while (lo <= hi) {
                    int64_t mid = (lo + hi) >> 1;
                    int cm = a.C.col[mid];
                    if (cm == f) { cv = a.C.val[mid]; break; }
                    if (cm < f) lo = mid + 1; else hi = mid - 1;
                }
                y[i] = cv;
            }
            __syncwarp();
            // A^(m) = L D L^T, forward elimination of y
            bool ok = true;
            for (int kk = 0; kk < s; ++kk) {
                const double d = M[kk * (kk + 1) / 2 + kk];
                if (!(d < 0.0) || !isfinite(d)) { ok = false; break; }
                const double inv = rcp_rn(d);
                if (lane == 0) dv[kk] = inv;
                const int n = s - kk - 1;
                for (int t = lane; t < n; t += 32) {
                    const int i = kk + 1 + t;
                    lc[i] = M[i * (i + 1) / 2 + kk] * inv;
                }
                __syncwarp();
                const int ntri = n * (n + 1) / 2;
                for (int t = lane; t < ntri + n; t += 32) {
                    if (t < ntri) {
                        const int ii = dyn_tri_row(t);
                        const int jj = t - ii * (ii + 1) / 2;
                        const int i = kk + 1 + ii, j = kk + 1 + jj;
                        M[i * (i + 1) / 2 + j] -= lc[i] * M[j * (j + 1) / 2 + kk];
                    } else {
                        const int i = kk + 1 + (t - ntri);
                        y[i] -= lc[i] * y[kk];
                    }
                }
                __syncwarp();
                for (int t = lane; t < n; t += 32) {
                    const int i = kk + 1 + t;
                    M[i * (i + 1) / 2 + kk] = lc[i];
                }
                __syncwarp();
            }
            if (!ok) {
                if (lane == 0) raise_err(a.err, EDFA_ERR_BREAKDOWN, m);
                fail = true;
                break;
            }
            for (int i = lane; i < s; i += 32) y[i] *= dv[i];
            __syncwarp();
            for (int kk = s - 1; kk >= 1; --kk) {
                for (int j = lane; j < kk; j += 32) y[j] -= M[kk * (kk + 1) / 2 + j] * y[kk];
                __syncwarp();
            }
            // y = (A^(m))^{-1} c_Q, so g~ = -y
            if (!(n_prog < a.n_ent && k < a.it_max)) break;
            // candidates: j outside Q with a stored A_jq, q in Q
            for (int t = lane; t < kDynCand; t += 32) tab[t] = -1;
            __syncwarp();
            for (int i = lane; i < s; i += 32) {
                const int f = q[i];
                for (int64_t p = a.A.rowptr[f]; p < a.A.rowptr[f + 1]; ++p) {
                    const int j = a.A.col[p];
                    if (dyn_find(q, s, j) >= 0) continue;
                    unsigned hsh = ((unsigned)j * 2654435761u) & (kDynCand - 1);
                    for (int probe = 0; probe < kDynCand; ++probe) {
                        int prev = atomicCAS(&tab[hsh], -1, j);
                        if (prev == -1 || prev == j) break;
                        hsh = (hsh + 1) & (kDynCand - 1);
                    }
                }
            }
            __syncwarp();
            int nc = 0;
            for (int b0 = 0; b0 < kDynCand; b0 += 32) {
                int v = tab[b0 + lane];
                unsigned bal = __ballot_sync(0xffffffffu, v >= 0);
                if (v >= 0) cand[nc + __popc(bal & ((1u << lane) - 1u))] = v;
                nc += __popc(bal);
            }
            __syncwarp();
            if (nc > kDynCand * 3 / 4) {
                if (lane == 0) raise_err(a.err, EDFA_ERR_BOUNDS, m);
                fail = true;
                break;
            }
            if (nc == 0) break;
            // prolonged residual at the candidates, ascending q within row j of A
            for (int t = lane; t < nc; t += 32) {
                const int j = cand[t];
                double r = 0.0;
                for (int64_t p = a.A.rowptr[j]; p < a.A.rowptr[j + 1]; ++p) {
                    int pos = dyn_find(q, s, a.A.col[p]);
                    if (pos >= 0) r = fma(a.A.val[p], -y[pos], r);
                }
                rv[t] = fabs(r);
            }
            __syncwarp();
            k += 1;
            const int want = min(a.n_add, a.n_ent - n_prog);
            int added = 0;
            while (added < want) {
                // largest remaining |r_j|, then the smallest j within a relative
                // kDynTie of it (rounding-order ties count as ties)
                double rmax = -1.0;
                for (int t = lane; t < nc; t += 32)
                    if (cand[t] >= 0 && rv[t] > rmax) rmax = rv[t];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
                if (rmax < 0.0) break;
                const double floor_r = rmax * (1.0 - kDynTie);
                int bj = INT_MAX, bt = -1;
                for (int t = lane; t < nc; t += 32)
                    if (cand[t] >= 0 && rv[t] >= floor_r && cand[t] < bj) { bj = cand[t]; bt = t; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
                    int t2 = __shfl_xor_sync(0xffffffffu, bt, o);
                    if (j2 < bj) { bj = j2; bt = t2; }
                }
                if (bt < 0) break;
                if (s + 1 > P) {
                    if (lane == 0) raise_err(a.err, EDFA_ERR_BOUNDS, m);
                    fail = true;
                    break;
                }
                // sorted insert of bj into q (lane 0), mark the candidate taken
                if (lane == 0) {
                    int pos = s;
                    while (pos > 0 && q[pos - 1] > bj) { q[pos] = q[pos - 1]; --pos; }
                    q[pos] = bj;
                    cand[bt] = -1;
                }
                __syncwarp();
                s += 1;
                added += 1;
            }
            if (fail) break;
            n_prog += added;
            __syncwarp();
        }
        if (fail) s = 0;
        int32_t* out = a.qpad + (size_t)m * P;
        for (int i = lane; i < s; i += 32) out[i] = q[i];
        if (lane == 0) {
            a.cnt[m] = s;
            atomicMax(a.qmax, s);
        }
        __syncwarp();
    }
}

__global__ void k_qpad_compact(int32_t Ne, int cap, const int32_t* qpad, const int64_t* qptr, int32_t* qidx)
{
    int64_t m = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (m >= Ne) return;
    const int64_t b = qptr[m];
    const int s = (int)(qptr[m + 1] - b);
    for (int i = lane; i < s; i += 32) qidx[b + i] = qpad[(size_t)m * cap + i];
}

__global__ void k_row_len_max(int32_t n, const int64_t* rowptr, int* out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, (int)(rowptr[i + 1] - rowptr[i]));
}

int build_qsets_dynamic(edfa_handle_s* h, cudaStream_t s)
{
    const int32_t Ne = h->Ne;
    int* dmax = nullptr;
    if (cudaMallocAsync((void**)&dmax, 2 * sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemsetAsync(dmax, 0, 2 * sizeof(int), s);
    if (Ne > 0) (edfa::count_launch(), k_row_len_max<<<(Ne + 255) / 256, 256, 0, s>>>(Ne, h->C.rowptr, dmax));
    int c0 = 0;
    cudaMemcpyAsync(&c0, dmax, sizeof(int), cudaMemcpyDeviceToHost, s);
    int rc = check_err(h, s);
    if (rc) return rc;
    const int cap = c0 + (h->opt.n_ent > 0 ? h->opt.n_ent : 0);
    const int P = cap > 0 ? cap : 1;
    const size_t per_warp = ((size_t)P * (P + 1) / 2 + 3 * P + kDynCand) * sizeof(double) +
                            ((size_t)P + 2 * kDynCand) * sizeof(int);
    const size_t smem = per_warp * kDynWarps;
    if (smem > 220 * 1024) return EDFA_ERR_BOUNDS;
    if (cudaFuncSetAttribute(k_qsets_dynamic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return EDFA_ERR_CUDA;
    rc = dalloc_t(h, &h->qptr, (size_t)Ne + 1);
    if (rc) return rc;
    int32_t* qpad = nullptr;
    if (cudaMallocAsync((void**)&qpad, (size_t)(Ne > 0 ? Ne : 1) * P * sizeof(int32_t), s) != cudaSuccess)
        return EDFA_ERR_OOM;
    cudaMemsetAsync(h->qptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    DynArgs a{};
    a.Ne = Ne;
    a.cap = P;
    a.n_add = h->opt.n_add;
    a.n_ent = h->opt.n_ent;
    a.it_max = h->opt.it_max;
    a.A = csr_of(h->A);
    a.C = csr_of(h->C);
    a.qpad = qpad;
    a.cnt = h->qptr;
    a.qmax = dmax + 1;
    a.err = h->err;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_qsets_dynamic, kDynWarps * 32, smem);
    if (per < 1) per = 1;
    long long grid = (long long)per * h->nsm;
    long long need = (Ne + kDynWarps - 1) / kDynWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    (edfa::count_launch(), k_qsets_dynamic<<<(unsigned)grid, kDynWarps * 32, smem, s>>>(a));
    rc = scan_i64(h, h->qptr, Ne, s);
    if (rc) return rc;
    int64_t tot = 0;
    int qm = 0;
    cudaMemcpyAsync(&tot, h->qptr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&qm, dmax + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    rc = check_err(h, s);
    if (rc) { cudaFreeAsync(qpad, s); cudaFreeAsync(dmax, s); return rc; }
    h->qtot = tot;
    h->qmax = qm;
    rc = dalloc_t(h, &h->qidx, (size_t)(tot > 0 ? tot : 1));
    if (rc) return rc;
    if (Ne > 0)
        (edfa::count_launch(), k_qpad_compact<<<(unsigned)((Ne + 7) / 8), 256, 0, s>>>(Ne, P, qpad, h->qptr, h->qidx));
    cudaFreeAsync(qpad, s);
    cudaFreeAsync(dmax, s);
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

}  // namespace edfa
