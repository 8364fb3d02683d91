// Approximate Schur complement (Eq. sparse_S):
//   form 0 (one-sided):  H~ = C X~            (X~ = -F~)
//   form 1 (two-sided):  H~ = G~ A F~ = -(G~ A) X~
//   S~ = D - H~  on pattern(H~) u pattern(D) u diagonal, columns ascending.
// The pattern is structural: a position is kept whenever a product term
// reaches it, even if the values cancel.
//
// Two passes, one warp per row of S~: a shared-memory hash set collects the
// column candidates (cells m whose set Q^(m) meets the faces reached from row
// E), pass 0 counts them, pass 1 sorts them and computes every entry as an
// ordered merge of two ascending index lists (no atomics in the value path,
// so the result is deterministic).
#include <climits>

#include "internal.cuh"

namespace edfa {

constexpr int kHS = 1024;      // hash capacity (columns of one S~ row, before load-factor limit)
constexpr int kUCap = 512;     // two-sided: faces reached by G~_E A

// ------------------------------------------------------------ X~ rows
__global__ void k_q_count(const int32_t* qidx, int64_t tot, unsigned long long* cnt)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < tot) atomicAdd(&cnt[qidx[p]], 1ull);
}

__global__ void k_q_fill(int32_t Ne, const int64_t* qptr, const int32_t* qidx, unsigned long long* cursor,
                         int32_t* xr_cell)
{
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= Ne) return;
    for (int64_t p = qptr[m]; p < qptr[m + 1]; ++p) {
        unsigned long long pos = atomicAdd(&cursor[qidx[p]], 1ull);
        xr_cell[pos] = (int32_t)m;
    }
}

__global__ void k_row_sort2(const int64_t* ptr, int32_t* col, int64_t n)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t b = ptr[r], e = ptr[r + 1];
    for (int64_t p = b + 1; p < e; ++p) {
        int32_t v = col[p];
        int64_t q = p - 1;
        while (q >= b && col[q] > v) { col[q + 1] = col[q]; --q; }
        col[q + 1] = v;
    }
}

// ------------------------------------------------------------ helpers
__device__ __forceinline__ bool hs_insert(int* tab, int key)
{
    unsigned h = ((unsigned)key * 2654435761u) & (kHS - 1);
    for (int probe = 0; probe < kHS; ++probe) {
        int prev = atomicCAS(&tab[h], -1, key);
        if (prev == -1) return true;
        if (prev == key) return false;
        h = (h + 1) & (kHS - 1);
    }
    return false;
}

template <class T>
struct SchurArgs {
    int form;
    int32_t Ne;
    Csr<T> A, C;
    Csr<double> D;
    const int64_t* xptr;  // X~ column m on (xptr, xidx): Q^(m), or what pre-filtration kept of it
    const int32_t* xidx;
    const T* xval;
    const int64_t* gptr;  // G~ row m on (gptr, gidx) (two-sided form)
    const int32_t* gidx;
    const T* gval;
    const int64_t* xr_ptr;
    const int32_t* xr_cell;
    int64_t* cnt;        // pass 0
    int* rowmax;
    const int64_t* s_ptr;  // pass 1
    int32_t* s_col;
    T* h_val;
    int64_t* d_map;
    DevErr* err;
};

// binary search of key in sorted a[0..n)
__device__ __forceinline__ int bsearch_i(const int* a, int n, int key)
{
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ void warp_bitonic(int* a, int n2, int lane)
{
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n2; i += 32) {
                int ixj = i ^ j;
                if (ixj > i) {
                    int x = a[i], y = a[ixj];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[ixj] = x; }
                }
            }
            __syncwarp();
        }
}

// compact the hash table into out[0..n) ascending; returns n, or -1 (nothing
// written) when n exceeds cap (cap a power of two)
__device__ int hs_compact_sort(const int* tab, int* out, int cap, int lane)
{
    int n = 0;
    for (int base = 0; base < kHS; base += 32) n += __popc(__ballot_sync(0xffffffffu, tab[base + lane] >= 0));
    if (n > cap) return -1;
    n = 0;
    for (int base = 0; base < kHS; base += 32) {
        int v = tab[base + lane];
        bool has = v >= 0;
        unsigned b = __ballot_sync(0xffffffffu, has);
        if (has) out[n + __popc(b & ((1u << lane) - 1u))] = v;
        n += __popc(b);
    }
    __syncwarp();
    int n2 = 32;
    while (n2 < n) n2 <<= 1;
    for (int i = n + lane; i < n2; i += 32) out[i] = INT_MAX;
    __syncwarp();
    warp_bitonic(out, n2, lane);
    return n;
}

template <class T, int PASS, int kSWarps>
__global__ void __launch_bounds__(kSWarps * 32) k_schur(SchurArgs<T> a)
{
    __shared__ int s_tab[kSWarps][kHS];
    __shared__ int s_key[kSWarps][kHS];
    __shared__ int s_u[kSWarps][kUCap];
    __shared__ T s_uv[kSWarps][kUCap];
    __shared__ int s_cnt[kSWarps];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* tab = s_tab[wid];
    int* key = s_key[wid];
    int* ul = s_u[wid];
    T* uv = s_uv[wid];
    for (int64_t E = (int64_t)blockIdx.x * kSWarps + wid; E < a.Ne; E += (int64_t)gridDim.x * kSWarps) {
        for (int i = lane; i < kHS; i += 32) tab[i] = -1;
        if (lane == 0) s_cnt[wid] = 0;
        __syncwarp();
        int nu = 0;
        bool overflow = false;
        if (a.form == 1) {
            // faces g reached by G~_E A: A-neighbours of Q^(E)
            int* ut = key;  // reuse as a second hash table
            for (int i = lane; i < kHS; i += 32) ut[i] = -1;
            __syncwarp();
            for (int64_t p = a.gptr[E]; p < a.gptr[E + 1]; ++p) {
                int f = a.gidx[p];
                for (int64_t q = a.A.rowptr[f] + lane; q < a.A.rowptr[f + 1]; q += 32) hs_insert(ut, a.A.col[q]);
            }
            __syncwarp();
            nu = hs_compact_sort(ut, ul, kUCap, lane);
            if (nu < 0) { overflow = true; nu = 0; }
            // u_g = sum_{f in Q^(E)} G~[E,f] A[f,g]  (A symmetric: row g of A), ascending f
            const int64_t qb = a.gptr[E], qe = a.gptr[E + 1];
            for (int t = lane; t < nu; t += 32) {
                int gidx = ul[t];
                int64_t pa = a.A.rowptr[gidx], ea = a.A.rowptr[gidx + 1];
                int64_t pq = qb;
                T acc = T(0);
                while (pa < ea && pq < qe) {
                    int ca = a.A.col[pa], cq = a.gidx[pq];
                    if (ca == cq) { acc = fma(a.gval[pq], a.A.val[pa], acc); ++pa; ++pq; }
                    else if (ca < cq) ++pa;
                    else ++pq;
                }
                uv[t] = acc;
            }
            for (int i = lane; i < kHS; i += 32) key[i] = -1;
            __syncwarp();
        }
        // column candidates
        if (lane == 0) { if (hs_insert(tab, (int)E)) atomicAdd(&s_cnt[wid], 1); }
        for (int64_t p = a.D.rowptr[E] + lane; p < a.D.rowptr[E + 1]; p += 32)
            if (hs_insert(tab, a.D.col[p])) atomicAdd(&s_cnt[wid], 1);
        if (a.form == 0) {
            for (int64_t p = a.C.rowptr[E]; p < a.C.rowptr[E + 1]; ++p) {
                int f = a.C.col[p];
                for (int64_t t = a.xr_ptr[f] + lane; t < a.xr_ptr[f + 1]; t += 32)
                    if (hs_insert(tab, a.xr_cell[t])) atomicAdd(&s_cnt[wid], 1);
            }
        } else {
            for (int t0 = 0; t0 < nu; ++t0) {
                int gidx = ul[t0];
                for (int64_t t = a.xr_ptr[gidx] + lane; t < a.xr_ptr[gidx + 1]; t += 32)
                    if (hs_insert(tab, a.xr_cell[t])) atomicAdd(&s_cnt[wid], 1);
            }
        }
        __syncwarp();
        int cnt = s_cnt[wid];
        if (cnt > kHS * 3 / 4) overflow = true;
        if (overflow) {
            if (lane == 0) raise_err(a.err, EDFA_ERR_BOUNDS, E);
            if (PASS == 0 && lane == 0) a.cnt[E] = 0;
            __syncwarp();
            continue;
        }
        if (PASS == 0) {
            if (lane == 0) { a.cnt[E] = cnt; atomicMax(a.rowmax, cnt); }
            __syncwarp();
            continue;
        }
        int n = hs_compact_sort(tab, key, kHS, lane);
        const int64_t sb = a.s_ptr[E];
        for (int t = lane; t < n; t += 32) {
            const int m = key[t];
            a.s_col[sb + t] = m;
            const int64_t qb = a.xptr[m], qe = a.xptr[m + 1];
            T acc = T(0);
            if (a.form == 0) {
                // H~[E,m] = sum over f in C_E and Q^(m), ascending f
                int64_t pc = a.C.rowptr[E], ec = a.C.rowptr[E + 1], pq = qb;
                while (pc < ec && pq < qe) {
                    int cc = a.C.col[pc], cq = a.xidx[pq];
                    if (cc == cq) { acc = fma(a.C.val[pc], a.xval[pq], acc); ++pc; ++pq; }
                    else if (cc < cq) ++pc;
                    else ++pq;
                }
            } else {
                // H~[E,m] = -sum_{g in Q^(m)} u_g X~[g,m]
                for (int64_t pq = qb; pq < qe; ++pq) {
                    int pos = bsearch_i(ul, nu, a.xidx[pq]);
                    if (pos >= 0) acc = fma(-uv[pos], a.xval[pq], acc);
                }
            }
            a.h_val[sb + t] = acc;
        }
        for (int64_t p = a.D.rowptr[E] + lane; p < a.D.rowptr[E + 1]; p += 32)
            a.d_map[p] = sb + bsearch_i(key, n, a.D.col[p]);
        __syncwarp();
    }
}

template <class T>
__global__ void k_stage2(int64_t s_nnz, const T* h_val, T* s_val)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s_nnz; k += (int64_t)gridDim.x * blockDim.x)
        s_val[k] = -h_val[k];
}

template <class T>
__global__ void k_stage2_d(int64_t d_nnz, const double* d_val, const int64_t* d_map, T* s_val)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < d_nnz; p += (int64_t)gridDim.x * blockDim.x)
        s_val[d_map[p]] += (T)d_val[p];
}

template <class T>
static int schur_t(edfa_handle_s* h, const T* xval, const T* gval, T** h_val, cudaStream_t s)
{
    const int32_t Ne = h->Ne, Nf = h->Nf;
    // X~ row pattern
    int rc = dalloc_t(h, &h->xr_ptr, (size_t)Nf + 1);
    if (!rc) rc = dalloc_t(h, &h->xr_cell, (size_t)(h->x_tot > 0 ? h->x_tot : 1));
    if (rc) return rc;
    cudaMemsetAsync(h->xr_ptr, 0, ((size_t)Nf + 1) * sizeof(int64_t), s);
    if (h->x_tot > 0)
        (edfa::count_launch(), k_q_count<<<(unsigned)((h->x_tot + 255) / 256), 256, 0, s>>>(h->x_idx, h->x_tot, (unsigned long long*)h->xr_ptr));
    rc = scan_i64(h, h->xr_ptr, Nf, s);
    if (rc) return rc;
    unsigned long long* cursor = nullptr;
    if (cudaMallocAsync((void**)&cursor, ((size_t)Nf + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemcpyAsync(cursor, h->xr_ptr, ((size_t)Nf + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (Ne > 0) (edfa::count_launch(), k_q_fill<<<(Ne + 255) / 256, 256, 0, s>>>(Ne, h->x_ptr, h->x_idx, cursor, h->xr_cell));
    if (Nf > 0) (edfa::count_launch(), k_row_sort2<<<(Nf + 255) / 256, 256, 0, s>>>(h->xr_ptr, h->xr_cell, Nf));
    cudaFreeAsync(cursor, s);

    SchurArgs<T> a{};
    a.form = h->opt.schur_form;
    a.Ne = Ne;
    if constexpr (sizeof(T) == 8) {
        a.A = csr_of(h->A);
        a.C = csr_of(h->C);
    } else {
        a.A = Csr<float>{h->A.nrows, h->A.ncols, h->A.nnz, h->A.rowptr, h->A.col, h->a32};
        a.C = Csr<float>{h->C.nrows, h->C.ncols, h->C.nnz, h->C.rowptr, h->C.col, h->c32};
    }
    a.D = csr_of(h->D);
    a.xptr = h->x_ptr;
    a.xidx = h->x_idx;
    a.xval = xval;
    a.gptr = h->g_ptr;
    a.gidx = h->g_idx;
    a.gval = gval;
    a.xr_ptr = h->xr_ptr;
    a.xr_cell = h->xr_cell;
    a.err = h->err;
    rc = dalloc_t(h, &h->s_ptr, (size_t)Ne + 1);
    if (rc) return rc;
    int* rowmax = nullptr;
    if (cudaMallocAsync((void**)&rowmax, sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemsetAsync(rowmax, 0, sizeof(int), s);
    cudaMemsetAsync(h->s_ptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    a.cnt = h->s_ptr;
    a.rowmax = rowmax;
    // autotuned tile: warps (rows) per block of the Schur kernel, timed on a
    // prefix sample of the rows with the counting pass
    int sw = 2;
    if (Ne >= 32768) {
        SchurArgs<T> sample = a;
        sample.Ne = 8192;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        const int cands[2] = {1, 2};
        for (int c : cands) {
            for (int rep = 0; rep < 2; ++rep) {
                if (rep == 1) cudaEventRecord(e0, s);
                if (c == 1) (edfa::count_launch(), k_schur<T, 0, 1><<<(unsigned)(h->nsm * 8), 32, 0, s>>>(sample));
                else (edfa::count_launch(), k_schur<T, 0, 2><<<(unsigned)(h->nsm * 4), 64, 0, s>>>(sample));
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; sw = c; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaMemsetAsync(rowmax, 0, sizeof(int), s);
        cudaMemsetAsync(h->s_ptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    }
    h->stats.tuned_schur_warps = sw;
    int per = 0;
    if (sw == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_schur<T, 0, 1>, 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_schur<T, 0, 2>, 64, 0);
    if (per < 1) per = 1;
    long long grid = (long long)per * h->nsm;
    long long need = (Ne + sw - 1) / sw;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (sw == 1) (edfa::count_launch(), k_schur<T, 0, 1><<<(unsigned)grid, 32, 0, s>>>(a));
    else (edfa::count_launch(), k_schur<T, 0, 2><<<(unsigned)grid, 64, 0, s>>>(a));
    rc = scan_i64(h, h->s_ptr, Ne, s);
    if (rc) return rc;
    int64_t nnz = 0;
    cudaMemcpyAsync(&nnz, h->s_ptr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(rowmax, s);
    rc = check_err(h, s);
    if (rc) return rc;
    h->s_nnz = nnz;
    rc = dalloc_t(h, &h->s_col, (size_t)(nnz > 0 ? nnz : 1));
    if (!rc) rc = dalloc_t(h, h_val, (size_t)(nnz > 0 ? nnz : 1));
    if (!rc) rc = dalloc_t(h, &h->d_map, (size_t)(h->D.nnz > 0 ? h->D.nnz : 1));
    if (rc) return rc;
    a.s_ptr = h->s_ptr;
    a.s_col = h->s_col;
    a.h_val = *h_val;
    a.d_map = h->d_map;
    if (sw == 1) (edfa::count_launch(), k_schur<T, 1, 1><<<(unsigned)grid, 32, 0, s>>>(a));
    else (edfa::count_launch(), k_schur<T, 1, 2><<<(unsigned)grid, 64, 0, s>>>(a));
    if (cudaGetLastError() != cudaSuccess) return EDFA_ERR_CUDA;
    // post-filtration of H~ (Algorithm 1, Stage 1): compacts the S~ pattern
    if (h->opt.filtration == EDFA_FILT_POST_H) return postfilter_h<T>(h, *h_val, s);
    return EDFA_OK;
}

int build_schur(edfa_handle_s* h, cudaStream_t s)
{
    if (h->opt.precision == 1) {
        int rc = schur_t<float>(h, h->xf32, h->gf32, &h->h_val32, s);
        if (!rc) rc = dalloc_t(h, &h->s_val32, (size_t)(h->s_nnz > 0 ? h->s_nnz : 1));
        return rc;
    }
    int rc = schur_t<double>(h, h->xf64, h->gf64, &h->h_val, s);
    if (!rc) rc = dalloc_t(h, &h->s_val, (size_t)(h->s_nnz > 0 ? h->s_nnz : 1));
    return rc;
}

int stage2_values(edfa_handle_s* h, cudaStream_t s)
{
    int64_t g = (h->s_nnz + 255) / 256;
    if (g > 65535) g = 65535;
    if (g < 1) g = 1;
    int64_t gd = (h->D.nnz + 255) / 256;
    if (gd > 65535) gd = 65535;
    if (gd < 1) gd = 1;
    if (h->opt.precision == 1) {
        (edfa::count_launch(), k_stage2<float><<<(unsigned)g, 256, 0, s>>>(h->s_nnz, h->h_val32, h->s_val32));
        (edfa::count_launch(), k_stage2_d<float><<<(unsigned)gd, 256, 0, s>>>(h->D.nnz, h->D.val, h->d_map, h->s_val32));
    } else {
        (edfa::count_launch(), k_stage2<double><<<(unsigned)g, 256, 0, s>>>(h->s_nnz, h->h_val, h->s_val));
        (edfa::count_launch(), k_stage2_d<double><<<(unsigned)gd, 256, 0, s>>>(h->D.nnz, h->D.val, h->d_map, h->s_val));
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

}  // namespace edfa
