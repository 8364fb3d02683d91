// Approximate Schur complement (Eq. sparse_S):
//   form 0 (one-sided):  H~ = C X~            (X~ = -F~)
//   form 1 (two-sided):  H~ = G~ A F~ = -(G~ A) X~
//   S~ = D - H~  on pattern(H~) u pattern(D) u diagonal, columns ascending.
// The pattern is structural: a position is kept whenever a product term
// reaches it, even if the values cancel.
//
// Two passes, one warp per row of S~: a shared-memory hash set collects the
// column candidates (cells m whose set Q^(m) meets the faces reached from row
// E; in the one-sided form the (cell, X~ value) pairs of all faces of the row
// are loaded at once, the lanes taking the flattened list) and pass 0 counts
// them.  The numeric pass (k_schur_num) sorts them, maps
// every column to its position through the same hash, and forms the row as a
// row-wise (Gustavson) product: for every face f of row E of C in ascending
// order, the lanes take the cells m of row f of X~ (distinct within one f) and
// add C[E,f] X~[f,m] into a shared-memory accumulator, with a warp barrier
// between faces.  Every entry is thus summed over ascending f, the order of
// the plain definition; no atomics touch values, so the result is
// deterministic.  X~ is read through a row-major copy (cells and values of
// every face row) made once per build.
#include <climits>
#include <mutex>
#include <utility>
#include <vector>

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

// row-major copy of X~ with its values: face row f lists (m, X~[f,m])
template <class T>
__global__ void k_q_fill_vals(int32_t Ne, const int64_t* qptr, const int32_t* qidx, const T* xv,
                              unsigned long long* cursor, int32_t* xr_cell, T* xr_val)
{
    int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= Ne) return;
    for (int64_t p = qptr[m]; p < qptr[m + 1]; ++p) {
        unsigned long long pos = atomicAdd(&cursor[qidx[p]], 1ull);
        xr_cell[pos] = (int32_t)m;
        xr_val[pos] = xv[p];
    }
}

// sort (col, val) pairs of every row by col (insertion sort, rows are short)
template <class T>
__global__ void k_row_sort_pairs(const int64_t* ptr, int32_t* col, T* val, int64_t n)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t b = ptr[r], e = ptr[r + 1];
    for (int64_t p = b + 1; p < e; ++p) {
        int32_t v = col[p];
        T w = val[p];
        int64_t q = p - 1;
        while (q >= b && col[q] > v) { col[q + 1] = col[q]; val[q + 1] = val[q]; --q; }
        col[q + 1] = v;
        val[q + 1] = w;
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

// counting pass: the number of columns of every row of S~ (and the longest)
template <class T, int kSWarps>
__global__ void __launch_bounds__(kSWarps * 32) k_schur_count(SchurArgs<T> a)
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
        const int64_t cb = a.C.rowptr[E];
        const int nf = (int)(a.C.rowptr[E + 1] - cb);
        if (a.form == 0 && nf <= 32) {
            // the cells of all faces' X~ rows at once (flattened, as in the
            // numeric pass), not face after face
            int64_t fb = 0;
            int flen = 0;
            if (lane < nf) {
                const int f = a.C.col[cb + lane];
                fb = a.xr_ptr[f];
                flen = (int)(a.xr_ptr[f + 1] - fb);
            }
            int inc = flen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const int fpre = inc - flen;
            const int L = __shfl_sync(0xffffffffu, inc, 31);
            for (int k0 = 0; k0 < L; k0 += 32) {
                const int k = k0 + lane;
                int lo = 0, hi = nf - 1;
#pragma unroll
                for (int step = 0; step < 5; ++step) {
                    const int mid = (lo + hi + 1) >> 1;
                    const int pm = __shfl_sync(0xffffffffu, fpre, mid);
                    if (lo < hi) {
                        if (pm <= k) lo = mid; else hi = mid - 1;
                    }
                }
                const int64_t ob = __shfl_sync(0xffffffffu, fb, lo);
                const int op = __shfl_sync(0xffffffffu, fpre, lo);
                if (k < L && hs_insert(tab, a.xr_cell[ob + (k - op)])) atomicAdd(&s_cnt[wid], 1);
            }
        } else if (a.form == 0) {
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
            if (lane == 0) a.cnt[E] = 0;
            __syncwarp();
            continue;
        }
        if (lane == 0) { a.cnt[E] = cnt; atomicMax(a.rowmax, cnt); }
        __syncwarp();
    }
}

// ------------------------------------------------------------ numeric pass
// hash of capacity cap (a power of two): insert / slot lookup
__device__ __forceinline__ bool hsc_insert(int* tab, int cap, int key)
{
    unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(cap - 1);
    for (int probe = 0; probe < cap; ++probe) {
        int prev = atomicCAS(&tab[h], -1, key);
        if (prev == -1) return true;
        if (prev == key) return false;
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return false;
}

__device__ __forceinline__ int hsc_slot(const int* tab, int cap, int key)
{
    unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(cap - 1);
    for (int probe = 0; probe < cap; ++probe) {
        const int k = tab[h];
        if (k == key) return (int)h;
        if (k < 0) return -1;
        h = (h + 1) & (unsigned)(cap - 1);
    }
    return -1;
}

// compact the keys of tab[0..cap) into out ascending (out holds cap entries)
__device__ int hsc_compact_sort(const int* tab, int cap, int* out, int lane)
{
    int n = 0;
    for (int base = 0; base < cap; base += 32) {
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

constexpr int kNumWarps = 8;  // rows (warps) per block of the numeric pass

template <class T, int FORM>
__host__ __device__ constexpr size_t num_warp_bytes(int hs)
{
    // one-sided form: also the flattened (cell, X~ value) list of the row's
    // faces, hs entries
    return ((size_t)hs * sizeof(T) + (size_t)hs * 12 + (size_t)(FORM ? (hs > kHS ? hs : kHS) : hs) * 4 +
            (FORM ? (size_t)kUCap * (4 + sizeof(T)) : (size_t)hs * (4 + sizeof(T))) + 15) & ~(size_t)15;
}

template <class T, int FORM>
__global__ void __launch_bounds__(kNumWarps * 32, 2)
k_schur_num(SchurArgs<T> a, const T* __restrict__ xr_val, int hs)
{
    extern __shared__ __align__(16) unsigned char nsm_raw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wb = nsm_raw + wid * num_warp_bytes<T, FORM>(hs);
    T* acc = (T*)wb;              // [hs] accumulator by position
    int* tab = (int*)(acc + hs);  // [hs] column hash
    int* pos = tab + hs;          // [hs] position of the column in each slot
    int* key = pos + hs;          // [hs] sorted columns (two-sided: [max(hs, kHS)], also the face hash)
    const int kc = FORM ? (hs > kHS ? hs : kHS) : hs;
    int* ul = key + kc;           // two-sided: faces g of G~_E A
    T* uv = (T*)(ul + kUCap);     // and their values u_g
    T* flv = acc;                 // one-sided: X~ values of the flattened list [hs]
    int* flc = ul;                // and their cells [hs]
    if (FORM == 0) {
        flv = (T*)(((uintptr_t)(key + kc) + 7) & ~(uintptr_t)7);
        flc = (int*)(flv + hs);
    }
    const int64_t nw = (int64_t)gridDim.x * kNumWarps;
    for (int64_t E = (int64_t)blockIdx.x * kNumWarps + wid; E < a.Ne; E += nw) {
        for (int i = lane; i < hs; i += 32) tab[i] = -1;
        int nu = 0;
        bool bad = false;
        if (FORM == 1) {
            for (int i = lane; i < kHS; i += 32) key[i] = -1;
            __syncwarp();
            for (int64_t p = a.gptr[E]; p < a.gptr[E + 1]; ++p) {
                const int f = a.gidx[p];
                for (int64_t q = a.A.rowptr[f] + lane; q < a.A.rowptr[f + 1]; q += 32) hs_insert(key, a.A.col[q]);
            }
            __syncwarp();
            nu = hs_compact_sort(key, ul, kUCap, lane);
            if (nu < 0) { bad = true; nu = 0; }
            const int64_t qb = a.gptr[E], qe = a.gptr[E + 1];
            for (int t = lane; t < nu; t += 32) {
                const int g = ul[t];
                int64_t pa = a.A.rowptr[g], ea = a.A.rowptr[g + 1], pq = qb;
                T u = T(0);
                while (pa < ea && pq < qe) {
                    const int ca = a.A.col[pa], cq = a.gidx[pq];
                    if (ca == cq) { u = fma(a.gval[pq], a.A.val[pa], u); ++pa; ++pq; }
                    else if (ca < cq) ++pa;
                    else ++pq;
                }
                uv[t] = u;
            }
        }
        __syncwarp();
        // columns: E, the row of D, every cell reached by a product term
        if (lane == 0) hsc_insert(tab, hs, (int)E);
        for (int64_t p = a.D.rowptr[E] + lane; p < a.D.rowptr[E + 1]; p += 32) hsc_insert(tab, hs, a.D.col[p]);
        // one-sided form, rows with at most 32 faces: lane j holds face j of the
        // row of C (its value, the start and length of its X~ row, the prefix
        // of the lengths), and the (cell, value) pairs of all faces are loaded
        // at once, flattened, instead of face after face
        const int64_t cb = a.C.rowptr[E];
        const int nf = (int)(a.C.rowptr[E + 1] - cb);
        bool flat = FORM == 0 && nf <= 32;
        T fc = T(0);
        int64_t fb = 0;
        int flen = 0, fpre = 0, L = 0;
        if (flat) {
            if (lane < nf) {
                const int f = a.C.col[cb + lane];
                fc = a.C.val[cb + lane];
                fb = a.xr_ptr[f];
                flen = (int)(a.xr_ptr[f + 1] - fb);
            }
            int inc = flen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            fpre = inc - flen;
            L = __shfl_sync(0xffffffffu, inc, 31);
            flat = L <= hs;
        }
        if (FORM == 0 && flat) {
            for (int k0 = 0; k0 < L; k0 += 32) {
                const int k = k0 + lane;
                int lo = 0, hi = nf - 1;  // face of entry k: last j with fpre_j <= k
#pragma unroll
                for (int step = 0; step < 5; ++step) {
                    const int mid = (lo + hi + 1) >> 1;
                    const int pm = __shfl_sync(0xffffffffu, fpre, mid);
                    if (lo < hi) {
                        if (pm <= k) lo = mid; else hi = mid - 1;
                    }
                }
                const int64_t ob = __shfl_sync(0xffffffffu, fb, lo);
                const int op = __shfl_sync(0xffffffffu, fpre, lo);
                if (k < L) {
                    const int64_t t = ob + (k - op);
                    const int cell = a.xr_cell[t];
                    flc[k] = cell;
                    flv[k] = xr_val[t];
                    hsc_insert(tab, hs, cell);
                }
            }
        } else if (FORM == 0) {
            for (int64_t p = a.C.rowptr[E]; p < a.C.rowptr[E + 1]; ++p) {
                const int f = a.C.col[p];
                for (int64_t t = a.xr_ptr[f] + lane; t < a.xr_ptr[f + 1]; t += 32) hsc_insert(tab, hs, a.xr_cell[t]);
            }
        } else {
            for (int t0 = 0; t0 < nu; ++t0) {
                const int g = ul[t0];
                for (int64_t t = a.xr_ptr[g] + lane; t < a.xr_ptr[g + 1]; t += 32) hsc_insert(tab, hs, a.xr_cell[t]);
            }
        }
        __syncwarp();
        const int n = hsc_compact_sort(tab, hs, key, lane);
        const int64_t sb = a.s_ptr[E];
        if (bad || n != (int)(a.s_ptr[E + 1] - sb)) {
            // the counting pass saw another set (or the face list overflowed)
            if (lane == 0) raise_err(a.err, EDFA_ERR_BOUNDS, E);
            __syncwarp();
            continue;
        }
        for (int t = lane; t < n; t += 32) {
            const int sl = hsc_slot(tab, hs, key[t]);
            if (sl >= 0) pos[sl] = t;
            acc[t] = T(0);
        }
        __syncwarp();
        // Gustavson product, faces in ascending order
        if (FORM == 0 && flat) {
            for (int j = 0; j < nf; ++j) {
                const T c = __shfl_sync(0xffffffffu, fc, j);
                const int pj = __shfl_sync(0xffffffffu, fpre, j);
                const int lj = __shfl_sync(0xffffffffu, flen, j);
                for (int k = pj + lane; k < pj + lj; k += 32) {
                    const int sl = hsc_slot(tab, hs, flc[k]);
                    if (sl < 0) continue;
                    const int q = pos[sl];
                    acc[q] = fma(c, flv[k], acc[q]);
                }
                __syncwarp();
            }
        } else if (FORM == 0) {
            for (int64_t p = a.C.rowptr[E]; p < a.C.rowptr[E + 1]; ++p) {
                const int f = a.C.col[p];
                const T c = a.C.val[p];
                for (int64_t t = a.xr_ptr[f] + lane; t < a.xr_ptr[f + 1]; t += 32) {
                    const int sl = hsc_slot(tab, hs, a.xr_cell[t]);
                    if (sl < 0) continue;  // cannot happen: every cell was inserted above
                    const int q = pos[sl];
                    acc[q] = fma(c, xr_val[t], acc[q]);
                }
                __syncwarp();
            }
        } else {
            for (int t0 = 0; t0 < nu; ++t0) {
                const int g = ul[t0];
                const T u = uv[t0];
                for (int64_t t = a.xr_ptr[g] + lane; t < a.xr_ptr[g + 1]; t += 32) {
                    const int sl = hsc_slot(tab, hs, a.xr_cell[t]);
                    if (sl < 0) continue;
                    const int q = pos[sl];
                    acc[q] = fma(-u, xr_val[t], acc[q]);
                }
                __syncwarp();
            }
        }
        for (int t = lane; t < n; t += 32) {
            a.s_col[sb + t] = key[t];
            a.h_val[sb + t] = acc[t];
        }
        for (int64_t p = a.D.rowptr[E] + lane; p < a.D.rowptr[E + 1]; p += 32) {
            const int sl = hsc_slot(tab, hs, a.D.col[p]);
            a.d_map[p] = sb + (sl >= 0 ? pos[sl] : 0);
        }
        __syncwarp();
    }
}

template <class T, int FORM>
static int launch_schur_num(edfa_handle_s* h, const SchurArgs<T>& a, const T* xr_val, int hs, cudaStream_t s)
{
    const size_t smem = num_warp_bytes<T, FORM>(hs) * kNumWarps;
    auto fn = k_schur_num<T, FORM>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return EDFA_ERR_BOUNDS;
    }
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kNumWarps * 32, smem);
    if (per < 1) return EDFA_ERR_BOUNDS;
    long long grid = (long long)per * h->nsm;
    const long long need = (a.Ne + kNumWarps - 1) / kNumWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    (edfa::count_launch(), fn<<<(unsigned)grid, kNumWarps * 32, smem, s>>>(a, xr_val, hs));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
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
    T* xr_val = nullptr;  // X~ values in row-major order, for the numeric pass only
    if (cudaMallocAsync((void**)&cursor, ((size_t)Nf + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&xr_val, (size_t)(h->x_tot > 0 ? h->x_tot : 1) * sizeof(T), s) != cudaSuccess)
        return EDFA_ERR_OOM;
    cudaMemcpyAsync(cursor, h->xr_ptr, ((size_t)Nf + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (Ne > 0)
        (edfa::count_launch(), k_q_fill_vals<T><<<(Ne + 255) / 256, 256, 0, s>>>(Ne, h->x_ptr, h->x_idx, xval, cursor,
                                                                               h->xr_cell, xr_val));
    if (Nf > 0)
        (edfa::count_launch(), k_row_sort_pairs<T><<<(Nf + 255) / 256, 256, 0, s>>>(h->xr_ptr, h->xr_cell, xr_val, Nf));
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
    // prefix sample of the rows with the counting pass (once per process for a
    // given precision, form and longest X~ set)
    int sw = 2;
    static std::mutex tune_mu;
    static std::vector<std::pair<long long, int>> tuned;
    const long long tkey = ((long long)sizeof(T) << 40) | ((long long)a.form << 32) | (long long)h->qmax;
    bool have = false;
    {
        std::lock_guard<std::mutex> lock(tune_mu);
        for (auto& kv : tuned)
            if (kv.first == tkey) { sw = kv.second; have = true; }
    }
    if (Ne >= 32768 && !have) {
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
                if (c == 1) (edfa::count_launch(), k_schur_count<T, 1><<<(unsigned)(h->nsm * 8), 32, 0, s>>>(sample));
                else (edfa::count_launch(), k_schur_count<T, 2><<<(unsigned)(h->nsm * 4), 64, 0, s>>>(sample));
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
        std::lock_guard<std::mutex> lock(tune_mu);
        tuned.push_back({tkey, sw});
    }
    h->stats.tuned_schur_warps = sw;
    int per = 0;
    if (sw == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_schur_count<T, 1>, 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_schur_count<T, 2>, 64, 0);
    if (per < 1) per = 1;
    long long grid = (long long)per * h->nsm;
    long long need = (Ne + sw - 1) / sw;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (sw == 1) (edfa::count_launch(), k_schur_count<T, 1><<<(unsigned)grid, 32, 0, s>>>(a));
    else (edfa::count_launch(), k_schur_count<T, 2><<<(unsigned)grid, 64, 0, s>>>(a));
    rc = scan_i64(h, h->s_ptr, Ne, s);
    if (rc) return rc;
    int64_t nnz = 0;
    int rmax = 0;
    cudaMemcpyAsync(&nnz, h->s_ptr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&rmax, rowmax, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(rowmax, s);
    rc = check_err(h, s);
    if (rc) { cudaFreeAsync(xr_val, s); return rc; }
    h->s_nnz = nnz;
    rc = dalloc_t(h, &h->s_col, (size_t)(nnz > 0 ? nnz : 1));
    if (!rc) rc = dalloc_t(h, h_val, (size_t)(nnz > 0 ? nnz : 1));
    if (!rc) rc = dalloc_t(h, &h->d_map, (size_t)(h->D.nnz > 0 ? h->D.nnz : 1));
    if (rc) return rc;
    a.s_ptr = h->s_ptr;
    a.s_col = h->s_col;
    a.h_val = *h_val;
    a.d_map = h->d_map;
    // numeric pass: hash capacity at least twice the longest row
    int hs = 64;
    while (hs < 2 * rmax) hs <<= 1;
    rc = a.form == 1 ? launch_schur_num<T, 1>(h, a, xr_val, hs, s) : launch_schur_num<T, 0>(h, a, xr_val, hs, s);
    cudaFreeAsync(xr_val, s);
    if (rc) return rc;
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
