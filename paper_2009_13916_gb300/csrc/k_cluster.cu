// Both S~ triangular solves of the preconditioner application (Eq. EDFA_prec,
// the Schur-complement block: w = L_S^{-1} r', z_p = U_S^{-1} w) in ONE
// launch of one 16-CTA thread-block cluster.
//
// Why: S~ has N_e rows and hundreds of dependency levels with only a few
// hundred rows each, so its sweeps are bound by the latency of passing values
// between levels.  Cross-SM polling through L2 costs ~1.5-2 us per level on
// GB300; a cluster barrier costs ~0.2 us, and a distributed-shared-memory read
// a fraction of a microsecond.  So the whole solution vector lives in the
// cluster's shared memory (16 x up to ~140 KB), each level ends with one
// cluster barrier, and the dependencies of a row are read straight from the
// shared memory of the CTA that owns them.
//
// Data layout (built once per S~ pattern, values refreshed after every
// numeric factorization):
//  * every forward level, sorted by row index, is cut into 16 contiguous
//    blocks; CTA r owns block r (its value slots follow in level order), and
//    the dependency encoding slot * 16 + owner locates a value anywhere in the
//    cluster;
//  * for every (phase, level, CTA) the rows that CTA computes are packed into
//    one or more self-contained chunks of at most kChunk bytes:
//       int4 header {nrows, nentries, 0, 0}
//       int4 rows[nrows]     {slot, count, first entry, 0}
//       T    dinv[nrows]     1/U_ii (backward phase; 1 in the forward phase)
//       int  dep[nentries]   forward-plan position t of each dependency
//       T    val[nentries]   L_ij (forward) or U_ij (backward)
//    every part padded to 16 bytes;
//  * each CTA's chunks are contiguous in processing order (forward levels,
//    then backward levels); a uint16 per chunk gives its size in 16-byte
//    units, bit 15 marking the last chunk of a level.
// The kernel streams a CTA's chunks through a ring of kRing shared-memory
// slots with cp.async.bulk (TMA) copies completing on mbarriers, issued
// kRing chunks ahead.  These copies run in the async proxy, so the release
// semantics of the cluster barrier do not wait for them, and after each
// barrier only shared-memory reads and the arithmetic remain on the critical
// path.  Both sweeps run in place: the forward result w_i stays in the owner's
// slot and the backward sweep overwrites it with z_i.
//
// Safety: every mbarrier wait is bounded (kSpinLimit polls, giving up early
// once any thread has recorded an error); a CTA whose initial copy timed out
// keeps taking part in every cluster barrier without touching data, so no
// CTA of the cluster can be left waiting; all dependency slots are bounds
// checked against the slot capacity before the remote read.
#include <cooperative_groups.h>

#include <climits>

#include "internal.cuh"

namespace edfa {

namespace cgx = cooperative_groups;

constexpr int kCl = 16;           // CTAs per cluster (non-portable cluster size)
constexpr int kClThreads = 512;   // 16 warps per CTA
constexpr int kRing = 4;          // staged chunks in flight per CTA
constexpr int kChunk = 16384;     // bytes per chunk slot
constexpr int kClLpr = 8;         // lanes per row

__host__ __device__ __forceinline__ int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }

template <class T>
__host__ __device__ __forceinline__ int64_t chunk_bytes(int64_t nr, int64_t ne)
{
    return 16 + 16 * nr + pad16(nr * (int64_t)sizeof(T)) + pad16(4 * ne) + pad16(ne * (int64_t)sizeof(T));
}

// ------------------------------------------------------------ plan build
__device__ __forceinline__ int level_of(const int64_t* loff, int nlev, int64_t t)
{
    int lo = 0, hi = nlev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (loff[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Owner blocks.  The rows of every forward level are sorted by index and
// cut into 16 contiguous blocks, CTA r taking block r: the level stays
// balanced over the cluster, and since the rows of neighbouring levels that
// a row depends on have nearby indices, most dependencies land in the same
// CTA (about 70% on 3-D brick workloads against 1/16 for a round-robin deal)
// and are read from local rather than distributed shared memory, whose
// request rate (~1.6 ns per scattered load per SM) bounds the sweep.
constexpr int kSortMax = 8192;  // longer levels keep their order (still balanced)

__global__ void __launch_bounds__(1024) k_cp_sort_levels(int32_t* __restrict__ perm, const int64_t* __restrict__ loff)
{
    __shared__ int32_t key[kSortMax];
    const int L = blockIdx.x;
    const int64_t b = loff[L];
    const int m = (int)(loff[L + 1] - b);
    if (m <= 1 || m > kSortMax) return;
    int P = 1;
    while (P < m) P <<= 1;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const int v = k < m ? perm[b + k] : -1;
        key[k] = v < 0 ? INT_MAX : v;
    }
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const bool up = (t & kk) == 0;
                    const int a = key[t], c = key[u];
                    if ((a > c) == up) {
                        key[t] = c;
                        key[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < m; k += blockDim.x) perm[b + k] = key[k] == INT_MAX ? -1 : key[k];
}

// rows of forward level L (its padding trails the rows) and the size of every
// CTA's block of it: cnt[r * nlf + L]
__global__ void k_cp_level_counts(int nlf, const int32_t* __restrict__ perm, const int64_t* __restrict__ loff,
                                  int32_t* __restrict__ cL, int64_t* __restrict__ cnt)
{
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nlf) return;
    int c = 0;
    for (int64_t p = loff[L]; p < loff[L + 1]; ++p) c += perm[p] >= 0;
    cL[L] = c;
    for (int r = 0; r < kCl; ++r)
        cnt[(int64_t)r * nlf + L] = ((int64_t)(r + 1) * c + kCl - 1) / kCl - ((int64_t)r * c + kCl - 1) / kCl;
}

// posf[i] = slot * 16 + owner for every row (G: exclusive scan of cnt)
__global__ void k_cp_assign(int64_t nsf, int nlf, const int32_t* __restrict__ perm, const int64_t* __restrict__ loff,
                            const int32_t* __restrict__ cL, const int64_t* __restrict__ G, int32_t* __restrict__ posf)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nsf) return;
    const int i = perm[t];
    if (i < 0) return;
    int lo = 0, hi = nlf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (loff[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int L = lo;
    const int64_t k = t - loff[L];
    const int64_t c = cL[L];
    const int r = (int)(k * kCl / c);
    const int64_t first = ((int64_t)r * c + kCl - 1) / kCl;
    const int64_t slot = (G[(int64_t)r * nlf + L] - G[(int64_t)r * nlf]) + (k - first);
    posf[i] = (int32_t)(slot * kCl + r);
}

__global__ void k_cp_totals(int nlf, const int64_t* __restrict__ G, int64_t* __restrict__ tot)
{
    const int r = threadIdx.x;
    if (r < kCl) tot[r] = G[(int64_t)(r + 1) * nlf] - G[(int64_t)r * nlf];
}

__global__ void k_cp_rowof(int32_t n, const int32_t* __restrict__ posf, int32_t cap, int32_t* __restrict__ rowof)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = posf[i];
    rowof[(int64_t)(p & (kCl - 1)) * cap + (p >> 4)] = (int32_t)i;
}

struct ListGeom {
    const int32_t *permf, *permb;
    const int64_t *loff_f, *loff_b;
    int64_t nsf, nsb;
    int nlf, nlb;
};

// list id of (phase, level, CTA): CTA-major so that the chunks of one CTA are
// contiguous in processing order
template <int FILL>
__global__ void k_cp_lists(ListGeom G, const int32_t* __restrict__ posf, unsigned long long* __restrict__ cnt,
                           int32_t* __restrict__ lrows)
{
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= G.nsf + G.nsb) return;
    const int bwd = u >= G.nsf;
    const int64_t t = bwd ? u - G.nsf : u;
    const int i = bwd ? G.permb[t] : G.permf[t];
    if (i < 0) return;
    const int L = bwd ? level_of(G.loff_b, G.nlb, t) : level_of(G.loff_f, G.nlf, t);
    const int r = posf[i] & (kCl - 1);
    const int64_t list = (int64_t)r * (G.nlf + G.nlb) + (bwd ? G.nlf + L : L);
    if (FILL) {
        const unsigned long long pos = atomicAdd(&cnt[list], 1ull);
        lrows[pos] = i;
    } else {
        atomicAdd(&cnt[list], 1ull);
    }
}

__device__ __forceinline__ int64_t row_lo(int bwd, int i, const int64_t* rowptr, const int64_t* diag)
{
    return bwd ? diag[i] + 1 : rowptr[i];
}
__device__ __forceinline__ int64_t row_hi(int bwd, int i, const int64_t* rowptr, const int64_t* diag)
{
    return bwd ? rowptr[i + 1] : diag[i];
}

// greedy chunking of list rows [p, pend): returns the end q of the chunk
// starting at p and its row / entry counts (a single row always fits)
template <class T>
__device__ __forceinline__ int64_t next_chunk(int64_t p, int64_t pend, int bwd, const int32_t* lrows,
                                              const int64_t* rowptr, const int64_t* diag, int64_t& nr, int64_t& ne)
{
    nr = 0;
    ne = 0;
    int64_t q = p;
    while (q < pend) {
        const int i = lrows[q];
        const int64_t c = row_hi(bwd, i, rowptr, diag) - row_lo(bwd, i, rowptr, diag);
        if (nr > 0 && chunk_bytes<T>(nr + 1, ne + c) > kChunk) break;
        ++nr;
        ne += c;
        ++q;
    }
    return q;
}

template <class T>
__global__ void k_cp_size(int64_t nlists, int nlt, int nlf, const int64_t* __restrict__ lofs,
                          const int32_t* __restrict__ lrows, const int64_t* __restrict__ rowptr,
                          const int64_t* __restrict__ diag, int64_t* __restrict__ lbyte, int64_t* __restrict__ lchunk,
                          int* __restrict__ bad)
{
    const int64_t list = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (list >= nlists) return;
    const int bwd = (int)(list % nlt) >= nlf;
    const int64_t pend = lofs[list + 1];
    int64_t p = lofs[list], bytes = 0, nch = 0;
    do {
        int64_t nr, ne;
        const int64_t q = next_chunk<T>(p, pend, bwd, lrows, rowptr, diag, nr, ne);
        const int64_t b = chunk_bytes<T>(nr, ne);
        if (b > kChunk) atomicExch(bad, 1);  // a row longer than one chunk slot
        bytes += b;
        ++nch;
        p = q;
    } while (p < pend);
    lbyte[list] = bytes;
    lchunk[list] = nch;
}

__global__ void k_cp_meta(int nlt, const int64_t* __restrict__ lbyte, const int64_t* __restrict__ lchunk,
                          int64_t* __restrict__ meta)
{
    const int r = threadIdx.x;
    if (r >= kCl) return;
    const int64_t c0 = lchunk[(int64_t)r * nlt];
    meta[2 * r] = lbyte[(int64_t)r * nlt];
    meta[2 * r + 1] = lchunk[(int64_t)(r + 1) * nlt] - c0;
}

template <class T>
__global__ void k_cp_write(int64_t nlists, int nlt, int nlf, const int64_t* __restrict__ lofs,
                           const int32_t* __restrict__ lrows, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const int64_t* __restrict__ diag, const T* __restrict__ lu,
                           const T* __restrict__ dinv, const int32_t* __restrict__ posf,
                           const int64_t* __restrict__ lbyte, const int64_t* __restrict__ lchunk,
                           unsigned char* __restrict__ chunks, uint16_t* __restrict__ sz, int32_t szstride)
{
    const int64_t list = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (list >= nlists) return;
    const int bwd = (int)(list % nlt) >= nlf;
    const int64_t r = list / nlt;
    int64_t cl = lchunk[list] - lchunk[r * nlt];
    unsigned char* base = chunks + lbyte[list];
    const int64_t pend = lofs[list + 1];
    int64_t p = lofs[list];
    do {
        int64_t nr, ne;
        const int64_t q = next_chunk<T>(p, pend, bwd, lrows, rowptr, diag, nr, ne);
        const int64_t cb = chunk_bytes<T>(nr, ne);
        *(int4*)base = make_int4((int)nr, (int)ne, 0, 0);
        int4* rec = (int4*)(base + 16);
        T* dv = (T*)(base + 16 + 16 * nr);
        int32_t* dep = (int32_t*)(base + 16 + 16 * nr + pad16(nr * (int64_t)sizeof(T)));
        T* val = (T*)((unsigned char*)dep + pad16(4 * ne));
        int e = 0;
        for (int64_t k = 0; k < nr; ++k) {
            const int i = lrows[p + k];
            const int64_t lo = row_lo(bwd, i, rowptr, diag), hi = row_hi(bwd, i, rowptr, diag);
            rec[k] = make_int4(posf[i] >> 4, (int)(hi - lo), e, 0);
            dv[k] = bwd ? dinv[i] : T(1);
            for (int64_t pp = lo; pp < hi; ++pp, ++e) {
                dep[e] = posf[col[pp]];
                val[e] = lu[pp];
            }
        }
        p = q;
        sz[r * szstride + cl] = (uint16_t)((cb >> 4) | (p >= pend ? 0x8000 : 0));
        ++cl;
        base += cb;
    } while (p < pend);
}

// right-hand side of the forward S~ sweep in slot order:
// bslot[owner * cap + slot] = base_i - (M v)_i   (M v omitted when mptr is null)
template <class T, class TB>
__global__ void k_cp_rhs(int32_t n, const int32_t* __restrict__ posf, int32_t cap, const TB* __restrict__ base,
                         const int64_t* __restrict__ mptr, const int32_t* __restrict__ mcol, const T* __restrict__ mval,
                         const T* __restrict__ mv, T* __restrict__ bslot)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc = T(0), a2 = T(0);
    if (mptr) {
        int64_t p = mptr[i];
        const int64_t e = mptr[i + 1];
        for (; p + 1 < e; p += 2) {
            acc = fma(mval[p], mv[mcol[p]], acc);
            a2 = fma(mval[p + 1], mv[mcol[p + 1]], a2);
        }
        if (p < e) acc = fma(mval[p], mv[mcol[p]], acc);
    }
    const int q = posf[i];
    bslot[(int64_t)(q & (kCl - 1)) * cap + (q >> 4)] = (T)base[i] - (acc + a2);
}

// ------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; gives up early once any
// thread has recorded an error
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const DevErr* err)
{
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && err_set(err)) return false;
    }
    return false;
}

// ------------------------------------------------------------ the sweep kernel
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// load of a value in the shared memory of CTA `rank` of the cluster
__device__ __forceinline__ double ld_dsmem(uint32_t addr, uint32_t rank, double)
{
    double v;
    asm volatile(
        "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %1, %2;\n\tld.shared::cluster.f64 %0, [ra];\n\t}"
        : "=d"(v)
        : "r"(addr), "r"(rank));
    return v;
}
__device__ __forceinline__ float ld_dsmem(uint32_t addr, uint32_t rank, float)
{
    float v;
    asm volatile(
        "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %1, %2;\n\tld.shared::cluster.f32 %0, [ra];\n\t}"
        : "=f"(v)
        : "r"(addr), "r"(rank));
    return v;
}

// The first KMAX x LPR dependencies of one row, staged in registers before
// the cluster barrier that releases them.
template <class T, int KMAX>
struct RowRegs {
    int k;       // row within the chunk, -1 when this lane group has none
    int sl;      // value slot of the row
    int cnt, eo; // dependency count and first entry
    T dv;
    int t[KMAX];
    T v[KMAX];
};

template <class T, int LPR, int KMAX>
__device__ __forceinline__ void stage_row(RowRegs<T, KMAX>& R, const unsigned char* ck, int nr, int ne, int k, int gl,
                                          int cap, DevErr* err)
{
    R.k = -1;
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        R.t[q] = -1;
        R.v[q] = T(0);
    }
    if (k >= nr) return;
    const int4 rr = ((const int4*)(ck + 16))[k];
    if (rr.x < 0 || rr.x >= cap || rr.y < 0 || rr.z < 0 || rr.z + rr.y > ne) {
        raise_err(err, EDFA_ERR_BOUNDS, k);
        return;
    }
    R.k = k;
    R.sl = rr.x;
    R.cnt = rr.y;
    R.eo = rr.z;
    R.dv = ((const T*)(ck + 16 + 16 * nr))[k];
    const int32_t* dep = (const int32_t*)(ck + 16 + 16 * nr + pad16((int64_t)nr * sizeof(T)));
    const T* val = (const T*)((const unsigned char*)dep + pad16(4 * (int64_t)ne));
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int p = gl + q * LPR;
        if (p < R.cnt) {
            R.t[q] = dep[R.eo + p];
            R.v[q] = val[R.eo + p];
        }
    }
}

// finish a staged row: remote reads (all issued before the first use), the
// tail of rows longer than KMAX x LPR, the lane-group reduction, the update
template <class T>
__device__ __forceinline__ T ld_value(const T* xs, uint32_t xs_s, int t, int cap, int rank)
{
    const int sl = t >> 4, r = t & (kCl - 1);
    if ((unsigned)sl >= (unsigned)cap) return T(0);
    if (r == rank) return xs[sl];
    return ld_dsmem(xs_s + (uint32_t)(sl * (int)sizeof(T)), (uint32_t)r, T(0));
}

template <class T, int LPR, int KMAX>
__device__ __forceinline__ void finish_row(const RowRegs<T, KMAX>& R, const unsigned char* ck, int nr, int ne, T* xs,
                                           int cap, bool bwd, int gl, int rank)
{
    const uint32_t xs_s = smem_u32(xs);
    T x[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) x[q] = ld_value(xs, xs_s, R.t[q], cap, rank);
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < KMAX; ++q) acc = fma(R.v[q], x[q], acc);
    if (R.k >= 0 && R.cnt > KMAX * LPR) {
        const int32_t* dep = (const int32_t*)(ck + 16 + 16 * nr + pad16((int64_t)nr * sizeof(T)));
        const T* val = (const T*)((const unsigned char*)dep + pad16(4 * (int64_t)ne));
        for (int p = gl + KMAX * LPR; p < R.cnt; p += LPR) {
            acc = fma(val[R.eo + p], ld_value(xs, xs_s, dep[R.eo + p], cap, rank), acc);
        }
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (R.k >= 0 && gl == 0) {
        T y = xs[R.sl] - acc;
        if (bwd) y *= R.dv;
        xs[R.sl] = y;
    }
}

template <class T, class TO, int LPR>
__global__ void __launch_bounds__(kClThreads, 1)
k_s_cluster(const T* __restrict__ bslot, const unsigned char* __restrict__ chunks, const uint16_t* __restrict__ sz,
            const int64_t* __restrict__ meta, int32_t szstride, int32_t cap, int nlf, int nlb,
            const int32_t* __restrict__ rowof, TO* __restrict__ out, DevErr* err)
{
    constexpr int KMAX = 32 / LPR;
    constexpr int RPW = 32 / LPR;
    constexpr int NW = kClThreads / 32;
    extern __shared__ __align__(128) unsigned char sm[];
    const int rank = (int)cgx::this_cluster().block_rank();
    T* xs = (T*)sm;
    unsigned char* ring = sm + pad16((int64_t)cap * sizeof(T));
    uint16_t* szt = (uint16_t*)(ring + kRing * kChunk);
    uint64_t* bar = (uint64_t*)((unsigned char*)szt + pad16((int64_t)szstride * 2));
    const int64_t byte0 = meta[2 * rank];
    int nch = (int)meta[2 * rank + 1];
    if (nch > szstride) nch = szstride;
    // the TMA producer is lane 0 of the last warp, which holds rows only in
    // levels with more than (NW - 1) x RPW rows on this CTA
    const bool prod = threadIdx.x == kClThreads - 32;
    if (prod) {
        for (int k = 0; k <= kRing; ++k) mbar_init(smem_u32(bar + k), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (prod) {
        const uint32_t xsb = (uint32_t)((int64_t)cap * sizeof(T));
        const uint32_t szb = (uint32_t)pad16((int64_t)nch * 2);
        mbar_expect_tx(smem_u32(bar + kRing), xsb + szb);
        bulk_g2s(smem_u32(xs), bslot + (int64_t)rank * cap, xsb, smem_u32(bar + kRing));
        bulk_g2s(smem_u32(szt), sz + (int64_t)rank * szstride, szb, smem_u32(bar + kRing));
    }
    const bool ok0 = mbar_wait(smem_u32(bar + kRing), 0, err);
    const int dead = __syncthreads_or(!ok0);
    if (dead && prod) raise_err(err, EDFA_ERR_TIMEOUT, -1);

    // producer state: chunks issued so far and the next source byte
    int issued = 0;
    int64_t pbyte = byte0;
    bool pstop = dead != 0;
    auto issue = [&](int consumed) {
        while (!pstop && issued < nch && issued < consumed + kRing) {
            const uint32_t b = (uint32_t)(szt[issued] & 0x7fff) * 16u;
            if (b < 16u || b > (uint32_t)kChunk) {
                raise_err(err, EDFA_ERR_BOUNDS, issued);
                pstop = true;
                break;
            }
            const int slot = issued % kRing;
            mbar_expect_tx(smem_u32(bar + slot), b);
            bulk_g2s(smem_u32(ring + slot * kChunk), chunks + pbyte, b, smem_u32(bar + slot));
            pbyte += b;
            ++issued;
        }
    };

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane / LPR, gl = lane % LPR;
    const int kfirst = wid * RPW + g;  // this lane group's row in the first pass over a chunk
    // staging of chunk c: wait for its copy, read its header, stage the first-pass row
    int c = 0;
    int cnr = 0, cne = 0;
    bool cok = false;
    RowRegs<T, KMAX> R;
    auto stage = [&](int cc) {
        cok = false;
        cnr = cne = 0;
        R.k = -1;
        if (dead || cc >= nch) return;
        const bool got = mbar_wait(smem_u32(bar + cc % kRing), (uint32_t)((cc / kRing) & 1), err);
        if (!got) {
            raise_err(err, EDFA_ERR_TIMEOUT, cc);
            if (prod) pstop = true;
            return;
        }
        const unsigned char* ck = ring + (cc % kRing) * kChunk;
        const int4 hd = *(const int4*)ck;
        if (hd.x < 0 || hd.y < 0 || chunk_bytes<T>(hd.x, hd.y) > kChunk) {
            raise_err(err, EDFA_ERR_BOUNDS, cc);
            return;
        }
        cnr = hd.x;
        cne = hd.y;
        cok = true;
        stage_row<T, LPR, KMAX>(R, ck, cnr, cne, kfirst, gl, cap, err);
    };

    // a lane group's staged row is used only if its whole warp staged the chunk
    // (keeps the shuffles of the reduction convergent after a timed-out wait)
    auto stage_all = [&](int cc) {
        stage(cc);
        cok = __all_sync(0xffffffffu, cok);
    };
    if (prod) issue(0);
    stage_all(0);
    cluster_arrive();  // every CTA runs and holds its right-hand side before any remote read
    cluster_wait();

    const int nlev = nlf + nlb;
    for (int L = 0; L < nlev; ++L) {
        const bool bwd = L >= nlf;
        if (!dead) {
            for (;;) {
                if (c >= nch) {
                    if (prod) raise_err(err, EDFA_ERR_BOUNDS, c);
                    break;
                }
                const bool last = (szt[c] & 0x8000) != 0;
                // warps without a row skip the arithmetic: FP64 issue slots are
                // scarce on this part and shared by all warps of the SM
                if (cok && wid * RPW < cnr) {
                    const unsigned char* ck = ring + (c % kRing) * kChunk;
                    finish_row<T, LPR, KMAX>(R, ck, cnr, cne, xs, cap, bwd, gl, rank);
                    // further passes over chunks with more rows than lane groups
                    for (int k0 = wid * RPW + NW * RPW; k0 < cnr; k0 += NW * RPW) {
                        RowRegs<T, KMAX> Q;
                        stage_row<T, LPR, KMAX>(Q, ck, cnr, cne, k0 + g, gl, cap, err);
                        finish_row<T, LPR, KMAX>(Q, ck, cnr, cne, xs, cap, bwd, gl, rank);
                    }
                }
                ++c;
                if (last) break;
                __syncthreads();  // chunk c-1 read by every warp: its slot may be refilled
                if (prod) issue(c);
                stage_all(c);
            }
        }
        cluster_arrive();
        if (L + 1 < nlev) stage_all(c);  // overlaps the barrier
        cluster_wait();
        if (prod) issue(c);
    }
    // copies still in flight can only follow an error: wait (bounded) for them
    // before the CTA's shared memory is released
    if (prod) {
        for (int q = issued - kRing < 0 ? 0 : issued - kRing; q < issued; ++q)
            mbar_wait(smem_u32(bar + q % kRing), (uint32_t)((q / kRing) & 1), err);
    }
    for (int sl = threadIdx.x; sl < cap; sl += blockDim.x) {
        const int i = rowof[(int64_t)rank * cap + sl];
        if (i >= 0) out[i] = (TO)xs[sl];
    }
}

// ------------------------------------------------------------ dataflow variant
// The same two sweeps without a barrier per level: every row polls the values
// it depends on directly in the distributed shared memory (a slot holds the
// all-ones NaN until its row is done; no arithmetic produces that pattern),
// so a level costs one value hop instead of a cluster barrier plus the skew
// of the slowest CTA.  Rows are claimed in level order through a per-CTA
// ticket, a warp's rows always of one level (every (CTA, phase, level) list is
// padded to whole warps), so no row waits on a row of its own warp; claiming
// in level order keeps it deadlock free: the in-flight row of smallest
// (phase, level) has all its dependencies done.  Between the phases one
// cluster-wide step moves every w_i into its backward record and resets the
// slots to the sentinel.
//
// Per row, LPR lanes share the dependencies, which the record lists in
// ascending dependency level (oldest first).  Each lane consumes its
// dependencies strictly in that order as they become ready, accumulating
// r_i - sum l_ij x_j as it goes, so when the last (newest) dependency
// arrives only one FMA, log2(LPR) shuffle-adds and the 1/U_ii product remain:
// on GB300 every FP64 warp instruction occupies its SM sub-partition for
// ~33 ns, so the work left after the critical dependency, not the dot
// product as a whole, sets the time per level.  Lanes with several pending
// dependencies back off between polls; a lane waiting on its last one spins.
//
// Row record (kDfDeps dependencies inline, older ones in an overflow array):
//   0: int slot, int count, int64 overflow offset
//  16: T aux (forward: right-hand side; backward: w_i / U_ii), 24: T 1/U_ii
//  (backward values are stored as U_ij / U_ii)
//  32: int dep[kDfDeps] (slot * 16 + owner)
// 160: T val[kDfDeps]
// A padding record has slot -1 and no dependencies.
constexpr int kDfDeps = 32;

template <class T>
__host__ __device__ constexpr int df_rb()
{
    return 160 + kDfDeps * (int)sizeof(T);
}

__device__ __forceinline__ bool df_sent(double v) { return __double_as_longlong(v) == -1ll; }
__device__ __forceinline__ bool df_sent(float v) { return __float_as_int(v) == -1; }
template <class T>
__device__ __forceinline__ T df_sentinel();
template <>
__device__ __forceinline__ double df_sentinel<double>() { return __longlong_as_double(-1ll); }
template <>
__device__ __forceinline__ float df_sentinel<float>() { return __int_as_float(-1); }

__device__ __forceinline__ double df_ld_local(uint32_t a, double)
{
    double v;
    asm volatile("ld.volatile.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float df_ld_local(uint32_t a, float)
{
    float v;
    asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double df_ld_remote(uint32_t a, uint32_t rank, double)
{
    double v;
    asm volatile(
        "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %1, %2;\n\tld.relaxed.cluster.shared::cluster.f64 %0, [ra];\n\t}"
        : "=d"(v)
        : "r"(a), "r"(rank));
    return v;
}
__device__ __forceinline__ float df_ld_remote(uint32_t a, uint32_t rank, float)
{
    float v;
    asm volatile(
        "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %1, %2;\n\tld.relaxed.cluster.shared::cluster.f32 %0, [ra];\n\t}"
        : "=f"(v)
        : "r"(a), "r"(rank));
    return v;
}
__device__ __forceinline__ void df_st(uint32_t a, double v)
{
    asm volatile("st.relaxed.cluster.shared::cta.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void df_st(uint32_t a, float v)
{
    asm volatile("st.relaxed.cluster.shared::cta.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// value of dependency t (slot * 16 + owner), or the sentinel while not ready
template <class T>
__device__ __forceinline__ T df_value(uint32_t xs_s, int t, int rank)
{
    const uint32_t a = xs_s + (uint32_t)((t >> 4) * (int)sizeof(T));
    const int r = t & (kCl - 1);
    return r == rank ? df_ld_local(a, T(0)) : df_ld_remote(a, (uint32_t)r, T(0));
}

template <class T, int LPR, int SLEEP>
__device__ __forceinline__ void df_row(const unsigned char* __restrict__ rc, uint32_t xs_s, int cap, int rank,
                                       bool bwd, int gl, unsigned gmask, const int32_t* __restrict__ ovf_dep,
                                       const T* __restrict__ ovf_val, DevErr* err)
{
    constexpr int KMAX = kDfDeps / LPR;
    const int4 hd = *(const int4*)rc;
    const int slot = hd.x, cnt = hd.y;
    if ((unsigned)slot >= (unsigned)cap) return;  // padding record (whole lane group)
    const long long ovf = (long long)(((unsigned long long)(unsigned)hd.w << 32) | (unsigned)hd.z);
    const T aux = *(const T*)(rc + 16);
    const T dv = *(const T*)(rc + 24);
    const int32_t* dep = (const int32_t*)(rc + 32);
    const T* val = (const T*)(rc + 160);
    const int nin = cnt < kDfDeps ? cnt : kDfDeps;
    // this lane's inline dependencies, oldest first: positions gl, gl + LPR, ...
    int t[KMAX];
    T v[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        const int p = gl + q * LPR;
        const bool on = p < nin;
        t[q] = on ? dep[p] : 0;
        v[q] = on ? val[p] : T(0);
        if (on && (unsigned)(t[q] >> 4) >= (unsigned)cap) {
            raise_err(err, EDFA_ERR_BOUNDS, slot);
            v[q] = T(0);
            t[q] = 0;
        }
    }
    const int mine = nin > gl ? (nin - gl + LPR - 1) / LPR : 0;
    T acc = gl == 0 ? aux : T(0);
    // overflow dependencies (the oldest of long rows) first, one at a time
    for (int p = kDfDeps + gl; p < cnt; p += LPR) {
        const int tt = ovf_dep[ovf + p - kDfDeps];
        const T vv = ovf_val[ovf + p - kDfDeps];
        if ((unsigned)(tt >> 4) >= (unsigned)cap) {
            raise_err(err, EDFA_ERR_BOUNDS, slot);
            continue;
        }
        T y = df_value<T>(xs_s, tt, rank);
        for (unsigned it = 0; df_sent(y) && it < kSpinLimit; ++it) {
            if ((it & 255u) == 255u && err_set(err)) break;
            if (SLEEP > 0) __nanosleep(SLEEP);
            y = df_value<T>(xs_s, tt, rank);
        }
        if (!df_sent(y)) acc = fma(-vv, y, acc);
    }
    // inline dependencies: one batch of polls, then consumed strictly in order;
    // a dependency still pending is re-polled alone (the group votes, so rows of
    // other lane groups in the warp go on independently)
    T x[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX; ++q) x[q] = q < mine ? df_value<T>(xs_s, t[q], rank) : T(0);
    bool live = true;
#pragma unroll
    for (int q = 0; q < KMAX; ++q) {
        if (q * LPR >= nin) break;  // uniform over the group
        for (unsigned it = 0; __any_sync(gmask, q < mine && df_sent(x[q])); ++it) {
            // give up together (the decision is voted, so the group stays converged)
            if (__any_sync(gmask, it >= kSpinLimit || ((it & 255u) == 255u && err_set(err)))) {
                if (it >= kSpinLimit && gl == 0) raise_err(err, EDFA_ERR_TIMEOUT, slot);
                live = false;
                break;
            }
            // the last dependency spins; earlier ones leave the request slots of
            // the distributed shared memory to the rows on the critical path
            if (SLEEP > 0 && q + 1 < mine) __nanosleep(SLEEP);
            // refresh every dependency still pending from q on, so that the
            // later ones are known by the time q arrives
#pragma unroll
            for (int qq = q; qq < KMAX; ++qq)
                if (qq < mine && df_sent(x[qq])) x[qq] = df_value<T>(xs_s, t[qq], rank);
        }
        if (!live) break;
        if (q < mine) acc = fma(-v[q], x[q], acc);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o);
    // backward rows: the record holds U_ij / U_ii and the scaled w_i / U_ii,
    // so no product remains after the last dependency
    (void)dv;
    if (gl == 0) df_st(xs_s + (uint32_t)(slot * (int)sizeof(T)), acc);
}

template <class T, class TO, int LPR, int THREADS, int SLEEP>
__global__ void __launch_bounds__(THREADS, 1)
k_s_df(unsigned char* __restrict__ rec, const int64_t* __restrict__ rmeta, int32_t cap,
       const int32_t* __restrict__ ovf_dep, const T* __restrict__ ovf_val, const int64_t* __restrict__ bidx,
       const int32_t* __restrict__ rowof, TO* __restrict__ out, DevErr* err)
{
    constexpr int RPW = 32 / LPR;
    constexpr int RB = df_rb<T>();
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ int ticket[2];
    T* xs = (T*)sm;
    const uint32_t xs_s = smem_u32(xs);
    const int rank = (int)cgx::this_cluster().block_rank();
    for (int sl = threadIdx.x; sl < cap; sl += blockDim.x) xs[sl] = df_sentinel<T>();
    if (threadIdx.x < 2) ticket[threadIdx.x] = 0;
    cluster_arrive();  // every slot of the cluster holds the sentinel before any poll
    cluster_wait();
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, gl = lane % LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (g * LPR));
    for (int ph = 0; ph < 2; ++ph) {
        const int64_t pbase = rmeta[4 * rank + 2 * ph], nr = rmeta[4 * rank + 2 * ph + 1];
        for (;;) {
            int k0 = 0;
            if (lane == 0) k0 = atomicAdd(&ticket[ph], RPW);
            k0 = __shfl_sync(0xffffffffu, k0, 0);
            if (k0 >= nr) break;
            const int k = k0 + g;
            if (k < nr)
                df_row<T, LPR, SLEEP>(rec + (pbase + k) * RB, xs_s, cap, rank, ph == 1, gl, gmask, ovf_dep, ovf_val,
                                      err);
            __syncwarp();
        }
        cluster_arrive();  // every row of this phase is done in the whole cluster
        cluster_wait();
        if (ph == 0) {
            // w_i into the backward records, then every slot back to the sentinel
            for (int sl = threadIdx.x; sl < cap; sl += blockDim.x) {
                const int64_t p = bidx[(int64_t)rank * cap + sl];
                if (p >= 0) *(T*)(rec + p * RB + 16) = xs[sl] * *(const T*)(rec + p * RB + 24);
            }
            __syncthreads();
            for (int sl = threadIdx.x; sl < cap; sl += blockDim.x) xs[sl] = df_sentinel<T>();
            cluster_arrive();
            cluster_wait();
        }
    }
    for (int sl = threadIdx.x; sl < cap; sl += blockDim.x) {
        const int i = rowof[(int64_t)rank * cap + sl];
        if (i >= 0) out[i] = (TO)xs[sl];
    }
}

// ---- dataflow plan: dependency levels, record indices, overflow, records
// lvl[off + i] = level of row i in a sweep plan (perm, loff)
__global__ void k_df_levels(int64_t nslots, int nlev, const int32_t* __restrict__ perm,
                            const int64_t* __restrict__ loff, int32_t* __restrict__ lvl)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nslots) return;
    const int i = perm[t];
    if (i >= 0) lvl[i] = level_of(loff, nlev, t);
}

__global__ void k_df_idx(int64_t nrec, int nlt, int nlf, const int64_t* __restrict__ lofs,
                         const int32_t* __restrict__ lrows, const int32_t* __restrict__ posf, int32_t cap,
                         int64_t* __restrict__ fidx, int64_t* __restrict__ bidx)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrec) return;
    const int i = lrows[p];
    if (i < 0) return;
    const int q = posf[i];
    const int r = q & (kCl - 1);
    if (p < lofs[(int64_t)r * nlt + nlf]) fidx[i] = p;
    else bidx[(int64_t)r * cap + (q >> 4)] = p;
}

__global__ void k_df_ovf_count(int64_t nrec, int nlt, int nlf, const int64_t* __restrict__ lofs,
                               const int32_t* __restrict__ lrows, const int32_t* __restrict__ posf,
                               const int64_t* __restrict__ rowptr, const int64_t* __restrict__ diag,
                               int64_t* __restrict__ ovc)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrec) return;
    const int i = lrows[p];
    if (i < 0) {
        ovc[p] = 0;
        return;
    }
    const int r = posf[i] & (kCl - 1);
    const int bwd = p >= lofs[(int64_t)r * nlt + nlf];
    const int64_t c = row_hi(bwd, i, rowptr, diag) - row_lo(bwd, i, rowptr, diag);
    ovc[p] = c > kDfDeps ? c - kDfDeps : 0;
}

__global__ void k_df_rmeta(int nlt, int nlf, const int64_t* __restrict__ lofs, int64_t* __restrict__ rmeta)
{
    const int r = threadIdx.x;
    if (r >= kCl) return;
    const int64_t a = lofs[(int64_t)r * nlt], b = lofs[(int64_t)r * nlt + nlf], c = lofs[(int64_t)(r + 1) * nlt];
    rmeta[4 * r] = a;
    rmeta[4 * r + 1] = b - a;
    rmeta[4 * r + 2] = b;
    rmeta[4 * r + 3] = c - b;
}

// Records of one numeric factor.  The dependencies of a row are ordered by
// their level in the sweep (ascending, ties by column), the oldest of a long
// row (beyond kDfDeps) in the overflow array; rows longer than kDfSortMax keep
// column order.
constexpr int kDfSortMax = 64;

template <class T>
__global__ void k_df_write(int64_t nrec, int nlt, int nlf, int32_t n, const int64_t* __restrict__ lofs,
                           const int32_t* __restrict__ lrows, const int32_t* __restrict__ posf,
                           const int32_t* __restrict__ lvl, const int64_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const int64_t* __restrict__ diag, const T* __restrict__ lu,
                           const T* __restrict__ dinv, const int64_t* __restrict__ ovoff, unsigned char* __restrict__ rec,
                           int32_t* __restrict__ ovf_dep, T* __restrict__ ovf_val)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nrec) return;
    const int i = lrows[p];
    unsigned char* rc = rec + p * df_rb<T>();
    if (i < 0) {
        *(int4*)rc = make_int4(-1, 0, 0, 0);
        return;
    }
    const int q = posf[i];
    const int r = q & (kCl - 1);
    const int bwd = p >= lofs[(int64_t)r * nlt + nlf];
    const int64_t lo = row_lo(bwd, i, rowptr, diag), hi = row_hi(bwd, i, rowptr, diag);
    const int cnt = (int)(hi - lo);
    const long long ov = ovoff[p];
    *(int4*)rc = make_int4(q >> 4, cnt, (int)(unsigned)(ov & 0xffffffffll), (int)(ov >> 32));
    *(T*)(rc + 24) = bwd ? dinv[i] : T(1);
    int32_t* dep = (int32_t*)(rc + 32);
    T* val = (T*)(rc + 160);
    const int nov = cnt > kDfDeps ? cnt - kDfDeps : 0;
    // order: by level of the dependency, then by column (insertion sort of
    // entry offsets); output position u < nov goes to the overflow array
    unsigned char ord[kDfSortMax];
    const bool sorted = cnt <= kDfSortMax;
    if (sorted) {
        const int32_t* lv = lvl + (bwd ? n : 0);
        for (int k = 0; k < cnt; ++k) {
            const int key = lv[col[lo + k]];
            int u = k;
            while (u > 0 && lv[col[lo + ord[u - 1]]] > key) {
                ord[u] = ord[u - 1];
                --u;
            }
            ord[u] = (unsigned char)k;
        }
    }
    for (int u = 0; u < cnt; ++u) {
        const int k = sorted ? ord[u] : (u < nov ? kDfDeps + u : u - nov);
        const int d = posf[col[lo + k]];
        const T w = bwd ? lu[lo + k] * dinv[i] : lu[lo + k];
        if (u < nov) {
            ovf_dep[ov + u] = d;
            ovf_val[ov + u] = w;
        } else {
            dep[u - nov] = d;
            val[u - nov] = w;
        }
    }
}

// forward right-hand side into the forward records: aux_i = base_i - (M v)_i,
// four consecutive lanes per row (coalesced runs of the row of M)
template <class T, class TB>
__global__ void k_df_rhs(int32_t n, const int64_t* __restrict__ fidx, unsigned char* __restrict__ rec,
                         const TB* __restrict__ base, const int64_t* __restrict__ mptr,
                         const int32_t* __restrict__ mcol, const T* __restrict__ mval, const T* __restrict__ mv)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t >> 2;
    const int gl = (int)(t & 3);
    T acc = T(0);
    if (mptr && i < n)
        for (int64_t p = mptr[i] + gl; p < mptr[i + 1]; p += 4) acc = fma(mval[p], mv[mcol[p]], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (gl == 0 && i < n) *(T*)(rec + fidx[i] * df_rb<T>() + 16) = (T)base[i] - acc;
}

// ------------------------------------------------------------ host side
// launch shape of the dataflow kernel: 16 lanes per row (two rows per warp),
// 1024 threads per CTA, no back-off between polls.  Measured on the 64^3
// workload (FP64 / FP32 ms for both sweeps): 16 lanes 1.59 / 1.30, 8 lanes
// 1.73 / 1.43, 32 lanes 2.38 / 1.49, 4 lanes 3.04 / 2.64; 512 threads per CTA
// and 32-64 ns back-off were slower in every shape.
constexpr int kDfLpr = 16;
constexpr int kDfThreads = 1024;
constexpr int kDfSleep = 0;

static cudaLaunchConfig_t cluster_cfg(size_t smem, int threads, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// can one 16-CTA cluster of this kernel with this much shared memory per CTA
// be scheduled?  (sets the kernel's cluster and shared-memory attributes)
static bool cluster_schedulable(const void* fn, int threads, size_t smem)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the attribute is an upper bound shared by every handle: set it to the
    // device maximum less the kernel's static shared memory
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if ((int64_t)smem > dyn_max ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_cfg(smem, threads, nullptr, attr);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return ncl > 0;
}

// owner blocks, value slots and the per-(phase, level, CTA) row lists shared
// by both cluster variants; returns the slot capacity (0: does not fit)
// round the row count of every (CTA, phase, level) list up to a multiple of
// pad (padding rows are -1 at the end of the list)
__global__ void k_cp_pad_lists(int64_t nlists, int64_t* __restrict__ cnt, int pad)
{
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l < nlists) cnt[l] = (cnt[l] + pad - 1) / pad * pad;
}

template <class T>
static int plan_common(edfa_handle_s* h, int64_t min_extra_smem, int32_t* cap_out, cudaStream_t s, int pad = 1)
{
    ClusterPlan& cp = h->cp;
    Factor& f = h->fs;
    const int64_t nsf = f.fwd.nslots, nsb = f.bwd.nslots;
    const int nlf = f.fwd.nlevels, nlb = f.bwd.nlevels, nlt = nlf + nlb;
    *cap_out = 0;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    // quick reject before any work: the values alone must fit
    if (pad16(((int64_t)f.n + kCl - 1) / kCl * sizeof(T)) + min_extra_smem > optin) return EDFA_OK;

    // owner blocks: sort every forward level by row index (the order of rows
    // within a level is free for the sweeps), then deal index blocks
    if (nlf > 0) (edfa::count_launch(), k_cp_sort_levels<<<nlf, 1024, 0, s>>>(f.fwd.perm, f.fwd.loff));
    int rc = dalloc_t(h, &cp.posf, (size_t)f.n);
    if (rc) return rc;
    int32_t* cL = nullptr;
    int64_t *G = nullptr, *tot = nullptr;
    if (cudaMallocAsync((void**)&cL, (size_t)nlf * sizeof(int32_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&G, ((size_t)kCl * nlf + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&tot, kCl * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    (edfa::count_launch(), k_cp_level_counts<<<(unsigned)((nlf + 127) / 128), 128, 0, s>>>(nlf, f.fwd.perm, f.fwd.loff,
                                                                                           cL, G));
    rc = scan_i64(h, G, (int64_t)kCl * nlf, s);
    if (rc) return rc;
    (edfa::count_launch(), k_cp_assign<<<(unsigned)((nsf + 255) / 256), 256, 0, s>>>(nsf, nlf, f.fwd.perm, f.fwd.loff,
                                                                                     cL, G, cp.posf));
    (edfa::count_launch(), k_cp_totals<<<1, 32, 0, s>>>(nlf, G, tot));
    int64_t htot[kCl];
    cudaMemcpyAsync(htot, tot, sizeof htot, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(cL, s);
    cudaFreeAsync(G, s);
    cudaFreeAsync(tot, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
    int64_t mx = 0;
    for (int r = 0; r < kCl; ++r) mx = htot[r] > mx ? htot[r] : mx;
    const int32_t cap = (int32_t)((mx + 3) & ~(int64_t)3);  // 16-byte rows for 4- and 8-byte values
    if (pad16((int64_t)cap * sizeof(T)) + min_extra_smem > optin) return EDFA_OK;
    rc = dalloc_t(h, &cp.rowof, (size_t)kCl * cap);
    if (rc) return rc;
    cudaMemsetAsync(cp.rowof, 0xFF, (size_t)kCl * cap * sizeof(int32_t), s);
    (edfa::count_launch(), k_cp_rowof<<<(unsigned)((f.n + 255) / 256), 256, 0, s>>>(f.n, cp.posf, cap, cp.rowof));

    const int64_t nlists = (int64_t)kCl * nlt;
    rc = dalloc_t(h, &cp.lofs, (size_t)nlists + 1);
    if (rc) return rc;
    ListGeom lg{f.fwd.perm, f.bwd.perm, f.fwd.loff, f.bwd.loff, nsf, nsb, nlf, nlb};
    const unsigned gl = (unsigned)((nsf + nsb + 255) / 256);
    cudaMemsetAsync(cp.lofs, 0, ((size_t)nlists + 1) * sizeof(int64_t), s);
    (edfa::count_launch(), k_cp_lists<0><<<gl, 256, 0, s>>>(lg, cp.posf, (unsigned long long*)cp.lofs, nullptr));
    if (pad > 1)
        (edfa::count_launch(), k_cp_pad_lists<<<(unsigned)((nlists + 255) / 256), 256, 0, s>>>(nlists, cp.lofs, pad));
    rc = scan_i64(h, cp.lofs, nlists, s);
    if (rc) return rc;
    int64_t nrec = 0;
    cudaMemcpyAsync(&nrec, cp.lofs + nlists, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
    rc = dalloc_t(h, &cp.lrows, (size_t)(nrec > 0 ? nrec : 1));
    if (rc) return rc;
    cudaMemsetAsync(cp.lrows, 0xFF, (size_t)(nrec > 0 ? nrec : 1) * sizeof(int32_t), s);
    cp.nrec = nrec;
    unsigned long long* cursor = nullptr;
    if (cudaMallocAsync((void**)&cursor, ((size_t)nlists + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemcpyAsync(cursor, cp.lofs, ((size_t)nlists + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    (edfa::count_launch(), k_cp_lists<1><<<gl, 256, 0, s>>>(lg, cp.posf, cursor, cp.lrows));
    cudaFreeAsync(cursor, s);
    cp.cap = cap;
    cp.nlf = nlf;
    cp.nlb = nlb;
    cp.nlists = nlists;
    *cap_out = cap;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// level-synchronous variant: packed chunks streamed by TMA
template <class T>
static int plan_levelsync_t(edfa_handle_s* h, cudaStream_t s)
{
    ClusterPlan& cp = h->cp;
    const Factor& f = h->fs;
    const int64_t ring = (int64_t)kRing * kChunk + 16 * (kRing + 1);
    int32_t cap = 0;
    int rc = plan_common<T>(h, ring + 16, &cap, s);
    if (rc || cap == 0) return rc;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    const int64_t fixed = pad16((int64_t)cap * sizeof(T)) + ring;
    const void* fn = (const void*)k_s_cluster<T, T, kClLpr>;
    if (!cluster_schedulable(fn, kClThreads, (size_t)(fixed + 16))) return EDFA_OK;
    const int nlt = cp.nlf + cp.nlb;
    const int64_t nlists = cp.nlists;
    rc = dalloc_t(h, &cp.lbyte, (size_t)nlists + 1);
    if (!rc) rc = dalloc_t(h, &cp.lchunk, (size_t)nlists + 1);
    if (!rc) rc = dalloc_t(h, &cp.meta, 2 * kCl);
    if (rc) return rc;
    int* bad = nullptr;
    if (cudaMallocAsync((void**)&bad, sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    const unsigned gL = (unsigned)((nlists + 127) / 128);
    (edfa::count_launch(), k_cp_size<T><<<gL, 128, 0, s>>>(nlists, nlt, cp.nlf, cp.lofs, cp.lrows, f.rowptr, f.diag,
                                                          cp.lbyte, cp.lchunk, bad));
    rc = scan_i64(h, cp.lbyte, nlists, s);
    if (!rc) rc = scan_i64(h, cp.lchunk, nlists, s);
    if (rc) return rc;
    (edfa::count_launch(), k_cp_meta<<<1, 32, 0, s>>>(nlt, cp.lbyte, cp.lchunk, cp.meta));
    int64_t meta[2 * kCl];
    int hbad = 0;
    int64_t total = 0;
    cudaMemcpyAsync(meta, cp.meta, sizeof meta, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&total, cp.lbyte + nlists, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(bad, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
    if (hbad) return EDFA_OK;
    int64_t maxch = 0;
    for (int r = 0; r < kCl; ++r) maxch = meta[2 * r + 1] > maxch ? meta[2 * r + 1] : maxch;
    const int32_t szstride = (int32_t)((maxch + 7) & ~(int64_t)7);
    const int64_t smem = fixed + pad16((int64_t)szstride * 2);
    if (smem > optin) return EDFA_OK;
    if (!cluster_schedulable(fn, kClThreads, (size_t)smem)) return EDFA_OK;
    rc = dalloc(h, (void**)&cp.chunks, (size_t)total);
    if (!rc) rc = dalloc_t(h, &cp.sz, (size_t)kCl * szstride);
    if (!rc) rc = dalloc(h, &cp.bslot, (size_t)kCl * cap * sizeof(T));
    if (rc) return rc;
    cp.szstride = szstride;
    cp.smem = (size_t)smem;
    cp.bytes = total;
    cp.state = 1;
    cp.kind = 2;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// dataflow variant: fixed-size row records in processing order
template <class T>
static int plan_dataflow_t(edfa_handle_s* h, cudaStream_t s)
{
    ClusterPlan& cp = h->cp;
    const Factor& f = h->fs;
    int32_t cap = 0;
    int rc = plan_common<T>(h, 64, &cap, s, 32 / kDfLpr);
    if (rc || cap == 0) return rc;
    const size_t smem = (size_t)pad16((int64_t)cap * sizeof(T));
    if (!cluster_schedulable((const void*)k_s_df<T, T, kDfLpr, kDfThreads, kDfSleep>, kDfThreads, smem))
        return EDFA_OK;
    const int nlt = cp.nlf + cp.nlb;
    const int64_t nrec = cp.nrec;
    rc = dalloc_t(h, &cp.fidx, (size_t)f.n);
    if (!rc) rc = dalloc_t(h, &cp.bidx, (size_t)kCl * cap);
    if (!rc) rc = dalloc_t(h, &cp.rmeta, 4 * kCl);
    if (!rc) rc = dalloc_t(h, &cp.ovoff, (size_t)nrec + 1);
    if (!rc) rc = dalloc_t(h, &cp.lvl, (size_t)2 * f.n);
    if (rc) return rc;
    cudaMemsetAsync(cp.bidx, 0xFF, (size_t)kCl * cap * sizeof(int64_t), s);
    // dependency levels of every row in both sweeps (order of the record entries)
    if (f.fwd.nslots > 0)
        (edfa::count_launch(), k_df_levels<<<(unsigned)((f.fwd.nslots + 255) / 256), 256, 0, s>>>(
            f.fwd.nslots, f.fwd.nlevels, f.fwd.perm, f.fwd.loff, cp.lvl));
    if (f.bwd.nslots > 0)
        (edfa::count_launch(), k_df_levels<<<(unsigned)((f.bwd.nslots + 255) / 256), 256, 0, s>>>(
            f.bwd.nslots, f.bwd.nlevels, f.bwd.perm, f.bwd.loff, cp.lvl + f.n));
    const unsigned gr = (unsigned)((nrec + 255) / 256);
    if (nrec > 0) {
        (edfa::count_launch(), k_df_idx<<<gr, 256, 0, s>>>(nrec, nlt, cp.nlf, cp.lofs, cp.lrows, cp.posf, cap,
                                                         cp.fidx, cp.bidx));
        (edfa::count_launch(), k_df_ovf_count<<<gr, 256, 0, s>>>(nrec, nlt, cp.nlf, cp.lofs, cp.lrows, cp.posf,
                                                               f.rowptr, f.diag, cp.ovoff));
    }
    rc = scan_i64(h, cp.ovoff, nrec, s);
    if (rc) return rc;
    (edfa::count_launch(), k_df_rmeta<<<1, 32, 0, s>>>(nlt, cp.nlf, cp.lofs, cp.rmeta));
    int64_t novf = 0;
    cudaMemcpyAsync(&novf, cp.ovoff + nrec, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
    rc = dalloc(h, (void**)&cp.rec, (size_t)(nrec > 0 ? nrec : 1) * df_rb<T>());
    if (!rc) rc = dalloc_t(h, &cp.ovf_dep, (size_t)(novf > 0 ? novf : 1));
    if (!rc) rc = dalloc(h, &cp.ovf_val, (size_t)(novf > 0 ? novf : 1) * sizeof(T));
    if (rc) return rc;
    cudaMemsetAsync(cp.rec, 0, (size_t)(nrec > 0 ? nrec : 1) * df_rb<T>(), s);
    cp.smem = smem;
    cp.bytes = nrec * df_rb<T>() + novf * (4 + (int64_t)sizeof(T));
    cp.state = 1;
    cp.kind = 1;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int cluster_plan_build(edfa_handle_s* h, cudaStream_t s)
{
    h->cp.state = 0;
    const Factor& f = h->fs;
    const int mode = h->opt.sweep_mode;
    if (mode == 1 || f.n <= 0 || f.fwd.nlevels <= 0 || f.bwd.nlevels <= 0) return EDFA_OK;
    const bool f32 = h->opt.precision == 1;
    if (mode == 2) return f32 ? plan_levelsync_t<float>(h, s) : plan_levelsync_t<double>(h, s);
    return f32 ? plan_dataflow_t<float>(h, s) : plan_dataflow_t<double>(h, s);
}

template <class T>
static int fill_t(edfa_handle_s* h, const T* lu, const T* dinv, cudaStream_t s)
{
    ClusterPlan& cp = h->cp;
    const Factor& f = h->fs;
    const int nlt = cp.nlf + cp.nlb;
    if (cp.kind == 2) {
        const unsigned gL = (unsigned)((cp.nlists + 127) / 128);
        (edfa::count_launch(), k_cp_write<T><<<gL, 128, 0, s>>>(cp.nlists, nlt, cp.nlf, cp.lofs, cp.lrows, f.rowptr,
                                                               f.col, f.diag, lu, dinv, cp.posf, cp.lbyte, cp.lchunk,
                                                               cp.chunks, cp.sz, cp.szstride));
    } else {
        const int64_t nrec = cp.nrec;
        if (nrec > 0)
        (edfa::count_launch(), k_df_write<T><<<(unsigned)((nrec + 127) / 128), 128, 0, s>>>(
            nrec, nlt, cp.nlf, f.n, cp.lofs, cp.lrows, cp.posf, cp.lvl, f.rowptr, f.col, f.diag, lu, dinv, cp.ovoff, cp.rec,
            cp.ovf_dep, (T*)cp.ovf_val));
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int cluster_plan_fill(edfa_handle_s* h, cudaStream_t s)
{
    ClusterPlan& cp = h->cp;
    if (cp.state != 1) return EDFA_OK;
    const Factor& f = h->fs;
    if (h->opt.precision == 1) return fill_t<float>(h, f.lu32, f.dinv32, s);
    return fill_t<double>(h, f.lu64, f.dinv64, s);
}

template <class T>
int s_cluster_solve(edfa_handle_s* h, const double* rp, const int64_t* mptr, const int32_t* mcol, const T* mval,
                    const T* mv, T* out, cudaStream_t s, cudaEvent_t* pe)
{
    ClusterPlan& cp = h->cp;
    const Factor& f = h->fs;
    cudaLaunchAttribute attr[1];
    cudaError_t e;
    if (cp.kind == 2) {
        (edfa::count_launch(), k_cp_rhs<T, double><<<(unsigned)((f.n + 255) / 256), 256, 0, s>>>(
            f.n, cp.posf, cp.cap, rp, mptr, mcol, mval, mv, (T*)cp.bslot));
        cudaLaunchConfig_t cfg = cluster_cfg(cp.smem, kClThreads, s, attr);
        if (pe) cudaEventRecord(pe[0], s);
        edfa::count_launch();
        e = cudaLaunchKernelEx(&cfg, k_s_cluster<T, T, kClLpr>, (const T*)cp.bslot, (const unsigned char*)cp.chunks,
                               (const uint16_t*)cp.sz, (const int64_t*)cp.meta, cp.szstride, cp.cap, cp.nlf, cp.nlb,
                               (const int32_t*)cp.rowof, out, h->err);
    } else {
        (edfa::count_launch(), k_df_rhs<T, double><<<(unsigned)((4 * (int64_t)f.n + 255) / 256), 256, 0, s>>>(
            f.n, cp.fidx, cp.rec, rp, mptr, mcol, mval, mv));
        cudaLaunchConfig_t cfg = cluster_cfg(cp.smem, kDfThreads, s, attr);
        if (pe) cudaEventRecord(pe[0], s);
        edfa::count_launch();
        e = cudaLaunchKernelEx(&cfg, k_s_df<T, T, kDfLpr, kDfThreads, kDfSleep>, cp.rec, (const int64_t*)cp.rmeta, cp.cap,
                               (const int32_t*)cp.ovf_dep, (const T*)cp.ovf_val, (const int64_t*)cp.bidx,
                               (const int32_t*)cp.rowof, out, h->err);
    }
    if (pe) cudaEventRecord(pe[1], s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EDFA_ERR_CUDA;
    }
    return EDFA_OK;
}

template int s_cluster_solve<double>(edfa_handle_s*, const double*, const int64_t*, const int32_t*, const double*,
                                     const double*, double*, cudaStream_t, cudaEvent_t*);
template int s_cluster_solve<float>(edfa_handle_s*, const double*, const int64_t*, const int32_t*, const float*,
                                    const float*, float*, cudaStream_t, cudaEvent_t*);

}  // namespace edfa
