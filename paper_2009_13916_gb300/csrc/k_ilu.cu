// ILU(0) in the natural ordering (the inner preconditioners standing for
// A~^{-1} and S~^{-1} in Eq. (EDFA_prec)) and its triangular sweeps.
//
// Design (GB300): the dependency depth of a natural-order sweep is fixed by
// the pattern (193 levels for the 64^3 face block, ~700 for S~), so the
// sweeps are latency-bound.  Every kernel here is sync-free: rows are handed
// out in dependency-level order through a global ticket, and a row waits only
// for the rows it reads.  The sweeps poll the result values themselves (the
// output vector is pre-filled with an all-ones NaN that no arithmetic
// produces), so one L2 round trip resolves a dependency.  Rows of one level are
// padded to whole warps so that no warp ever waits on itself.
//
// Every wait is bounded (kSpinLimit polls); on timeout the kernel records
// EDFA_ERR_TIMEOUT and finishes.
#include <climits>

#include <cooperative_groups.h>

#include <cstring>

#include "internal.cuh"

// lanes per row of the sweeps over A~ and S~ (1 = thread per row) and the
// dependencies a thread-per-row sweep holds in registers per round
#ifndef EDFA_LPR_A
#define EDFA_LPR_A 4
#endif
#ifndef EDFA_LPR_S
#define EDFA_LPR_S 8
#endif
#ifndef EDFA_KMAX_ROW
#define EDFA_KMAX_ROW 8
#endif

namespace edfa {

constexpr int kFacWarps = 2;
constexpr int kSweepThreads = 64;

// next c work items for this warp (the counter is zeroed before each launch)
__device__ __forceinline__ long long claim(unsigned long long* ticket, int c)
{
    unsigned long long v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(ticket, (unsigned long long)c);
    v = __shfl_sync(0xffffffffu, v, 0);
    return (long long)v;
}

// ------------------------------------------------------------ levels
// level(i) = 1 + max level(j) over the stored j < i (fwd) or j > i (bwd).
// Computed by frontier expansion (Kahn's algorithm) in one persistent launch
// of a single 16-CTA thread-block cluster: every row keeps a count of its
// unfinished dependencies; the rows of level L decrement the counts of their
// dependents, and a row whose count reaches zero joins level L+1.  One cluster
// barrier (~0.2 us) per level instead of a grid-wide barrier (several us),
// O(nnz) work, no polling of unfinished rows.

// dependency counts and the dependents pattern (transpose of the dependency part)
template <int FWD>
__global__ void k_dep_count(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            int* indeg, unsigned long long* dcnt)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int j = col[p];
        if (FWD ? (j < i) : (j > i)) {
            ++c;
            atomicAdd(&dcnt[j], 1ull);
        }
    }
    indeg[i] = c;
}

template <int FWD>
__global__ void k_dep_fill(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           unsigned long long* cursor, int32_t* dcol)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int j = col[p];
        if (FWD ? (j < i) : (j > i)) dcol[atomicAdd(&cursor[j], 1ull)] = (int32_t)i;
    }
}

constexpr int kKahnCtas = 16, kKahnThreads = 1024;

// G lanes per frontier row: the decrements of one row's dependents are issued
// together (one atomic round trip per row, not one per dependent), and the
// rows that become ready are appended with one atomic per warp.
template <int G>
__global__ void __launch_bounds__(kKahnThreads, 1)
k_kahn(int32_t n, const int64_t* __restrict__ dptr, const int32_t* __restrict__ dcol, int* indeg, int* level,
       int32_t* order, int* cnt, int* nlev_out)
{
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = tid - lane; i0 < n; i0 += nth) {  // warp-uniform trip count
        const int64_t i = i0 + lane;
        const bool ready = i < n && indeg[i] == 0;
        const unsigned m = __ballot_sync(0xffffffffu, ready);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&cnt[0], __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ready) {
            level[i] = 0;
            order[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
        }
    }
    cl.sync();
    const int64_t ngroups = nth / G;
    const int64_t grp = tid / G;
    const int gl = (int)(tid % G);
    int64_t start = 0;
    int L = 0;
    // every CTA reads the same count after the same barrier, so all leave the
    // loop together; at most n levels
    while (L < n) {
        const int c = __ldcg(&cnt[L]);  // completed by other SMs before the barrier
        if (c == 0) break;
        const int64_t end = start + c;
        // warp-uniform trip count: every lane of a warp runs the same rounds
        const int64_t rounds = (c + ngroups - 1) / ngroups;
        for (int64_t rd = 0; rd < rounds; ++rd) {
            const int64_t p = start + rd * ngroups + grp;
            bool fin_any = false;
            int fin_i[1] = {-1};
            if (p < end) {
                const int j = __ldcg(order + p);
                const int64_t q0 = dptr[j], q1 = dptr[j + 1];
                for (int64_t q = q0 + gl; q < q1; q += G) {
                    const int i = dcol[q];
                    if (atomicSub(&indeg[i], 1) == 1) {
                        level[i] = L + 1;
                        // rare second completion in the same lane: append directly
                        if (fin_any) order[end + atomicAdd(&cnt[L + 1], 1)] = (int32_t)i;
                        else { fin_any = true; fin_i[0] = i; }
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, fin_any);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&cnt[L + 1], __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (fin_any) order[end + base + __popc(m & ((1u << lane) - 1u))] = (int32_t)fin_i[0];
        }
        cl.sync();
        start = end;
        ++L;
    }
    if (tid == 0) *nlev_out = L;
}

__global__ void k_level_hist(int32_t n, const int* level, unsigned long long* hist)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&hist[level[i]], 1ull);
}

__global__ void k_level_pad(int32_t nlev, int64_t* hist, int g)
{
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l < nlev) hist[l] = (hist[l] + g - 1) / g * g;
}

__global__ void k_level_scatter(int32_t n, const int* level, const int64_t* off, unsigned long long* cursor,
                                int32_t* perm)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = level[i];
    unsigned long long k = atomicAdd(&cursor[l], 1ull);
    perm[off[l] + (int64_t)k] = (int32_t)i;
}

// grid of a sync-free kernel: at most `warps_per_sm` resident warps per SM
// (0 = default), never more than the occupancy limit
static int resident_grid(edfa_handle_s* h, const void* fn, int threads, size_t smem, int warps_per_sm = 0)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
    if (per < 1) per = 1;
    int want = warps_per_sm > 0 ? warps_per_sm : 16;
    int bl = want * 32 / threads;
    if (bl < 1) bl = 1;
    if (bl < per) per = bl;
    return per * h->nsm;
}

static int make_plan(edfa_handle_s* h, SweepPlan& plan, int32_t n, const int64_t* rowptr, const int32_t* col,
                     int fwd, int pad, cudaStream_t s)
{
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int *level = nullptr, *indeg = nullptr, *cnt = nullptr, *misc = nullptr;
    int64_t* dptr = nullptr;
    int32_t *dcol = nullptr, *order = nullptr;
    unsigned long long* dcur = nullptr;
    if (cudaMallocAsync((void**)&level, nn * sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&indeg, nn * sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&cnt, (nn + 2) * sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&misc, 4 * sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&dptr, (nn + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&dcur, (nn + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&order, nn * sizeof(int32_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemsetAsync(dptr, 0, (nn + 1) * sizeof(int64_t), s);
    cudaMemsetAsync(cnt, 0, (nn + 2) * sizeof(int), s);
    cudaMemsetAsync(misc, 0, 4 * sizeof(int), s);
    const unsigned gb = (unsigned)((n + 255) / 256);
    if (n > 0) {
        if (fwd) (edfa::count_launch(), k_dep_count<1><<<gb, 256, 0, s>>>(n, rowptr, col, indeg, (unsigned long long*)dptr));
        else (edfa::count_launch(), k_dep_count<0><<<gb, 256, 0, s>>>(n, rowptr, col, indeg, (unsigned long long*)dptr));
    }
    int rc = scan_i64(h, dptr, n, s);
    if (rc) return rc;
    int64_t ndep = 0;
    cudaMemcpyAsync(&ndep, dptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (cudaMallocAsync((void**)&dcol, (size_t)(ndep > 0 ? ndep : 1) * sizeof(int32_t), s) != cudaSuccess)
        return EDFA_ERR_OOM;
    cudaMemcpyAsync(dcur, dptr, (nn + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (n > 0) {
        if (fwd) (edfa::count_launch(), k_dep_fill<1><<<gb, 256, 0, s>>>(n, rowptr, col, dcur, dcol));
        else (edfa::count_launch(), k_dep_fill<0><<<gb, 256, 0, s>>>(n, rowptr, col, dcur, dcol));
    }
    // frontier expansion in one 16-CTA cluster; lanes per frontier row from
    // the mean number of dependents
    int* nlev_d = misc + 2;
    if (n > 0) {
        const double avg = (double)ndep / (double)n;
        auto fn = avg > 12.0 ? k_kahn<32> : avg > 6.0 ? k_kahn<16> : avg > 3.0 ? k_kahn<8> : k_kahn<4>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kKahnCtas, 1, 1);
        cfg.blockDim = dim3(kKahnThreads, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kKahnCtas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        edfa::count_launch();
        if (cudaLaunchKernelEx(&cfg, fn, (int32_t)n, (const int64_t*)dptr, (const int32_t*)dcol, indeg, level,
                               order, cnt, nlev_d) != cudaSuccess) {
            cudaGetLastError();
            return EDFA_ERR_CUDA;
        }
    }
    int nlev = 0;
    cudaMemcpyAsync(&nlev, nlev_d, sizeof(int), cudaMemcpyDeviceToHost, s);
    rc = check_err(h, s);
    if (rc) return rc;
    if (n == 0) nlev = 0;
    cudaFreeAsync(indeg, s);
    cudaFreeAsync(cnt, s);
    cudaFreeAsync(misc, s);
    cudaFreeAsync(dptr, s);
    cudaFreeAsync(dcur, s);
    cudaFreeAsync(dcol, s);
    cudaFreeAsync(order, s);
    int64_t* off = nullptr;
    unsigned long long* cursor = nullptr;
    if (cudaMallocAsync((void**)&off, ((size_t)nlev + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&cursor, ((size_t)nlev + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemsetAsync(off, 0, ((size_t)nlev + 1) * sizeof(int64_t), s);
    cudaMemsetAsync(cursor, 0, ((size_t)nlev + 1) * sizeof(int64_t), s);
    if (n > 0) (edfa::count_launch(), k_level_hist<<<(n + 255) / 256, 256, 0, s>>>(n, level, (unsigned long long*)off));
    if (nlev > 0) (edfa::count_launch(), k_level_pad<<<(nlev + 255) / 256, 256, 0, s>>>(nlev, off, pad));
    rc = scan_i64(h, off, nlev, s);
    if (rc) return rc;
    int64_t nslots = 0;
    cudaMemcpyAsync(&nslots, off + nlev, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    rc = dalloc_t(h, &plan.perm, (size_t)(nslots > 0 ? nslots : 1));
    if (rc) return rc;
    cudaMemsetAsync(plan.perm, 0xFF, (size_t)(nslots > 0 ? nslots : 1) * sizeof(int32_t), s);
    if (n > 0) (edfa::count_launch(), k_level_scatter<<<(n + 255) / 256, 256, 0, s>>>(n, level, off, cursor, plan.perm));
    plan.nslots = nslots;
    plan.nlevels = nlev;
    rc = dalloc_t(h, &plan.loff, (size_t)nlev + 1);
    if (rc) return rc;
    cudaMemcpyAsync(plan.loff, off, ((size_t)nlev + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(off, s);
    cudaFreeAsync(cursor, s);
    cudaFreeAsync(level, s);
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

__global__ void k_find_diag(int32_t n, const int64_t* rowptr, const int32_t* col, int64_t* diag, DevErr* err)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t d = -1;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
        if (col[p] == i) d = p;
    if (d < 0) raise_err(err, EDFA_ERR_BREAKDOWN, i);
    diag[i] = d;
}

// longest row of a pattern (picks the layout of the numeric factorisation)
__global__ void k_row_maxlen(int32_t n, const int64_t* __restrict__ rowptr, int* out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, (int)(rowptr[i + 1] - rowptr[i]));
}

// the parts of the symbolic set-up that do not depend on how the level plans
// are obtained: pattern, diagonal positions, longest row, value arrays
int factor_plan_common(edfa_handle_s* h, Factor& f, int32_t n, int64_t nnz, const int64_t* rowptr,
                       const int32_t* col, cudaStream_t s)
{
    f.n = n;
    f.nnz = nnz;
    f.rowptr = rowptr;
    f.col = col;
    int rc = dalloc_t(h, &f.diag, (size_t)(n > 0 ? n : 1));
    if (rc) return rc;
    if (n > 0) (edfa::count_launch(), k_find_diag<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, col, f.diag, h->err));
    {
        // longest row: picks the shared-memory layout of the numeric factorisation
        int* d = nullptr;
        if (cudaMallocAsync((void**)&d, sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
        cudaMemsetAsync(d, 0, sizeof(int), s);
        if (n > 0) (edfa::count_launch(), k_row_maxlen<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, d));
        int r = 0;
        cudaMemcpyAsync(&r, d, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(d, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
        f.fac_R = r;
    }
    const bool f32 = h->opt.precision == 1;
    if (f32) {
        rc = dalloc_t(h, &f.lu32, (size_t)(nnz > 0 ? nnz : 1));
        if (!rc) rc = dalloc_t(h, &f.dinv32, (size_t)(n > 0 ? n : 1));
    } else {
        rc = dalloc_t(h, &f.lu64, (size_t)(nnz > 0 ? nnz : 1));
        if (!rc) rc = dalloc_t(h, &f.dinv64, (size_t)(n > 0 ? n : 1));
    }
    return rc;
}

int factor_plan(edfa_handle_s* h, Factor& f, int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                cudaStream_t s)
{
    int rc = factor_plan_common(h, f, n, nnz, rowptr, col, s);
    if (rc) return rc;
    rc = make_plan(h, f.fwd, n, rowptr, col, 1, 32, s);
    if (rc) return rc;
    return make_plan(h, f.bwd, n, rowptr, col, 0, 32, s);
}

// ------------------------------------------------------------ factorisation
// ILU(0), IKJ order (Saad, Alg. 10.4): row i, for each stored k < i in
// ascending order: l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for stored
// j > k present in row k.  One warp per row, rows taken in level order.
// Per row the warp
//   1. stages the row in shared memory with a column -> position hash,
//   2. before any wait, gathers the U columns of every row it depends on (the
//      pattern is fixed) with one burst of 16-byte cp.async.cg copies (L2,
//      never a stale L1 line) and maps them to positions in row i,
//   3. polls its dependencies (lanes in parallel, no sleep) and gathers 1/u_kk
//      and the U values of each one as soon as it has finished,
//   4. eliminates every finished dependency that has no unfinished one before
//      it in column order: a sequential loop over k whose inner updates are
//      one lane per U entry; then back to 3.
// The operations and their order are those of the IKJ loop; only the waits
// move.  The critical path through the level DAG is one row latency per
// level, and after the last dependency finishes only one poll, one gather
// and the elimination of the last few k remain.  Rows whose U data exceed the
// shared buffers read the U parts from global memory in step 4 instead.
// Three shared-memory layouts per warp, picked by the longest row: up to 256
// entries with up to 1280 gathered U entries and a 512-slot hash (~35 KB per
// warp); up to 64 entries (S~ of the face-neighbour sets: <= 63), ~20 KB; and
// up to 32 entries (the face block: <= 11), ~5 KB; the smaller the layout, the
// more rows are in flight.
template <int R_, int U_, int HB_>
struct FacLayout {
    static constexpr int R = R_, U = U_, HB = HB_, H = 1 << HB_;
};
using FacWide = FacLayout<256, 1280, 9>;
using FacMedium = FacLayout<64, 1280, 7>;
using FacNarrow = FacLayout<32, 256, 7>;

template <class T, class L>
struct alignas(16) FacSmem {
    T rv[L::R];        // the row being factored
    T dk[L::R];        // 1 / u_kk of every dependency
    T uv[L::U];        // U values of the dependencies
    int uc[L::U];      // U columns of the dependencies
    long long ub[L::R];  // first U entry of every dependency
    int rc[L::R];      // row columns
    int oc[L::R + 1];  // dependency u's columns start at uc[oc[u] + sc[u]]
    int ov[L::R + 1];  // ... and its values at uv[ov[u] + sv[u]]
    int sc[L::R];
    int sv[L::R];
    int ul[L::R];      // U length of every dependency
    int rd[L::R];      // dependency state: 0 pending, 1 finished, 2 U values gathered
    int hk[L::H];      // hash keys (column, -1 empty)
    int hp[L::H];      // hash values (position in the row)
};

template <class L>
__device__ __forceinline__ int fac_hslot(int j) { return (int)(((unsigned)j * 2654435769u) >> (32 - L::HB)); }

template <class T, class L>
__device__ __forceinline__ int fac_lookup(const FacSmem<T, L>& S, int j)
{
    int sl = fac_hslot<L>(j);
    for (int it = 0; it < L::H; ++it) {
        const int k = S.hk[sl];
        if (k == j) return S.hp[sl];
        if (k < 0) return -1;
        sl = (sl + 1) & (L::H - 1);
    }
    return -1;
}



__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}

// copy nblk 16-byte blocks starting at element `first` of a global array of
// `total` elements (E per block) to shared memory, all by the calling lane; a
// block reaching past the end of the array is copied element by element
template <class V>
__device__ __forceinline__ void gather_blocks(V* dst, const V* src, long long first, int nblk, long long total,
                                              bool async_ok)
{
    constexpr int E = 16 / (int)sizeof(V);
    for (int q = 0; q < nblk; ++q) {
        const long long g0 = first + (long long)q * E;
        if (async_ok && g0 + E <= total) {
            cp_async16(dst + q * E, src + g0);
        } else {
            for (int e = 0; e < E; ++e)
                if (g0 + e < total) dst[q * E + e] = __ldcg(src + g0 + e);
        }
    }
}

template <class T, class L>
__global__ void __launch_bounds__(kFacWarps * 32, 16)
k_ilu0(int32_t n, int64_t nnz, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
       const int64_t* __restrict__ diag, const T* __restrict__ vals, T* lu, T* dinv, const int32_t* perm,
       int64_t nslots, int* flags, int epoch, unsigned long long* ticket, int async_ok, DevErr* err)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FacSmem<T, L>& S = reinterpret_cast<FacSmem<T, L>*>(fsm_raw)[wid];
    constexpr int VPB = 16 / (int)sizeof(T);
    for (;;) {
        long long t = claim(ticket, 1);
        if (t >= nslots) break;
        int i = perm[t];
        if (i < 0) continue;
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        const int len = (int)(e - b);
        const int dpos = (int)(diag[i] - b);
        if (len > L::R) {
            if (lane == 0) { raise_err(err, EDFA_ERR_BOUNDS, i); st_release(flags + i, epoch); }
            continue;
        }
        // 1. the row and its column hash
        for (int k = lane; k < L::H; k += 32) S.hk[k] = -1;
        __syncwarp();
        for (int u = lane; u < len; u += 32) {
            const int j = col[b + u];
            S.rv[u] = vals[b + u];
            S.rc[u] = j;
            int sl = fac_hslot<L>(j);
            for (int it = 0; it < L::H; ++it) {
                if (atomicCAS(&S.hk[sl], -1, j) == -1) { S.hp[sl] = u; break; }
                sl = (sl + 1) & (L::H - 1);
            }
        }
        __syncwarp();
        // 2. what does not change while the rows above are factored: the U
        // ranges of the dependencies, their aligned blocks, their U columns
        // (gathered in one burst) and the target position of every U entry in
        // row i, all before any wait
        int totc = 0, totv = 0;
        for (int base0 = 0; base0 < dpos; base0 += 32) {
            const int u = base0 + lane;
            int pc = 0, pv = 0;
            if (u < dpos) {
                const int k = S.rc[u];
                const long long ubk = diag[k] + 1;
                const int ulen = (int)(rowptr[k + 1] - ubk);
                S.ub[u] = ubk;
                S.ul[u] = ulen;
                S.rd[u] = 0;
                const int sc = (int)(ubk & 3), sv = (int)(ubk % VPB);
                S.sc[u] = sc;
                S.sv[u] = sv;
                pc = (sc + ulen + 3) & ~3;
                pv = (sv + ulen + VPB - 1) / VPB * VPB;
            }
            int xc = pc, xv = pv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int yc = __shfl_up_sync(0xffffffffu, xc, o);
                const int yv = __shfl_up_sync(0xffffffffu, xv, o);
                if (lane >= o) { xc += yc; xv += yv; }
            }
            if (u < dpos) { S.oc[u] = totc + xc - pc; S.ov[u] = totv + xv - pv; }
            totc += __shfl_sync(0xffffffffu, xc, 31);
            totv += __shfl_sync(0xffffffffu, xv, 31);
        }
        if (lane == 0) { S.oc[dpos] = totc; S.ov[dpos] = totv; }
        __syncwarp();
        const bool in_smem = totc <= L::U && totv <= L::U;
        if (in_smem) {
            for (int u = lane; u < dpos; u += 32)
                gather_blocks(S.uc + S.oc[u], col, S.ub[u] - S.sc[u], (S.oc[u + 1] - S.oc[u]) / 4, nnz, async_ok != 0);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            // padding entries get a position too, never used
            for (int q = lane; q < totc; q += 32) S.uc[q] = fac_lookup(S, S.uc[q]);
        }
        __syncwarp();
        // 3. progressive elimination: poll the pending dependencies (relaxed,
        // then one acquire fence per round: acquire loads in a spin loop would
        // keep invalidating the L1 of every warp on the SM), gather 1/u_kk and
        // the U values of those that finished, and eliminate the longest
        // finished prefix in ascending column order, the order of the IKJ loop.
        // Bounded: no sleep between polls (one row latency per level).
        int done = 0;
        unsigned spins = 0;
        while (done < dpos) {
            bool fresh = false;
            for (int u = done + lane; u < dpos; u += 32)
                if (S.rd[u] == 0 && ld_relaxed_i32(flags + S.rc[u]) == epoch) {
                    S.rd[u] = 1;
                    fresh = true;
                }
            if (!__any_sync(0xffffffffu, fresh)) {
                ++spins;  // warp-uniform
                if (__any_sync(0xffffffffu, spins >= (kSpinLimit << 2) || ((spins & 255u) == 255u && err_set(err)))) {
                    if (lane == 0 && spins >= (kSpinLimit << 2)) raise_err(err, EDFA_ERR_TIMEOUT, i);
                    break;
                }
                continue;
            }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            __syncwarp();
            for (int u = done + lane; u < dpos; u += 32) {
                if (S.rd[u] != 1) continue;
                // the copies first, so that the load of 1/u_kk overlaps them
                if (in_smem)
                    gather_blocks(S.uv + S.ov[u], (const T*)lu, S.ub[u] - S.sv[u], (S.ov[u + 1] - S.ov[u]) / VPB, nnz,
                                  async_ok != 0);
                S.dk[u] = ld_cg(dinv + S.rc[u]);
                S.rd[u] = 2;
            }
            if (in_smem) asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            // 4. eliminate the finished prefix: l_ik on lane 0 (no other lane
            // touches a_ik in this step), the updates a_ij -= l_ik u_kj one
            // lane per U entry
            for (; done < dpos && S.rd[done] == 2; ++done) {
                const int tt = done;
                T lik = T(0);
                if (lane == 0) {
                    lik = S.rv[tt] * S.dk[tt];
                    S.rv[tt] = lik;
                }
                lik = __shfl_sync(0xffffffffu, lik, 0);
                const int n_u = S.ul[tt];
                if (in_smem) {
                    const int c0 = S.oc[tt] + S.sc[tt], v0 = S.ov[tt] + S.sv[tt];
                    for (int q = lane; q < n_u; q += 32) {
                        const int pos = S.uc[c0 + q];
                        if (pos >= 0) S.rv[pos] -= lik * S.uv[v0 + q];
                    }
                } else {
                    const long long ubk = S.ub[tt];
                    for (int q = lane; q < n_u; q += 32) {
                        const int pos = fac_lookup(S, __ldcg(col + ubk + q));
                        if (pos >= 0) S.rv[pos] -= lik * ld_cg(lu + ubk + q);
                    }
                }
                __syncwarp();
            }
        }
        const T piv = S.rv[dpos];
        for (int u = lane; u < len; u += 32) lu[b + u] = S.rv[u];
        if (lane == 0) {
            if (!(piv != T(0)) || !isfinite((double)piv)) raise_err(err, EDFA_ERR_BREAKDOWN, i);
            dinv[i] = T(1) / piv;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(flags + i, epoch);
        __syncwarp();
    }
}

// ILU(0) of an ordered factor, one launch per colour: every dependency of a
// row of colour c lies in an earlier colour, finished by an earlier launch,
// so nothing is awaited and nothing is staged ahead.  A warp per row keeps the
// row, a column -> position hash and its dependencies' 1/u_kk and U ranges in
// shared memory (~3 KB, so up to 64 warps per SM) and reads the dependencies'
// U rows through the caches.  The arithmetic and its order are those of
// k_ilu0 (l_ik = a_ik (1/u_kk), then a_ij -= l_ik u_kj, dependencies in
// ascending column order), so the factors are the same.
template <int R_, int HB_>
struct McFacLayout {
    static constexpr int R = R_, HB = HB_, H = 1 << HB_;
};

template <class T, class L>
struct alignas(16) McFacSmem {
    T rv[L::R];          // the row being factored
    T dk[L::R];          // 1 / u_kk of every dependency
    long long ub[L::R];  // first U entry of every dependency
    int ul[L::R];        // its U length
    int rc[L::R];        // row columns
    int hk[L::H];        // hash keys (column, -1 empty)
    int hp[L::H];        // hash values (position in the row)
};

constexpr int kMcFacWarps = 8;

template <class T, class L>
__global__ void __launch_bounds__(kMcFacWarps * 32)
k_ilu0_colour(int32_t r0, int32_t r1, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
              const int64_t* __restrict__ diag, const T* __restrict__ vals, T* lu, T* dinv, DevErr* err)
{
    extern __shared__ __align__(16) unsigned char mfs_raw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    McFacSmem<T, L>& S = reinterpret_cast<McFacSmem<T, L>*>(mfs_raw)[wid];
    const int64_t nw = (int64_t)gridDim.x * kMcFacWarps;
    for (int64_t i = r0 + (int64_t)blockIdx.x * kMcFacWarps + wid; i < r1; i += nw) {
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        const int len = (int)(e - b);
        const int dpos = (int)(diag[i] - b);
        if (len > L::R) {
            if (lane == 0) raise_err(err, EDFA_ERR_BOUNDS, i);
            continue;
        }
        for (int k = lane; k < L::H; k += 32) S.hk[k] = -1;
        __syncwarp();
        for (int u = lane; u < len; u += 32) {
            const int j = col[b + u];
            S.rv[u] = vals[b + u];
            S.rc[u] = j;
            int sl = (int)(((unsigned)j * 2654435769u) >> (32 - L::HB));
            for (int it = 0; it < L::H; ++it) {
                if (atomicCAS(&S.hk[sl], -1, j) == -1) { S.hp[sl] = u; break; }
                sl = (sl + 1) & (L::H - 1);
            }
        }
        // the dependencies' 1/u_kk and U ranges, all lanes at once
        for (int u = lane; u < dpos; u += 32) {
            const int k = S.rc[u];
            const long long ubk = diag[k] + 1;
            S.ub[u] = ubk;
            S.ul[u] = (int)(rowptr[k + 1] - ubk);
            S.dk[u] = dinv[k];
        }
        __syncwarp();
        for (int t = 0; t < dpos; ++t) {
            const T lik = S.rv[t] * S.dk[t];
            __syncwarp();
            if (lane == 0) S.rv[t] = lik;
            const long long ubk = S.ub[t];
            const int n_u = S.ul[t];
            for (int q = lane; q < n_u; q += 32) {
                const int j = col[ubk + q];
                int sl = (int)(((unsigned)j * 2654435769u) >> (32 - L::HB));
                int pos = -1;
                for (int it = 0; it < L::H; ++it) {
                    const int kk = S.hk[sl];
                    if (kk == j) { pos = S.hp[sl]; break; }
                    if (kk < 0) break;
                    sl = (sl + 1) & (L::H - 1);
                }
                if (pos >= 0) S.rv[pos] -= lik * lu[ubk + q];
            }
            __syncwarp();
        }
        const T piv = S.rv[dpos];
        for (int u = lane; u < len; u += 32) lu[b + u] = S.rv[u];
        if (lane == 0) {
            if (!(piv != T(0)) || !isfinite((double)piv)) raise_err(err, EDFA_ERR_BREAKDOWN, i);
            dinv[i] = T(1) / piv;
        }
        __syncwarp();
    }
}

template <class T, class L>
static void ilu0_colour_launch(edfa_handle_s* h, const Factor& f, const Ordering& o, const T* vals, T* lu, T* dinv,
                               cudaStream_t s)
{
    auto fn = k_ilu0_colour<T, L>;
    const size_t smem = sizeof(McFacSmem<T, L>) * kMcFacWarps;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kMcFacWarps * 32, smem);
    if (per < 1) per = 1;
    for (int c = 0; c < o.ncolours; ++c) {
        const int32_t r0 = o.cstart[c], r1 = o.cstart[c + 1];
        if (r1 <= r0) continue;
        int64_t blocks = ((int64_t)(r1 - r0) + kMcFacWarps - 1) / kMcFacWarps;
        if (blocks > (int64_t)per * h->nsm) blocks = (int64_t)per * h->nsm;
        (edfa::count_launch(), fn<<<(unsigned)blocks, kMcFacWarps * 32, smem, s>>>(r0, r1, f.rowptr, f.col, f.diag, vals,
                                                                                  lu, dinv, h->err));
    }
}

int factor_numeric(edfa_handle_s* h, Factor& f, const double* vals64, const float* vals32, cudaStream_t s)
{
    if (f.n == 0) return EDFA_OK;
    if (f.ord && f.fac_R <= 128) {
        using L64 = McFacLayout<64, 7>;
        using L128 = McFacLayout<128, 8>;
        if (h->opt.precision == 1) {
            if (f.fac_R <= 64) ilu0_colour_launch<float, L64>(h, f, *f.ord, vals32, f.lu32, f.dinv32, s);
            else ilu0_colour_launch<float, L128>(h, f, *f.ord, vals32, f.lu32, f.dinv32, s);
        } else {
            if (f.fac_R <= 64) ilu0_colour_launch<double, L64>(h, f, *f.ord, vals64, f.lu64, f.dinv64, s);
            else ilu0_colour_launch<double, L128>(h, f, *f.ord, vals64, f.lu64, f.dinv64, s);
        }
        return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
    }
    h->epoch += 1;
    if (h->epoch == INT_MAX) {
        h->epoch = 1;
        int32_t nmax = h->Nf > h->Ne ? h->Nf : h->Ne;
        cudaMemsetAsync(h->flags, 0, (size_t)nmax * sizeof(int), s);
    }
    cudaMemsetAsync(h->ticket, 0, sizeof(unsigned long long), s);
    // 16-byte copies need 16-byte aligned column and value arrays
    const bool f32 = h->opt.precision == 1;
    const int async_ok = ((uintptr_t)f.col % 16 == 0) && ((uintptr_t)(f32 ? (void*)f.lu32 : (void*)f.lu64) % 16 == 0);
    // resident warps: about six dependency levels of rows in flight, so that
    // the preparation of a row (step 2) is done before its dependencies are;
    // a wide DAG such as the face block fills the SMs, a narrow one such as
    // S~ is capped by the shared memory per warp (64^3, FP64: 6 levels 9.0 ms,
    // 4 levels 9.5 ms, 2.5 levels 12.2 ms)
    const double per_level = f.fwd.nlevels > 0 ? (double)f.n / f.fwd.nlevels : (double)f.n;
    int wps = (int)(6.0 * per_level / h->nsm);
    if (wps < 6) wps = 6;
    if (wps > 32) wps = 32;
    auto launch = [&](auto tag, auto lay) -> void {
        using TT = decltype(tag);
        using LL = decltype(lay);
        auto fn = k_ilu0<TT, LL>;
        const size_t smem = sizeof(FacSmem<TT, LL>) * kFacWarps;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = resident_grid(h, (const void*)fn, kFacWarps * 32, smem, wps);
        const TT* vals;
        TT *lu, *dinv;
        if constexpr (sizeof(TT) == 8) { vals = (const TT*)vals64; lu = (TT*)f.lu64; dinv = (TT*)f.dinv64; }
        else { vals = (const TT*)vals32; lu = (TT*)f.lu32; dinv = (TT*)f.dinv32; }
        (edfa::count_launch(), fn<<<grid, kFacWarps * 32, smem, s>>>(f.n, f.nnz, f.rowptr, f.col, f.diag, vals, lu, dinv,
                                                                     f.fwd.perm, f.fwd.nslots, h->flags, h->epoch,
                                                                     h->ticket, async_ok, h->err));
    };
    const bool narrow = f.fac_R <= FacNarrow::R;
    const bool medium = !narrow && f.fac_R <= FacMedium::R;
    if (f32) {
        if (narrow) launch(float(0), FacNarrow{});
        else if (medium) launch(float(0), FacMedium{});
        else launch(float(0), FacWide{});
    } else {
        if (narrow) launch(double(0), FacNarrow{});
        else if (medium) launch(double(0), FacMedium{});
        else launch(double(0), FacWide{});
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ sweeps
// Sentinel: all-ones bit pattern (a NaN no arithmetic produces).
__device__ __forceinline__ bool is_sentinel(double v) { return __double_as_longlong(v) == -1ll; }
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_int(v) == -1; }

__device__ __forceinline__ double ld_poll(const double* p)
{
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_poll(const float* p)
{
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed(double* p, double v)
{
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(float* p, float v)
{
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// a poll of a result stored as TO, read in the working precision T; the
// sentinel is tested on the stored bits, before any conversion (a conversion
// of a NaN need not keep its payload)
template <class T, class TO>
__device__ __forceinline__ bool poll_ready(const TO* p, T& v)
{
    const TO x = ld_poll(p);
    v = (T)x;
    return !is_sentinel(x);
}

template <class T>
__device__ __forceinline__ T wait_value(const T* p, DevErr* err, long long who)
{
    T v = ld_poll(p);
    unsigned it = 0, ns = kBackoffMin;
    while (is_sentinel(v) && it < kSpinLimit) {
        __nanosleep(ns);
        if (ns < kBackoffMax) ns <<= 1;
        v = ld_poll(p);
        ++it;
        if ((it & 255u) == 0u && err_set(err)) break;
    }
    if (is_sentinel(v)) { raise_err(err, EDFA_ERR_TIMEOUT, who); v = T(0); }
    return v;
}

template <class TI>
__device__ __forceinline__ double to_d(TI v) { return (double)v; }

// One sweep over a level-ordered plan; LPR lanes per row.
//   FWD=1: out_i = rhs_i - sum_{j<i} L_ij out_j          (unit lower L)
//   FWD=0: out_i = dinv_i (rhs_i - sum_{j>i} U_ij out_j)
// rhs_i = base_i - sum_p M_ip v_p  when a coupling matrix M is given (fused
// SpMV of the block apply), else base_i.
// Latency: everything that does not depend on this sweep's results (column
// indices, factor values, the coupling term, base_i) is loaded first; then the
// polls of up to KMAX dependencies per lane are issued back to back, so a row
// whose dependencies are ready costs one L2 round trip.
template <class T, class TB, class TO, int FWD, int LPR, int KMAX>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep(const int32_t* __restrict__ perm, int64_t nslots, const int64_t* __restrict__ rowptr,
        const int32_t* __restrict__ col, const T* __restrict__ lu, const int64_t* __restrict__ diag,
        const T* __restrict__ dinv, const TB* __restrict__ base, const int64_t* __restrict__ mptr,
        const int32_t* __restrict__ mcol, const T* __restrict__ mval, const TO* __restrict__ mv, TO* out,
        unsigned long long* ticket, DevErr* err)
{
    constexpr int RPW = 32 / LPR;  // rows per warp
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, gl = lane % LPR;
    for (;;) {
        long long t0 = claim(ticket, RPW);
        if (t0 >= nslots) break;
        long long t = t0 + g;
        int i = (t < nslots) ? perm[t] : -1;
        T acc = T(0);
        T bi = T(0), di = T(1);
        if (i >= 0) {
            bi = (T)to_d(base[i]);
            if (!FWD) di = dinv[i];
            const int64_t b = rowptr[i], e = rowptr[i + 1];
            const int64_t d = diag[i];
            const int64_t lo = FWD ? b : d + 1, hi = FWD ? d : e;
            if (mptr) {
                const int64_t mb = mptr[i], me = mptr[i + 1];
                for (int64_t p = mb + gl; p < me; p += 4 * LPR) {
                    int c[4];
                    T w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        int64_t q = p + u * LPR;
                        c[u] = q < me ? mcol[q] : -1;
                        w[u] = q < me ? mval[q] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c[u] >= 0) acc = fma(w[u], (T)mv[c[u]], acc);
                }
            }
            T lacc = T(0);
            for (int64_t c0 = lo; c0 < hi; c0 += KMAX * LPR) {
                int cj[KMAX];
                T lv[KMAX];
#pragma unroll
                for (int k = 0; k < KMAX; ++k) {
                    int64_t p = c0 + gl + k * LPR;
                    cj[k] = p < hi ? col[p] : -1;
                    lv[k] = p < hi ? lu[p] : T(0);
                }
                T xv[KMAX];
                unsigned pending = 0;
#pragma unroll
                for (int k = 0; k < KMAX; ++k) {
                    xv[k] = T(0);
                    if (cj[k] >= 0 && !poll_ready(out + cj[k], xv[k])) pending |= 1u << k;
                }
                // poll every still-pending dependency in the same round, without
                // sleeping: a level completes with its slowest row, and measured
                // per-level times on GB300 were ~30% lower without back-off
                unsigned it = 0;
                while (pending && it < (kSpinLimit << 2)) {
#pragma unroll
                    for (int k = 0; k < KMAX; ++k)
                        if (((pending >> k) & 1u) && poll_ready(out + cj[k], xv[k])) pending &= ~(1u << k);
                    ++it;
                    if ((it & 255u) == 0u && err_set(err)) break;
                }
                if (pending) {
                    raise_err(err, EDFA_ERR_TIMEOUT, i);
#pragma unroll
                    for (int k = 0; k < KMAX; ++k)
                        if ((pending >> k) & 1u) xv[k] = T(0);
                }
                // products summed as a tree: short dependent FP64 chain once
                // the last dependency has arrived
                T pr[KMAX];
#pragma unroll
                for (int k = 0; k < KMAX; ++k) pr[k] = lv[k] * xv[k];
#pragma unroll
                for (int w = 1; w < KMAX; w <<= 1)
#pragma unroll
                    for (int k = 0; k + w < KMAX; k += 2 * w) pr[k] += pr[k + w];
                lacc += pr[0];
            }
            acc += lacc;
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i >= 0 && gl == 0) {
            T r = bi - acc;
            if (!FWD) r *= di;
            st_relaxed(out + i, (TO)r);
        }
    }
}

// Thread-per-row sweep (same contract as k_sweep): a thread owns one row; the
// products of dependencies that are already final are summed while the late
// ones are polled, and the row is finished and stored from inside the polling
// loop as soon as its last dependency arrives, so only ~3 dependent FP64
// operations follow the last arrival (no shuffle reduction, and no thread waits
// for another row of its warp before storing).
template <class T, class TB, class TO, int FWD, int KMAX>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_row(const int32_t* __restrict__ perm, int64_t nslots, const int64_t* __restrict__ rowptr,
            const int32_t* __restrict__ col, const T* __restrict__ lu, const int64_t* __restrict__ diag,
            const T* __restrict__ dinv, const TB* __restrict__ base, const int64_t* __restrict__ mptr,
            const int32_t* __restrict__ mcol, const T* __restrict__ mval, const TO* __restrict__ mv, TO* out,
            unsigned long long* ticket, DevErr* err)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        long long t0 = claim(ticket, 32);
        if (t0 >= nslots) break;
        const long long t = t0 + lane;
        const int i = (t < nslots) ? perm[t] : -1;
        if (i < 0) continue;
        const T bi = (T)to_d(base[i]);
        const T di = FWD ? T(1) : dinv[i];
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        const int64_t d = diag[i];
        const int64_t lo = FWD ? b : d + 1, hi = FWD ? d : e;
        T acc = T(0);
        if (mptr) {
            const int64_t mb = mptr[i], me = mptr[i + 1];
            T a2 = T(0);
            int64_t p = mb;
            for (; p + 1 < me; p += 2) {
                acc = fma(mval[p], (T)mv[mcol[p]], acc);
                a2 = fma(mval[p + 1], (T)mv[mcol[p + 1]], a2);
            }
            if (p < me) acc = fma(mval[p], (T)mv[mcol[p]], acc);
            acc += a2;
        }
        bool done = false;
        for (int64_t c0 = lo; c0 < hi || !done; c0 += KMAX) {
            int cj[KMAX];
            T lv[KMAX], xv[KMAX];
            unsigned pending = 0;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                const int64_t p = c0 + k;
                cj[k] = p < hi ? col[p] : -1;
                lv[k] = p < hi ? lu[p] : T(0);
            }
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                xv[k] = T(0);
                if (cj[k] >= 0 && !poll_ready(out + cj[k], xv[k])) pending |= 1u << k;
            }
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (cj[k] >= 0 && !((pending >> k) & 1u)) acc = fma(lv[k], xv[k], acc);
            const bool last = c0 + KMAX >= hi;
            unsigned it = 0;
            while (pending && it < (kSpinLimit << 2)) {
#pragma unroll
                for (int k = 0; k < KMAX; ++k)
                    if ((pending >> k) & 1u) {
                        T v;
                        if (poll_ready(out + cj[k], v)) {
                            acc = fma(lv[k], v, acc);
                            pending &= ~(1u << k);
                        }
                    }
                ++it;
                if (last && !pending) {
                    st_relaxed(out + i, (TO)((bi - acc) * di));
                    done = true;
                }
                if ((it & 255u) == 0u && err_set(err)) break;
            }
            if (pending) {
                raise_err(err, EDFA_ERR_TIMEOUT, i);
                pending = 0;
            }
            if (last && !done) {
                st_relaxed(out + i, (TO)((bi - acc) * di));
                done = true;
            }
        }
    }
}

// an event pair for a launcher that records both events itself
static cudaEvent_t* prof_begin_pair(edfa_handle_s* h, int kind) { return prof_begin(h, kind, (cudaStream_t)-1); }

template <class T, class TB, class TO, int FWD, int LPR>
static int launch_sweep(edfa_handle_s* h, const Factor& f, const TB* base, const int64_t* mptr, const int32_t* mcol,
                        const T* mval, const TO* mv, TO* out, cudaStream_t s)
{
    const SweepPlan& p = FWD ? f.fwd : f.bwd;
    if (f.n == 0) return EDFA_OK;
    cudaMemsetAsync(out, 0xFF, (size_t)f.n * sizeof(TO), s);
    cudaMemsetAsync(h->ticket, 0, sizeof(unsigned long long), s);
    const T* lu = nullptr;
    const T* dinv = nullptr;
    if constexpr (sizeof(T) == 8) { lu = (const T*)f.lu64; dinv = (const T*)f.dinv64; }
    else { lu = (const T*)f.lu32; dinv = (const T*)f.dinv32; }
    auto fn = (LPR == 1) ? k_sweep_row<T, TB, TO, FWD, (EDFA_KMAX_ROW)>
                         : k_sweep<T, TB, TO, FWD, (LPR > 1 ? LPR : 2), (LPR >= 32 ? 1 : (LPR >= 16 ? 2 : 4))>;
    // resident warps: enough to hold ~3 dependency levels of rows in flight
    // (fewer warps means fewer pollers competing for L2), 2..16 per SM
    int wps = h->opt.sweep_warps_per_sm;
    if (wps <= 0) {
        // 8 warps per SM, more when a level holds many more rows than that
        // (wide levels of batched systems are throughput-bound)
        constexpr int RPW = 32 / (LPR > 1 ? LPR : 1);
        const double per_level = p.nlevels > 0 ? (double)p.nslots / p.nlevels : 1.0;
        wps = (int)(per_level / RPW / h->nsm);
        if (wps < 8) wps = 8;
        if (wps > 64) wps = 64;
    }
    int grid = resident_grid(h, (const void*)fn, kSweepThreads, 0, wps);
    cudaEvent_t* pe = prof_begin(h, (&f == &h->fs ? 2 : 0) + (FWD ? 0 : 1), s);
    (edfa::count_launch(), fn<<<grid, kSweepThreads, 0, s>>>(p.perm, p.nslots, f.rowptr, f.col, lu, f.diag, dinv, base, mptr, mcol, mval, mv, out,
                            h->ticket, h->err));
    if (pe) cudaEventRecord(pe[1], s);
    return EDFA_OK;
}

// ------------------------------------------------------------ multicolour sweeps
// Sweep of an ordered factor, one launch per colour: the rows of a colour are
// contiguous in the ordered numbering and depend only on rows of earlier
// colours (forward) or later colours (backward), which earlier launches have
// written, so a launch is a plain row-parallel pass (no tickets, no polling).
//   FWD=1: out_i = rhs_i - sum_{j<i} L_ij out_j
//   FWD=0: out_i = dinv_i (rhs_i - sum_{j>i} U_ij out_j)
// rhs_i = base_{bperm[i]} - sum_p M_ip v_p (bperm, the coupling M: optional);
// with sperm the result is also written, as FP64, to scat[sperm[i]] (the
// natural numbering).  LPR lanes per row, four entries per lane in flight,
// rows of a colour in order, the factor entries streamed once; the grid is one
// resident wave, since a colour holds a few hundred thousand rows at most.
constexpr int kMcThreads = 256;

// rows [r0, r1) of one colour, grid-stride over warps
template <class T, class TB, class TO, int FWD, int LPR>
__device__ __forceinline__ void mc_rows(int64_t r0, int64_t r1, int64_t warp, int64_t nwarps,
                                        const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                        const T* __restrict__ lu, const int64_t* __restrict__ diag,
                                        const T* __restrict__ dinv, const TB* __restrict__ base,
                                        const int32_t* __restrict__ bperm, const int64_t* __restrict__ mptr,
                                        const int32_t* __restrict__ mcol, const T* __restrict__ mval,
                                        const TO* __restrict__ mv, TO* out, const int32_t* __restrict__ sperm,
                                        double* scat)
{
    constexpr int RPW = 32 / LPR;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, gl = lane % LPR;
    for (int64_t i0 = r0 + warp * RPW; i0 < r1; i0 += nwarps * RPW) {
        const int64_t i = i0 + g;
        const bool live = i < r1;
        T acc = T(0), bi = T(0), di = T(1);
        if (live) {
            // the row's own data first (independent loads)
            const int64_t lo = FWD ? rowptr[i] : diag[i] + 1;
            const int64_t hi = FWD ? diag[i] : rowptr[i + 1];
            bi = (T)to_d(base[bperm ? bperm[i] : i]);
            if (!FWD) di = dinv[i];
            int64_t mb = 0, me = 0;
            if (mptr) { mb = mptr[i]; me = mptr[i + 1]; }
            for (int64_t p0 = lo; p0 < hi; p0 += U * LPR) {
                int c[U];
                T w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t p = p0 + gl + u * LPR;
                    c[u] = p < hi ? col[p] : -1;
                    w[u] = p < hi ? lu[p] : T(0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (c[u] >= 0) acc = fma(w[u], (T)out[c[u]], acc);
            }
            for (int64_t p0 = mb; p0 < me; p0 += U * LPR) {
                int c[U];
                T w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t p = p0 + gl + u * LPR;
                    c[u] = p < me ? mcol[p] : -1;
                    w[u] = p < me ? mval[p] : T(0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (c[u] >= 0) acc = fma(w[u], (T)mv[c[u]], acc);
            }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (live && gl == 0) {
            T r = bi - acc;
            if (!FWD) r *= di;
            out[i] = (TO)r;
            if (sperm) scat[sperm[i]] = (double)r;
        }
    }
}

template <class T, class TB, class TO, int FWD, int LPR>
__global__ void __launch_bounds__(kMcThreads)
k_mc_sweep(int32_t r0, int32_t r1, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
           const T* __restrict__ lu, const int64_t* __restrict__ diag, const T* __restrict__ dinv,
           const TB* __restrict__ base, const int32_t* __restrict__ bperm, const int64_t* __restrict__ mptr,
           const int32_t* __restrict__ mcol, const T* __restrict__ mval, const TO* __restrict__ mv, TO* out,
           const int32_t* __restrict__ sperm, double* scat)
{
    const int64_t warp = ((int64_t)blockIdx.x * kMcThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kMcThreads) >> 5;
    mc_rows<T, TB, TO, FWD, LPR>(r0, r1, warp, nwarps, rowptr, col, lu, diag, dinv, base, bperm, mptr, mcol,
                                        mval, mv, out, sperm, scat);
}

// blocks of the cooperative sweeps: 512 threads, two per SM (the register
// budget of that shape holds the kernel without spills)
constexpr int kMcAllThreads = 512;

// All colours of one sweep in one cooperative launch without barriers
// (dataflow): the row groups of RPW consecutive ordered rows (never straddling
// two colours: every colour's rows are split into its own groups) are dealt to
// the warps statically in processing order (colours ascending forward,
// descending backward), and a row waits only for the results it reads, which
// it polls in `out` (filled with the all-ones pattern before the launch;
// arithmetic never produces it).  Deadlock free: a warp takes its groups in
// processing order, a group depends only on groups earlier in that order, and
// all warps are resident (cooperative launch); the earliest unfinished group
// therefore has its inputs.  Every wait is bounded (a timeout records
// EDFA_ERR_TIMEOUT and the value reads as 0).  tstart[l] = first group of the
// l-th colour in processing order.
template <class T, class TB, class TO, int FWD, int LPR>
__global__ void __launch_bounds__(kMcAllThreads, 2)
k_mc_sweep_df(int ncol, const int64_t* __restrict__ tstart, const int32_t* __restrict__ cstart,
              const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const T* __restrict__ lu,
              const int64_t* __restrict__ diag, const T* __restrict__ dinv, const TB* __restrict__ base,
              const int32_t* __restrict__ bperm, const int64_t* __restrict__ mptr, const int32_t* __restrict__ mcol,
              const T* __restrict__ mval, const TO* __restrict__ mv, TO* out, const int32_t* __restrict__ sperm,
              double* scat, DevErr* err)
{
    constexpr int RPW = 32 / LPR;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR, gl = lane % LPR;
    const int64_t warp = ((int64_t)blockIdx.x * kMcAllThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kMcAllThreads) >> 5;
    const int64_t ntasks = tstart[ncol];
    for (int64_t t = warp; t < ntasks; t += nwarps) {
        int lo = 0, hi = ncol - 1;  // colour position: last l with tstart[l] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tstart[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int c = FWD ? lo : ncol - 1 - lo;
        const int64_t i = (int64_t)cstart[c] + (t - tstart[lo]) * RPW + g;
        const bool live = i < cstart[c + 1];
        T acc = T(0), bi = T(0), di = T(1);
        if (live) {
            const int64_t rlo = FWD ? rowptr[i] : diag[i] + 1;
            const int64_t rhi = FWD ? diag[i] : rowptr[i + 1];
            bi = (T)to_d(base[bperm ? bperm[i] : i]);
            if (!FWD) di = dinv[i];
            int64_t mb = 0, me = 0;
            if (mptr) { mb = mptr[i]; me = mptr[i + 1]; }
            for (int64_t p0 = mb; p0 < me; p0 += U * LPR) {
                int cc[U];
                T w[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t p = p0 + gl + u * LPR;
                    cc[u] = p < me ? mcol[p] : -1;
                    w[u] = p < me ? mval[p] : T(0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (cc[u] >= 0) acc = fma(w[u], (T)mv[cc[u]], acc);
            }
            for (int64_t p0 = rlo; p0 < rhi; p0 += U * LPR) {
                int cc[U];
                T w[U], x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t p = p0 + gl + u * LPR;
                    cc[u] = p < rhi ? col[p] : -1;
                    w[u] = p < rhi ? lu[p] : T(0);
                }
                unsigned pending = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    x[u] = T(0);
                    if (cc[u] >= 0 && !poll_ready(out + cc[u], x[u])) pending |= 1u << u;
                }
                unsigned it = 0;
                while (pending && it < (kSpinLimit << 2)) {
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (((pending >> u) & 1u) && poll_ready(out + cc[u], x[u])) pending &= ~(1u << u);
                    ++it;
                    if ((it & 255u) == 0u && err_set(err)) break;
                }
                if (pending) {
                    raise_err(err, EDFA_ERR_TIMEOUT, i);
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if ((pending >> u) & 1u) x[u] = T(0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (cc[u] >= 0) acc = fma(w[u], x[u], acc);
            }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (live && gl == 0) {
            T r = bi - acc;
            if (!FWD) r *= di;
            if (sperm) scat[sperm[i]] = (double)r;
            st_relaxed(out + i, (TO)r);
        }
    }
}

// Sweeps of a block multicolour ordering (blocks of NB rows, LPR lanes per row,
// 32 / (NB LPR) blocks per warp).  Block j of block colour c holds the rows
// i_k = cstart[c NB + k] + j at positions k = 0 .. NB - 1 (some may be absent
// in the one short block).  Blocks of one block colour are not coupled, so a
// row's entries split into external ones (other block colours: earlier in the
// sweep, polled like the dataflow sweep's) and internal ones (the rows of its
// own block, whose columns lie in the colour range of its block colour).  The
// lanes of a row walk it, sum the external part and the coupling term and keep
// the internal coefficients in shared memory by position; then the warp solves
// its blocks' small triangular systems in registers, position after position
// (ascending forward, descending backward): the rows of that position are
// final, are broadcast within their block, and the later rows add their term.
// The internal chains cost shuffles, not memory round trips, and every warp-wide
// FP64 instruction of that phase serves all the warp's blocks.  Tasks = groups
// of 32 / (NB LPR) blocks, dealt to the warps in processing order (block colours
// ascending forward, descending backward); deadlock free like the dataflow
// sweep.
template <class T, class TB, class TO, int FWD, int NB, int LPR>
__global__ void __launch_bounds__(kMcAllThreads, 2)
k_mc_sweep_blk(int ncol, int nbc, const int64_t* __restrict__ bstart, const int32_t* __restrict__ cstart,
               const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const T* __restrict__ lu,
               const int64_t* __restrict__ diag, const T* __restrict__ dinv, const TB* __restrict__ base,
               const int32_t* __restrict__ bperm, const int64_t* __restrict__ mptr, const int32_t* __restrict__ mcol,
               const T* __restrict__ mval, const TO* __restrict__ mv, TO* out, const int32_t* __restrict__ sperm,
               double* scat, DevErr* err)
{
    constexpr int RPW = 32 / LPR;  // rows per warp
    constexpr int NBW = RPW / NB;  // blocks per warp
    constexpr int U = 4;
    __shared__ T wsh[kMcAllThreads / 32][RPW][NB + 1];  // [warp][row][column position]
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int g = lane / LPR, gl = lane % LPR;  // row of the warp, lane within the row
    const int q = g / NB, kown = g % NB;
    const int64_t warp = ((int64_t)blockIdx.x * kMcAllThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kMcAllThreads) >> 5;
    const int64_t ntasks = bstart[nbc];
    T* W = wsh[wl][g];
    for (int64_t t = warp; t < ntasks; t += nwarps) {
        int lo = 0, hi = nbc - 1;  // block colour position: last l with bstart[l] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bstart[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int cb = FWD ? lo : nbc - 1 - lo;
        const int64_t j = (t - bstart[lo]) * NBW + q;  // this lane's block within its block colour
        const int c0 = cb * NB, c1 = c0 + NB < ncol ? c0 + NB : ncol;
        const int64_t in_lo = cstart[c0], in_hi = cstart[c1];  // the block colour's rows
        if (gl == 0) {
#pragma unroll
            for (int k = 0; k < NB; ++k) W[k] = T(0);
        }
        __syncwarp();
        const int cp = c0 + kown;
        int64_t i = -1;
        bool live = false;
        if (cp < c1) {
            i = (int64_t)cstart[cp] + j;
            live = i < cstart[cp + 1];
        }
        T acc = T(0), bi = T(0), di = T(1);
        if (live) {
            const int64_t rlo = FWD ? rowptr[i] : diag[i] + 1;
            const int64_t rhi = FWD ? diag[i] : rowptr[i + 1];
            bi = (T)to_d(base[bperm ? bperm[i] : i]);
            if (!FWD) di = dinv[i];
            if (mptr) {
                const int64_t mb = mptr[i], me = mptr[i + 1];
                for (int64_t p0 = mb; p0 < me; p0 += U * LPR) {
                    int cc[U];
                    T w[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int64_t p = p0 + gl + u * LPR;
                        cc[u] = p < me ? mcol[p] : -1;
                        w[u] = p < me ? mval[p] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (cc[u] >= 0) acc = fma(w[u], (T)mv[cc[u]], acc);
                }
            }
            for (int64_t p0 = rlo; p0 < rhi; p0 += U * LPR) {
                int cc[U];
                T w[U], x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t p = p0 + gl + u * LPR;
                    cc[u] = p < rhi ? col[p] : -1;
                    w[u] = p < rhi ? lu[p] : T(0);
                }
                // internal entries: coefficient by position (the position of
                // column cc is the k with cstart[c0 + k] + j == cc)
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (cc[u] >= in_lo && cc[u] < in_hi) {
                        bool found = false;
                        for (int k = 0; k < NB && c0 + k < c1; ++k)
                            if ((int64_t)cstart[c0 + k] + j == cc[u]) { W[k] = w[u]; found = true; break; }
                        if (!found) raise_err(err, EDFA_ERR_BOUNDS, i);  // not a block colouring
                        cc[u] = -1;
                    }
                unsigned pending = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    x[u] = T(0);
                    if (cc[u] >= 0 && !poll_ready(out + cc[u], x[u])) pending |= 1u << u;
                }
                unsigned it = 0;
                while (pending && it < (kSpinLimit << 2)) {
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (((pending >> u) & 1u) && poll_ready(out + cc[u], x[u])) pending &= ~(1u << u);
                    ++it;
                    if ((it & 255u) == 0u && err_set(err)) break;
                }
                if (pending) {
                    raise_err(err, EDFA_ERR_TIMEOUT, i);
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if ((pending >> u) & 1u) x[u] = T(0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (cc[u] >= 0) acc = fma(w[u], x[u], acc);
            }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncwarp();
        // the blocks' triangular systems, position after position (backward:
        // in the scaled form x = d bi - d acc, d = 1/U_ii, with the internal
        // coefficients scaled by d once, so a position costs one add and one
        // FMA on the FP64 pipe, forward and backward)
        if (!FWD) {
            bi *= di;
            acc *= di;
            if (gl == 0) {
#pragma unroll
                for (int k = 0; k < NB; ++k) W[k] *= di;
            }
            __syncwarp();
        }
        T xv = T(0);
#pragma unroll
        for (int s2 = 0; s2 < NB; ++s2) {
            const int k = FWD ? s2 : NB - 1 - s2;
            const T r = bi - acc;
            const int src = (q * NB + k) * LPR;
            const T xk = __shfl_sync(0xffffffffu, r, src);
            const int kl = __shfl_sync(0xffffffffu, live ? 1 : 0, src);
            if (kown == k) xv = r;
            if (kl) acc = fma(W[k], xk, acc);
        }
        if (live && gl == 0) {
            if (sperm) scat[sperm[i]] = (double)xv;
            st_relaxed(out + i, (TO)xv);
        }
        __syncwarp();
    }
}

template <class T, class TB, class TO, int FWD, int LPR>
static void mc_launch(edfa_handle_s* h, const Factor& f, const Ordering& o, const T* lu, const T* dinv,
                      const TB* base, const int32_t* bperm, const int64_t* mptr, const int32_t* mcol, const T* mval,
                      const TO* mv, TO* out, const int32_t* sperm, double* scat, bool prefilled, cudaStream_t s)
{
    // one cooperative dataflow launch for all colours when the device supports it
    if (o.ncolours > 1 && o.tstart_dev && h->coop_ok) {
        auto fd = k_mc_sweep_df<T, TB, TO, FWD, LPR>;
        static thread_local int per_dev = -1, per_sm = 0;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev != per_dev) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fd, kMcAllThreads, 0);
            per_dev = dev;
        }
        if (per_sm >= 1) {
            constexpr int li = LPR == 1 ? 0 : LPR == 2 ? 1 : LPR == 4 ? 2 : 3;
            const int64_t* ts = o.tstart_dev + ((int64_t)(FWD ? 0 : 1) * 4 + li) * (o.ncolours + 1);
            if (!prefilled) cudaMemsetAsync(out, 0xFF, (size_t)f.n * sizeof(TO), s);
            int ncol = o.ncolours;
            void* args[] = {(void*)&ncol, (void*)&ts, (void*)&o.cstart_dev, (void*)&f.rowptr, (void*)&f.col,
                            (void*)&lu, (void*)&f.diag, (void*)&dinv, (void*)&base, (void*)&bperm, (void*)&mptr,
                            (void*)&mcol, (void*)&mval, (void*)&mv, (void*)&out, (void*)&sperm, (void*)&scat,
                            (void*)&h->err};
            edfa::count_launch();
            if (cudaLaunchCooperativeKernel((const void*)fd, dim3((unsigned)(h->nsm * per_sm)), dim3(kMcAllThreads),
                                            args, 0, s) == cudaSuccess)
                return;
            cudaGetLastError();
        }
    }
    auto fn = k_mc_sweep<T, TB, TO, FWD, LPR>;
    static thread_local int per_dev = -1, per_sm = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != per_dev) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMcThreads, 0);
        if (per_sm < 1) per_sm = 1;
        per_dev = dev;
    }
    constexpr int RPW = 32 / LPR;
    for (int k = 0; k < o.ncolours; ++k) {
        const int c = FWD ? k : o.ncolours - 1 - k;
        const int32_t r0 = o.cstart[c], r1 = o.cstart[c + 1];
        if (r1 <= r0) continue;
        int64_t blocks = ((int64_t)(r1 - r0) + RPW * (kMcThreads / 32) - 1) / (RPW * (kMcThreads / 32));
        const int64_t cap = (int64_t)h->nsm * per_sm;
        if (blocks > cap) blocks = cap;
        (edfa::count_launch(), fn<<<(unsigned)blocks, kMcThreads, 0, s>>>(r0, r1, f.rowptr, f.col, lu, f.diag, dinv,
                                                                          base, bperm, mptr, mcol, mval, mv, out,
                                                                          sperm, scat));
    }
}

// one cooperative launch of the block sweep; false when that is not possible
template <class T, class TB, class TO, int FWD, int NB, int LPR>
static bool blk_launch(edfa_handle_s* h, const Factor& f, const Ordering& o, const T* lu, const T* dinv,
                       const TB* base, const int32_t* bperm, const int64_t* mptr, const int32_t* mcol, const T* mval,
                       const TO* mv, TO* out, const int32_t* sperm, double* scat, bool prefilled, cudaStream_t s)
{
    auto fb = k_mc_sweep_blk<T, TB, TO, FWD, NB, LPR>;
    static thread_local int per_dev = -1, per_sm = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != per_dev) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fb, kMcAllThreads, 0);
        per_dev = dev;
    }
    if (per_sm < 1) return false;
    const int64_t* bs = o.bstart_dev + ((int64_t)(FWD ? 0 : 1) * 2 + (LPR == 1 ? 0 : 1)) * (o.nbcolours + 1);
    if (!prefilled) cudaMemsetAsync(out, 0xFF, (size_t)f.n * sizeof(TO), s);
    int ncol = o.ncolours, nbc = o.nbcolours;
    void* args[] = {(void*)&ncol, (void*)&nbc, (void*)&bs, (void*)&o.cstart_dev, (void*)&f.rowptr, (void*)&f.col,
                    (void*)&lu, (void*)&f.diag, (void*)&dinv, (void*)&base, (void*)&bperm, (void*)&mptr,
                    (void*)&mcol, (void*)&mval, (void*)&mv, (void*)&out, (void*)&sperm, (void*)&scat, (void*)&h->err};
    edfa::count_launch();
    if (cudaLaunchCooperativeKernel((const void*)fb, dim3((unsigned)(h->nsm * per_sm)), dim3(kMcAllThreads), args, 0,
                                    s) == cudaSuccess)
        return true;
    cudaGetLastError();
    return false;
}

// lanes per row from the average length of the rows' halves plus the coupling
template <class T, class TB, class TO, int FWD>
static int mc_sweep(edfa_handle_s* h, const Factor& f, const Ordering& o, const TB* base, const int32_t* bperm,
                    const int64_t* mptr, const int32_t* mcol, const T* mval, int64_t mnnz, const TO* mv, TO* out,
                    const int32_t* sperm, double* scat, cudaStream_t s, bool prefilled = false)
{
    if (f.n == 0) return EDFA_OK;
    const T* lu = nullptr;
    const T* dinv = nullptr;
    if constexpr (sizeof(T) == 8) { lu = (const T*)f.lu64; dinv = (const T*)f.dinv64; }
    else { lu = (const T*)f.lu32; dinv = (const T*)f.dinv32; }
    const double avg = ((double)(f.nnz - f.n) / 2.0 + (mptr ? (double)mnnz : 0.0)) / (double)f.n;
    cudaEvent_t* pe = prof_begin(h, (&f == &h->fs ? 2 : 0) + (FWD ? 0 : 1), s);
    if (o.bstart_dev && h->coop_ok) {
        // block multicolour ordering: whole blocks per warp, one or two lanes
        // per row (with long rows this still beats the dataflow sweep over
        // block size times the colours: 64^3 full tensor, rows of ~60)
        bool ok = false;
        // one lane per row for short rows, two for longer ones; in FP64 the
        // block solve's instructions weigh more (they serve half the blocks
        // with two lanes per row), so the rows must be longer to gain
        const bool two = avg > (sizeof(T) == 8 ? 12.0 : 8.0);
        if (o.block == 4 && two)
            ok = blk_launch<T, TB, TO, FWD, 4, 2>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm,
                                                  scat, prefilled, s);
        else if (o.block == 4)
            ok = blk_launch<T, TB, TO, FWD, 4, 1>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm,
                                                  scat, prefilled, s);
        else if (o.block == 8 && two)
            ok = blk_launch<T, TB, TO, FWD, 8, 2>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm,
                                                  scat, prefilled, s);
        else if (o.block == 8)
            ok = blk_launch<T, TB, TO, FWD, 8, 1>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm,
                                                  scat, prefilled, s);
        if (ok) {
            if (pe) cudaEventRecord(pe[1], s);
            return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
        }
    }
    if (avg <= 4.0)
        mc_launch<T, TB, TO, FWD, 1>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm, scat,
                                       prefilled, s);
    else if (avg <= 12.0)
        mc_launch<T, TB, TO, FWD, 2>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm, scat,
                                       prefilled, s);
    else if (avg <= 32.0)
        mc_launch<T, TB, TO, FWD, 4>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm, scat,
                                       prefilled, s);
    else
        mc_launch<T, TB, TO, FWD, 8>(h, f, o, lu, dinv, base, bperm, mptr, mcol, mval, mv, out, sperm, scat,
                                       prefilled, s);
    if (pe) cudaEventRecord(pe[1], s);
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// sweep of the A~ factor: chain-decomposed when its DAG collapses to a few
// phases of chains (k_chain.cu), else the level-scheduled sync-free sweep
template <class T, class TB, class TO, int FWD>
static int a_sweep(edfa_handle_s* h, const TB* base, const int64_t* mptr, const int32_t* mcol, const T* mval,
                   const TO* mv, TO* out, cudaStream_t s)
{
    const Factor& f = h->fa;
    if ((FWD ? f.chf.ok : f.chb.ok) != 0) {
        cudaEvent_t* pe = prof_begin(h, FWD ? 0 : 1, s);
        const int rc = chain_sweep<T, TB, TO, FWD>(h, f, base, mptr, mcol, mval, mv, out, s);
        if (pe) cudaEventRecord(pe[1], s);
        return rc;
    }
    return launch_sweep<T, TB, TO, FWD, EDFA_LPR_A>(h, f, base, mptr, mcol, mval, mv, out, s);
}

// ------------------------------------------------------------ block apply
// z = P^{-1} r, Eq. (EDFA_prec):
//   y    = A~^{-1} r_pi                  (L sweep, U sweep of ILU(0)(A))
//   z_p  = S~^{-1} (r_p - C y)           (C y fused into the L sweep of S~)
//   z_pi = A~^{-1} (r_pi - B z_p)        (B z_p fused into the L sweep of A)
// variant 1 (upper block triangular): z_p = S~^{-1} r_p, then z_pi as above.
// The same application with ordered inner factors (edfa_options.ordering):
// the ILU(0) factors of P_a A P_a^T (P_a = identity without an ordering of
// A~) and P_s S~ P_s^T; the right-hand sides are read through the orderings,
// C and B enter as P_s C P_a^T and P_a B P_s^T, and the last sweep of each
// block writes its result back to the natural numbering:
//   y    = A_o^{-1} P_a r_pi
//   z_o  = S_o^{-1} (P_s r_p - C_o y),      z_p  = P_s^T z_o
//   v    = A_o^{-1} (P_a r_pi - B_o z_o),   z_pi = P_a^T v
template <class T>
static int apply_ordered(edfa_handle_s* h, const double* r, double* z, cudaStream_t s)
{
    const int32_t Nf = h->Nf;
    const bool oa = h->oa.on != 0;
    const int32_t* ap = oa ? h->oa.perm : nullptr;
    const int32_t* sp = h->os.perm;
    T* u1 = (T*)h->tmp1;
    T* u2 = (T*)h->tmp2;
    T* zo = (T*)h->tmp3;
    const T* cval;
    const T* bval;
    if constexpr (sizeof(T) == 8) { cval = (const T*)h->co.v64; bval = (const T*)h->bo.v64; }
    else { cval = (const T*)h->co.v32; bval = (const T*)h->bo.v32; }
    const T* none = nullptr;
    int rc;
    if (h->opt.variant == 0) {
        rc = oa ? mc_sweep<T, double, T, 1>(h, h->fa, h->oa, r, ap, nullptr, nullptr, none, 0, none, u2, nullptr,
                                           nullptr, s)
                : a_sweep<T, double, T, 1>(h, r, nullptr, nullptr, none, none, u2, s);
        if (rc) return rc;
        rc = oa ? mc_sweep<T, T, T, 0>(h, h->fa, h->oa, (const T*)u2, nullptr, nullptr, nullptr, none, 0, none, u1,
                                      nullptr, nullptr, s)
                : a_sweep<T, T, T, 0>(h, u2, nullptr, nullptr, none, none, u1, s);
        if (rc) return rc;
        rc = mc_sweep<T, double, T, 1>(h, h->fs, h->os, r + Nf, sp, h->co.ptr, h->co.col, cval, h->co.nnz,
                                       (const T*)u1, u2, nullptr, nullptr, s);
    } else {
        rc = mc_sweep<T, double, T, 1>(h, h->fs, h->os, r + Nf, sp, nullptr, nullptr, none, 0, none, u2, nullptr,
                                       nullptr, s);
    }
    if (rc) return rc;
    rc = mc_sweep<T, T, T, 0>(h, h->fs, h->os, (const T*)u2, nullptr, nullptr, nullptr, none, 0, none, zo, sp,
                              z + Nf, s);
    if (rc) return rc;
    rc = oa ? mc_sweep<T, double, T, 1>(h, h->fa, h->oa, r, ap, h->bo.ptr, h->bo.col, bval, h->bo.nnz,
                                       (const T*)zo, u2, nullptr, nullptr, s)
            : a_sweep<T, double, T, 1>(h, r, h->bo.ptr, h->bo.col, bval, (const T*)zo, u2, s);
    if (rc) return rc;
    if (oa) rc = mc_sweep<T, T, T, 0>(h, h->fa, h->oa, (const T*)u2, nullptr, nullptr, nullptr, none, 0, none, u1, ap,
                                      z, s);
    else rc = a_sweep<T, T, double, 0>(h, u2, nullptr, nullptr, none, (const double*)nullptr, z, s);
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// The same application with r and z in the ordered numbering,
// r = [P_a r_pi; P_s r_p] and z = [P_a z_pi; P_s z_p]: the sweeps read their
// right-hand sides and write their results in place, with no gather or
// scatter through the permutations.  With both orderings on, the six sweep
// outputs of one application are distinct buffers (tmp2, tmp1, tmp4, z_o,
// tmp5, z), so that all of them can be filled with the all-ones pattern before
// the application starts (`prefilled`: by the Krylov update that precedes it)
// instead of by one memset before every sweep.
template <class T>
static bool ordered_prefill_ok(edfa_handle_s* h)
{
    return h->opt.ordering == 2 && h->oa.on && h->os.on && h->coop_ok && h->tmp4 && h->tmp5;
}

template <class T>
static int apply_ordered_numbering(edfa_handle_s* h, const double* r, double* z, bool prefilled, cudaStream_t s)
{
    const int32_t Nf = h->Nf, Ne = h->Ne;
    const bool oa = h->oa.on != 0;
    if (prefilled && !ordered_prefill_ok<T>(h)) return EDFA_ERR_INVALID;
    const bool pf = prefilled;
    T* u1 = (T*)h->tmp1;
    T* u2 = (T*)h->tmp2;
    // S~ forward and the second A~ forward get buffers of their own when both
    // orderings are on (prefilled applications need six distinct outputs)
    T* us = oa && h->tmp4 ? (T*)h->tmp4 : u2;
    T* ua = oa && h->tmp5 ? (T*)h->tmp5 : u2;
    T* zo;  // z_o in the working precision
    if constexpr (sizeof(T) == 8) zo = (T*)(z + Nf);
    else zo = (T*)h->tmp3;
    const T* cval;
    const T* bval;
    if constexpr (sizeof(T) == 8) { cval = (const T*)h->co.v64; bval = (const T*)h->bo.v64; }
    else { cval = (const T*)h->co.v32; bval = (const T*)h->bo.v32; }
    const T* none = nullptr;
    int rc;
    if (h->opt.variant == 0) {
        rc = oa ? mc_sweep<T, double, T, 1>(h, h->fa, h->oa, r, nullptr, nullptr, nullptr, none, 0, none, u2, nullptr,
                                           nullptr, s, pf)
                : a_sweep<T, double, T, 1>(h, r, nullptr, nullptr, none, none, u2, s);
        if (rc) return rc;
        rc = oa ? mc_sweep<T, T, T, 0>(h, h->fa, h->oa, (const T*)u2, nullptr, nullptr, nullptr, none, 0, none, u1,
                                      nullptr, nullptr, s, pf)
                : a_sweep<T, T, T, 0>(h, u2, nullptr, nullptr, none, none, u1, s);
        if (rc) return rc;
        rc = mc_sweep<T, double, T, 1>(h, h->fs, h->os, r + Nf, nullptr, h->co.ptr, h->co.col, cval, h->co.nnz,
                                       (const T*)u1, us, nullptr, nullptr, s, pf);
    } else {
        rc = mc_sweep<T, double, T, 1>(h, h->fs, h->os, r + Nf, nullptr, nullptr, nullptr, none, 0, none, us, nullptr,
                                       nullptr, s, pf);
    }
    if (rc) return rc;
    rc = mc_sweep<T, T, T, 0>(h, h->fs, h->os, (const T*)us, nullptr, nullptr, nullptr, none, 0, none, zo, nullptr,
                              nullptr, s, pf);
    if (rc) return rc;
    rc = oa ? mc_sweep<T, double, T, 1>(h, h->fa, h->oa, r, nullptr, h->bo.ptr, h->bo.col, bval, h->bo.nnz,
                                       (const T*)zo, ua, nullptr, nullptr, s, pf)
            : a_sweep<T, double, T, 1>(h, r, h->bo.ptr, h->bo.col, bval, (const T*)zo, ua, s);
    if (rc) return rc;
    const double* dnone = nullptr;
    rc = oa ? mc_sweep<T, T, double, 0>(h, h->fa, h->oa, (const T*)ua, nullptr, nullptr, nullptr, none, 0, dnone, z,
                                       nullptr, nullptr, s, pf)
            : a_sweep<T, T, double, 0>(h, ua, nullptr, nullptr, none, dnone, z, s);
    if constexpr (sizeof(T) == 4) {
        if (rc) return rc;
        rc = to_f64_launch(zo, z + Nf, Ne, s);
    }
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

template <class T>
static int apply_impl(edfa_handle_s* h, const double* r, double* z, cudaStream_t s)
{
    if (h->opt.ordering >= 1) return apply_ordered<T>(h, r, z, s);
    const int32_t Nf = h->Nf, Ne = h->Ne;
    const double* rpi = r;
    const double* rp = r + Nf;
    double* zpi = z;
    double* zp = z + Nf;
    T* u1 = (T*)h->tmp1;  // length Nf
    T* u2 = (T*)h->tmp2;  // length max(Nf, Ne)
    const T* bval;
    const T* cval;
    if constexpr (sizeof(T) == 8) { bval = (const T*)h->B.val; cval = (const T*)h->C.val; }
    else { bval = (const T*)h->b32; cval = (const T*)h->c32; }
    int rc;
    if (h->opt.variant == 0) {
        // y = A~^{-1} r_pi
        rc = a_sweep<T, double, T, 1>(h, rpi, nullptr, nullptr, (const T*)nullptr, (const T*)nullptr, u2, s);
        if (rc) return rc;
        rc = a_sweep<T, T, T, 0>(h, u2, nullptr, nullptr, (const T*)nullptr, (const T*)nullptr, u1, s);
        if (rc) return rc;
    }
    // z_p = U_S^{-1} L_S^{-1} (r_p - C y)   (C y omitted in the upper-triangular variant);
    // the FP64 path writes z_p directly, the FP32 path into a working-precision copy
    T* zpw;
    if constexpr (sizeof(T) == 8) zpw = zp;
    else zpw = (T*)h->tmp3;
    const bool cpl = h->opt.variant == 0;
    if (h->cp.state == 1) {
        rc = s_cluster_solve<T>(h, rp, cpl ? h->C.rowptr : nullptr, cpl ? h->C.col : nullptr, cpl ? cval : nullptr,
                                cpl ? (const T*)u1 : nullptr, zpw, s, prof_begin_pair(h, 4));
        if (rc) return rc;
    } else {
        if (cpl) rc = launch_sweep<T, double, T, 1, EDFA_LPR_S>(h, h->fs, rp, h->C.rowptr, h->C.col, cval, u1, u2, s);
        else rc = launch_sweep<T, double, T, 1, EDFA_LPR_S>(h, h->fs, rp, nullptr, nullptr, (const T*)nullptr, (const T*)nullptr, u2, s);
        if (rc) return rc;
        rc = launch_sweep<T, T, T, 0, EDFA_LPR_S>(h, h->fs, u2, nullptr, nullptr, (const T*)nullptr, (const T*)nullptr, zpw, s);
        if (rc) return rc;
    }
    // v = L_A^{-1} (r_pi - B z_p), z_pi = U_A^{-1} v
    rc = a_sweep<T, double, T, 1>(h, rpi, h->B.rowptr, h->B.col, bval, (const T*)zpw, u2, s);
    if (rc) return rc;
    rc = a_sweep<T, T, double, 0>(h, u2, nullptr, nullptr, (const T*)nullptr, (const double*)nullptr, zpi, s);
    if constexpr (sizeof(T) == 4) {
        if (rc) return rc;
        rc = to_f64_launch(zpw, zp, Ne, s);
    }
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

__global__ void k_f32_to_f64(const float* in, double* out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

int to_f64_launch(const float* in, double* out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return EDFA_OK;
    int64_t g = (n + 255) / 256;
    if (g > 65535) g = 65535;
    (edfa::count_launch(), k_f32_to_f64<<<(unsigned)g, 256, 0, s>>>(in, out, n));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ wait self-test
// The forward sync-free sweep kernel of the S~ factor run on a 2 x 2 unit lower
// triangular system (row 1 depends on row 0) with a level plan that leaves out
// row 0: row 1's bounded wait for x_0 can never end, so it runs to its poll
// budget, records EDFA_ERR_TIMEOUT with detail 1 and the kernel finishes.
static int wait_selftest(cudaStream_t s, long long* detail, float* ms)
{
    constexpr int LPR = EDFA_LPR_S, RPW = 32 / LPR;
    auto fn = k_sweep<double, double, double, 1, LPR, (LPR >= 32 ? 1 : (LPR >= 16 ? 2 : 4))>;
    struct Buf {
        int64_t rowptr[3], diag[2];
        int32_t col[3], perm[RPW];
        double lu[3], base[2], out[2];
        unsigned long long ticket;
        DevErr err;
    } hb{};
    hb.rowptr[0] = 0; hb.rowptr[1] = 1; hb.rowptr[2] = 3;
    hb.col[0] = 0; hb.col[1] = 0; hb.col[2] = 1;
    hb.diag[0] = 0; hb.diag[1] = 2;
    hb.lu[0] = 1.0; hb.lu[1] = 0.5; hb.lu[2] = 1.0;
    hb.base[0] = 1.0; hb.base[1] = 1.0;
    hb.perm[0] = 1;  // the only planned row; row 0 is never computed
    for (int k = 1; k < RPW; ++k) hb.perm[k] = -1;
    memset(hb.out, 0xFF, sizeof hb.out);  // the "not yet computed" pattern
    Buf* db = nullptr;
    if (cudaMalloc((void**)&db, sizeof(Buf)) != cudaSuccess) { cudaGetLastError(); return EDFA_ERR_OOM; }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = EDFA_OK;
    if (cudaMemcpyAsync(db, &hb, sizeof(Buf), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = EDFA_ERR_CUDA;
    if (!rc) {
        cudaEventRecord(e0, s);
        (edfa::count_launch(), fn<<<1, kSweepThreads, 0, s>>>(db->perm, RPW, db->rowptr, db->col, db->lu, db->diag,
                                                                nullptr, db->base, nullptr, nullptr, nullptr,
                                                                nullptr, db->out, &db->ticket, &db->err));
        cudaEventRecord(e1, s);
        DevErr e{};
        cudaMemcpyAsync(&e, &db->err, sizeof(DevErr), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = EDFA_ERR_CUDA;
        else {
            rc = e.code;
            *detail = e.detail;
            cudaEventElapsedTime(ms, e0, e1);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(db);
    return rc;
}

int apply_prec(edfa_handle_s* h, const double* r, double* z, cudaStream_t s)
{
    if (h->opt.precision == 1) return apply_impl<float>(h, r, z, s);
    return apply_impl<double>(h, r, z, s);
}

int apply_prec_ordered_numbering(edfa_handle_s* h, const double* r, double* z, int prefilled, cudaStream_t s)
{
    if (h->opt.ordering < 1) return EDFA_ERR_INVALID;
    if (h->opt.precision == 1) return apply_ordered_numbering<float>(h, r, z, prefilled != 0, s);
    return apply_ordered_numbering<double>(h, r, z, prefilled != 0, s);
}

int ordered_prefill_list(edfa_handle_s* h, double* z, FillList& fl)
{
    fl = FillList{};
    const bool f32 = h->opt.precision == 1;
    if (!(f32 ? ordered_prefill_ok<float>(h) : ordered_prefill_ok<double>(h))) return 0;
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    const int64_t Nf = h->Nf, Ne = h->Ne;
    fl.add(h->tmp2, Nf * (int64_t)esz);  // A~ forward
    fl.add(h->tmp1, Nf * (int64_t)esz);  // A~ backward
    fl.add(h->tmp4, Ne * (int64_t)esz);  // S~ forward
    if (f32) fl.add(h->tmp3, Ne * (int64_t)esz);  // S~ backward (working precision)
    fl.add(h->tmp5, Nf * (int64_t)esz);  // second A~ forward
    fl.add(z, (Nf + (f32 ? 0 : Ne)) * (int64_t)sizeof(double));  // second A~ backward (and S~ backward in FP64)
    return fl.n;
}

}  // namespace edfa

extern "C" int edfa_selftest_wait_timeout(float* ms, edfa_stream stream)
{
    long long detail = -1;
    float t = 0.f;
    int rc = edfa::wait_selftest((cudaStream_t)stream, &detail, &t);
    edfa::set_detail(detail);
    if (ms) *ms = t;
    return rc;
}
