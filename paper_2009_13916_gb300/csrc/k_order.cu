// Multicolour orderings of the inner ILU(0) factorisations (opt-in,
// edfa_options.ordering).  The paper leaves the inner preconditioners and
// their ordering open (Sec. 3, inner preconditioners; Sec. 4 uses incomplete
// factorisations with partial fill-in).  In the natural order the triangular
// solves of ILU(0) are chains of hundreds of dependency levels; after a
// multicolour ordering the rows of one colour depend only on rows of earlier
// colours, so a sweep has at most as many levels as there are colours.
//
// Colouring (Jones & Plassmann 1993) of the graph of M + M^T (an edge {i, j},
// i != j, wherever M_ij or M_ji is stored): vertex v has priority
// SplitMix64-finaliser(v + 1) (Steele, Lea & Flood 2014; a bijection, so no
// ties) and takes the smallest colour not used by its neighbours of higher
// priority.  Rounds: every uncoloured vertex whose higher-priority neighbours
// are all coloured takes its colour; a colour, once written, is final, so
// whatever a round reads (a final colour or "not yet") the result is that
// fixed point, whatever the timing.  Ordering: rows sorted by (colour, index).
// Block variant (edfa_options.s_block = b > 1): the vertices are the blocks of
// b consecutive rows (priority of block + 1; an edge where M + M^T couples two
// blocks), and row r of block B takes colour c(B) b + r - B b, so the rows of
// one colour stay independent and a block keeps its rows' natural order.
// The ordered matrices P M Q^T are built once per pattern with a map to the
// original entries, so new values only need a gather.
#include "internal.cuh"

namespace edfa {

__device__ __forceinline__ unsigned long long jp_priority(int32_t v)
{
    unsigned long long z = ((unsigned long long)v + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------ transpose pattern
__global__ void k_tp_count(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           unsigned long long* cnt)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) atomicAdd(&cnt[col[p]], 1ull);
}

__global__ void k_tp_fill(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          unsigned long long* cursor, int32_t* tcol)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) tcol[atomicAdd(&cursor[col[p]], 1ull)] = (int32_t)r;
}

// ------------------------------------------------------------ colouring rounds
// the priorities, computed once per colouring (a round reads a neighbour's
// priority instead of recomputing its hash)
__global__ void k_jp_prio(int32_t n, unsigned long long* prio)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        prio[i] = jp_priority((int32_t)i);
}

// A group of G lanes examines one vertex v: every lane takes every G-th entry
// of the rows of v in M and in M^T, and the group combines the lanes' findings
// (G consecutive lanes, G a power of two uniform over the warp, group mask gm).
__device__ __forceinline__ bool grp_any(bool x, unsigned gm) { return (__ballot_sync(0xffffffffu, x) & gm) != 0u; }

__device__ __forceinline__ unsigned long long grp_or(unsigned long long x, int G)
{
    for (int o = G / 2; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// The vertices of the colouring are blocks of b consecutive rows (b = 1: the
// rows themselves); the entries of block B's rows are the contiguous range
// rp[B b] .. rp[min(B b + b, n)) of the CSR arrays, and entry u belongs to
// block u / b.

// some neighbouring block of B (in M and M^T) has higher priority and no colour yet
__device__ __forceinline__ bool jp_blocked(int32_t B, unsigned long long pv, const int64_t* rp, const int32_t* cl,
                                           const unsigned long long* prio, const int* colour, int gl, int G, int b,
                                           int32_t n)
{
    const int64_t r0 = (int64_t)B * b, r1 = r0 + b < n ? r0 + b : n;
    for (int64_t p = rp[r0] + gl; p < rp[r1]; p += G) {
        const int32_t U = cl[p] / b;
        if (U != B && __ldcg(colour + U) < 0 && prio[U] > pv) return true;
    }
    return false;
}

// colours below 64 of the higher-priority neighbouring blocks, as a bit set
__device__ __forceinline__ unsigned long long jp_used(int32_t B, unsigned long long pv, const int64_t* rp,
                                                      const int32_t* cl, const unsigned long long* prio,
                                                      const int* colour, int gl, int G, int b, int32_t n)
{
    unsigned long long used = 0ull;
    const int64_t r0 = (int64_t)B * b, r1 = r0 + b < n ? r0 + b : n;
    for (int64_t p = rp[r0] + gl; p < rp[r1]; p += G) {
        const int32_t U = cl[p] / b;
        if (U == B) continue;
        const int c = __ldcg(colour + U);
        if (c >= 0 && c < 64 && prio[U] > pv) used |= 1ull << c;
    }
    return used;
}

__device__ __forceinline__ bool jp_uses(int32_t B, unsigned long long pv, const int64_t* rp, const int32_t* cl,
                                        const unsigned long long* prio, const int* colour, int c, int gl, int G, int b,
                                        int32_t n)
{
    const int64_t r0 = (int64_t)B * b, r1 = r0 + b < n ? r0 + b : n;
    for (int64_t p = rp[r0] + gl; p < rp[r1]; p += G) {
        const int32_t U = cl[p] / b;
        if (U != B && __ldcg(colour + U) == c && prio[U] > pv) return true;
    }
    return false;
}

// row r of block B: colour c(B) b + r - B b
__global__ void k_block_row_colours(int32_t n, int b, const int* bcolour, int* colour, int* maxcol)
{
    int m = -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = bcolour[i / b] * b + (int)(i % b);
        colour[i] = c;
        m = c > m ? c : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(maxcol, m);
}

__global__ void k_jp_iota(int32_t n, int32_t* wl)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        wl[i] = (int32_t)i;
}

// One round over the worklist of still uncoloured vertices: a vertex whose
// higher-priority neighbours are all coloured takes the smallest colour they
// do not use, the others go to the next round's list (appended a warp at a
// time; the list's order does not matter, the colouring is the greedy one in
// priority order whatever the order of work).  Long lists take one lane per
// vertex (most vertices stop at their first blocking neighbour); short lists,
// the last rounds, where a round lasts as long as its slowest vertex, take 8
// or 32 lanes per vertex, by the mean row length.  The counts rotate over
// three words: round r reads wcnt[r % 3], appends to wcnt[(r + 1) % 3] and
// clears wcnt[(r + 2) % 3] for round r + 1.  A round with an empty list does
// nothing.
__global__ void k_jp_round(const int64_t* __restrict__ rp, const int32_t* __restrict__ cl,
                           const int64_t* __restrict__ tp, const int32_t* __restrict__ tc,
                           const unsigned long long* __restrict__ prio, int* colour, const int32_t* __restrict__ wl_in,
                           int32_t* wl_out, unsigned* wcnt, int r, int gwide, int* maxcol, int b, int32_t n)
{
    const unsigned m = wcnt[r % 3];
    unsigned* out_cnt = wcnt + (r + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) wcnt[(r + 2) % 3] = 0u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int G = (int64_t)m >= nwarps * 32 ? 1 : gwide;  // uniform over the grid
    const int VPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G, gl = lane % G;
    const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (gi * G));
    for (int64_t w0 = warp * VPW; w0 < m; w0 += nwarps * VPW) {
        const int64_t i = w0 + gi;
        const bool live = i < m;
        const int32_t v = live ? wl_in[i] : 0;
        const unsigned long long pv = live ? prio[v] : 0ull;
        bool blk = live && (jp_blocked(v, pv, rp, cl, prio, colour, gl, G, b, n) ||
                            jp_blocked(v, pv, tp, tc, prio, colour, gl, G, b, n));
        blk = grp_any(blk, gm);
        const bool go = live && !blk;
        unsigned long long used = 0ull;
        if (go) used = jp_used(v, pv, rp, cl, prio, colour, gl, G, b, n) | jp_used(v, pv, tp, tc, prio, colour, gl, G, b, n);
        used = grp_or(used, G);
        int c = 0;
        if (go) {
            if (~used != 0ull) c = __ffsll((long long)~used) - 1;
            else c = 64;
        }
        // the rare vertex whose higher-priority neighbours hold all colours
        // below 64 (every lane of the warp takes part in the group votes)
        bool more = go && c >= 64;
        while (__any_sync(0xffffffffu, more)) {
            bool hit = more && (jp_uses(v, pv, rp, cl, prio, colour, c, gl, G, b, n) ||
                                jp_uses(v, pv, tp, tc, prio, colour, c, gl, G, b, n));
            hit = grp_any(hit, gm);
            if (more && hit) ++c;
            else more = false;
        }
        if (go && gl == 0) {
            atomicMax(maxcol, c);
            __stcg(colour + v, c);
        }
        const bool defer = live && blk && gl == 0;
        const unsigned bal = __ballot_sync(0xffffffffu, defer);
        if (bal) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(out_cnt, (unsigned)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (defer) wl_out[base + __popc(bal & ((1u << lane) - 1u))] = v;
        }
    }
}

// ------------------------------------------------------------ rows sorted by (colour, index)
constexpr int kOrdChunk = 1024;  // vertices per block in the placement kernels
constexpr int kOrdMaxColours = 256;

// cnt[c * nchunks + b] = vertices of colour c in chunk b
__global__ void __launch_bounds__(kOrdChunk) k_col_chunk_count(int32_t n, const int* colour, int ncol, int64_t nchunks,
                                                              int64_t* cnt)
{
    __shared__ int h[kOrdMaxColours];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kOrdChunk + threadIdx.x;
    if (v < n) atomicAdd(&h[colour[v]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) cnt[(int64_t)c * nchunks + blockIdx.x] = h[c];
}

// every vertex goes to position offset(colour, chunk) + (vertices of its colour
// before it in the chunk); the rank inside the chunk is counted per warp
// (matching lanes before it) plus the earlier warps' counts of that colour
__global__ void __launch_bounds__(kOrdChunk) k_col_chunk_place(int32_t n, const int* colour, int ncol, int64_t nchunks,
                                                              const int64_t* off, int32_t* perm, int32_t* iperm)
{
    __shared__ int wc[kOrdChunk / 32][kOrdMaxColours];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kOrdChunk / 32) * ncol; k += blockDim.x) wc[k / ncol][k % ncol] = 0;
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kOrdChunk + threadIdx.x;
    const bool live = v < n;
    const int c = live ? colour[v] : -1 - lane;  // distinct dummies never match a colour
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int rank = __popc(same & ((1u << lane) - 1u));
    if (live && rank == 0) wc[w][c] = __popc(same);
    __syncthreads();
    if (live) {
        int before = 0;
        for (int k = 0; k < w; ++k) before += wc[k][c];
        const int64_t pos = off[(int64_t)c * nchunks + blockIdx.x] + before + rank;
        perm[pos] = (int32_t)v;
        iperm[v] = (int32_t)pos;
    }
}

// exclusive scan of the (colour-major) chunk counts, in one block
__global__ void k_col_offsets(int64_t m, int64_t* a)
{
    __shared__ long long part[1024];
    const int64_t per = (m + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = b + per < m ? b + per : m;
    long long s = 0;
    for (int64_t i = b; i < e; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (unsigned k = 0; k < blockDim.x; ++k) {
            long long t = part[k];
            part[k] = run;
            run += t;
        }
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        long long t = a[i];
        a[i] = run;
        run += t;
    }
}

// first ordered row of every colour (the offset of its first chunk)
__global__ void k_col_starts(int ncol, int64_t nchunks, const int64_t* off, int32_t* starts)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncol) starts[c] = (int32_t)off[(int64_t)c * nchunks];
}

// ------------------------------------------------------------ P M Q^T patterns
// row lengths of the permuted matrix: new row k is old row rperm[k]
__global__ void k_perm_len(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ rperm,
                           int64_t* len)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = rperm ? rperm[k] : (int32_t)k;
        len[k] = rowptr[r + 1] - rowptr[r];
    }
}

constexpr int kPermWarps = 4;
constexpr int kPermRowCache = 1024;  // columns of a row cached in shared memory per warp

// one warp per new row: columns renamed through cmap (old column -> new), and
// every entry placed at its rank among the row's new columns (distinct), so
// the row comes out sorted; map[pos] = position of the entry in the original
__global__ void __launch_bounds__(kPermWarps * 32) k_perm_fill(int32_t n, const int64_t* __restrict__ rowptr,
                                                               const int32_t* __restrict__ col,
                                                               const int32_t* __restrict__ rperm,
                                                               const int32_t* __restrict__ cmap,
                                                               const int64_t* __restrict__ nptr, int32_t* ncol,
                                                               int64_t* nmap)
{
    __shared__ int32_t cache[kPermWarps][kPermRowCache];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t k = (int64_t)blockIdx.x * kPermWarps + w; k < n; k += (int64_t)gridDim.x * kPermWarps) {
        const int32_t r = rperm ? rperm[k] : (int32_t)k;
        const int64_t b = rowptr[r], e = rowptr[r + 1];
        const int len = (int)(e - b);
        const bool cached = len <= kPermRowCache;
        if (cached)
            for (int q = lane; q < len; q += 32) cache[w][q] = cmap ? cmap[col[b + q]] : col[b + q];
        __syncwarp();
        for (int q = lane; q < len; q += 32) {
            const int32_t c = cached ? cache[w][q] : (cmap ? cmap[col[b + q]] : col[b + q]);
            int rank = 0;
            for (int t = 0; t < len; ++t) {
                const int32_t ct = cached ? cache[w][t] : (cmap ? cmap[col[b + t]] : col[b + t]);
                rank += ct < c;
            }
            ncol[nptr[k] + rank] = c;
            nmap[nptr[k] + rank] = b + q;
        }
        __syncwarp();
    }
}

template <class TI, class TO>
__global__ void k_gather_vals(int64_t n, const int64_t* __restrict__ map, const TI* __restrict__ in, TO* out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (TO)in[map[k]];
}

static unsigned grid_for(edfa_handle_s* h, int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)h->nsm * 32;
    if (g > cap) g = cap;
    return (unsigned)(g > 0 ? g : 1);
}

// ------------------------------------------------------------ host side
int order_colour(edfa_handle_s* h, Ordering& o, int32_t n, const int64_t* rowptr, const int32_t* col, int64_t nnz,
                 cudaStream_t s, int32_t block)
{
    const int b = block > 1 ? block : 1;
    o.on = 0;
    o.n = n;
    o.ncolours = 0;
    int rc;
    if ((rc = dalloc_t(h, &o.perm, (size_t)(n > 0 ? n : 1)))) return rc;
    if ((rc = dalloc_t(h, &o.iperm, (size_t)(n > 0 ? n : 1)))) return rc;
    if (n == 0) {
        o.on = 1;
        o.cstart.assign(1, 0);
        if ((rc = dalloc_t(h, &o.cstart_dev, 1))) return rc;
        cudaMemsetAsync(o.cstart_dev, 0, sizeof(int32_t), s);
        return EDFA_OK;
    }
    // transpose pattern (rows unordered), colours, counters
    int64_t *tp = nullptr, *cur = nullptr, *cnt = nullptr;
    int32_t* tc = nullptr;
    int* colour = nullptr;
    int* bcolour = nullptr;  // colours of the blocks (b > 1; the row colours follow from them)
    unsigned long long* misc = nullptr;  // [0] vertices left uncoloured by a round, [1] max colour (int)
    unsigned long long* prio = nullptr;
    int32_t* wl = nullptr;  // [2 n] worklists of uncoloured vertices
    unsigned* wcnt = nullptr;  // [3] their lengths, rotating
    auto done = [&](int code) {
        cudaFreeAsync(tp, s); cudaFreeAsync(cur, s); cudaFreeAsync(tc, s); cudaFreeAsync(colour, s);
        cudaFreeAsync(misc, s); cudaFreeAsync(cnt, s); cudaFreeAsync(prio, s); cudaFreeAsync(wl, s);
        cudaFreeAsync(wcnt, s);
        if (bcolour) cudaFreeAsync(bcolour, s);
        return code;
    };
    const int32_t nb = (int32_t)(((int64_t)n + b - 1) / b);  // vertices of the colouring
    if (cudaMallocAsync((void**)&tp, ((size_t)n + 1) * sizeof(int64_t), s) != cudaSuccess ||
        cudaMallocAsync((void**)&cur, ((size_t)n + 1) * sizeof(int64_t), s) != cudaSuccess ||
        cudaMallocAsync((void**)&tc, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t), s) != cudaSuccess ||
        cudaMallocAsync((void**)&colour, (size_t)n * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&misc, 2 * sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMallocAsync((void**)&prio, (size_t)nb * sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMallocAsync((void**)&wl, (size_t)2 * nb * sizeof(int32_t), s) != cudaSuccess ||
        cudaMallocAsync((void**)&wcnt, 3 * sizeof(unsigned), s) != cudaSuccess ||
        (b > 1 && cudaMallocAsync((void**)&bcolour, (size_t)nb * sizeof(int), s) != cudaSuccess)) {
        cudaGetLastError();
        return done(EDFA_ERR_OOM);
    }
    cudaMemsetAsync(tp, 0, ((size_t)n + 1) * sizeof(int64_t), s);
    const unsigned g = grid_for(h, n);
    (edfa::count_launch(), k_tp_count<<<g, 256, 0, s>>>(n, rowptr, col, (unsigned long long*)tp));
    if ((rc = scan_i64(h, tp, n, s))) return done(rc);
    cudaMemcpyAsync(cur, tp, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    (edfa::count_launch(), k_tp_fill<<<g, 256, 0, s>>>(n, rowptr, col, (unsigned long long*)cur, tc));
    int* vcol = b > 1 ? bcolour : colour;  // colours of the vertices of the colouring
    (edfa::count_launch(), k_jp_prio<<<g, 256, 0, s>>>(nb, prio));
    cudaMemsetAsync(vcol, 0xFF, (size_t)nb * sizeof(int), s);
    cudaMemsetAsync(misc, 0, 2 * sizeof(unsigned long long), s);
    // rounds until a round leaves no vertex uncoloured; every round colours at
    // least the uncoloured vertex of highest priority, so n rounds always end it
    (edfa::count_launch(), k_jp_iota<<<g, 256, 0, s>>>(nb, wl));
    {
        const unsigned init[3] = {(unsigned)nb, 0u, 0u};
        cudaMemcpyAsync(wcnt, init, sizeof init, cudaMemcpyHostToDevice, s);
    }
    int64_t rounds = 0;
    int per_check = 8;
    unsigned left = 1;
    const unsigned gr = grid_for(h, nb, 128);
    // lanes per vertex from the mean number of entries of its rows in M and M^T
    const bool wide = nb > 0 && 2.0 * (double)nnz / (double)nb > 48.0;
    while (left > 0) {
        if (rounds > (int64_t)nb + 1) return done(EDFA_ERR_TIMEOUT);
        for (int k = 0; k < per_check; ++k, ++rounds) {
            const int32_t* win = wl + (rounds & 1) * (int64_t)nb;
            int32_t* wout = wl + ((rounds + 1) & 1) * (int64_t)nb;
            (edfa::count_launch(), k_jp_round<<<gr, 128, 0, s>>>(rowptr, col, tp, tc, prio, vcol, win, wout, wcnt,
                                                                 (int)(rounds % 3), wide ? 32 : 8, (int*)(misc + 1), b,
                                                                 n));
        }
        if (per_check < 64) per_check *= 2;
        cudaMemcpyAsync(&left, wcnt + rounds % 3, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return done(EDFA_ERR_CUDA);
    }
    if (b > 1) {
        cudaMemsetAsync(misc + 1, 0, sizeof(unsigned long long), s);
        (edfa::count_launch(), k_block_row_colours<<<g, 256, 0, s>>>(n, b, bcolour, colour, (int*)(misc + 1)));
    }
    int maxcol = 0;
    cudaMemcpyAsync(&maxcol, (int*)(misc + 1), sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return done(EDFA_ERR_CUDA);
    const int ncol = maxcol + 1;
    if (ncol > kOrdMaxColours) {
        set_detail(ncol);
        return done(EDFA_ERR_BOUNDS);
    }
    // rows sorted by (colour, index)
    const int64_t nchunks = ((int64_t)n + kOrdChunk - 1) / kOrdChunk;
    if (cudaMallocAsync((void**)&cnt, (size_t)(ncol * nchunks + 1) * sizeof(int64_t), s) != cudaSuccess) {
        cudaGetLastError();
        return done(EDFA_ERR_OOM);
    }
    (edfa::count_launch(), k_col_chunk_count<<<(unsigned)nchunks, kOrdChunk, 0, s>>>(n, colour, ncol, nchunks, cnt));
    (edfa::count_launch(), k_col_offsets<<<1, 1024, 0, s>>>((int64_t)ncol * nchunks, cnt));
    (edfa::count_launch(), k_col_chunk_place<<<(unsigned)nchunks, kOrdChunk, 0, s>>>(n, colour, ncol, nchunks, cnt,
                                                                                      o.perm, o.iperm));
    // colour starts to the host (the colour array is free again: reuse it)
    (edfa::count_launch(), k_col_starts<<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(ncol, nchunks, cnt, colour));
    o.cstart.assign((size_t)ncol + 1, n);
    cudaMemcpyAsync(o.cstart.data(), colour, (size_t)ncol * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return done(EDFA_ERR_CUDA);
    if ((rc = dalloc_t(h, &o.cstart_dev, (size_t)ncol + 1))) return done(rc);
    cudaMemcpyAsync(o.cstart_dev, o.cstart.data(), ((size_t)ncol + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    // row groups per colour for the dataflow sweeps
    {
        std::vector<int64_t> ts((size_t)2 * 4 * (ncol + 1), 0);
        for (int dir = 0; dir < 2; ++dir)
            for (int li = 0; li < 4; ++li) {
                const int rpw = 32 >> li;
                int64_t* t = ts.data() + ((size_t)dir * 4 + li) * (ncol + 1);
                for (int l = 0; l < ncol; ++l) {
                    const int c = dir == 0 ? l : ncol - 1 - l;
                    t[l + 1] = t[l] + ((int64_t)o.cstart[c + 1] - o.cstart[c] + rpw - 1) / rpw;
                }
            }
        if ((rc = dalloc_t(h, &o.tstart_dev, ts.size()))) return done(rc);
        cudaMemcpyAsync(o.tstart_dev, ts.data(), ts.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        // blocks per block colour (every block has a row at position 0)
        o.block = b;
        o.nbcolours = 0;
        o.bstart_dev = nullptr;
        if (b == 4 || b == 8) {
            const int nbc = (ncol + b - 1) / b;
            std::vector<int64_t> bs((size_t)2 * 2 * (nbc + 1), 0);
            for (int dir = 0; dir < 2; ++dir)
                for (int li = 0; li < 2; ++li) {
                    const int bpw = 32 / (b << li);  // blocks per warp with 1 or 2 lanes per row
                    int64_t* t = bs.data() + ((size_t)dir * 2 + li) * (nbc + 1);
                    for (int l = 0; l < nbc; ++l) {
                        const int c = dir == 0 ? l : nbc - 1 - l;
                        const int64_t nblk = (int64_t)o.cstart[(size_t)c * b + 1] - o.cstart[(size_t)c * b];
                        t[l + 1] = t[l] + (nblk + bpw - 1) / bpw;  // tasks of bpw blocks
                    }
                }
            if ((rc = dalloc_t(h, &o.bstart_dev, bs.size()))) return done(rc);
            cudaMemcpyAsync(o.bstart_dev, bs.data(), bs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
            o.nbcolours = nbc;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return done(EDFA_ERR_CUDA);
    }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    h->coop_ok = coop != 0;  // else per-colour launches
    o.on = 1;
    o.ncolours = ncol;
    return done(cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA);
}

int order_matrix(edfa_handle_s* h, OrderedCsr& m, int32_t nrows, const int64_t* rowptr, const int32_t* col,
                 int64_t nnz, const int32_t* rperm, const int32_t* cmap, cudaStream_t s)
{
    m.nnz = nnz;
    int rc;
    if ((rc = dalloc_t(h, &m.ptr, (size_t)nrows + 1))) return rc;
    if ((rc = dalloc_t(h, &m.col, (size_t)(nnz > 0 ? nnz : 1)))) return rc;
    if ((rc = dalloc_t(h, &m.map, (size_t)(nnz > 0 ? nnz : 1)))) return rc;
    m.v64 = nullptr;
    m.v32 = nullptr;
    if (nrows == 0) {
        cudaMemsetAsync(m.ptr, 0, sizeof(int64_t), s);
        return EDFA_OK;
    }
    (edfa::count_launch(), k_perm_len<<<grid_for(h, nrows), 256, 0, s>>>(nrows, rowptr, rperm, m.ptr));
    if ((rc = scan_i64(h, m.ptr, nrows, s))) return rc;
    const int64_t nb = ((int64_t)nrows + kPermWarps - 1) / kPermWarps;
    const unsigned gb = (unsigned)(nb < (int64_t)h->nsm * 64 ? nb : (int64_t)h->nsm * 64);
    (edfa::count_launch(), k_perm_fill<<<gb, kPermWarps * 32, 0, s>>>(nrows, rowptr, col, rperm, cmap, m.ptr, m.col,
                                                                      m.map));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int order_values(edfa_handle_s* h, OrderedCsr& m, const double* src64, const float* src32, cudaStream_t s)
{
    const size_t cap = (size_t)(m.nnz > 0 ? m.nnz : 1);
    int rc;
    const unsigned g = grid_for(h, m.nnz);
    if (src64) {
        if (!m.v64 && (rc = dalloc_t(h, &m.v64, cap))) return rc;
        if (m.nnz > 0) (edfa::count_launch(), k_gather_vals<double, double><<<g, 256, 0, s>>>(m.nnz, m.map, src64, m.v64));
    }
    if (src32) {
        if (!m.v32 && (rc = dalloc_t(h, &m.v32, cap))) return rc;
        if (m.nnz > 0) (edfa::count_launch(), k_gather_vals<float, float><<<g, 256, 0, s>>>(m.nnz, m.map, src32, m.v32));
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ level plans from colours
// The colours of an ordered factor are a valid level schedule: every
// dependency of a row of colour c lies in an earlier colour (forward) or a
// later one (backward), and the rows of a colour are contiguous.  Level l of
// the plan is colour l (forward) or nc - 1 - l (backward), padded to whole
// warps like the plans of the level analysis.
__global__ void k_plan_colours(int64_t nslots, int nlev, const int64_t* __restrict__ loff,
                               const int32_t* __restrict__ cstart, int fwd, int32_t* perm)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nslots; t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nlev - 1;  // last level whose start is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (loff[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int c = fwd ? lo : nlev - 1 - lo;
        const int64_t k = t - loff[lo];
        const int32_t cnt = cstart[c + 1] - cstart[c];
        perm[t] = k < cnt ? (int32_t)(cstart[c] + k) : -1;
    }
}

static int plan_from_colours(edfa_handle_s* h, SweepPlan& plan, const Ordering& o, int fwd, cudaStream_t s)
{
    const int nc = o.ncolours;
    std::vector<int64_t> loff((size_t)nc + 1, 0);
    for (int l = 0; l < nc; ++l) {
        const int c = fwd ? l : nc - 1 - l;
        const int64_t cnt = o.cstart[c + 1] - o.cstart[c];
        loff[l + 1] = loff[l] + (cnt + 31) / 32 * 32;
    }
    plan.nlevels = nc;
    plan.nslots = loff[nc];
    int rc;
    if ((rc = dalloc_t(h, &plan.loff, (size_t)nc + 1))) return rc;
    if ((rc = dalloc_t(h, &plan.perm, (size_t)(plan.nslots > 0 ? plan.nslots : 1)))) return rc;
    const int32_t* cs = o.cstart_dev;
    cudaMemcpyAsync(plan.loff, loff.data(), ((size_t)nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (plan.nslots > 0)
        (edfa::count_launch(), k_plan_colours<<<grid_for(h, plan.nslots), 256, 0, s>>>(plan.nslots, nc, plan.loff, cs,
                                                                                    fwd, plan.perm));
    // the host vector must outlive the copy
    return cudaStreamSynchronize(s) == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// Symbolic factor set-up of an ordered matrix: diagonal positions, longest
// row and value arrays as factor_plan does, with the level plans taken from
// the colours instead of a level analysis.
static int factor_plan_ordered(edfa_handle_s* h, Factor& f, const Ordering& o, int32_t n, int64_t nnz,
                               const int64_t* rowptr, const int32_t* col, cudaStream_t s)
{
    int rc = factor_plan_common(h, f, n, nnz, rowptr, col, s);
    if (rc) return rc;
    f.ord = &o;
    if ((rc = plan_from_colours(h, f.fwd, o, 1, s))) return rc;
    return plan_from_colours(h, f.bwd, o, 0, s);
}

// faces through the face ordering (identity without one), cells through the
// cell ordering: forward out[k] = in[perm[k]], backward out[perm[k]] = in[k]
__global__ void k_order_vec(int32_t Nf, int32_t Ne, const int32_t* __restrict__ ap, const int32_t* __restrict__ sp,
                            const double* __restrict__ in, double* out, int to_ordered)
{
    const int64_t n = (int64_t)Nf + Ne;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t o;
        if (k < Nf) o = ap ? ap[k] : k;
        else o = Nf + sp[k - Nf];
        if (to_ordered) out[k] = in[o];
        else out[o] = in[k];
    }
}

int order_vector(edfa_handle_s* h, const double* in, double* out, int to_ordered, cudaStream_t s)
{
    const int64_t n = (int64_t)h->Nf + h->Ne;
    if (n > 0)
        (edfa::count_launch(), k_order_vec<<<grid_for(h, n), 256, 0, s>>>(h->Nf, h->Ne, h->oa.on ? h->oa.perm : nullptr,
                                                                          h->os.perm, in, out, to_ordered));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// Stage-2 symbolic work with an ordering of S~: the colouring of the
// factorised S~ pattern, P_s S~ P_s^T, the couplings in the ordered numbering
// (P_s C P_a^T for the right-hand side of the S~ sweep, P_a B P_s^T for the
// second A~ sweep; P_a = identity without an ordering of A~), P_s D P_s^T
// (for the block product in the ordered numbering) and the level plans of the
// ordered factor.
int order_stage2_symbolic(edfa_handle_s* h, cudaStream_t s)
{
    int rc;
    const int32_t Ne = h->Ne, Nf = h->Nf;
    if ((rc = order_colour(h, h->os, Ne, h->sf_ptr, h->sf_col, h->sf_nnz, s, h->opt.s_block))) return rc;
    if ((rc = order_matrix(h, h->so, Ne, h->sf_ptr, h->sf_col, h->sf_nnz, h->os.perm, h->os.iperm, s))) return rc;
    const int32_t* ap = h->oa.on ? h->oa.perm : nullptr;
    const int32_t* aip = h->oa.on ? h->oa.iperm : nullptr;
    if ((rc = order_matrix(h, h->co, Ne, h->C.rowptr, h->C.col, h->C.nnz, h->os.perm, aip, s))) return rc;
    if ((rc = order_values(h, h->co, h->C.val, h->c32, s))) return rc;
    if ((rc = order_matrix(h, h->bo, Nf, h->B.rowptr, h->B.col, h->B.nnz, ap, h->os.iperm, s))) return rc;
    if ((rc = order_values(h, h->bo, h->B.val, h->b32, s))) return rc;
    if ((rc = order_matrix(h, h->dord, Ne, h->D.rowptr, h->D.col, h->D.nnz, h->os.perm, h->os.iperm, s))) return rc;
    if ((rc = order_values(h, h->dord, h->D.val, nullptr, s))) return rc;
    // value arrays of the ordered S~ now, inside the symbolic step, so that a
    // pattern rebuilt by a later Stage 2 releases them with the rest of its plan
    const bool f32 = h->opt.precision == 1;
    if ((rc = order_values(h, h->so, f32 ? nullptr : h->sf_val, f32 ? h->sf_val32 : nullptr, s))) return rc;
    h->cp = ClusterPlan{};
    h->cp.state = 0;
    return factor_plan_ordered(h, h->fs, h->os, Ne, h->so.nnz, h->so.ptr, h->so.col, s);
}

// numeric ILU(0) of S~ (ordered when an ordering of S~ is on)
int stage2_numeric(edfa_handle_s* h, cudaStream_t s)
{
    if (h->opt.ordering >= 1) {
        int rc = order_values(h, h->so, h->opt.precision == 1 ? nullptr : h->sf_val,
                              h->opt.precision == 1 ? h->sf_val32 : nullptr, s);
        if (!rc) rc = order_values(h, h->dord, h->D.val, nullptr, s);  // D may have new values
        if (rc) return rc;
        return factor_numeric(h, h->fs, h->so.v64, h->so.v32, s);
    }
    return factor_numeric(h, h->fs, h->sf_val, h->sf_val32, s);
}

// the A~ factor with an ordering of the faces: colouring of A's pattern,
// P_a A P_a^T, its level plans and numeric ILU(0)
int order_a_factor(edfa_handle_s* h, cudaStream_t s)
{
    int rc;
    const int32_t Nf = h->Nf;
    if ((rc = order_colour(h, h->oa, Nf, h->A.rowptr, h->A.col, h->A.nnz, s))) return rc;
    if ((rc = order_matrix(h, h->ao, Nf, h->A.rowptr, h->A.col, h->A.nnz, h->oa.perm, h->oa.iperm, s))) return rc;
    if ((rc = order_values(h, h->ao, h->A.val, h->opt.precision == 1 ? h->a32 : nullptr, s))) return rc;
    if ((rc = factor_plan_ordered(h, h->fa, h->oa, Nf, h->ao.nnz, h->ao.ptr, h->ao.col, s))) return rc;
    return factor_numeric(h, h->fa, h->ao.v64, h->ao.v32, s);
}

}  // namespace edfa
