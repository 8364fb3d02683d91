// Kernels of the outer flexible GMRES (FP64): the block-system SpMV, the
// classical Gram-Schmidt multi-dot / update pair (a second pass when the
// reorthogonalisation test asks for it, decided on the device) and small vector
// operations.  Reductions are two-level with a
// fixed tree, so results do not depend on scheduling.
//
// FP64 on GB300 issues at ~2 FMA/clk/SM (a warp instruction occupies its SM
// sub-partition for ~33 ns), so these kernels use one thread per row /
// element, no shuffle reductions in the inner loops (every FP64 instruction
// does useful work on all 32 lanes), and the dot kernels reduce across warps
// once per block rather than once per vector.
#include "internal.cuh"

namespace edfa {

constexpr int kKT = 256;           // threads per block
constexpr int kChunk = kKT * 8;    // vector elements per block in the dot kernels

// y = [A B; C D] x.  Face rows (A and B) and cell rows (C and D) have their
// own number of lanes per row, LF and LC, from their mean lengths (a face row
// of the channelised workload holds ~5 entries, a full-tensor cell row ~43):
// the first nbf blocks take the face rows, the rest the cell rows.  A warp
// load touches 32 / L rows in L * 8-byte runs; each lane keeps four entries'
// loads in flight, and a log2(L)-step shuffle reduction closes the row.
constexpr int kSpU = 4;

template <int L>
__device__ __forceinline__ double row_dot(const Csr<double>& M, int64_t r, const double* __restrict__ x, int gl,
                                          double acc)
{
    const int64_t b = M.rowptr[r], e = M.rowptr[r + 1];
    for (int64_t p0 = b; p0 < e; p0 += kSpU * L) {
        int c[kSpU];
        double w[kSpU];
#pragma unroll
        for (int u = 0; u < kSpU; ++u) {
            const int64_t p = p0 + gl + u * L;
            c[u] = p < e ? __ldg(M.col + p) : -1;
            w[u] = p < e ? __ldg(M.val + p) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kSpU; ++u)
            if (c[u] >= 0) acc = fma(w[u], x[c[u]], acc);
    }
    return acc;
}

template <int L>
__device__ __forceinline__ void spmv_rows(int64_t r0, int64_t nrows, int64_t t, const Csr<double>& M1,
                                          const double* x1, const Csr<double>& M2, const double* x2, double* y)
{
    const int64_t r = r0 + t / L;
    const int gl = (int)(t % L);
    double acc = 0.0;
    if (r < r0 + nrows) {
        acc = row_dot<L>(M1, r - r0, x1, gl, acc);
        acc = row_dot<L>(M2, r - r0, x2, gl, acc);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (gl == 0 && r < r0 + nrows) y[r] = acc;
}

template <int LF, int LC>
__global__ void __launch_bounds__(kKT)
k_block_spmv(int32_t Nf, int32_t Ne, Csr<double> A, Csr<double> B, Csr<double> C, Csr<double> D,
             const double* __restrict__ x, double* __restrict__ y, int64_t nbf)
{
    const double* xp = x + Nf;
    if ((int64_t)blockIdx.x < nbf)
        spmv_rows<LF>(0, Nf, (int64_t)blockIdx.x * kKT + threadIdx.x, A, x, B, xp, y);
    else
        spmv_rows<LC>(Nf, Ne, ((int64_t)blockIdx.x - nbf) * kKT + threadIdx.x, C, x, D, xp, y);
}

// lanes per row from the mean row length: a row shared by more lanes costs
// log2(lanes) FP64 adds to reduce, and on this part an FP64 instruction costs
// its share of the pipe whatever the number of active lanes
static int lanes_for(double avg) { return avg <= 6.0 ? 1 : avg <= 16.0 ? 2 : avg <= 40.0 ? 4 : 8; }

template <int LF, int LC>
static void spmv_launch(edfa_handle_s* h, const Csr<double>* M, const double* x, double* y, cudaStream_t s)
{
    const int64_t nbf = ((int64_t)h->Nf * LF + kKT - 1) / kKT;
    const int64_t nbc = ((int64_t)h->Ne * LC + kKT - 1) / kKT;
    (edfa::count_launch(), k_block_spmv<LF, LC><<<(unsigned)(nbf + nbc), kKT, 0, s>>>(h->Nf, h->Ne, M[0], M[1], M[2],
                                                                                      M[3], x, y, nbf));
}

template <int LF>
static void spmv_dispatch_c(edfa_handle_s* h, int lc, const Csr<double>* M, const double* x, double* y,
                            cudaStream_t s)
{
    switch (lc) {
    case 1: spmv_launch<LF, 1>(h, M, x, y, s); break;
    case 2: spmv_launch<LF, 2>(h, M, x, y, s); break;
    case 4: spmv_launch<LF, 4>(h, M, x, y, s); break;
    default: spmv_launch<LF, 8>(h, M, x, y, s); break;
    }
}

// y = [A B; C D] x with the four blocks given
static int block_matvec(edfa_handle_s* h, const Csr<double>* M, const double* x, double* y, cudaStream_t s)
{
    int64_t n = (int64_t)h->Nf + h->Ne;
    if (n == 0) return EDFA_OK;
    const int lf = lanes_for(h->Nf > 0 ? (double)(M[0].nnz + M[1].nnz) / h->Nf : 1.0);
    const int lc = lanes_for(h->Ne > 0 ? (double)(M[2].nnz + M[3].nnz) / h->Ne : 1.0);
    switch (lf) {
    case 1: spmv_dispatch_c<1>(h, lc, M, x, y, s); break;
    case 2: spmv_dispatch_c<2>(h, lc, M, x, y, s); break;
    case 4: spmv_dispatch_c<4>(h, lc, M, x, y, s); break;
    default: spmv_dispatch_c<8>(h, lc, M, x, y, s); break;
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int matvec(edfa_handle_s* h, const double* x, double* y, cudaStream_t s)
{
    const Csr<double> M[4] = {csr_of(h->A), csr_of(h->B), csr_of(h->C), csr_of(h->D)};
    return block_matvec(h, M, x, y, s);
}

// the same product with x and y in the numbering of an ordered handle (faces
// through the face ordering, identity without one; cells through the cell
// ordering): the blocks P_a A P_a^T, P_a B P_s^T, P_s C P_a^T, P_s D P_s^T
int matvec_ordered_numbering(edfa_handle_s* h, const double* x, double* y, cudaStream_t s)
{
    const int32_t Nf = h->Nf, Ne = h->Ne;
    const Csr<double> A = h->oa.on ? Csr<double>{Nf, Nf, h->ao.nnz, h->ao.ptr, h->ao.col, h->ao.v64} : csr_of(h->A);
    const Csr<double> M[4] = {A, Csr<double>{Nf, Ne, h->bo.nnz, h->bo.ptr, h->bo.col, h->bo.v64},
                              Csr<double>{Ne, Nf, h->co.nnz, h->co.ptr, h->co.col, h->co.v64},
                              Csr<double>{Ne, Ne, h->dord.nnz, h->dord.ptr, h->dord.col, h->dord.v64}};
    return block_matvec(h, M, x, y, s);
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[kKT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kKT / 32 ? ws[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// part[i * nchunks + chunk] = V_i[chunk] . w[chunk] for i < nv; when with_self,
// part[nv * nchunks + chunk] = w[chunk] . w[chunk].  Each thread keeps its
// kPer elements of w in registers and takes eight vectors at a time (8 kPer
// independent loads in flight); a transposed butterfly reduces the eight dot
// products across the warp with 9 FP64 adds (instead of 8 x 5 for separate
// reductions; the FP64 pipe of this part makes every add count), and the
// cross-warp sums of all vectors are formed once at the end.  When gate is non-null and *gate == 0 the kernel does nothing (the
// second Gram-Schmidt pass was found unnecessary on the device).
constexpr int kPer = kChunk / kKT;
constexpr int kMaxVec = 128;

__global__ void __launch_bounds__(kKT)
k_multidot(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w, int64_t n,
           double* part, int nchunks, int with_self, const int* gate)
{
    __shared__ double wp[kMaxVec][kKT / 32];
    if (gate && *gate == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    double wr[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) wr[k] = base + (int64_t)k * kKT < n ? w[base + (int64_t)k * kKT] : 0.0;
    const int nt = nv + with_self;
    for (int i0 = 0; i0 < nt; i0 += 8) {
        double a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            a[j] = 0.0;
            const int i = i0 + j;
            if (i < nv) {
                const double* vi = V + (int64_t)i * ld + base;
#pragma unroll
                for (int k = 0; k < kPer; ++k)
                    if (base + (int64_t)k * kKT < n) a[j] = fma(__ldg(vi + (int64_t)k * kKT), wr[k], a[j]);
            } else if (i < nt) {
#pragma unroll
                for (int k = 0; k < kPer; ++k) a[j] = fma(wr[k], wr[k], a[j]);
            }
        }
        // transposed butterfly over eight vectors (9 FP64 adds): the lower half
        // of the warp keeps vectors 0-3, the upper 4-7; then bit 3 of the lane
        // halves that again, then bit 2; the last two steps sum within quads
        const bool up = lane >= 16;
        double b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            b[q] = (up ? a[4 + q] : a[q]) + __shfl_xor_sync(0xffffffffu, up ? a[q] : a[4 + q], 16);
        const bool h8 = (lane & 8) != 0;
        const double c0 = (h8 ? b[2] : b[0]) + __shfl_xor_sync(0xffffffffu, h8 ? b[0] : b[2], 8);
        const double c1 = (h8 ? b[3] : b[1]) + __shfl_xor_sync(0xffffffffu, h8 ? b[1] : b[3], 8);
        const bool h4 = (lane & 4) != 0;
        double d = (h4 ? c1 : c0) + __shfl_xor_sync(0xffffffffu, h4 ? c0 : c1, 4);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        const int v = i0 + (up ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
        if ((lane & 3) == 0 && v < nt) wp[v][wid] = d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += kKT) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kKT / 32; ++q) t += wp[i][q];
        part[(int64_t)i * nchunks + blockIdx.x] = t;
    }
}

// out[i] = sum_c part[i * nchunks + c] in a fixed order; when add != null also
// out_sum[i] = add[i] + out[i].  With a gate reading 0 the parts are not
// summed: out[i] = 0 and out_sum[i] = add[i] (a skipped second pass), and a
// norm request (add == null, out_sum == null) leaves out untouched.
__global__ void __launch_bounds__(kKT)
k_reduce_parts(const double* part, int nchunks, double* out, const double* add, double* out_sum, const int* gate)
{
    const int i = blockIdx.x;
    if (gate && *gate == 0) {
        if (threadIdx.x == 0 && add) {
            out[i] = 0.0;
            out_sum[i] = add[i];
        }
        return;
    }
    double acc = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += kKT) acc += part[(int64_t)i * nchunks + c];
    double t = block_sum(acc);
    if (threadIdx.x == 0) {
        out[i] = t;
        if (add) out_sum[i] = add[i] + t;
    }
}

// Reorthogonalisation test (Rutishauser's criterion, the DGKS test of Daniel,
// Gragg, Kaufman & Stewart 1976 with the factor 10): a second classical
// Gram-Schmidt pass runs when the first one shrank the norm by more than a
// factor of 10, ||w1|| < ||w|| / 10.  With the DGKS factor 1/sqrt(2) the second
// pass ran in almost every iteration of these solves; with 10 it runs in a few
// per cent, the FP64 work of the orthogonalisation halves and the iteration
// counts stay those of modified Gram-Schmidt.
__global__ void k_dgks(const double* nrm2_after, const double* nrm2_before, int* gate)
{
    if (threadIdx.x == 0) *gate = (*nrm2_after < 0.01 * *nrm2_before) ? 1 : 0;
}

// v = alpha * w
__global__ void k_scale_const(const double* w, double* v, int64_t n, double alpha)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = alpha * w[e];
}

// w -= sum_i h_i V_i ; optional partial squared norm of the result.  kPer
// independent elements per thread: one coalesced load per element and vector,
// kPer independent FMA chains
// the all-ones pattern into the buffers of fl, grid-stride over their words
__device__ __forceinline__ void fill_words(const FillList& fl)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int b = 0; b < fl.n; ++b)
        for (int64_t q = t0; q < fl.words[b]; q += stride) fl.p[b][q] = 0xFFFFFFFFu;
}

__global__ void k_fill(FillList fl) { fill_words(fl); }

__global__ void __launch_bounds__(kKT)
k_update(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ hcoef, double* w, int64_t n,
         double* part_norm, const int* gate, FillList fill)
{
    __shared__ double sh[kMaxVec];
    if (gate && *gate == 0) return;
    // the fill stores go out first: they overlap the FP64-bound update
    fill_words(fill);
    for (int i = threadIdx.x; i < nv && i < kMaxVec; i += kKT) sh[i] = -hcoef[i];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    double v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) v[k] = base + (int64_t)k * kKT < n ? w[base + (int64_t)k * kKT] : 0.0;
    for (int i = 0; i < nv; ++i) {
        const double hi = sh[i];
        const double* vi = V + (int64_t)i * ld + base;
#pragma unroll
        for (int k = 0; k < kPer; ++k)
            if (base + (int64_t)k * kKT < n) v[k] = fma(hi, __ldg(vi + (int64_t)k * kKT), v[k]);
    }
    double nacc = 0.0;
#pragma unroll
    for (int k = 0; k < kPer; ++k)
        if (base + (int64_t)k * kKT < n) {
            w[base + (int64_t)k * kKT] = v[k];
            nacc = fma(v[k], v[k], nacc);
        }
    if (part_norm) {
        double t = block_sum(nacc);
        if (threadIdx.x == 0) part_norm[blockIdx.x] = t;
    }
}

// v = w / nrm  where nrm = sqrt(*nrm2) is also stored into *out_norm; the
// square root and the reciprocal (multi-instruction FP64 sequences) are taken
// once per block, not once per thread
__global__ void k_scale_from(const double* w, double* v, int64_t n, const double* nrm2, double* out_norm)
{
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        const double nr = sqrt(*nrm2);
        if (blockIdx.x == 0 && out_norm) *out_norm = nr;
        s_inv = nr > 0.0 ? 1.0 / nr : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = w[e] * inv;
}

// x += sum_i y_i Z_i
__global__ void __launch_bounds__(kKT)
k_combine(const double* __restrict__ Z, int64_t ld, int k, const double* __restrict__ y, double* x, int64_t n)
{
    __shared__ double sy[128];
    for (int i = threadIdx.x; i < k && i < 128; i += kKT) sy[i] = y[i];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double v = x[e];
        for (int i = 0; i < k; ++i) v = fma(sy[i], __ldg(Z + (int64_t)i * ld + e), v);
        x[e] = v;
    }
}

// r = b - r (in place), partial squared norms per chunk
__global__ void __launch_bounds__(kKT) k_residual(const double* b, double* r, int64_t n, double* part)
{
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    double acc = 0.0;
    for (int k = threadIdx.x; k < kChunk; k += kKT) {
        int64_t e = base + k;
        if (e >= n) break;
        double v = b[e] - r[e];
        r[e] = v;
        acc = fma(v, v, acc);
    }
    double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ------------------------------------------------------------ Bi-CGStab vectors
// p = r + beta (p - omega v)
__global__ void k_bcg_p(const double* __restrict__ r, double* __restrict__ p, const double* __restrict__ v,
                        double beta, double omega, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = r[e] + beta * (p[e] - omega * v[e]);
}

// s = r - alpha v, partial ||s||^2 per chunk
__global__ void __launch_bounds__(kKT)
k_bcg_s(const double* __restrict__ r, const double* __restrict__ v, double alpha, double* __restrict__ sv, int64_t n,
        double* part)
{
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    double acc = 0.0;
    for (int k = threadIdx.x; k < kChunk; k += kKT) {
        const int64_t e = base + k;
        if (e >= n) break;
        const double x = r[e] - alpha * v[e];
        sv[e] = x;
        acc = fma(x, x, acc);
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// x += alpha ph + omega sh ; r = s - omega t
__global__ void k_bcg_xr(double* __restrict__ x, const double* __restrict__ ph, const double* __restrict__ sh,
                         const double* __restrict__ sv, const double* __restrict__ t, double alpha, double omega,
                         double* __restrict__ r, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        x[e] += alpha * ph[e] + omega * sh[e];
        r[e] = sv[e] - omega * t[e];
    }
}

// x += a y
__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ y, double a, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] += a * y[e];
}

// ------------------------------------------------------------ launchers
struct Kry {
    static int nchunks(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }
};

int kry_multidot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* part, double* out,
                 const double* add, double* out_sum, int with_self, cudaStream_t s, const int* gate)
{
    if (nv + with_self > kMaxVec) return EDFA_ERR_INVALID;
    int nc = Kry::nchunks(n);
    (edfa::count_launch(), k_multidot<<<nc, kKT, 0, s>>>(V, ld, nv, w, n, part, nc, with_self, gate));
    (edfa::count_launch(), k_reduce_parts<<<nv + with_self, kKT, 0, s>>>(part, nc, out, add, out_sum, gate));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_fill(const FillList& fl, cudaStream_t s)
{
    if (fl.n == 0) return EDFA_OK;
    (edfa::count_launch(), k_fill<<<4096, kKT, 0, s>>>(fl));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_update(const double* V, int64_t ld, int nv, const double* hcoef, double* w, int64_t n, double* part,
               double* nrm2_out, cudaStream_t s, const int* gate, const FillList* fill)
{
    if (nv > kMaxVec) return EDFA_ERR_INVALID;
    int nc = Kry::nchunks(n);
    const FillList fl = fill ? *fill : FillList{};
    (edfa::count_launch(), k_update<<<nc, kKT, 0, s>>>(V, ld, nv, hcoef, w, n, nrm2_out ? part : nullptr, gate, fl));
    if (nrm2_out) (edfa::count_launch(), k_reduce_parts<<<1, kKT, 0, s>>>(part, nc, nrm2_out, nullptr, nullptr, gate));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_dgks(const double* nrm2_after, const double* nrm2_before, int* gate, cudaStream_t s)
{
    (edfa::count_launch(), k_dgks<<<1, 32, 0, s>>>(nrm2_after, nrm2_before, gate));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_scale_from(const double* w, double* v, int64_t n, const double* nrm2, double* out_norm, cudaStream_t s)
{
    int64_t g = (n + kKT - 1) / kKT;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    (edfa::count_launch(), k_scale_from<<<(unsigned)g, kKT, 0, s>>>(w, v, n, nrm2, out_norm));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_combine(const double* Z, int64_t ld, int k, const double* y, double* x, int64_t n, cudaStream_t s)
{
    int64_t g = (n + kKT - 1) / kKT;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    (edfa::count_launch(), k_combine<<<(unsigned)g, kKT, 0, s>>>(Z, ld, k, y, x, n));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_residual(const double* b, double* r, int64_t n, double* part, double* nrm2_out, cudaStream_t s)
{
    int nc = Kry::nchunks(n);
    (edfa::count_launch(), k_residual<<<nc, kKT, 0, s>>>(b, r, n, part));
    (edfa::count_launch(), k_reduce_parts<<<1, kKT, 0, s>>>(part, nc, nrm2_out, nullptr, nullptr, nullptr));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_scale_const(const double* w, double* v, int64_t n, double alpha, cudaStream_t s)
{
    int64_t g = (n + kKT - 1) / kKT;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    (edfa::count_launch(), k_scale_const<<<(unsigned)g, kKT, 0, s>>>(w, v, n, alpha));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int64_t kry_part_size(int64_t n, int nvmax) { return (int64_t)Kry::nchunks(n) * (nvmax + 2); }

}  // namespace edfa

namespace edfa {

static unsigned flat_blocks(int64_t n)
{
    int64_t g = (n + kKT - 1) / kKT;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (unsigned)g;
}

int kry_bcg_p(const double* r, double* p, const double* v, double beta, double omega, int64_t n, cudaStream_t s)
{
    (edfa::count_launch(), k_bcg_p<<<flat_blocks(n), kKT, 0, s>>>(r, p, v, beta, omega, n));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_bcg_s(const double* r, const double* v, double alpha, double* sv, int64_t n, double* part, double* nrm2_out,
              cudaStream_t s)
{
    const int nc = Kry::nchunks(n);
    (edfa::count_launch(), k_bcg_s<<<nc, kKT, 0, s>>>(r, v, alpha, sv, n, part));
    (edfa::count_launch(), k_reduce_parts<<<1, kKT, 0, s>>>(part, nc, nrm2_out, nullptr, nullptr, nullptr));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_bcg_xr(double* x, const double* ph, const double* sh, const double* sv, const double* t, double alpha,
               double omega, double* r, int64_t n, cudaStream_t s)
{
    (edfa::count_launch(), k_bcg_xr<<<flat_blocks(n), kKT, 0, s>>>(x, ph, sh, sv, t, alpha, omega, r, n));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_axpy(double* x, const double* y, double a, int64_t n, cudaStream_t s)
{
    (edfa::count_launch(), k_axpy<<<flat_blocks(n), kKT, 0, s>>>(x, y, a, n));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

}  // namespace edfa
