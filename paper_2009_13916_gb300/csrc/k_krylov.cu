// Kernels of the outer flexible GMRES (FP64): the block-system SpMV, the
// classical Gram-Schmidt multi-dot / update pair (applied twice per Arnoldi
// step, CGS2) and small vector operations.  Reductions are two-level with a
// fixed tree, so results do not depend on scheduling.
//
// FP64 on GB300 issues at ~2 FMA/clk/SM, so these kernels use one thread per
// row / element and no shuffle reductions in the inner loops: every FP64
// instruction does useful work on all 32 lanes.
#include "internal.cuh"

namespace edfa {

constexpr int kKT = 256;           // threads per block
constexpr int kChunk = kKT * 8;    // vector elements per block in the dot kernels

// y = [A B; C D] x, one thread per row
__global__ void __launch_bounds__(kKT)
k_block_spmv(int32_t Nf, int32_t Ne, Csr<double> A, Csr<double> B, Csr<double> C, Csr<double> D,
             const double* __restrict__ x, double* __restrict__ y)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= (int64_t)Nf + Ne) return;
    const double* xp = x + Nf;
    double acc = 0.0;
    if (r < Nf) {
        for (int64_t p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) acc = fma(__ldg(A.val + p), x[__ldg(A.col + p)], acc);
        for (int64_t p = B.rowptr[r]; p < B.rowptr[r + 1]; ++p) acc = fma(__ldg(B.val + p), xp[__ldg(B.col + p)], acc);
    } else {
        int64_t e = r - Nf;
        for (int64_t p = C.rowptr[e]; p < C.rowptr[e + 1]; ++p) acc = fma(__ldg(C.val + p), x[__ldg(C.col + p)], acc);
        for (int64_t p = D.rowptr[e]; p < D.rowptr[e + 1]; ++p) acc = fma(__ldg(D.val + p), xp[__ldg(D.col + p)], acc);
    }
    y[r] = acc;
}

int matvec(edfa_handle_s* h, const double* x, double* y, cudaStream_t s)
{
    int64_t n = (int64_t)h->Nf + h->Ne;
    if (n == 0) return EDFA_OK;
    (edfa::count_launch(), k_block_spmv<<<(unsigned)((n + kKT - 1) / kKT), kKT, 0, s>>>(h->Nf, h->Ne, csr_of(h->A), csr_of(h->B),
                                                                  csr_of(h->C), csr_of(h->D), x, y));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
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
// part[nv * nchunks + chunk] = w[chunk] . w[chunk]
__global__ void __launch_bounds__(kKT)
k_multidot(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w, int64_t n,
           double* part, int nchunks, int with_self)
{
    __shared__ double sw[kChunk];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    for (int k = threadIdx.x; k < kChunk; k += kKT) sw[k] = (base + k < n) ? w[base + k] : 0.0;
    __syncthreads();
    for (int i = 0; i < nv + with_self; ++i) {
        const double* vi = (i < nv) ? V + (int64_t)i * ld : nullptr;
        double acc = 0.0;
        for (int k = threadIdx.x; k < kChunk; k += kKT) {
            if (base + k < n) acc = fma(vi ? __ldg(vi + base + k) : sw[k], sw[k], acc);
        }
        double t = block_sum(acc);
        if (threadIdx.x == 0) part[(int64_t)i * nchunks + blockIdx.x] = t;
    }
}

// out[i] = sum_c part[i * nchunks + c] in a fixed order; when add != null also
// out_sum[i] = add[i] + out[i]
__global__ void __launch_bounds__(kKT)
k_reduce_parts(const double* part, int nchunks, double* out, const double* add, double* out_sum)
{
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += kKT) acc += part[(int64_t)i * nchunks + c];
    double t = block_sum(acc);
    if (threadIdx.x == 0) {
        out[i] = t;
        if (add) out_sum[i] = add[i] + t;
    }
}

// v = alpha * w
__global__ void k_scale_const(const double* w, double* v, int64_t n, double alpha)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = alpha * w[e];
}

// w -= sum_i h_i V_i ; optional partial squared norm of the result
__global__ void __launch_bounds__(kKT)
k_update(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ hcoef, double* w, int64_t n,
         double* part_norm)
{
    __shared__ double sh[128];
    for (int i = threadIdx.x; i < nv && i < 128; i += kKT) sh[i] = hcoef[i];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    double nacc = 0.0;
    for (int k = threadIdx.x; k < kChunk; k += kKT) {
        int64_t e = base + k;
        if (e >= n) break;
        double v = w[e];
        for (int i = 0; i < nv; ++i) v = fma(-sh[i], __ldg(V + (int64_t)i * ld + e), v);
        w[e] = v;
        nacc = fma(v, v, nacc);
    }
    if (part_norm) {
        double t = block_sum(nacc);
        if (threadIdx.x == 0) part_norm[blockIdx.x] = t;
    }
}

// v = w / nrm  where nrm = sqrt(*nrm2) is also stored into *out_norm
__global__ void k_scale_from(const double* w, double* v, int64_t n, const double* nrm2, double* out_norm)
{
    double nr = sqrt(*nrm2);
    if (blockIdx.x == 0 && threadIdx.x == 0 && out_norm) *out_norm = nr;
    double inv = nr > 0.0 ? 1.0 / nr : 0.0;
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

// ------------------------------------------------------------ launchers
struct Kry {
    static int nchunks(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }
};

int kry_multidot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* part, double* out,
                 const double* add, double* out_sum, int with_self, cudaStream_t s)
{
    int nc = Kry::nchunks(n);
    (edfa::count_launch(), k_multidot<<<nc, kKT, 0, s>>>(V, ld, nv, w, n, part, nc, with_self));
    (edfa::count_launch(), k_reduce_parts<<<nv + with_self, kKT, 0, s>>>(part, nc, out, add, out_sum));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int kry_update(const double* V, int64_t ld, int nv, const double* hcoef, double* w, int64_t n, double* part,
               double* nrm2_out, cudaStream_t s)
{
    int nc = Kry::nchunks(n);
    (edfa::count_launch(), k_update<<<nc, kKT, 0, s>>>(V, ld, nv, hcoef, w, n, nrm2_out ? part : nullptr));
    if (nrm2_out) (edfa::count_launch(), k_reduce_parts<<<1, kKT, 0, s>>>(part, nc, nrm2_out, nullptr, nullptr));
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
    (edfa::count_launch(), k_reduce_parts<<<1, kKT, 0, s>>>(part, nc, nrm2_out, nullptr, nullptr));
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
