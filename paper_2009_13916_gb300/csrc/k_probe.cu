// Arithmetic-rate probe: the FP64 and FP32 fused multiply-add throughput of the
// device, measured with CUDA events, as the denominator of the ALU roofline of
// the local-solve kernel (the dense per-cell factorisations are FP64-pipe
// bound, not bound by memory).  Not part of the preconditioner.
#include "internal.cuh"

namespace edfa {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

// kProbeChains independent FMA chains per thread, `iters` steps each; the sum
// is stored only under a condition the values never meet, which keeps the
// chains live without a store per thread.
template <class T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T* sink, int iters, T seed)
{
    T a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = seed + (T)(threadIdx.x & 7) + (T)k;
    const T m = (T)0.9999, c = (T)0.0001;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    if (s == (T)-12345.0) sink[0] = s;
}

template <class T>
static int probe(int nsm, int iters, double* rate, cudaStream_t s)
{
    T* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(T)) != cudaSuccess) { cudaGetLastError(); return EDFA_ERR_OOM; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = nsm * kProbeBlocksPerSm;
    (edfa::count_launch(), k_fma_probe<T><<<grid, kProbeThreads, 0, s>>>(sink, iters / 8, (T)1));  // warm-up
    cudaEventRecord(e0, s);
    (edfa::count_launch(), k_fma_probe<T><<<grid, kProbeThreads, 0, s>>>(sink, iters, (T)1));
    cudaEventRecord(e1, s);
    int rc = cudaStreamSynchronize(s) == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
    float ms = 0.f;
    if (!rc) cudaEventElapsedTime(&ms, e0, e1);
    *rate = ms > 0.f ? (double)grid * kProbeThreads * kProbeChains * (double)iters / (ms * 1e-3) : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

}  // namespace edfa

extern "C" int edfa_probe_fma_rate(int32_t precision, double* fma_per_s, edfa_stream stream)
{
    if (!fma_per_s || (precision != 0 && precision != 1)) return EDFA_ERR_INVALID;
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return EDFA_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm < 1) nsm = 1;
    // about 30 ms at the nominal rates of the part (FP64 ~0.6, FP32 ~40 T FMA/s)
    const int iters = precision == 0 ? 16384 : 1 << 20;
    return precision == 0 ? edfa::probe<double>(nsm, iters, fma_per_s, (cudaStream_t)stream)
                          : edfa::probe<float>(nsm, iters, fma_per_s, (cudaStream_t)stream);
}
