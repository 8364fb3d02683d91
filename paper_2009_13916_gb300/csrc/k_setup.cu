// Input validation, prefix scans, the cell->face pattern B^T and the static
// restriction sets Q^(m) (Sec. 3, Eq. r_r^m; static technique; base pattern
// Q_{A_ppi} = stored columns of row m of A_ppi).
#include <climits>
#include <mutex>

#include "internal.cuh"

namespace edfa {

// ------------------------------------------------------------ validation
// One thread per row: monotone row pointers, columns in range and strictly
// ascending, finite values, and (need_diag) a stored diagonal.
__global__ void k_validate(Csr<double> M, int need_diag, DevErr* err)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > M.nrows) return;
    if (i == 0 && M.rowptr[0] != 0) raise_err(err, EDFA_ERR_INVALID, 0);
    if (i == M.nrows) {
        if (M.rowptr[M.nrows] != M.nnz) raise_err(err, EDFA_ERR_INVALID, M.nrows);
        return;
    }
    int64_t b = M.rowptr[i], e = M.rowptr[i + 1];
    if (e < b || b < 0 || e > M.nnz) { raise_err(err, EDFA_ERR_INVALID, i); return; }
    int prev = -1;
    int has_diag = 0;
    for (int64_t p = b; p < e; ++p) {
        int c = M.col[p];
        double v = M.val[p];
        if (c <= prev || c >= M.ncols || !isfinite(v)) { raise_err(err, EDFA_ERR_INVALID, i); return; }
        if (c == i) has_diag = 1;
        prev = c;
    }
    if (need_diag && !has_diag) raise_err(err, EDFA_ERR_INVALID, i);
}

int launch_validate(edfa_handle_s* h, const edfa_csr& M, int need_diag, cudaStream_t s)
{
    if (M.nrows < 0 || M.ncols < 0 || M.nnz < 0) return EDFA_ERR_INVALID;
    if (M.nrows > 0 && (!M.rowptr || (M.nnz > 0 && (!M.col || !M.val)))) return EDFA_ERR_INVALID;
    int64_t n = (int64_t)M.nrows + 1;
    (edfa::count_launch(), k_validate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(csr_of(M), need_diag, h->err));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* total)
{
    __shared__ long long warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    long long base = wid > 0 ? warp_sums[wid - 1] : 0;
    if (total) *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void k_scan_reduce(const int64_t* in, int64_t n, int64_t* part)
{
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    long long s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    long long tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_parts(int64_t* part, int64_t nparts)
{
    // single block: sequential over chunks of kScanThreads
    long long carry = 0;
    for (int64_t b = 0; b < nparts; b += kScanThreads) {
        int64_t i = b + threadIdx.x;
        long long v = i < nparts ? part[i] : 0;
        long long tot;
        long long ex = block_exclusive_scan(v, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

__global__ void k_scan_apply(int64_t* data, int64_t n, const int64_t* part)
{
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    long long v[kScanItems];
    long long s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        v[k] = i < n ? data[i] : 0;
        s += v[k];
    }
    long long ex = block_exclusive_scan(s, nullptr) + part[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < n) data[i] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) data[n] = part[gridDim.x];
}

int scan_i64(edfa_handle_s* h, int64_t* data, int64_t n, cudaStream_t s)
{
    (void)h;
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb == 0) nb = 1;
    int64_t* part = nullptr;
    if (cudaMallocAsync((void**)&part, (nb + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    (edfa::count_launch(), k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, part));
    (edfa::count_launch(), k_scan_parts<<<1, kScanThreads, 0, s>>>(part, nb));
    (edfa::count_launch(), k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, part));
    cudaFreeAsync(part, s);
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ B^T pattern
__global__ void k_col_count(Csr<double> M, unsigned long long* cnt)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < M.nnz) atomicAdd(&cnt[M.col[p]], 1ull);
}

__global__ void k_col_fill(Csr<double> M, unsigned long long* cursor, int32_t* out_col)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= M.nrows) return;
    for (int64_t p = M.rowptr[r]; p < M.rowptr[r + 1]; ++p) {
        unsigned long long pos = atomicAdd(&cursor[M.col[p]], 1ull);
        out_col[pos] = (int32_t)r;
    }
}

__global__ void k_row_sort(const int64_t* ptr, int32_t* col, int64_t n)
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

int build_bt(edfa_handle_s* h, cudaStream_t s)
{
    const int32_t Ne = h->Ne;
    int rc = dalloc_t(h, &h->bt_ptr, (size_t)Ne + 1);
    if (rc) return rc;
    rc = dalloc_t(h, &h->bt_col, (size_t)(h->B.nnz > 0 ? h->B.nnz : 1));
    if (rc) return rc;
    cudaMemsetAsync(h->bt_ptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    Csr<double> B = csr_of(h->B);
    if (B.nnz > 0)
        (edfa::count_launch(), k_col_count<<<(unsigned)((B.nnz + 255) / 256), 256, 0, s>>>(B, (unsigned long long*)h->bt_ptr));
    rc = scan_i64(h, h->bt_ptr, Ne, s);
    if (rc) return rc;
    unsigned long long* cursor = nullptr;
    if (cudaMallocAsync((void**)&cursor, ((size_t)Ne + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemcpyAsync(cursor, h->bt_ptr, ((size_t)Ne + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (B.nrows > 0) (edfa::count_launch(), k_col_fill<<<(unsigned)((B.nrows + 255) / 256), 256, 0, s>>>(B, cursor, h->bt_col));
    if (Ne > 0) (edfa::count_launch(), k_row_sort<<<(unsigned)((Ne + 255) / 256), 256, 0, s>>>(h->bt_ptr, h->bt_col, Ne));
    cudaFreeAsync(cursor, s);
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ Q sets
constexpr int kQBuf = 256;       // candidate capacity per cell (before de-duplication)
constexpr int kQWarps = 8;       // warps per block

struct QArgs {
    int mode;
    double thresh;
    int32_t Ne;
    Csr<double> A, B, C;
    const int64_t* bt_ptr;
    const int32_t* bt_col;
    const int64_t* gq_ptr;  // given sets
    const int32_t* gq_idx;
    int64_t* cnt;           // pass 0 output [Ne]
    const int64_t* qptr;    // pass 1 input
    int32_t* qidx;          // pass 1 output
    int* qmax;
    DevErr* err;
};

__device__ __forceinline__ void q_append(int* cand, int* ncand, int v)
{
    int pos = atomicAdd(ncand, 1);
    if (pos < kQBuf) cand[pos] = v;
}

template <int PASS>
__global__ void __launch_bounds__(kQWarps * 32) k_qsets(QArgs a)
{
    __shared__ int s_cand[kQWarps][kQBuf];
    __shared__ int s_n[kQWarps];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* cand = s_cand[wid];
    for (int64_t m = (int64_t)blockIdx.x * kQWarps + wid; m < a.Ne; m += (int64_t)gridDim.x * kQWarps) {
        if (lane == 0) s_n[wid] = 0;
        __syncwarp();
        if (a.mode == EDFA_Q_CROW) {
            for (int64_t p = a.C.rowptr[m] + lane; p < a.C.rowptr[m + 1]; p += 32) q_append(cand, &s_n[wid], a.C.col[p]);
        } else if (a.mode == EDFA_Q_GIVEN) {
            int prev = -1;
            for (int64_t p = a.gq_ptr[m] + lane; p < a.gq_ptr[m + 1]; p += 32) {
                int f = a.gq_idx[p];
                if (f < 0 || f >= a.A.nrows) raise_err(a.err, EDFA_ERR_INVALID, m);
                q_append(cand, &s_n[wid], f);
            }
            (void)prev;
        } else {
            int64_t ob = a.bt_ptr[m], oe = a.bt_ptr[m + 1];
            for (int64_t p = ob + lane; p < oe; p += 32) {
                int f = a.bt_col[p];
                q_append(cand, &s_n[wid], f);
                if (a.mode == EDFA_Q_NBR) {
                    for (int64_t q = a.B.rowptr[f]; q < a.B.rowptr[f + 1]; ++q) {
                        int e2 = a.B.col[q];
                        if (e2 == m) continue;
                        for (int64_t t = a.bt_ptr[e2]; t < a.bt_ptr[e2 + 1]; ++t) q_append(cand, &s_n[wid], a.bt_col[t]);
                    }
                } else if (a.mode == EDFA_Q_THRESH) {
                    int64_t rb = a.A.rowptr[f], re = a.A.rowptr[f + 1];
                    double aii = 0.0;
                    for (int64_t q = rb; q < re; ++q)
                        if (a.A.col[q] == f) aii = fabs(a.A.val[q]);
                    for (int64_t q = rb; q < re; ++q)
                        if (fabs(a.A.val[q]) >= a.thresh * aii) q_append(cand, &s_n[wid], a.A.col[q]);
                }
            }
        }
        __syncwarp();
        int n = s_n[wid];
        if (n > kQBuf) {
            if (lane == 0) raise_err(a.err, EDFA_ERR_BOUNDS, m);
            n = kQBuf;
        }
        int n2 = 32;
        while (n2 < n) n2 <<= 1;
        for (int i = n + lane; i < n2; i += 32) cand[i] = INT_MAX;
        __syncwarp();
        // bitonic sort of cand[0..n2)
        for (int k = 2; k <= n2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < n2; i += 32) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        int x = cand[i], y = cand[ixj];
                        bool up = (i & k) == 0;
                        if ((x > y) == up) { cand[i] = y; cand[ixj] = x; }
                    }
                }
                __syncwarp();
            }
        // unique (ascending); candidates are ascending now
        int outpos = 0;
        for (int base = 0; base < n2; base += 32) {
            int i = base + lane;
            int v = cand[i];
            bool first = (i < n) && v != INT_MAX && (i == 0 || cand[i - 1] != v);
            unsigned b = __ballot_sync(0xffffffffu, first);
            if (PASS == 1 && first) a.qidx[a.qptr[m] + outpos + __popc(b & ((1u << lane) - 1u))] = v;
            outpos += __popc(b);
        }
        if (PASS == 0 && lane == 0) {
            a.cnt[m] = outpos;
            atomicMax(a.qmax, outpos);
        }
        __syncwarp();
    }
}

int build_qsets(edfa_handle_s* h, cudaStream_t s)
{
    const int32_t Ne = h->Ne;
    QArgs a{};
    a.mode = h->opt.qmode == EDFA_Q_DYNAMIC ? EDFA_Q_CROW : h->opt.qmode;
    a.thresh = h->opt.thresh;
    a.Ne = Ne;
    a.A = csr_of(h->A);
    a.B = csr_of(h->B);
    a.C = csr_of(h->C);
    a.bt_ptr = h->bt_ptr;
    a.bt_col = h->bt_col;
    a.gq_ptr = h->opt.qptr;
    a.gq_idx = h->opt.qidx;
    a.err = h->err;
    int rc = dalloc_t(h, &h->qptr, (size_t)Ne + 1);
    if (rc) return rc;
    int* qmax = nullptr;
    if (cudaMallocAsync((void**)&qmax, sizeof(int), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemsetAsync(qmax, 0, sizeof(int), s);
    cudaMemsetAsync(h->qptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    a.cnt = h->qptr;
    a.qmax = qmax;
    unsigned grid = (unsigned)((Ne + kQWarps - 1) / kQWarps);
    unsigned cap = (unsigned)h->nsm * 16;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    (edfa::count_launch(), k_qsets<0><<<grid, kQWarps * 32, 0, s>>>(a));
    rc = scan_i64(h, h->qptr, Ne, s);
    if (rc) return rc;
    int64_t tot = 0;
    int qm = 0;
    cudaMemcpyAsync(&tot, h->qptr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&qm, qmax, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(qmax, s);
    rc = check_err(h, s);
    if (rc) return rc;
    h->qtot = tot;
    h->qmax = qm;
    rc = dalloc_t(h, &h->qidx, (size_t)(tot > 0 ? tot : 1));
    if (rc) return rc;
    a.qptr = h->qptr;
    a.qidx = h->qidx;
    (edfa::count_launch(), k_qsets<1><<<grid, kQWarps * 32, 0, s>>>(a));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ FP32 copies
__global__ void k_to_f32(const double* in, float* out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

int to_f32(const double* in, float* out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return EDFA_OK;
    int64_t g = (n + 255) / 256;
    if (g > 65535) g = 65535;
    (edfa::count_launch(), k_to_f32<<<(unsigned)g, 256, 0, s>>>(in, out, n));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

}  // namespace edfa

// ------------------------------------------------------------ no-allocation variant
// edfa_qsets_noalloc: the static restriction sets with all working memory
// taken from one fixed file-scope device array instead of cudaMalloc.  The
// kernels are the ones the handle path uses.
namespace edfa {

static __device__ __align__(256) unsigned char g_qsets_scratch[EDFA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

// device address of the fixed array on the current device (looked up once per device)
static int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EDFA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_qsets_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EDFA_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return EDFA_OK;
}

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// same three kernels as scan_i64, with the block partials in caller storage
static int scan_i64_into(int64_t* data, int64_t n, int64_t* part, cudaStream_t s)
{
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb == 0) nb = 1;
    (edfa::count_launch(), k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, part));
    (edfa::count_launch(), k_scan_parts<<<1, kScanThreads, 0, s>>>(part, nb));
    (edfa::count_launch(), k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, part));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

}  // namespace edfa

extern "C" int edfa_qsets_noalloc(const edfa_csr* A, const edfa_csr* B, const edfa_csr* C, int32_t qmode,
                                  double thresh, int64_t* qptr, int32_t* qidx, int64_t qidx_capacity,
                                  int64_t* qtot, edfa_stream stream)
{
    using namespace edfa;
    set_detail(-1);
    if (!A || !B || !C || !qptr || !qtot || qidx_capacity < 0) return EDFA_ERR_INVALID;
    if (qmode != EDFA_Q_OWN && qmode != EDFA_Q_NBR && qmode != EDFA_Q_CROW && qmode != EDFA_Q_THRESH)
        return EDFA_ERR_INVALID;
    if (qmode == EDFA_Q_THRESH && !(thresh >= 0.0)) return EDFA_ERR_INVALID;
    const int32_t Nf = A->nrows, Ne = B->ncols;
    if (Nf < 0 || Ne < 0 || A->ncols != Nf || B->nrows != Nf || C->nrows != Ne || C->ncols != Nf ||
        A->nnz < 0 || B->nnz < 0 || C->nnz < 0)
        return EDFA_ERR_INVALID;
    // scratch layout, checked against the fixed size before any device work
    const int64_t nb = ((int64_t)Ne + kScanChunk - 1) / kScanChunk + 1;
    const size_t off_btp = 0;
    const size_t off_btc = off_btp + round256(((size_t)Ne + 1) * sizeof(int64_t));
    const size_t off_cur = off_btc + round256((size_t)(B->nnz > 0 ? B->nnz : 1) * sizeof(int32_t));
    const size_t off_part = off_cur + round256(((size_t)Ne + 1) * sizeof(int64_t));
    const size_t off_misc = off_part + round256(((size_t)nb + 1) * sizeof(int64_t));
    const size_t need = off_misc + round256(sizeof(DevErr) + sizeof(int));
    if (need > (size_t)EDFA_NOALLOC_SCRATCH_BYTES) {
        set_detail((long long)need);
        return EDFA_ERR_BOUNDS;
    }
    if ((Nf > 0 && (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val)))) ||
        (Nf > 0 && (!B->rowptr || (B->nnz > 0 && (!B->col || !B->val)))) ||
        (Ne > 0 && (!C->rowptr || (C->nnz > 0 && (!C->col || !C->val)))))
        return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int rc = scratch_address((void**)&base);
    if (rc) return rc;
    int64_t* bt_ptr = (int64_t*)(base + off_btp);
    int32_t* bt_col = (int32_t*)(base + off_btc);
    unsigned long long* cursor = (unsigned long long*)(base + off_cur);
    int64_t* part = (int64_t*)(base + off_part);
    DevErr* err = (DevErr*)(base + off_misc);
    int* qmax = (int*)(base + off_misc + sizeof(DevErr));
    int nsm = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm < 1) nsm = 1;

    // state that must start at zero
    cudaMemsetAsync(base + off_misc, 0, sizeof(DevErr) + sizeof(int), s);
    cudaMemsetAsync(bt_ptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    cudaMemsetAsync(qptr, 0, ((size_t)Ne + 1) * sizeof(int64_t), s);
    // input validation (the checks edfa_build makes: A must store its
    // diagonal), read back before any kernel uses the blocks' indices as
    // addresses
    const edfa_csr* mats[3] = {A, B, C};
    for (int k = 0; k < 3; ++k) {
        int64_t n = (int64_t)mats[k]->nrows + 1;
        (edfa::count_launch(),
         k_validate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(csr_of(*mats[k]), k == 0 ? 1 : 0, err));
    }
    {
        DevErr ve{};
        cudaMemcpyAsync(&ve, err, sizeof(DevErr), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
        if (ve.code != 0) {
            set_detail(ve.detail);
            return ve.code;
        }
    }
    // B^T pattern: the faces of each cell
    Csr<double> Bc = csr_of(*B);
    if (Bc.nnz > 0)
        (edfa::count_launch(), k_col_count<<<(unsigned)((Bc.nnz + 255) / 256), 256, 0, s>>>(Bc, (unsigned long long*)bt_ptr));
    if ((rc = scan_i64_into(bt_ptr, Ne, part, s))) return rc;
    cudaMemcpyAsync(cursor, bt_ptr, ((size_t)Ne + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (Bc.nrows > 0) (edfa::count_launch(), k_col_fill<<<(unsigned)((Bc.nrows + 255) / 256), 256, 0, s>>>(Bc, cursor, bt_col));
    if (Ne > 0) (edfa::count_launch(), k_row_sort<<<(unsigned)((Ne + 255) / 256), 256, 0, s>>>(bt_ptr, bt_col, Ne));
    // counting pass, offsets, total
    QArgs a{};
    a.mode = qmode;
    a.thresh = thresh;
    a.Ne = Ne;
    a.A = csr_of(*A);
    a.B = Bc;
    a.C = csr_of(*C);
    a.bt_ptr = bt_ptr;
    a.bt_col = bt_col;
    a.err = err;
    a.cnt = qptr;
    a.qmax = qmax;
    unsigned grid = (unsigned)((Ne + kQWarps - 1) / kQWarps);
    unsigned cap = (unsigned)nsm * 16;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    (edfa::count_launch(), k_qsets<0><<<grid, kQWarps * 32, 0, s>>>(a));
    if ((rc = scan_i64_into(qptr, Ne, part, s))) return rc;
    int64_t tot = 0;
    DevErr e{};
    cudaMemcpyAsync(&tot, qptr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&e, err, sizeof(DevErr), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
    if (e.code != 0) {
        set_detail(e.detail);
        return e.code;
    }
    *qtot = tot;
    if (tot > qidx_capacity) {
        set_detail(tot);
        return EDFA_ERR_BOUNDS;
    }
    if (tot > 0 && !qidx) return EDFA_ERR_INVALID;
    a.qptr = qptr;
    a.qidx = qidx;
    (edfa::count_launch(), k_qsets<1><<<grid, kQWarps * 32, 0, s>>>(a));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}
