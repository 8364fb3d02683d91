// Batched solve: many independent block systems concatenated block-diagonally
// into one handle (one persistent local-solve launch, one S~, one ILU plan over
// all systems), solved by one flexible GMRES(m) per system advanced in lock
// step.  The preconditioner application and the SpMV act on the whole
// block-diagonal system; every reduction is segmented per system (chunks of
// at most kBChunk entries never straddle two systems), and the Hessenberg /
// Givens updates, convergence tests and restarts run on the device, one
// thread per system.  A whole restart cycle (m Arnoldi steps + the solution
// update and true-residual test) is captured once as a CUDA graph and
// replayed until every system has converged or hit maxit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace edfa {

constexpr int kBT = 256;
constexpr int kBChunk = 2048;

struct BState {
    int nsys, m;
    double rtol;
    int maxit;
    // per system
    double *bnorm, *beta, *H, *cs, *sn, *g, *y, *h1, *h2, *hsum, *nrm2, *inv, *rn2, *true_rel;
    int *active, *conv, *kdone, *iters, *flags;  // flags[0] = systems still running
    int* gate;  // second Gram-Schmidt pass of the current step
};

// chunk table
struct BChunks {
    int64_t* start;
    int32_t* len;
    int32_t* sys;
    int64_t* sys_ptr;  // chunks of system i: [sys_ptr[i], sys_ptr[i+1])
    int nchunks;
};

__device__ __forceinline__ double bsum(double v)
{
    __shared__ double ws[kBT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kBT / 32 ? ws[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// part[c * stride + k] = V_k[chunk c] . w[chunk c] (k < nv); with_self adds w.w at k = nv
__global__ void __launch_bounds__(kBT)
k_bdot(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w, BChunks ch,
       const int* __restrict__ active, double* part, int stride, int with_self)
{
    const int c = blockIdx.x;
    const int sys = ch.sys[c];
    const int64_t st = ch.start[c];
    const int len = ch.len[c];
    const bool act = active[sys] != 0;
    if (!act) {  // block-uniform: zero parts without the reductions
        for (int k = threadIdx.x; k < nv + with_self; k += kBT) part[(int64_t)c * stride + k] = 0.0;
        return;
    }
    for (int k = 0; k < nv + with_self; ++k) {
        double acc = 0.0;
        {
            const double* vk = k < nv ? V + (int64_t)k * ld : w;
            for (int e = threadIdx.x; e < len; e += kBT) acc = fma(__ldg(vk + st + e), w[st + e], acc);
        }
        double t = bsum(acc);
        if (threadIdx.x == 0) part[(int64_t)c * stride + k] = t;
    }
}

// out[s * ostride + k] = sum over the system's chunks (fixed order); optional sum with add
__global__ void __launch_bounds__(kBT)
k_breduce(const double* part, int stride, int nk, BChunks ch, double* out, int ostride, const double* add,
          double* out_sum)
{
    const int s = blockIdx.x;
    const int64_t cb = ch.sys_ptr[s], ce = ch.sys_ptr[s + 1];
    for (int k = 0; k < nk; ++k) {
        double acc = 0.0;
        for (int64_t c = cb + threadIdx.x; c < ce; c += kBT) acc += part[c * stride + k];
        double t = bsum(acc);
        if (threadIdx.x == 0) {
            out[(int64_t)s * ostride + k] = t;
            if (add) out_sum[(int64_t)s * ostride + k] = add[(int64_t)s * ostride + k] + t;
        }
    }
}

// w -= sum_k coef[sys][k] V_k on active systems; partial squared norm per chunk
// of the active systems (the parts of the others are left as they are)
__global__ void __launch_bounds__(kBT)
k_bupdate(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ coef, int cstride,
          double* w, BChunks ch, const int* __restrict__ active, double* part_norm)
{
    __shared__ double sc[128];
    const int c = blockIdx.x;
    const int sys = ch.sys[c];
    const bool act = active[sys] != 0;
    for (int k = threadIdx.x; k < nv && k < 128; k += kBT) sc[k] = coef[(int64_t)sys * cstride + k];
    __syncthreads();
    const int64_t st = ch.start[c];
    const int len = ch.len[c];
    double nacc = 0.0;
    if (act) {
        for (int e = threadIdx.x; e < len; e += kBT) {
            double v = w[st + e];
            for (int k = 0; k < nv; ++k) v = fma(-sc[k], __ldg(V + (int64_t)k * ld + st + e), v);
            w[st + e] = v;
            nacc = fma(v, v, nacc);
        }
    }
    if (part_norm && act) {
        double t = bsum(nacc);
        if (threadIdx.x == 0) part_norm[c] = t;
    }
}

// Reorthogonalisation test per system (Rutishauser's criterion, as in the
// single-system solve): a second Gram-Schmidt pass for the active systems whose
// first pass shrank the norm by more than a factor of 10
__global__ void k_bgate(BState S, int nv)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.nsys) return;
    const int hs = S.m + 2;
    S.gate[s] = (S.active[s] && S.nrm2[s] < 0.01 * S.h1[(int64_t)s * hs + nv]) ? 1 : 0;
}

// v = w * inv[sys] (0 on inactive systems)
__global__ void __launch_bounds__(kBT)
k_bscale(const double* w, double* v, BChunks ch, const double* inv, const int* active)
{
    const int c = blockIdx.x;
    const int sys = ch.sys[c];
    const double f = active[sys] ? inv[sys] : 0.0;
    const int64_t st = ch.start[c];
    for (int e = threadIdx.x; e < ch.len[c]; e += kBT) v[st + e] = w[st + e] * f;
}

// Arnoldi column j of every active system: Givens rotations and convergence
__global__ void k_bgivens(BState S, int j)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.nsys || !S.active[s]) return;
    const int m = S.m, hs = m + 2;
    double* H = S.H + (int64_t)s * (m + 1) * m;
    double* cs = S.cs + (int64_t)s * m;
    double* sn = S.sn + (int64_t)s * m;
    double* g = S.g + (int64_t)s * (m + 1);
    const double* h = S.hsum + (int64_t)s * hs;
    const double hn = sqrt(S.nrm2[s]);
    for (int i = 0; i <= j; ++i) H[i * m + j] = h[i];
    H[(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
    }
    const double a = H[j * m + j], c = H[(j + 1) * m + j];
    const double den = sqrt(a * a + c * c);
    cs[j] = den > 0 ? a / den : 1.0;
    sn[j] = den > 0 ? c / den : 0.0;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    S.kdone[s] = j + 1;
    S.iters[s] += 1;
    S.inv[s] = hn > 0 ? 1.0 / hn : 0.0;
    const double est = fabs(g[j + 1]) / S.bnorm[s];
    if (est <= S.rtol || hn == 0.0 || j + 1 == m || S.iters[s] >= S.maxit) S.active[s] = 0;
}

// y = H^{-1} g on the kdone steps of the cycle (systems that were running)
__global__ void k_btri(BState S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.nsys || S.conv[s] || S.kdone[s] == 0) return;
    const int m = S.m, k = S.kdone[s];
    const double* H = S.H + (int64_t)s * (m + 1) * m;
    const double* g = S.g + (int64_t)s * (m + 1);
    double* y = S.y + (int64_t)s * m;
    for (int i = k - 1; i >= 0; --i) {
        double v = g[i];
        for (int l = i + 1; l < k; ++l) v -= H[i * m + l] * y[l];
        y[i] = H[i * m + i] != 0.0 ? v / H[i * m + i] : 0.0;
    }
}

// x += sum_{k < kdone} y_k Z_k on systems that ran in this cycle
__global__ void __launch_bounds__(kBT)
k_bcombine(const double* __restrict__ Z, int64_t ld, double* x, BChunks ch, BState S)
{
    __shared__ double sy[128];
    const int c = blockIdx.x;
    const int sys = ch.sys[c];
    const int k = S.conv[sys] ? 0 : S.kdone[sys];
    for (int i = threadIdx.x; i < k && i < 128; i += kBT) sy[i] = S.y[(int64_t)sys * S.m + i];
    __syncthreads();
    const int64_t st = ch.start[c];
    for (int e = threadIdx.x; e < ch.len[c]; e += kBT) {
        double v = x[st + e];
        for (int i = 0; i < k; ++i) v = fma(sy[i], __ldg(Z + (int64_t)i * ld + st + e), v);
        x[st + e] = v;
    }
}

// r = b - r in place, partial squared norms per chunk
__global__ void __launch_bounds__(kBT) k_bresid(const double* b, double* r, BChunks ch, double* part)
{
    const int c = blockIdx.x;
    const int64_t st = ch.start[c];
    double acc = 0.0;
    for (int e = threadIdx.x; e < ch.len[c]; e += kBT) {
        double v = b[st + e] - r[st + e];
        r[st + e] = v;
        acc = fma(v, v, acc);
    }
    double t = bsum(acc);
    if (threadIdx.x == 0) part[c] = t;
}

// end of a cycle: true residual test, restart of the systems still running
__global__ void k_bcycle_end(BState S, int first)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.nsys) return;
    if (first) {
        S.bnorm[s] = sqrt(S.rn2[s]);
        S.conv[s] = S.bnorm[s] == 0.0;
        S.iters[s] = 0;
        S.true_rel[s] = S.bnorm[s] == 0.0 ? 0.0 : 1.0;
    }
    int run = 0;
    if (!S.conv[s]) {
        const double rn = sqrt(S.rn2[s]);
        S.true_rel[s] = S.bnorm[s] > 0 ? rn / S.bnorm[s] : 0.0;
        if (!first && (S.true_rel[s] <= S.rtol || rn == 0.0)) {
            S.conv[s] = 1;
        } else if (S.iters[s] < S.maxit) {
            run = 1;
            S.beta[s] = rn;
            S.inv[s] = rn > 0 ? 1.0 / rn : 0.0;
            double* g = S.g + (int64_t)s * (S.m + 1);
            for (int i = 0; i <= S.m; ++i) g[i] = 0.0;
            g[0] = rn;
        }
    }
    S.active[s] = run;
    S.kdone[s] = 0;
    if (run) atomicAdd(S.flags, 1);
}

__global__ void k_bclear_flag(int* flags) { flags[0] = 0; }

}  // namespace edfa

using namespace edfa;

namespace {
struct BatchWork {
    int nsys = 0, m = 0;
    int64_t n = 0;
    std::vector<int64_t> fo, co;
    BChunks ch{};
    BState S{};
    double *V = nullptr, *Z = nullptr, *w = nullptr, *part = nullptr;
    double* pnorm = nullptr;  // per-chunk partial squared norms of w
    int pstride = 0;
    cudaGraphExec_t cycle = nullptr;
    cudaGraph_t graph = nullptr;
    const double* b = nullptr;
    double* x = nullptr;
    double rtol = 0;
    int maxit = 0;
};
}  // namespace

static int batch_prepare(edfa_handle_s* h, BatchWork& B, cudaStream_t s)
{
    // chunk table from the system offsets (faces first, then cells)
    std::vector<int64_t> cst;
    std::vector<int32_t> clen, csys;
    std::vector<int64_t> sptr(1, 0);
    for (int i = 0; i < B.nsys; ++i) {
        int64_t segs[2][2] = {{B.fo[i], B.fo[i + 1]}, {h->Nf + B.co[i], h->Nf + B.co[i + 1]}};
        for (auto& sg : segs)
            for (int64_t a = sg[0]; a < sg[1]; a += kBChunk) {
                cst.push_back(a);
                clen.push_back((int32_t)std::min<int64_t>(kBChunk, sg[1] - a));
                csys.push_back(i);
            }
        sptr.push_back((int64_t)cst.size());
    }
    const int nc = (int)cst.size();
    B.ch.nchunks = nc;
    B.pstride = B.m + 2;
    int rc = 0;
    rc |= dalloc_t(h, &B.ch.start, (size_t)std::max(nc, 1));
    rc |= dalloc_t(h, &B.ch.len, (size_t)std::max(nc, 1));
    rc |= dalloc_t(h, &B.ch.sys, (size_t)std::max(nc, 1));
    rc |= dalloc_t(h, &B.ch.sys_ptr, (size_t)B.nsys + 1);
    if (rc) return EDFA_ERR_OOM;
    cudaMemcpyAsync(B.ch.start, cst.data(), nc * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.ch.len, clen.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.ch.sys, csys.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.ch.sys_ptr, sptr.data(), (B.nsys + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    const int m = B.m, ns = B.nsys;
    BState& S = B.S;
    S.nsys = ns;
    S.m = m;
    double** dptrs[] = {&S.bnorm, &S.beta, &S.nrm2, &S.inv, &S.rn2, &S.true_rel};
    for (auto p : dptrs) rc |= dalloc_t(h, p, (size_t)ns);
    rc |= dalloc_t(h, &S.H, (size_t)ns * (m + 1) * m);
    rc |= dalloc_t(h, &S.cs, (size_t)ns * m);
    rc |= dalloc_t(h, &S.sn, (size_t)ns * m);
    rc |= dalloc_t(h, &S.g, (size_t)ns * (m + 1));
    rc |= dalloc_t(h, &S.y, (size_t)ns * m);
    rc |= dalloc_t(h, &S.h1, (size_t)ns * (m + 2));
    rc |= dalloc_t(h, &S.h2, (size_t)ns * (m + 2));
    rc |= dalloc_t(h, &S.hsum, (size_t)ns * (m + 2));
    int** iptrs[] = {&S.active, &S.conv, &S.kdone, &S.iters};
    for (auto p : iptrs) rc |= dalloc_t(h, p, (size_t)ns);
    rc |= dalloc_t(h, &S.flags, 4);
    rc |= dalloc_t(h, &B.V, (size_t)(m + 1) * B.n);
    rc |= dalloc_t(h, &B.Z, (size_t)m * B.n);
    rc |= dalloc_t(h, &B.w, (size_t)B.n);
    rc |= dalloc_t(h, &B.part, (size_t)nc * B.pstride);
    rc |= dalloc_t(h, &B.pnorm, (size_t)nc);
    rc |= dalloc_t(h, &S.gate, (size_t)B.nsys);
    return rc ? EDFA_ERR_OOM : EDFA_OK;
}

// enqueue the segmented reductions of one Arnoldi step j (CGS2)
static int batch_step(edfa_handle_s* h, BatchWork& B, int j, cudaStream_t s)
{
    const int64_t n = B.n;
    const int nc = B.ch.nchunks, ns = B.nsys, hs = B.m + 2;
    double* vj = B.V + (int64_t)j * n;
    double* zj = B.Z + (int64_t)j * n;
    int rc = apply_prec(h, vj, zj, s);
    if (!rc) rc = matvec(h, zj, B.w, s);
    if (rc) return rc;
    const int nv = j + 1;
    BState& S = B.S;
    // first pass (with ||w||^2 in h1[nv]), its squared norm, the per-system
    // test, and the second pass on the systems the test selects: for the
    // others the second dot products are zero (h2 = 0, hsum = h1) and the
    // norm parts of the first pass stay
    (edfa::count_launch(), k_bdot<<<nc, kBT, 0, s>>>(B.V, n, nv, B.w, B.ch, S.active, B.part, B.pstride, 1));
    (edfa::count_launch(), k_breduce<<<ns, kBT, 0, s>>>(B.part, B.pstride, nv + 1, B.ch, S.h1, hs, nullptr, nullptr));
    (edfa::count_launch(), k_bupdate<<<nc, kBT, 0, s>>>(B.V, n, nv, S.h1, hs, B.w, B.ch, S.active, B.pnorm));
    (edfa::count_launch(), k_breduce<<<ns, kBT, 0, s>>>(B.pnorm, 1, 1, B.ch, S.nrm2, 1, nullptr, nullptr));
    (edfa::count_launch(), k_bgate<<<(ns + 127) / 128, 128, 0, s>>>(S, nv));
    (edfa::count_launch(), k_bdot<<<nc, kBT, 0, s>>>(B.V, n, nv, B.w, B.ch, S.gate, B.part, B.pstride, 0));
    (edfa::count_launch(), k_breduce<<<ns, kBT, 0, s>>>(B.part, B.pstride, nv, B.ch, S.h2, hs, S.h1, S.hsum));
    (edfa::count_launch(), k_bupdate<<<nc, kBT, 0, s>>>(B.V, n, nv, S.h2, hs, B.w, B.ch, S.gate, B.pnorm));
    (edfa::count_launch(), k_breduce<<<ns, kBT, 0, s>>>(B.pnorm, 1, 1, B.ch, S.nrm2, 1, nullptr, nullptr));
    (edfa::count_launch(), k_bgivens<<<(ns + 127) / 128, 128, 0, s>>>(S, j));
    (edfa::count_launch(), k_bscale<<<nc, kBT, 0, s>>>(B.w, B.V + (int64_t)(j + 1) * n, B.ch, S.inv, S.active));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// solution update, true residual, restart of the running systems, v0 = r / beta
static int batch_cycle_end(edfa_handle_s* h, BatchWork& B, int first, cudaStream_t s)
{
    const int nc = B.ch.nchunks, ns = B.nsys;
    BState& S = B.S;
    int rc = EDFA_OK;
    if (!first) {
        (edfa::count_launch(), k_btri<<<(ns + 127) / 128, 128, 0, s>>>(S));
        (edfa::count_launch(), k_bcombine<<<nc, kBT, 0, s>>>(B.Z, B.n, B.x, B.ch, S));
        rc = matvec(h, B.x, B.w, s);
        if (rc) return rc;
    } else {
        cudaMemsetAsync(B.w, 0, (size_t)B.n * sizeof(double), s);
    }
    (edfa::count_launch(), k_bresid<<<nc, kBT, 0, s>>>(B.b, B.w, B.ch, B.part));
    (edfa::count_launch(), k_breduce<<<ns, kBT, 0, s>>>(B.part, 1, 1, B.ch, S.rn2, 1, nullptr, nullptr));
    (edfa::count_launch(), k_bclear_flag<<<1, 1, 0, s>>>(S.flags));
    (edfa::count_launch(), k_bcycle_end<<<(ns + 127) / 128, 128, 0, s>>>(S, first));
    (edfa::count_launch(), k_bscale<<<nc, kBT, 0, s>>>(B.w, B.V, B.ch, S.inv, S.active));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

extern "C" int edfa_solve_batched(edfa_handle h, int32_t nsys, const int64_t* face_off, const int64_t* cell_off,
                                  const double* b, double* x, int32_t restart, double rtol, int32_t maxit,
                                  int32_t* iterations, double* true_rel, int32_t* cycles, edfa_stream stream)
{
    if (!h || nsys < 1 || !face_off || !cell_off || restart < 1 || restart > 126 || !(rtol >= 0.0) || maxit < 0)
        return EDFA_ERR_INVALID;
    if (face_off[0] != 0 || cell_off[0] != 0 || face_off[nsys] != h->Nf || cell_off[nsys] != h->Ne)
        return EDFA_ERR_INVALID;
    for (int i = 0; i < nsys; ++i)
        if (face_off[i + 1] < face_off[i] || cell_off[i + 1] < cell_off[i]) return EDFA_ERR_INVALID;
    if (!b || !x) return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    BatchWork* Bp = (BatchWork*)h->batch;
    const bool reuse = Bp && Bp->nsys == nsys && Bp->m == restart &&
                       std::equal(Bp->fo.begin(), Bp->fo.end(), face_off) &&
                       std::equal(Bp->co.begin(), Bp->co.end(), cell_off);
    if (!reuse) {
        // a different layout: new workspace (device buffers stay owned by the handle)
        if (h->batch_del) h->batch_del(h->batch);
        Bp = new BatchWork();
        h->batch = Bp;
        h->batch_del = [](void* p) { delete (BatchWork*)p; };
        Bp->nsys = nsys;
        Bp->m = restart;
        Bp->n = (int64_t)h->Nf + h->Ne;
        Bp->fo.assign(face_off, face_off + nsys + 1);
        Bp->co.assign(cell_off, cell_off + nsys + 1);
        int rc0 = batch_prepare(h, *Bp, s);
        if (rc0) return rc0;
    }
    BatchWork& B = *Bp;
    B.b = b;
    B.x = x;
    int rc = EDFA_OK;
    B.S.rtol = rtol;
    B.S.maxit = maxit;
    cudaMemsetAsync(x, 0, (size_t)B.n * sizeof(double), s);
    cudaMemsetAsync(B.S.H, 0, sizeof(double) * (size_t)nsys * (restart + 1) * restart, s);
    // first cycle set-up: r = b, ||b|| per system, v0 = b / ||b||
    rc = batch_cycle_end(h, B, 1, s);
    if (rc) return rc;
    // capture one restart cycle
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return EDFA_ERR_CUDA;
    cudaEvent_t ready;
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    cudaEventRecord(ready, s);
    cudaStreamWaitEvent(cs, ready, 0);
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        for (int j = 0; j < restart && !rc; ++j) rc = batch_step(h, B, j, cs);
        if (!rc) rc = batch_cycle_end(h, B, 0, cs);
        ok = cudaStreamEndCapture(cs, &B.graph) == cudaSuccess && !rc;
    }
    if (ok) ok = cudaGraphInstantiate(&B.cycle, B.graph, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (B.graph) cudaGraphDestroy(B.graph);
        cudaStreamDestroy(cs);
        cudaEventDestroy(ready);
        return rc ? rc : EDFA_ERR_CUDA;
    }
    int running = 1, ncyc = 0;
    const int max_cycles = maxit / 1 + 2;
    while (running > 0 && ncyc < max_cycles) {
        cudaGraphLaunch(B.cycle, s);
        cudaMemcpyAsync(&running, B.S.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
        rc = check_err(h, s);
        if (rc) break;
        ++ncyc;
    }
    cudaGraphExecDestroy(B.cycle);
    cudaGraphDestroy(B.graph);
    cudaStreamDestroy(cs);
    cudaEventDestroy(ready);
    if (rc) return rc;
    std::vector<int> it(nsys), cv(nsys);
    std::vector<double> tr(nsys);
    cudaMemcpyAsync(it.data(), B.S.iters, nsys * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(cv.data(), B.S.conv, nsys * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(tr.data(), B.S.true_rel, nsys * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    bool all = true;
    for (int i = 0; i < nsys; ++i) {
        if (iterations) iterations[i] = it[i];
        if (true_rel) true_rel[i] = tr[i];
        if (!cv[i]) all = false;
    }
    if (cycles) *cycles = ncyc;
    return all ? EDFA_OK : EDFA_ERR_NOT_CONVERGED;
}
