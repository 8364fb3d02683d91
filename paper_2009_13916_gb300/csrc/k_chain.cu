// Chain-decomposed triangular sweeps (used for the ILU(0) factor of A~).
//
// The forward (backward) sweep of an ILU(0) factor is a DAG over rows.  On
// the face block of the MHFE system its levels are thin: every face row
// depends on at most one row of the level right before it -- the previous
// face on the same grid line -- and otherwise only on rows finished long ago.
// Such a DAG splits into a few PHASES of independent CHAINS:
//     phase(i) = pm         when exactly one dependency has the largest phase
//                           pm and row i is the chain successor of it,
//              = pm + 1     otherwise (row i heads a new chain),
// where a row gets at most one successor (the smallest competing row index,
// so the decomposition is deterministic).  Within a phase every dependency of
// a row except its chain predecessor lies in an earlier phase.  A sweep then
// runs phase by phase, one kernel per phase (k_ch_phase): for the chains of
// a block, all threads first form the off-chain sums
//     s_i = b_i - sum_{j != pred(i)} M_ij x_j   (- (B z)_i when fused)
// in parallel, then one lane per chain runs x_i = (s_i - m_i x_pred) [* 1/u_ii]
// with x_pred in a register -- one FMA per row on the chain.
// Instead of one inter-SM hand-off per level (~1.8 us x 193 levels on the
// 64^3 face block) a sweep costs 3 phases of a bandwidth-bound pass plus a
// register recurrence.  Factors whose DAG does not collapse (more than
// kChainMaxPhases phases) keep the level-scheduled sweeps.
//
// Layout: the rows of phase p sit at positions off_p + k * nc_p + c (chain c,
// step k), padded with -1 up to the phase's longest chain, so the recurrence
// reads consecutive addresses across the threads of a warp at every step.
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.cuh"

namespace edfa {

constexpr int kChainMaxPhases = 16;
constexpr int kChCtas = 16, kChThreads = 1024;

// phase / predecessor analysis, level by level inside one 16-CTA cluster.
// bid[j]: smallest row of the current level asking to continue j's chain;
// taken[j]: j already has its (unique) chain successor from an earlier level.
template <int FWD>
__global__ void __launch_bounds__(kChThreads, 1)
k_ch_analyse(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const int32_t* __restrict__ perm, const int64_t* __restrict__ loff, int nlev, int* __restrict__ phase,
             int* __restrict__ pred, int* __restrict__ bid, int* __restrict__ taken, int* __restrict__ cand,
             int* __restrict__ pmx)
{
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int L = 0; L < nlev; ++L) {
        const int64_t b = loff[L], e = loff[L + 1];
        // pass 1: largest dependency phase, its unique holder, bid for it
        for (int64_t t = b + tid; t < e; t += nth) {
            const int i = perm[t];
            if (i < 0) continue;
            int pm = -1, cj = -1, cnt = 0;
            const int64_t pe = rowptr[i + 1];
            // eight entries per round: their column and phase loads in flight together
            for (int64_t p0 = rowptr[i]; p0 < pe; p0 += 8) {
                int jj[8], ph[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = p0 + u < pe ? col[p0 + u] : -1;
                    jj[u] = (j >= 0 && (FWD ? (j < i) : (j > i))) ? j : -1;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) ph[u] = jj[u] >= 0 ? __ldcg(phase + jj[u]) : -1;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (jj[u] < 0) continue;
                    if (ph[u] > pm) { pm = ph[u]; cj = jj[u]; cnt = 1; }
                    else if (ph[u] == pm) ++cnt;
                }
            }
            const bool can = cnt == 1 && __ldcg(taken + cj) == 0;
            pmx[i] = pm;
            cand[i] = can ? cj : -1;
            if (can) atomicMin(bid + cj, i);
        }
        cl.sync();
        // pass 2: the smallest bidder continues the chain, the others start one
        for (int64_t t = b + tid; t < e; t += nth) {
            const int i = perm[t];
            if (i < 0) continue;
            const int pm = pmx[i], cj = cand[i];
            if (pm < 0) {
                phase[i] = 0;
                pred[i] = -1;
            } else if (cj >= 0 && __ldcg(bid + cj) == i) {
                phase[i] = pm;
                pred[i] = cj;
                taken[cj] = 1;
            } else {
                phase[i] = pm + 1;
                pred[i] = -1;
            }
        }
        cl.sync();
    }
}

// successor links from the confirmed predecessors (unique by construction)
__global__ void k_ch_succ(int32_t n, const int* __restrict__ pred, int* __restrict__ succ)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = pred[i];
    if (j >= 0 && j < n) succ[j] = (int)i;
}

// per head: chain length, per row: step index and head
__global__ void k_ch_walk(int32_t n, const int* __restrict__ pred, const int* __restrict__ succ,
                          int* __restrict__ kidx, int* __restrict__ head, int* __restrict__ clen)
{
    const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= n || pred[h] >= 0) return;
    int k = 0;
    for (int i = (int)h; i >= 0 && k <= n; i = succ[i], ++k) {
        kidx[i] = k;
        head[i] = (int)h;
    }
    clen[h] = k;
}

__global__ void k_ch_count_phases(int32_t n, const int* __restrict__ phase, int* __restrict__ nph)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicMax(nph, phase[i] + 1);
}

// chain index of every head within its phase (heads in ascending row order)
__global__ void k_ch_head_flags(int32_t n, int nph, const int* __restrict__ pred, const int* __restrict__ phase,
                                int64_t* __restrict__ flag)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool hd = pred[i] < 0;
    for (int p = 0; p < nph; ++p) flag[(int64_t)p * n + i] = (hd && phase[i] == p) ? 1 : 0;
}

__global__ void k_ch_phase_stats(int32_t n, const int* __restrict__ pred, const int* __restrict__ phase,
                                 const int* __restrict__ clen, unsigned* __restrict__ maxlen)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || pred[i] >= 0) return;
    atomicMax(maxlen + phase[i], (unsigned)clen[i]);
}

__global__ void k_ch_place(int32_t n, const int* __restrict__ phase, const int* __restrict__ kidx,
                           const int* __restrict__ head, const int64_t* __restrict__ flagscan,
                           const int64_t* __restrict__ poff, const int64_t* __restrict__ pnc, int32_t* __restrict__ rowat,
                           int64_t* __restrict__ posof)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = phase[i];
    const int h = head[i];
    // chain index = number of heads of phase p before h
    const int64_t c = flagscan[(int64_t)p * n + h] - flagscan[(int64_t)p * n];
    const int64_t pos = poff[p] + (int64_t)kidx[i] * pnc[p] + c;
    rowat[pos] = (int32_t)i;
    posof[i] = pos;
}

// ------------------------------------------------------------ values
// m[pos] = factor entry of row i at its chain predecessor, dv[pos] = 1/u_ii
template <class T, int FWD>
__global__ void k_ch_values(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const T* __restrict__ lu, const T* __restrict__ dinv, const int* __restrict__ pred,
                            const int64_t* __restrict__ posof, T* __restrict__ mv, T* __restrict__ dv)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = pred[i];
    T m = T(0);
    if (j >= 0)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] == j) m = lu[p];
    mv[posof[i]] = m;
    if (!FWD) dv[posof[i]] = dinv[i];
}

// ------------------------------------------------------------ sweep kernel
// One kernel per phase: a block owns 32 chains.  All its threads stage the
// off-chain sums s, the multipliers m (and 1/u_ii) and the row indices of up
// to `seg` steps of those chains in shared memory -- every global load of the
// segment in flight at once -- then warp 0 runs the 32 recurrences from
// shared memory, one lane per chain.
constexpr int kChPhThreads = 1024;
constexpr int kChCPB = 32;

template <class T, class TB, class TO, int FWD>
__global__ void __launch_bounds__(kChPhThreads)
k_ch_phase(int64_t off, int64_t nc, int maxlen, int seg, const int32_t* __restrict__ rowat,
           const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int64_t* __restrict__ diag,
           const T* __restrict__ lu, const T* __restrict__ mpre, const T* __restrict__ dvv, const TB* __restrict__ base,
           const int64_t* __restrict__ mptr, const int32_t* __restrict__ mcol, const T* __restrict__ mval,
           const TO* __restrict__ mvec, TO* __restrict__ x)
{
    extern __shared__ __align__(16) unsigned char chs[];
    T* ss = (T*)chs;
    T* sm = ss + (int64_t)seg * kChCPB;
    T* sd = sm + (int64_t)seg * kChCPB;
    int* sr = (int*)(sd + (int64_t)seg * kChCPB);
    const int64_t c0 = (int64_t)blockIdx.x * kChCPB;
    T xp = T(0);
    for (int k0 = 0; k0 < maxlen; k0 += seg) {
        const int kn = min(seg, maxlen - k0);
#pragma unroll 2
        for (int idx = threadIdx.x; idx < kn * kChCPB; idx += blockDim.x) {
            const int kk = idx / kChCPB, cl = idx % kChCPB;
            const int64_t c = c0 + cl;
            int i = -1;
            T sv = T(0), mv = T(0), dv = T(1);
            if (c < nc) {
                const int64_t pos = off + (int64_t)(k0 + kk) * nc + c;
                i = rowat[pos];
                if (i >= 0) {
                    const int pr = (k0 + kk) > 0 ? rowat[pos - nc] : -1;
                    const int64_t lo = FWD ? rowptr[i] : diag[i] + 1, hi = FWD ? diag[i] : rowptr[i + 1];
                    T acc = T(0), a2 = T(0);
                    int64_t p = lo;
                    for (; p + 1 < hi; p += 2) {
                        const int j0 = col[p], j1 = col[p + 1];
                        if (j0 != pr) acc = fma(lu[p], (T)x[j0], acc);
                        if (j1 != pr) a2 = fma(lu[p + 1], (T)x[j1], a2);
                    }
                    if (p < hi && col[p] != pr) acc = fma(lu[p], (T)x[col[p]], acc);
                    if (mptr)
                        for (int64_t r = mptr[i]; r < mptr[i + 1]; ++r) a2 = fma(mval[r], (T)mvec[mcol[r]], a2);
                    sv = (T)base[i] - (acc + a2);
                    mv = mpre[pos];
                    if (!FWD) dv = dvv[pos];
                }
            }
            ss[idx] = sv;
            sm[idx] = mv;
            sd[idx] = dv;
            sr[idx] = i;
        }
        __syncthreads();
        if (threadIdx.x < kChCPB) {
            for (int kk = 0; kk < kn; ++kk) {
                const int idx = kk * kChCPB + threadIdx.x;
                const int i = sr[idx];
                if (i >= 0) {
                    T y = ss[idx] - sm[idx] * xp;
                    if (!FWD) y *= sd[idx];
                    x[i] = (TO)y;
                    xp = y;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ host
static int build_dir(edfa_handle_s* h, Factor& f, ChainPlan& cpn, int fwd, cudaStream_t s)
{
    const SweepPlan& sp = fwd ? f.fwd : f.bwd;
    const int32_t n = f.n;
    cpn.ok = 0;
    if (n <= 0 || sp.nlevels <= 0) return EDFA_OK;
    const size_t nn = (size_t)n;
    int *phase = nullptr, *pred = nullptr, *succ = nullptr, *cand = nullptr, *pmx = nullptr, *kidx = nullptr,
        *head = nullptr, *clen = nullptr, *taken = nullptr;
    unsigned* maxlen = nullptr;
    int64_t* flag = nullptr;
    auto al = [&](void** p, size_t b) { return cudaMallocAsync(p, b, s) == cudaSuccess; };
    if (!al((void**)&phase, nn * 4) || !al((void**)&pred, nn * 4) || !al((void**)&succ, nn * 4) ||
        !al((void**)&cand, nn * 4) || !al((void**)&pmx, nn * 4) || !al((void**)&kidx, nn * 4) ||
        !al((void**)&head, nn * 4) || !al((void**)&clen, nn * 4) || !al((void**)&taken, nn * 4) ||
        !al((void**)&maxlen, kChainMaxPhases * 4))
        return EDFA_ERR_OOM;
    cudaMemsetAsync(phase, 0, nn * 4, s);
    cudaMemsetAsync(taken, 0, nn * 4, s);
    cudaMemsetAsync(succ, 0x7F, nn * 4, s);  // bids: large positive = none yet
    cudaMemsetAsync(maxlen, 0, kChainMaxPhases * 4, s);
    {
        auto fn = fwd ? k_ch_analyse<1> : k_ch_analyse<0>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kChCtas, 1, 1);
        cfg.blockDim = dim3(kChThreads, 1, 1);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kChCtas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        edfa::count_launch();
        if (cudaLaunchKernelEx(&cfg, fn, n, f.rowptr, f.col, (const int32_t*)sp.perm, (const int64_t*)sp.loff,
                               (int)sp.nlevels, phase, pred, succ, taken, cand, pmx) != cudaSuccess) {
            cudaGetLastError();
            return EDFA_ERR_CUDA;
        }
    }
    const unsigned g = (unsigned)((n + 255) / 256);
    cudaMemsetAsync(succ, 0xFF, nn * 4, s);
    (edfa::count_launch(), k_ch_succ<<<g, 256, 0, s>>>(n, pred, succ));
    (edfa::count_launch(), k_ch_walk<<<g, 256, 0, s>>>(n, pred, succ, kidx, head, clen));
    // number of phases
    int nph = 0;
    {
        int* dmax = nullptr;
        if (!al((void**)&dmax, sizeof(int))) return EDFA_ERR_OOM;
        cudaMemsetAsync(dmax, 0, sizeof(int), s);
        (edfa::count_launch(), k_ch_count_phases<<<g, 256, 0, s>>>(n, phase, dmax));
        cudaMemcpyAsync(&nph, dmax, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaFreeAsync(dmax, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return EDFA_ERR_CUDA;
    }
    int rc = EDFA_OK;
    if (nph >= 1 && nph <= kChainMaxPhases && nph * 8 <= sp.nlevels) {
        if (!al((void**)&flag, (size_t)nph * nn * 8 + 8)) return EDFA_ERR_OOM;
        (edfa::count_launch(), k_ch_head_flags<<<g, 256, 0, s>>>(n, nph, pred, phase, flag));
        rc = scan_i64(h, flag, (int64_t)nph * n, s);
        (edfa::count_launch(), k_ch_phase_stats<<<g, 256, 0, s>>>(n, pred, phase, clen, maxlen));
        int64_t fs[kChainMaxPhases + 1];
        unsigned ml[kChainMaxPhases];
        for (int p = 0; p <= nph && !rc; ++p)
            cudaMemcpyAsync(fs + p, flag + (int64_t)p * n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(ml, maxlen, sizeof(unsigned) * nph, cudaMemcpyDeviceToHost, s);
        if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = EDFA_ERR_CUDA;
        if (!rc) {
            int64_t poff[kChainMaxPhases + 1], pnc[kChainMaxPhases];
            poff[0] = 0;
            for (int p = 0; p < nph; ++p) {
                pnc[p] = fs[p + 1] - fs[p];
                cpn.nc[p] = pnc[p];
                cpn.maxlen[p] = (int)ml[p];
                cpn.off[p] = poff[p];
                poff[p + 1] = poff[p] + pnc[p] * (int64_t)ml[p];
            }
            cpn.nph = nph;
            cpn.npos = poff[nph];
            int64_t *dpoff = nullptr, *dpnc = nullptr;
            rc = dalloc_t(h, &cpn.rowat, (size_t)(cpn.npos > 0 ? cpn.npos : 1));
            if (!rc) rc = dalloc_t(h, &cpn.posof, nn);
            if (!rc) rc = dalloc_t(h, &cpn.pred, nn);
            if (!rc && !al((void**)&dpoff, sizeof poff)) rc = EDFA_ERR_OOM;
            if (!rc && !al((void**)&dpnc, sizeof pnc)) rc = EDFA_ERR_OOM;
            if (!rc) {
                const size_t esz = h->opt.precision == 1 ? sizeof(float) : sizeof(double);
                rc = dalloc(h, &cpn.m, (size_t)(cpn.npos > 0 ? cpn.npos : 1) * esz);
                if (!rc && !fwd) rc = dalloc(h, &cpn.dv, (size_t)(cpn.npos > 0 ? cpn.npos : 1) * esz);
            }
            if (!rc) {
                cudaMemsetAsync(cpn.rowat, 0xFF, (size_t)(cpn.npos > 0 ? cpn.npos : 1) * 4, s);
                cudaMemcpyAsync(dpoff, poff, sizeof poff, cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(dpnc, pnc, sizeof pnc, cudaMemcpyHostToDevice, s);
                // k_ch_place subtracts the phase's first flag: the scan is over
                // all phases back to back
                (edfa::count_launch(), k_ch_place<<<g, 256, 0, s>>>(n, phase, kidx, head, flag, dpoff, dpnc, cpn.rowat,
                                                                   cpn.posof));
                cudaMemcpyAsync(cpn.pred, pred, nn * 4, cudaMemcpyDeviceToDevice, s);
                cpn.ok = 1;
            }
            if (dpoff) cudaFreeAsync(dpoff, s);
            if (dpnc) cudaFreeAsync(dpnc, s);
        }
        cudaFreeAsync(flag, s);
    }
    cudaFreeAsync(phase, s);
    cudaFreeAsync(pred, s);
    cudaFreeAsync(succ, s);
    cudaFreeAsync(cand, s);
    cudaFreeAsync(pmx, s);
    cudaFreeAsync(kidx, s);
    cudaFreeAsync(head, s);
    cudaFreeAsync(clen, s);
    cudaFreeAsync(taken, s);
    cudaFreeAsync(maxlen, s);
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int chain_plan_build(edfa_handle_s* h, Factor& f, cudaStream_t s)
{
    int rc = build_dir(h, f, f.chf, 1, s);
    if (!rc) rc = build_dir(h, f, f.chb, 0, s);
    return rc;
}

int chain_plan_values(edfa_handle_s* h, Factor& f, cudaStream_t s)
{
    const unsigned g = (unsigned)((f.n + 255) / 256);
    const bool f32 = h->opt.precision == 1;
    for (int d = 0; d < 2; ++d) {
        ChainPlan& c = d == 0 ? f.chf : f.chb;
        if (!c.ok) continue;
        if (f32) {
            if (d == 0)
                (edfa::count_launch(), k_ch_values<float, 1><<<g, 256, 0, s>>>(f.n, f.rowptr, f.col, f.lu32, f.dinv32, c.pred,
                                                                              c.posof, (float*)c.m, (float*)c.dv));
            else
                (edfa::count_launch(), k_ch_values<float, 0><<<g, 256, 0, s>>>(f.n, f.rowptr, f.col, f.lu32, f.dinv32, c.pred,
                                                                              c.posof, (float*)c.m, (float*)c.dv));
        } else {
            if (d == 0)
                (edfa::count_launch(), k_ch_values<double, 1><<<g, 256, 0, s>>>(f.n, f.rowptr, f.col, f.lu64, f.dinv64,
                                                                               c.pred, c.posof, (double*)c.m,
                                                                               (double*)c.dv));
            else
                (edfa::count_launch(), k_ch_values<double, 0><<<g, 256, 0, s>>>(f.n, f.rowptr, f.col, f.lu64, f.dinv64,
                                                                               c.pred, c.posof, (double*)c.m,
                                                                               (double*)c.dv));
        }
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

template <class T, class TB, class TO, int FWD>
int chain_sweep(edfa_handle_s* h, const Factor& f, const TB* base, const int64_t* mptr, const int32_t* mcol,
                const T* mval, const TO* mvec, TO* out, cudaStream_t s)
{
    const ChainPlan& c = FWD ? f.chf : f.chb;
    const T* lu;
    if constexpr (sizeof(T) == 8) lu = (const T*)f.lu64;
    else lu = (const T*)f.lu32;
    auto fn = k_ch_phase<T, TB, TO, FWD>;
    static thread_local bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
        attr = true;
    }
    for (int p = 0; p < c.nph; ++p) {
        if (c.nc[p] == 0 || c.maxlen[p] == 0) continue;
        // staged steps per round: the whole chain when it fits 128 KB
        const int per_step = kChCPB * (3 * (int)sizeof(T) + 4);
        int seg = c.maxlen[p];
        if (seg * per_step > 128 * 1024) seg = 128 * 1024 / per_step;
        const size_t smem = (size_t)seg * per_step;
        (edfa::count_launch(), fn<<<(unsigned)((c.nc[p] + kChCPB - 1) / kChCPB), kChPhThreads, smem, s>>>(
            c.off[p], c.nc[p], c.maxlen[p], seg, c.rowat, f.rowptr, f.col, f.diag, lu, (const T*)c.m, (const T*)c.dv,
            base, mptr, mcol, mval, mvec, out));
    }
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

#define EDFA_CHAIN_INST(T, TB, TO, FWD)                                                                         \
    template int chain_sweep<T, TB, TO, FWD>(edfa_handle_s*, const Factor&, const TB*, const int64_t*, const int32_t*, \
                                             const T*, const TO*, TO*, cudaStream_t);
EDFA_CHAIN_INST(double, double, double, 1)
EDFA_CHAIN_INST(double, double, double, 0)
EDFA_CHAIN_INST(float, double, float, 1)
EDFA_CHAIN_INST(float, float, double, 0)
EDFA_CHAIN_INST(float, float, float, 0)
EDFA_CHAIN_INST(float, double, double, 1)
#undef EDFA_CHAIN_INST

}  // namespace edfa
