// Pre- and post-filtration of the approximate Schur complement (Sec. 3,
// implementation details; Algorithms 1 and 2).  An entry is discarded when
// its absolute value is below tau times the Euclidean norm of the vector it
// belongs to (a kept entry has |v| >= tau ||row||_2); diagonal entries of H~
// and S~ are always kept.
//   pre    (Stage 1): every column m of X~ on Q^(m) (and row m of G~), before
//                     the Schur product; X~ and G~ then carry own patterns
//   post_h (Stage 1): the rows of H~, computed on pattern(H~) u pattern(D) u
//                     diagonal; a dropped H~ entry at a position of D leaves
//                     the position with the value of D
//   post_s (Stage 2): the rows of S~ = D - H~; the pattern of S~ changes with
//                     D, so the ILU(0) level plans and the cluster records of
//                     S~ are rebuilt by every Stage 2
// One warp per vector: the squared norm is summed in FP64 by the lanes and a
// butterfly reduction, then the kept entries are compacted in order with
// ballots (two passes: count, fill).
#include "internal.cuh"

namespace edfa {

template <class T>
__device__ __forceinline__ double warp_sumsq(const T* v, int64_t b, int64_t e, int lane)
{
    double ss = 0.0;
    for (int64_t p = b + lane; p < e; p += 32) {
        const double x = (double)v[p];
        ss = fma(x, x, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    return ss;
}

// Pre-filtration of segments (column m of X~ or row m of G~ on Q^(m)).
// PASS 0: cnt[m] = kept entries; PASS 1: compacted (optr, oidx, oval).
template <class T, int PASS>
__global__ void k_segfilt(int32_t nseg, const int64_t* ptr, const int32_t* idx, const T* val, double tau,
                          int64_t* cnt_or_optr, int32_t* oidx, T* oval)
{
    const int lane = threadIdx.x & 31;
    const int64_t wpg = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < nseg; m += wpg) {
        const int64_t b = ptr[m], e = ptr[m + 1];
        const double lim = tau * sqrt(warp_sumsq(val, b, e, lane));
        int64_t o = PASS ? cnt_or_optr[m] : 0;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t p = base + lane;
            bool keep = false;
            T v = T(0);
            if (p < e) {
                v = val[p];
                keep = !(fabs((double)v) < lim);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (PASS == 1 && keep) {
                const int64_t q = o + __popc(bal & ((1u << lane) - 1u));
                oidx[q] = idx[p];
                oval[q] = v;
            }
            o += __popc(bal);
        }
        if (PASS == 0 && lane == 0) cnt_or_optr[m] = o;
    }
}

// Row filtration of a square CSR matrix (H~ or S~ on its pattern).  An entry
// keeps its value when it is diagonal or |v| >= tau ||row||_2; it keeps its
// position also when in_d marks it (a position of D: the value becomes 0).
// PASS 0: cnt[i] = kept positions; PASS 1: compacted (optr, ocol, oval) and
// newpos[p] = new position of old position p (-1 when dropped, may be null).
template <class T, int PASS>
__global__ void k_rowfilt(int32_t n, const int64_t* ptr, const int32_t* col, const T* val,
                          const unsigned char* in_d, double tau, int64_t* cnt_or_optr, int32_t* ocol, T* oval,
                          int64_t* newpos)
{
    const int lane = threadIdx.x & 31;
    const int64_t wpg = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += wpg) {
        const int64_t b = ptr[i], e = ptr[i + 1];
        const double lim = tau * sqrt(warp_sumsq(val, b, e, lane));
        int64_t o = PASS ? cnt_or_optr[i] : 0;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t p = base + lane;
            bool keep = false, keepv = false;
            T v = T(0);
            int c = 0;
            if (p < e) {
                v = val[p];
                c = col[p];
                keepv = c == (int)i || !(fabs((double)v) < lim);
                keep = keepv || (in_d != nullptr && in_d[p] != 0);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (PASS == 1 && p < e) {
                const int64_t q = o + __popc(bal & ((1u << lane) - 1u));
                if (keep) {
                    ocol[q] = c;
                    oval[q] = keepv ? v : T(0);
                }
                if (newpos) newpos[p] = keep ? q : -1;
            }
            o += __popc(bal);
        }
        if (PASS == 0 && lane == 0) cnt_or_optr[i] = o;
    }
}

__global__ void k_mark_d(int64_t nd, const int64_t* d_map, unsigned char* mask)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nd; k += (int64_t)gridDim.x * blockDim.x)
        mask[d_map[k]] = 1;
}

__global__ void k_remap_d(int64_t nd, int64_t* d_map, const int64_t* newpos)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nd; k += (int64_t)gridDim.x * blockDim.x)
        d_map[k] = newpos[d_map[k]];
}

static unsigned warp_grid(edfa_handle_s* h, int64_t nwarps)
{
    int64_t g = (nwarps + 7) / 8;  // 8 warps per 256-thread block
    const int64_t cap = (int64_t)h->nsm * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

static unsigned flat_grid(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 65535) g = 65535;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// compact one family of segments on (ptr, idx, val) into own arrays
template <class T>
static int seg_compact(edfa_handle_s* h, int32_t nseg, const int64_t* ptr, const int32_t* idx, const T* val,
                       int64_t** optr, int32_t** oidx, T** oval, int64_t* otot, cudaStream_t s)
{
    const double tau = h->opt.tau_filt;
    int rc = dalloc_t(h, optr, (size_t)nseg + 1);
    if (rc) return rc;
    const unsigned g = warp_grid(h, nseg);
    if (nseg > 0) (edfa::count_launch(), k_segfilt<T, 0><<<g, 256, 0, s>>>(nseg, ptr, idx, val, tau, *optr, nullptr, nullptr));
    rc = scan_i64(h, *optr, nseg, s);
    if (rc) return rc;
    int64_t tot = 0;
    cudaMemcpyAsync(&tot, *optr + nseg, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    rc = check_err(h, s);
    if (rc) return rc;
    rc = dalloc_t(h, oidx, (size_t)(tot > 0 ? tot : 1));
    if (!rc) rc = dalloc_t(h, oval, (size_t)(tot > 0 ? tot : 1));
    if (rc) return rc;
    if (nseg > 0) (edfa::count_launch(), k_segfilt<T, 1><<<g, 256, 0, s>>>(nseg, ptr, idx, val, tau, *optr, *oidx, *oval));
    *otot = tot;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

int prefilter(edfa_handle_s* h, cudaStream_t s)
{
    const bool two = h->opt.schur_form == 1;
    h->x_ptr = h->qptr;
    h->x_idx = h->qidx;
    h->x_tot = h->qtot;
    h->xf64 = h->xval;
    h->xf32 = h->xval32;
    h->g_ptr = h->qptr;
    h->g_idx = h->qidx;
    h->gf64 = h->gval;
    h->gf32 = h->gval32;
    if (h->opt.filtration != EDFA_FILT_PRE) return EDFA_OK;
    int64_t gt = 0;
    int rc;
    if (h->opt.precision == 1) {
        rc = seg_compact<float>(h, h->Ne, h->qptr, h->qidx, h->xval32, &h->x_ptr, &h->x_idx, &h->xf32, &h->x_tot, s);
        if (!rc && two)
            rc = seg_compact<float>(h, h->Ne, h->qptr, h->qidx, h->gval32, &h->g_ptr, &h->g_idx, &h->gf32, &gt, s);
    } else {
        rc = seg_compact<double>(h, h->Ne, h->qptr, h->qidx, h->xval, &h->x_ptr, &h->x_idx, &h->xf64, &h->x_tot, s);
        if (!rc && two)
            rc = seg_compact<double>(h, h->Ne, h->qptr, h->qidx, h->gval, &h->g_ptr, &h->g_idx, &h->gf64, &gt, s);
    }
    return rc;
}

// post-filtration of H~ on the S~ pattern: replaces (s_ptr, s_col, h_val,
// s_nnz) by the compacted pattern and moves d_map along
template <class T>
int postfilter_h(edfa_handle_s* h, T* h_val, cudaStream_t s)
{
    const int32_t Ne = h->Ne;
    const int64_t nnz = h->s_nnz, nd = h->D.nnz;
    unsigned char* in_d = nullptr;
    int64_t* newpos = nullptr;
    if (cudaMallocAsync((void**)&in_d, (size_t)(nnz > 0 ? nnz : 1), s) != cudaSuccess) return EDFA_ERR_OOM;
    if (cudaMallocAsync((void**)&newpos, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t), s) != cudaSuccess)
        return EDFA_ERR_OOM;
    cudaMemsetAsync(in_d, 0, (size_t)(nnz > 0 ? nnz : 1), s);
    if (nd > 0) (edfa::count_launch(), k_mark_d<<<flat_grid(nd), 256, 0, s>>>(nd, h->d_map, in_d));
    int64_t* optr = nullptr;
    int rc = dalloc_t(h, &optr, (size_t)Ne + 1);
    if (rc) return rc;
    const unsigned g = warp_grid(h, Ne);
    const double tau = h->opt.tau_filt;
    if (Ne > 0)
        (edfa::count_launch(), k_rowfilt<T, 0><<<g, 256, 0, s>>>(Ne, h->s_ptr, h->s_col, h_val, in_d, tau, optr, nullptr,
                                                                 nullptr, nullptr));
    rc = scan_i64(h, optr, Ne, s);
    if (rc) return rc;
    int64_t tot = 0;
    cudaMemcpyAsync(&tot, optr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    rc = check_err(h, s);
    if (rc) return rc;
    int32_t* ocol = nullptr;
    T* oval = nullptr;
    rc = dalloc_t(h, &ocol, (size_t)(tot > 0 ? tot : 1));
    if (!rc) rc = dalloc_t(h, &oval, (size_t)(tot > 0 ? tot : 1));
    if (rc) return rc;
    if (Ne > 0)
        (edfa::count_launch(), k_rowfilt<T, 1><<<g, 256, 0, s>>>(Ne, h->s_ptr, h->s_col, h_val, in_d, tau, optr, ocol,
                                                                 oval, newpos));
    if (nd > 0) (edfa::count_launch(), k_remap_d<<<flat_grid(nd), 256, 0, s>>>(nd, h->d_map, newpos));
    cudaFreeAsync(in_d, s);
    cudaFreeAsync(newpos, s);
    h->s_ptr = optr;
    h->s_col = ocol;
    h->s_nnz = tot;
    if constexpr (sizeof(T) == 8) h->h_val = (double*)oval;
    else h->h_val32 = (float*)oval;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

template int postfilter_h<double>(edfa_handle_s*, double*, cudaStream_t);
template int postfilter_h<float>(edfa_handle_s*, float*, cudaStream_t);

// The S~ the inner factorisation uses after the values of Stage 2: S~ itself,
// or (post-filtration of S~) its filtered copy, compacted into buffers of the
// unfiltered capacity.  Synchronises `s` once to read the filtered size.
int stage2_pattern(edfa_handle_s* h, cudaStream_t s)
{
    const bool f32 = h->opt.precision == 1;
    if (h->opt.filtration != EDFA_FILT_POST_S) {
        h->sf_nnz = h->s_nnz;
        h->sf_ptr = h->s_ptr;
        h->sf_col = h->s_col;
        h->sf_val = h->s_val;
        h->sf_val32 = h->s_val32;
        return EDFA_OK;
    }
    const int32_t Ne = h->Ne;
    const int64_t cap = h->s_nnz > 0 ? h->s_nnz : 1;
    int rc = EDFA_OK;
    if (!h->sf_cnt) {
        rc = dalloc_t(h, &h->sf_cnt, (size_t)Ne + 1);
        if (!rc) rc = dalloc_t(h, &h->sf_col, (size_t)cap);
        if (!rc) rc = f32 ? dalloc_t(h, &h->sf_val32, (size_t)cap) : dalloc_t(h, &h->sf_val, (size_t)cap);
        if (rc) return rc;
    }
    // the row pointers of the previous pattern belong to the previous plan
    // (owned_s2); a fresh array is taken for every Stage 2
    rc = dalloc_t(h, &h->sf_ptr, (size_t)Ne + 1);
    if (rc) return rc;
    h->owned_s2.push_back(h->owned.back());
    h->owned.pop_back();
    const unsigned g = warp_grid(h, Ne);
    const double tau = h->opt.tau_filt;
    if (f32) {
        if (Ne > 0)
            (edfa::count_launch(), k_rowfilt<float, 0><<<g, 256, 0, s>>>(Ne, h->s_ptr, h->s_col, h->s_val32, nullptr, tau,
                                                                         h->sf_ptr, nullptr, nullptr, nullptr));
    } else if (Ne > 0) {
        (edfa::count_launch(), k_rowfilt<double, 0><<<g, 256, 0, s>>>(Ne, h->s_ptr, h->s_col, h->s_val, nullptr, tau,
                                                                      h->sf_ptr, nullptr, nullptr, nullptr));
    }
    rc = scan_i64(h, h->sf_ptr, Ne, s);
    if (rc) return rc;
    if (f32) {
        if (Ne > 0)
            (edfa::count_launch(), k_rowfilt<float, 1><<<g, 256, 0, s>>>(Ne, h->s_ptr, h->s_col, h->s_val32, nullptr, tau,
                                                                         h->sf_ptr, h->sf_col, h->sf_val32, nullptr));
    } else if (Ne > 0) {
        (edfa::count_launch(), k_rowfilt<double, 1><<<g, 256, 0, s>>>(Ne, h->s_ptr, h->s_col, h->s_val, nullptr, tau,
                                                                      h->sf_ptr, h->sf_col, h->sf_val, nullptr));
    }
    int64_t tot = 0;
    cudaMemcpyAsync(&tot, h->sf_ptr + Ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    rc = check_err(h, s);
    if (rc) return rc;
    h->sf_nnz = tot;
    return EDFA_OK;
}

// Level plans and cluster records of the factorised S~ (sf_*).  With
// post-filtration of S~ every Stage 2 replaces them: the previous plan's
// buffers are released first (the stream has been synchronised by
// stage2_pattern, so no launch still reads them).
int stage2_symbolic(edfa_handle_s* h, cudaStream_t s)
{
    const bool replan = h->opt.filtration == EDFA_FILT_POST_S;
    if (replan) {
        // keep the row pointers of the current pattern (the last entry)
        DBuf cur{};
        if (!h->owned_s2.empty()) {
            cur = h->owned_s2.back();
            h->owned_s2.pop_back();
        }
        for (auto& b : h->owned_s2) cudaFree(b.p);
        h->owned_s2.clear();
        if (cur.p) h->owned_s2.push_back(cur);
        h->fs = Factor{};
        h->cp = ClusterPlan{};
    }
    const size_t mark = h->owned.size();
    int rc;
    if (h->opt.ordering >= 1) {
        rc = order_stage2_symbolic(h, s);
    } else {
        rc = factor_plan(h, h->fs, h->Ne, h->sf_nnz, h->sf_ptr, h->sf_col, s);
        if (!rc) rc = cluster_plan_build(h, s);
    }
    if (replan) {
        for (size_t k = mark; k < h->owned.size(); ++k) h->owned_s2.push_back(h->owned[k]);
        h->owned.resize(mark);
    }
    return rc;
}

}  // namespace edfa
