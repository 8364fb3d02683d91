// Internal declarations shared by the translation units of libedfa.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "edfa.h"

namespace edfa {

// ------------------------------------------------------------------ errors
// Device-side error record: the first failing thread wins the code; the detail
// (row/cell index) is written by the same thread.  Read by the host after a
// synchronisation point.
struct DevErr {
    int code;
    int pad;
    long long detail;
};

__device__ __forceinline__ void raise_err(DevErr* e, int code, long long detail)
{
    if (atomicCAS(&e->code, 0, code) == 0) e->detail = detail;
}

// Bounded spin budget for cross-warp waits (polling with nanosleep): about
// 2^20 polls of >= 20 ns, i.e. the wait gives up after some tens of ms,
// records EDFA_ERR_TIMEOUT and lets the kernel finish.  Every wait also gives
// up as soon as any thread has recorded an error, so a failure ends the whole
// kernel within one wait period.
constexpr unsigned kSpinLimit = 1u << 20;

__device__ __forceinline__ bool err_set(const DevErr* e)
{
    return *(volatile const int*)&e->code != 0;
}

// acquire load of a completion flag written by another SM
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// relaxed load of a flag (polling; pair with an acquire fence once it is seen)
__device__ __forceinline__ int ld_relaxed_i32(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polling back-off: the sleep between polls doubles from 32 ns up to 256 ns,
// which keeps thousands of waiting warps from flooding L2 with polls.
constexpr unsigned kBackoffMin = 32, kBackoffMax = 256;

// wait until *flag == epoch; returns false (and raises) on timeout
__device__ __forceinline__ bool wait_flag(const int* flag, int epoch, DevErr* err, long long who)
{
    if (ld_acquire(flag) == epoch) return true;
    unsigned ns = kBackoffMin;
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        __nanosleep(ns);
        if (ns < kBackoffMax) ns <<= 1;
        if (ld_acquire(flag) == epoch) return true;
        if ((it & 255u) == 255u && err_set(err)) return false;
    }
    raise_err(err, EDFA_ERR_TIMEOUT, who);
    return false;
}

template <class T>
__device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }

// 1/x rounded to nearest: the same value as the IEEE division 1/x, from the
// reciprocal intrinsics, which take fewer FP64 (FP32) instructions than a
// division; used for the pivots of the dense per-cell factorisations, where
// every warp-wide FP64 instruction occupies the narrow FP64 pipe of this part
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }

// ------------------------------------------------------------------ CSR
template <class T>
struct Csr {
    int32_t nrows, ncols;
    int64_t nnz;
    const int64_t* rowptr;
    const int32_t* col;
    const T* val;
};

inline Csr<double> csr_of(const edfa_csr& m)
{
    return Csr<double>{m.nrows, m.ncols, m.nnz, m.rowptr, m.col, m.val};
}

// --------------------------------------------------------- device buffers
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// ------------------------------------------------------------- sweeps
// A level-ordered triangular-sweep plan over a CSR pattern: rows grouped by
// dependency level (forward: on smaller columns, backward: on larger ones),
// each level padded with -1 to a multiple of 32 so that a warp never holds two
// rows of different levels.
struct SweepPlan {
    int32_t* perm = nullptr;  // [nslots]
    int64_t nslots = 0;
    int32_t nlevels = 0;
    int64_t* loff = nullptr;  // [nlevels+1] start of every (padded) level in perm
};

// Phases of independent chains of a triangular sweep (k_chain.cu): rows of
// phase p at positions off[p] + k * nc[p] + c (chain c, step k).
struct ChainPlan {
    int ok = 0;
    int nph = 0;
    int64_t npos = 0;
    int64_t off[16] = {}, nc[16] = {};
    int maxlen[16] = {};
    int32_t* rowat = nullptr;  // [npos] row at every position (-1: padding)
    int64_t* posof = nullptr;  // [n] position of every row
    int* pred = nullptr;       // [n] chain predecessor (-1: head)
    void* m = nullptr;         // [npos] factor entry at the chain predecessor
    void* dv = nullptr;        // [npos] 1/u_ii (backward only)
};

struct Factor {
    // pattern (not owned unless owned_pattern)
    int32_t n = 0;
    int64_t nnz = 0;
    const int64_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    int64_t* diag = nullptr;   // [n] position of the diagonal
    double* lu64 = nullptr;    // factor values (FP64 path)
    float* lu32 = nullptr;     // factor values (FP32 path)
    double* dinv64 = nullptr;  // 1 / U_ii
    float* dinv32 = nullptr;
    SweepPlan fwd, bwd;
    ChainPlan chf, chb;  // chain decomposition of the sweeps (k_chain.cu), used when ok
    int fac_R = 0;  // longest row (picks the shared-memory layout of the numeric factorisation)
    const struct Ordering* ord = nullptr;  // set for an ordered factor: factorised colour by colour
};

// Packed per-CTA level chunks of both S~ sweeps for the single-cluster solve
// (k_cluster.cu).  state: -1 not built, 0 not usable (falls back to the
// sync-free sweeps), 1 ready.
struct ClusterPlan {
    int state = -1;
    int32_t cap = 0;           // value slots per CTA
    int nlf = 0, nlb = 0;      // levels of the forward / backward plans
    int64_t nlists = 0;        // 16 x (nlf + nlb) row lists
    int64_t nrec = 0;          // rows of all lists, padding included
    int32_t* posf = nullptr;   // [n] slot * 16 + owner CTA of each row
    int32_t* rowof = nullptr;  // [16][cap] row held in each slot (-1: none)
    int64_t* lofs = nullptr;   // [nlists+1] first row of every list in lrows
    int32_t* lrows = nullptr;  // [2n]
    int64_t* lbyte = nullptr;  // [nlists+1] byte offset of every list's chunks
    int64_t* lchunk = nullptr; // [nlists+1] global index of every list's first chunk
    int64_t* meta = nullptr;   // [16][2] first byte and chunk count of every CTA
    unsigned char* chunks = nullptr;
    int64_t bytes = 0;
    uint16_t* sz = nullptr;    // [16][szstride] chunk sizes (16-byte units | 0x8000 on a level's last chunk)
    int32_t szstride = 0;
    void* bslot = nullptr;     // [16*cap] right-hand side in slot order
    size_t smem = 0;           // dynamic shared memory per CTA
    int kind = 0;              // 1 dataflow (row records), 2 level-synchronous (TMA chunks)
    // dataflow variant
    unsigned char* rec = nullptr;  // [2n] fixed-size row records in processing order
    int64_t* fidx = nullptr;       // [n] forward record of every row
    int64_t* bidx = nullptr;       // [16][cap] backward record of every slot (-1: none)
    int64_t* rmeta = nullptr;      // [16][4] first record and rows of each CTA, forward then backward
    int32_t* lvl = nullptr;        // [2n] forward and backward dependency level of every row
    int64_t* ovoff = nullptr;      // [2n+1] overflow offsets (dependencies beyond the inline ones)
    int32_t* ovf_dep = nullptr;
    void* ovf_val = nullptr;
};

// A multicolour ordering of the rows of a factorised matrix (k_order.cu).
struct Ordering {
    int on = 0;
    int32_t n = 0, ncolours = 0;
    int32_t* perm = nullptr;   // [n] ordered position -> original row
    int32_t* iperm = nullptr;  // [n] original row -> ordered position
    std::vector<int32_t> cstart;  // host: first ordered row of every colour, [ncolours + 1]
    int32_t* cstart_dev = nullptr;  // the same on the device
    // first row group of every colour in processing order, for groups of
    // 32, 16, 8 and 4 rows (1, 2, 4, 8 lanes per row): [dir][lanes][ncolours + 1],
    // dir 0 forward (colours ascending), 1 backward (descending)
    int64_t* tstart_dev = nullptr;
    // block multicolour ordering (block > 1): row r of block B has colour
    // c(B) block + r - B block, so block colour c spans colours c block ..
    // c block + block - 1; bstart_dev = first task (32 / (block lanes)
    // blocks) of every block colour in processing order, [dir][lanes][nbcolours
    // + 1] (dir 0 forward, 1 backward; 1 or 2 lanes per row), for the sweeps
    // that take whole blocks per warp (block 4 or 8)
    int32_t block = 1;
    int32_t nbcolours = 0;
    int64_t* bstart_dev = nullptr;
};

// Up to six device buffers to fill with the all-ones pattern, in 32-bit words
struct FillList {
    uint32_t* p[6] = {};
    int64_t words[6] = {};
    int n = 0;
    void add(void* ptr, int64_t bytes)
    {
        if (n < 6 && ptr && bytes > 0) { p[n] = (uint32_t*)ptr; words[n] = bytes / 4; ++n; }
    }
};

// An ordered copy P M Q^T of a CSR matrix: pattern, the position in M of every
// entry, and the gathered values (FP64 and/or FP32).
struct OrderedCsr {
    int64_t nnz = 0;
    int64_t* ptr = nullptr;
    int32_t* col = nullptr;
    int64_t* map = nullptr;
    double* v64 = nullptr;
    float* v32 = nullptr;
};

}  // namespace edfa

struct edfa_handle_s {
    int device = 0;
    int nsm = 0;
    edfa_options opt{};
    int32_t Nf = 0, Ne = 0;
    edfa_csr A{}, B{}, C{}, D{};
    // FP32 copies of the block values (precision 1)
    float *a32 = nullptr, *b32 = nullptr, *c32 = nullptr, *d32 = nullptr;
    // B^T pattern: faces of each cell
    int64_t* bt_ptr = nullptr;
    int32_t* bt_col = nullptr;
    // restriction sets
    int64_t* qptr = nullptr;
    int32_t* qidx = nullptr;
    int64_t qtot = 0;
    int32_t qmax = 0;
    double *xval = nullptr, *gval = nullptr;
    float *xval32 = nullptr, *gval32 = nullptr;
    // X~ and G~ as the Schur product reads them: the restriction sets and the
    // local solutions, or what pre-filtration kept of them (own patterns)
    int64_t* x_ptr = nullptr;
    int32_t* x_idx = nullptr;
    int64_t x_tot = 0;
    double* xf64 = nullptr;
    float* xf32 = nullptr;
    int64_t* g_ptr = nullptr;
    int32_t* g_idx = nullptr;
    double* gf64 = nullptr;
    float* gf32 = nullptr;
    // X~ rows: cells whose set holds each face
    int64_t* xr_ptr = nullptr;
    int32_t* xr_cell = nullptr;
    // S~ = D - H~
    int64_t s_nnz = 0;
    int64_t* s_ptr = nullptr;
    int32_t* s_col = nullptr;
    double *h_val = nullptr, *s_val = nullptr;
    float *h_val32 = nullptr, *s_val32 = nullptr;
    int64_t* d_map = nullptr;  // position of each D entry in S~
    // the S~ the inner ILU(0) factorises: (s_ptr, s_col, s_val) itself or,
    // with post-filtration of S~, a filtered copy rebuilt at every Stage 2
    int64_t sf_nnz = 0;
    int64_t* sf_ptr = nullptr;
    int32_t* sf_col = nullptr;
    double* sf_val = nullptr;
    float* sf_val32 = nullptr;
    int64_t* sf_cnt = nullptr;  // [Ne+1] row counts of the filtered copy
    // ILU(0) factors
    edfa::Factor fa, fs;
    // optional multicolour orderings of the factorised A~ (faces) and S~
    // (cells), the ordered matrices and the couplings in the ordered numbering
    // (P_s C P_a^T, P_a B P_s^T); P_s D P_s^T for the product of FGMRES in the
    // ordered numbering
    edfa::Ordering oa, os;
    edfa::OrderedCsr ao, so, co, bo, dord;
    double* ord_bx = nullptr;  // [2 (N_f + N_e)] b and x in the ordered numbering
    int coop_ok = 0;  // cooperative launches possible (the dataflow sweeps of ordered factors)
    edfa::ClusterPlan cp;
    // sweep synchronisation
    int* flags = nullptr;          // [max(Nf, Ne)] completion epochs
    unsigned long long* ticket = nullptr;  // work counter, zeroed before every sync-free launch
    int epoch = 0;
    // apply temporaries (length Nf + Ne) in the working precision
    void* tmp1 = nullptr;
    void* tmp2 = nullptr;
    void* tmp3 = nullptr;
    // two more sweep outputs of the in-place ordered application (ordering 2),
    // so that all six outputs of one application are distinct buffers
    void* tmp4 = nullptr;
    void* tmp5 = nullptr;
    // Krylov workspace
    int32_t kry_m = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *part = nullptr, *hbuf = nullptr;
    double* hbuf_host = nullptr;  // pinned
    int* kgate = nullptr;         // device flag: second Gram-Schmidt pass needed
    // Bi-CGStab workspace: r, r^, p, v, p^, s, s^, t (n each), partial sums, scalars
    double* bcg = nullptr;
    double* bcg_part = nullptr;
    double* bcg_sc = nullptr;
    // device error record and its pinned host mirror
    edfa::DevErr* err = nullptr;
    edfa::DevErr* err_host = nullptr;  // [3]: check_err, two FGMRES iteration slots
    cudaEvent_t ev[14] = {};
    // opt-in per-launch device timing: event pairs recorded around every sweep
    // launch (kind 0..4 = A forward, A backward, S~ forward, S~ backward, both S~ sweeps
    // in one cluster launch) and the first-pass Krylov kernels (5 multi-dot, 6 update,
    // 7 block SpMV)
    uint32_t profiling = 0;  // bit k: time the launches of kind k (edfa_set_profiling_mask)
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_used = 0;
    edfa_stats stats{};
    std::vector<double> hist;
    std::vector<edfa::DBuf> owned;  // every device allocation, released by edfa_free
    // allocations of the S~ factor plan (sweep levels, cluster records): kept
    // apart so that a Stage 2 that changes the pattern of S~ can replace them
    std::vector<edfa::DBuf> owned_s2;
    // workspace of the batched solve, reused across calls with the same layout
    void* batch = nullptr;
    void (*batch_del)(void*) = nullptr;
};

namespace edfa {

// process-wide count of kernel launches issued by the library
void count_launch();

// allocation helpers (record into h->owned)
int dalloc(edfa_handle_s* h, void** p, size_t bytes);
template <class T>
int dalloc_t(edfa_handle_s* h, T** p, size_t count)
{
    return dalloc(h, (void**)p, count * sizeof(T));
}
int check_err(edfa_handle_s* h, cudaStream_t s);  // sync + read device error record
// event pair of one timed launch when profiling is on (edfa_api.cu), else null
cudaEvent_t* prof_begin(edfa_handle_s* h, int kind, cudaStream_t s);
void set_detail(long long d);

// exclusive scan of int64 counts in place: out[i] = sum_{j<i} in[j]; out[n] = total.
int scan_i64(edfa_handle_s* h, int64_t* data, int64_t n, cudaStream_t s);

// launchers (return EDFA_* codes, enqueue only)
int launch_validate(edfa_handle_s* h, const edfa_csr& M, int need_diag, cudaStream_t s);
int build_bt(edfa_handle_s* h, cudaStream_t s);
int build_qsets(edfa_handle_s* h, cudaStream_t s);
int build_qsets_dynamic(edfa_handle_s* h, cudaStream_t s);
int run_local_solves(edfa_handle_s* h, cudaStream_t s);
int build_schur(edfa_handle_s* h, cudaStream_t s);
int stage2_values(edfa_handle_s* h, cudaStream_t s);
// filtration (k_filter.cu)
int prefilter(edfa_handle_s* h, cudaStream_t s);
template <class T>
int postfilter_h(edfa_handle_s* h, T* h_val, cudaStream_t s);
int stage2_pattern(edfa_handle_s* h, cudaStream_t s);
int stage2_symbolic(edfa_handle_s* h, cudaStream_t s);
int factor_plan(edfa_handle_s* h, Factor& f, int32_t n, int64_t nnz, const int64_t* rowptr,
                const int32_t* col, cudaStream_t s);
int factor_plan_common(edfa_handle_s* h, Factor& f, int32_t n, int64_t nnz, const int64_t* rowptr,
                       const int32_t* col, cudaStream_t s);
int factor_numeric(edfa_handle_s* h, Factor& f, const double* vals64, const float* vals32,
                   cudaStream_t s);
int apply_prec(edfa_handle_s* h, const double* r, double* z, cudaStream_t s);
// chain-decomposed sweeps (k_chain.cu)
int chain_plan_build(edfa_handle_s* h, Factor& f, cudaStream_t s);
int chain_plan_values(edfa_handle_s* h, Factor& f, cudaStream_t s);
template <class T, class TB, class TO, int FWD>
int chain_sweep(edfa_handle_s* h, const Factor& f, const TB* base, const int64_t* mptr, const int32_t* mcol,
                const T* mval, const TO* mvec, TO* out, cudaStream_t s);
// single-cluster S~ solves (k_cluster.cu)
int cluster_plan_build(edfa_handle_s* h, cudaStream_t s);
int cluster_plan_fill(edfa_handle_s* h, cudaStream_t s);
template <class T>
int s_cluster_solve(edfa_handle_s* h, const double* rp, const int64_t* mptr, const int32_t* mcol, const T* mval,
                    const T* mv, T* out, cudaStream_t s, cudaEvent_t* pe);
int matvec(edfa_handle_s* h, const double* x, double* y, cudaStream_t s);
// multicolour orderings (k_order.cu)
int order_colour(edfa_handle_s* h, Ordering& o, int32_t n, const int64_t* rowptr, const int32_t* col, int64_t nnz,
                 cudaStream_t s, int32_t block = 1);
int order_matrix(edfa_handle_s* h, OrderedCsr& m, int32_t nrows, const int64_t* rowptr, const int32_t* col,
                 int64_t nnz, const int32_t* rperm, const int32_t* cmap, cudaStream_t s);
int order_values(edfa_handle_s* h, OrderedCsr& m, const double* src64, const float* src32, cudaStream_t s);
int order_stage2_symbolic(edfa_handle_s* h, cudaStream_t s);
int order_a_factor(edfa_handle_s* h, cudaStream_t s);
int stage2_numeric(edfa_handle_s* h, cudaStream_t s);
// vectors between the natural and the ordered numbering (faces through P_a,
// identity without an ordering of A~; cells through P_s)
int order_vector(edfa_handle_s* h, const double* in, double* out, int to_ordered, cudaStream_t s);
// the block preconditioner and the block product with vectors in the ordered numbering
int apply_prec_ordered_numbering(edfa_handle_s* h, const double* r, double* z, int prefilled, cudaStream_t s);
// buffers the next in-place ordered application with output z writes through
// dataflow sweeps, to be filled with the all-ones pattern beforehand; returns
// the number of entries (0: nothing to prefill, the sweeps fill their own)
int ordered_prefill_list(edfa_handle_s* h, double* z, FillList& fl);
int matvec_ordered_numbering(edfa_handle_s* h, const double* x, double* y, cudaStream_t s);
int to_f32(const double* in, float* out, int64_t n, cudaStream_t s);
int to_f64_launch(const float* in, double* out, int64_t n, cudaStream_t s);

// Krylov building blocks (k_krylov.cu)
int kry_multidot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* part, double* out,
                 const double* add, double* out_sum, int with_self, cudaStream_t s, const int* gate = nullptr);
// fill the buffers of fl with the all-ones pattern (one launch)
int kry_fill(const FillList& fl, cudaStream_t s);
// w -= V h (and ||w||^2); with `fill` the same launch also fills those
// buffers with the all-ones pattern (the next application's sweep outputs)
int kry_update(const double* V, int64_t ld, int nv, const double* hcoef, double* w, int64_t n, double* part,
               double* nrm2_out, cudaStream_t s, const int* gate = nullptr, const FillList* fill = nullptr);
int kry_dgks(const double* nrm2_after, const double* nrm2_before, int* gate, cudaStream_t s);
int kry_scale_from(const double* w, double* v, int64_t n, const double* nrm2, double* out_norm, cudaStream_t s);
int kry_scale_const(const double* w, double* v, int64_t n, double alpha, cudaStream_t s);
int kry_combine(const double* Z, int64_t ld, int k, const double* y, double* x, int64_t n, cudaStream_t s);
int kry_residual(const double* b, double* r, int64_t n, double* part, double* nrm2_out, cudaStream_t s);
int64_t kry_part_size(int64_t n, int nvmax);
// Bi-CGStab vector updates (k_krylov.cu)
int kry_bcg_p(const double* r, double* p, const double* v, double beta, double omega, int64_t n, cudaStream_t s);
int kry_bcg_s(const double* r, const double* v, double alpha, double* sv, int64_t n, double* part, double* nrm2_out,
              cudaStream_t s);
int kry_bcg_xr(double* x, const double* ph, const double* sh, const double* sv, const double* t, double alpha,
               double omega, double* r, int64_t n, cudaStream_t s);
int kry_axpy(double* x, const double* y, double a, int64_t n, cudaStream_t s);

}  // namespace edfa
