// C ABI of libedfa.so: handle lifecycle, Stage 1 / Stage 2 orchestration
// (Algorithms 1 and 2), the preconditioner application and the outer flexible
// GMRES driver.  See include/edfa.h for argument meaning, layout, ownership and
// error behaviour.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>

#include "internal.cuh"

using namespace edfa;

static thread_local long long g_detail = -1;
static std::atomic<long long> g_launches{0};

namespace edfa {

void set_detail(long long d) { g_detail = d; }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// per-launch timing (edfa_set_profiling): a pair of events per timed launch,
// tagged 0 A fwd, 1 A bwd, 2 S fwd, 3 S bwd, 4 S fwd+bwd in one cluster launch,
// 5 first-pass multi-dot, 6 first-pass update, 7 block SpMV; returns null
// when profiling is off.  With s == -1 the caller records both events.
cudaEvent_t* prof_begin(edfa_handle_s* h, int kind, cudaStream_t s)
{
    if (!((h->profiling >> kind) & 1u)) return nullptr;
    if (h->prof_used * 2 + 2 > h->prof_ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            h->prof_ev.push_back(e);
        }
        h->prof_kind.resize(h->prof_ev.size() / 2);
    }
    cudaEvent_t* pe = &h->prof_ev[2 * h->prof_used];
    h->prof_kind[h->prof_used] = kind;
    h->prof_used++;
    if (s != (cudaStream_t)-1) cudaEventRecord(pe[0], s);
    return pe;
}

// fold the recorded event pairs into the stats (stream already synchronised)
static void prof_collect(edfa_handle_s* h)
{
    for (size_t k = 0; k < h->prof_used; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]) == cudaSuccess) {
            const int kind = h->prof_kind[k];
            if (kind < 5) {
                h->stats.sweep_ms[kind] += ms;
                h->stats.sweep_n[kind] += 1;
            } else {
                h->stats.kry_ms[kind - 5] += ms;
                h->stats.kry_n[kind - 5] += 1;
            }
        }
    }
    h->prof_used = 0;
}

int dalloc(edfa_handle_s* h, void** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return EDFA_ERR_OOM;
    }
    h->owned.push_back(DBuf{q, bytes});
    *p = q;
    return EDFA_OK;
}

int check_err(edfa_handle_s* h, cudaStream_t s)
{
    cudaMemcpyAsync(h->err_host, h->err, sizeof(DevErr), cudaMemcpyDeviceToHost, s);
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        fprintf(stderr, "edfa: CUDA error %s\n", cudaGetErrorString(ce));
        return EDFA_ERR_CUDA;
    }
    if (h->err_host->code != 0) {
        int code = h->err_host->code;
        set_detail(h->err_host->detail);
        cudaMemsetAsync(h->err, 0, sizeof(DevErr), s);
        cudaStreamSynchronize(s);
        h->err_host->code = 0;
        return code;
    }
    return EDFA_OK;
}

}  // namespace edfa

static void free_all(edfa_handle_s* h)
{
    if (!h) return;
    if (h->batch_del) h->batch_del(h->batch);
    for (auto& b : h->owned) cudaFree(b.p);
    h->owned.clear();
    for (auto& b : h->owned_s2) cudaFree(b.p);
    h->owned_s2.clear();
    if (h->err_host) cudaFreeHost(h->err_host);
    if (h->hbuf_host) cudaFreeHost(h->hbuf_host);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->prof_ev) cudaEventDestroy(e);
    delete h;
}

static bool csr_shape_ok(const edfa_csr* M, int32_t r, int32_t c)
{
    return M && M->nrows == r && M->ncols == c && M->nnz >= 0;
}

extern "C" {

void edfa_default_options(edfa_options* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->qmode = EDFA_Q_OWN;
    o->thresh = 0.05;
    o->n_add = 1;
    o->n_ent = 4;
    o->it_max = 100;
    o->schur_form = 0;
    o->variant = 0;
    o->precision = 0;
    o->warps_per_block = 0;
    o->filtration = EDFA_FILT_NONE;
    o->tau_filt = 0.0;
}

const char* edfa_strerror(int code)
{
    switch (code) {
    case EDFA_OK: return "ok";
    case EDFA_ERR_INVALID: return "invalid argument (sizes, pattern, option or non-finite value)";
    case EDFA_ERR_CUDA: return "CUDA runtime error";
    case EDFA_ERR_OOM: return "device allocation failed";
    case EDFA_ERR_BREAKDOWN: return "zero or wrong-signed pivot (local solve or ILU(0))";
    case EDFA_ERR_NOT_CONVERGED: return "FGMRES did not converge within maxit";
    case EDFA_ERR_TIMEOUT: return "bounded device wait timed out";
    case EDFA_ERR_BOUNDS: return "ragged set exceeds a fixed device capacity";
    case EDFA_ERR_UNSUPPORTED: return "option combination not supported";
    default: return "unknown error";
    }
}

int64_t edfa_last_error_detail(void) { return g_detail; }

#define TRY(x)                                   \
    do {                                         \
        int _rc = (x);                           \
        if (_rc != EDFA_OK) { free_all(h); return _rc; } \
    } while (0)

int edfa_build(edfa_handle* out, const edfa_csr* A, const edfa_csr* B, const edfa_csr* C, const edfa_csr* D,
               const edfa_options* opt, edfa_stream stream)
{
    g_detail = -1;
    if (!out || !A || !B || !C || !D) return EDFA_ERR_INVALID;
    *out = nullptr;
    const int32_t Nf = A->nrows, Ne = D->nrows;
    if (Nf < 0 || Ne < 0 || (int64_t)Nf + Ne >= INT32_MAX) return EDFA_ERR_INVALID;
    if (!csr_shape_ok(A, Nf, Nf) || !csr_shape_ok(B, Nf, Ne) || !csr_shape_ok(C, Ne, Nf) || !csr_shape_ok(D, Ne, Ne))
        return EDFA_ERR_INVALID;
    edfa_options o;
    if (opt) o = *opt; else edfa_default_options(&o);
    if (o.qmode < EDFA_Q_OWN || o.qmode > EDFA_Q_GIVEN) return EDFA_ERR_INVALID;
    if (o.sweep_mode < 0 || o.sweep_mode > 2) return EDFA_ERR_INVALID;
    if (o.qmode == EDFA_Q_GIVEN && (!o.qptr || !o.qidx)) return EDFA_ERR_INVALID;
    if (o.qmode == EDFA_Q_THRESH && !(o.thresh >= 0.0)) return EDFA_ERR_INVALID;
    if (o.qmode == EDFA_Q_DYNAMIC && (o.n_add < 0 || o.n_ent < 0 || o.it_max < 0)) return EDFA_ERR_INVALID;
    if (o.schur_form < 0 || o.schur_form > 1 || o.variant < 0 || o.variant > 1 || o.precision < 0 ||
        o.precision > 1)
        return EDFA_ERR_INVALID;
    if (o.filtration < EDFA_FILT_NONE || o.filtration > EDFA_FILT_POST_S || !(o.tau_filt >= 0.0) ||
        !std::isfinite(o.tau_filt))
        return EDFA_ERR_INVALID;
    if (o.ordering < 0 || o.ordering > 2 || o.s_block < 0 || o.s_block > 16) return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;

    edfa_handle_s* h = new (std::nothrow) edfa_handle_s();
    if (!h) return EDFA_ERR_OOM;
    h->opt = o;
    h->Nf = Nf;
    h->Ne = Ne;
    h->A = *A;
    h->B = *B;
    h->C = *C;
    h->D = *D;
    if (cudaGetDevice(&h->device) != cudaSuccess) { free_all(h); return EDFA_ERR_CUDA; }
    cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
    if (h->nsm < 1) h->nsm = 1;
    TRY(dalloc_t(h, &h->err, 1));
    if (cudaMallocHost((void**)&h->err_host, 3 * sizeof(DevErr)) != cudaSuccess) { free_all(h); return EDFA_ERR_OOM; }
    memset(h->err_host, 0, 3 * sizeof(DevErr));
    cudaMemsetAsync(h->err, 0, sizeof(DevErr), s);
    TRY(dalloc_t(h, &h->ticket, 1));
    const int32_t nmax = Nf > Ne ? Nf : Ne;
    TRY(dalloc_t(h, &h->flags, (size_t)(nmax > 0 ? nmax : 1)));
    cudaMemsetAsync(h->flags, 0, (size_t)(nmax > 0 ? nmax : 1) * sizeof(int), s);
    for (auto& e : h->ev) cudaEventCreate(&e);

    // inputs
    TRY(launch_validate(h, *A, 1, s));
    TRY(launch_validate(h, *B, 0, s));
    TRY(launch_validate(h, *C, 0, s));
    TRY(launch_validate(h, *D, 0, s));
    TRY(check_err(h, s));
    if (o.precision == 1) {
        TRY(dalloc_t(h, &h->a32, (size_t)(A->nnz > 0 ? A->nnz : 1)));
        TRY(dalloc_t(h, &h->b32, (size_t)(B->nnz > 0 ? B->nnz : 1)));
        TRY(dalloc_t(h, &h->c32, (size_t)(C->nnz > 0 ? C->nnz : 1)));
        TRY(to_f32(A->val, h->a32, A->nnz, s));
        TRY(to_f32(B->val, h->b32, B->nnz, s));
        TRY(to_f32(C->val, h->c32, C->nnz, s));
    }

    // Stage 1 (Algorithm 1)
    cudaEventRecord(h->ev[0], s);
    TRY(build_bt(h, s));
    if (o.qmode == EDFA_Q_DYNAMIC) TRY(build_qsets_dynamic(h, s));
    else TRY(build_qsets(h, s));
    cudaEventRecord(h->ev[1], s);
    TRY(run_local_solves(h, s));
    cudaEventRecord(h->ev[2], s);
    TRY(check_err(h, s));
    cudaEventRecord(h->ev[3], s);
    TRY(prefilter(h, s));
    TRY(build_schur(h, s));
    cudaEventRecord(h->ev[4], s);
    if (o.ordering == 2) {
        TRY(order_a_factor(h, s));
    } else {
        TRY(factor_plan(h, h->fa, Nf, A->nnz, A->rowptr, A->col, s));
        if (o.sweep_mode != 1) TRY(chain_plan_build(h, h->fa, s));
        TRY(factor_numeric(h, h->fa, A->val, h->a32, s));
        TRY(chain_plan_values(h, h->fa, s));
    }
    cudaEventRecord(h->ev[5], s);
    TRY(check_err(h, s));

    // Stage 2 (Algorithm 2) with the given D
    cudaEventRecord(h->ev[6], s);
    TRY(stage2_values(h, s));
    cudaEventRecord(h->ev[8], s);
    TRY(stage2_pattern(h, s));
    TRY(stage2_symbolic(h, s));
    cudaEventRecord(h->ev[9], s);
    TRY(stage2_numeric(h, s));
    cudaEventRecord(h->ev[10], s);
    TRY(cluster_plan_fill(h, s));
    cudaEventRecord(h->ev[7], s);

    // application temporaries
    const size_t esz = o.precision == 1 ? sizeof(float) : sizeof(double);
    TRY(dalloc(h, &h->tmp1, (size_t)(nmax > 0 ? nmax : 1) * esz));
    TRY(dalloc(h, &h->tmp2, (size_t)(nmax > 0 ? nmax : 1) * esz));
    TRY(dalloc(h, &h->tmp3, (size_t)(nmax > 0 ? nmax : 1) * esz));
    if (o.ordering == 2) {
        TRY(dalloc(h, &h->tmp4, (size_t)(nmax > 0 ? nmax : 1) * esz));
        TRY(dalloc(h, &h->tmp5, (size_t)(nmax > 0 ? nmax : 1) * esz));
    }
    TRY(check_err(h, s));

    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]); h->stats.ms_qsets = ms;
    cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]); h->stats.ms_local = ms;
    cudaEventElapsedTime(&ms, h->ev[3], h->ev[4]); h->stats.ms_schur = ms;
    cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]); h->stats.ms_ilu_a = ms;
    cudaEventElapsedTime(&ms, h->ev[6], h->ev[7]); h->stats.ms_stage2 = ms;
    cudaEventElapsedTime(&ms, h->ev[6], h->ev[8]); h->stats.ms_s_values = ms;
    cudaEventElapsedTime(&ms, h->ev[8], h->ev[9]); h->stats.ms_s_plan = ms;
    cudaEventElapsedTime(&ms, h->ev[9], h->ev[10]); h->stats.ms_s_factor = ms;
    cudaEventElapsedTime(&ms, h->ev[10], h->ev[7]); h->stats.ms_s_cluster = ms;
    h->stats.n_local = Ne;
    h->stats.q_total = h->qtot;
    h->stats.q_max = h->qmax;
    h->stats.s_nnz = h->sf_nnz;
    h->stats.s_cluster = h->cp.state == 1;
    h->stats.s_cluster_bytes = h->cp.state == 1 ? h->cp.bytes : 0;
    h->stats.levels_a = h->fa.fwd.nlevels;
    h->stats.levels_s = h->fs.fwd.nlevels;
    *out = h;
    return EDFA_OK;
}

#undef TRY

int edfa_setup(edfa_handle h, const edfa_csr* D, edfa_stream stream)
{
    g_detail = -1;
    if (!h || !D) return EDFA_ERR_INVALID;
    if (D->nrows != h->Ne || D->ncols != h->Ne || D->nnz != h->D.nnz) return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_validate(h, *D, 0, s);
    if (!rc) rc = check_err(h, s);
    if (rc) return rc;
    h->D = *D;
    const bool replan = h->opt.filtration == EDFA_FILT_POST_S;
    cudaEventRecord(h->ev[6], s);
    rc = stage2_values(h, s);
    cudaEventRecord(h->ev[8], s);
    // post-filtration of S~ changes its pattern with D: new levels and records
    if (!rc && replan) rc = stage2_pattern(h, s);
    if (!rc && replan) rc = stage2_symbolic(h, s);
    cudaEventRecord(h->ev[9], s);
    if (!rc) rc = stage2_numeric(h, s);
    cudaEventRecord(h->ev[10], s);
    if (!rc) rc = cluster_plan_fill(h, s);
    cudaEventRecord(h->ev[7], s);
    if (!rc) rc = check_err(h, s);
    if (rc) return rc;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[6], h->ev[7]);
    h->stats.ms_stage2 = ms;
    cudaEventElapsedTime(&ms, h->ev[6], h->ev[8]); h->stats.ms_s_values = ms;
    h->stats.ms_s_plan = 0;
    if (replan) {
        cudaEventElapsedTime(&ms, h->ev[8], h->ev[9]);
        h->stats.ms_s_plan = ms;
        h->stats.s_nnz = h->sf_nnz;
        h->stats.levels_s = h->fs.fwd.nlevels;
        h->stats.s_cluster = h->cp.state == 1;
        h->stats.s_cluster_bytes = h->cp.state == 1 ? h->cp.bytes : 0;
    }
    cudaEventElapsedTime(&ms, h->ev[9], h->ev[10]); h->stats.ms_s_factor = ms;
    cudaEventElapsedTime(&ms, h->ev[10], h->ev[7]); h->stats.ms_s_cluster = ms;
    return EDFA_OK;
}

int edfa_apply(edfa_handle h, const double* r, double* z, edfa_stream stream)
{
    if (!h || (!r && h->Nf + h->Ne > 0) || (!z && h->Nf + h->Ne > 0)) return EDFA_ERR_INVALID;
    return apply_prec(h, r, z, (cudaStream_t)stream);
}

int edfa_matvec(edfa_handle h, const double* x, double* y, edfa_stream stream)
{
    if (!h || (!x && h->Nf + h->Ne > 0) || (!y && h->Nf + h->Ne > 0)) return EDFA_ERR_INVALID;
    return matvec(h, x, y, (cudaStream_t)stream);
}

// Right-preconditioned flexible GMRES(m) (Saad, Alg. 9.6): Arnoldi with
// classical Gram-Schmidt in FP64 on the device, repeated once when the first
// pass shrank the norm by more than a factor of 10 (Rutishauser's criterion), the
// (m+1) x m Hessenberg least-squares problem by Givens rotations on the host
// (one (j+2)-value device->host read per inner iteration, read while the next
// iteration runs), x0 = 0, and the
// true residual ||b - A x|| checked at the end of every cycle; the outer loop
// restarts while it exceeds rtol ||b||.
int edfa_solve(edfa_handle h, const double* b, double* x, int32_t m, double rtol, int32_t maxit,
               edfa_solve_info* info, edfa_stream stream)
{
    g_detail = -1;
    if (!h || m < 1 || m > 126 || !(rtol >= 0.0) || maxit < 0) return EDFA_ERR_INVALID;
    const int64_t n = (int64_t)h->Nf + h->Ne;
    if (n > 0 && (!b || !x)) return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->kry_m < m) {
        // (re)allocate workspace; previous buffers stay owned until edfa_free
        if (dalloc_t(h, &h->V, (size_t)(m + 1) * n) || dalloc_t(h, &h->Z, (size_t)m * n) ||
            dalloc_t(h, &h->w, (size_t)(n > 0 ? n : 1)) || dalloc_t(h, &h->part, (size_t)kry_part_size(n, m + 1)) ||
            dalloc_t(h, &h->hbuf, (size_t)4 * (m + 2)) || dalloc_t(h, &h->kgate, 1))
            return EDFA_ERR_OOM;
        if (h->hbuf_host) cudaFreeHost(h->hbuf_host);
        if (cudaMallocHost((void**)&h->hbuf_host, sizeof(double) * 4 * (m + 2)) != cudaSuccess) return EDFA_ERR_OOM;
        h->kry_m = m;
    }
    // with an ordering the iteration runs in the ordered numbering: b is
    // permuted once, the preconditioner and the product work in place, and x is
    // permuted back at the end
    const bool ordn = h->opt.ordering >= 1 && n > 0;
    const double* bb = b;
    double* xx = x;
    if (ordn) {
        if (!h->ord_bx && dalloc_t(h, &h->ord_bx, (size_t)2 * n)) return EDFA_ERR_OOM;
        bb = h->ord_bx;
        xx = h->ord_bx + n;
    }
    // with both orderings the sweep outputs of the application of iteration
    // j + 1 are filled with the all-ones pattern by the update of iteration j
    // (the first of a cycle by a fill before it), not by a memset per sweep
    FillList probe_fl;
    const bool prefill = ordn && ordered_prefill_list(h, h->Z, probe_fl) > 0;
    auto prec = [&](const double* r, double* z) {
        return ordn ? apply_prec_ordered_numbering(h, r, z, prefill ? 1 : 0, s) : apply_prec(h, r, z, s);
    };
    auto mv = [&](const double* v, double* y) {
        return ordn ? matvec_ordered_numbering(h, v, y, s) : matvec(h, v, y, s);
    };
    double* h1 = h->hbuf;
    double* h2 = h->hbuf + (m + 2);
    double* hf = h->hbuf + 2 * (m + 2);
    double* misc = h->hbuf + 3 * (m + 2);  // [0] = squared norm, [1] = norm
    double* hh = h->hbuf_host;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
    h->hist.assign(1, 1.0);
    edfa_solve_info loc{};
    cudaEventRecord(h->ev[0], s);

    int rc = EDFA_OK;
    if (ordn && (rc = order_vector(h, b, h->ord_bx, 1, s))) return rc;
    // ||b||
    rc = kry_multidot(h->V, n, 0, bb, n, h->part, misc, nullptr, nullptr, 1, s);
    if (rc) return rc;
    cudaMemcpyAsync(hh, misc, sizeof(double), cudaMemcpyDeviceToHost, s);
    rc = check_err(h, s);
    if (rc) return rc;
    const double bnorm = std::sqrt(hh[0]);
    cudaMemsetAsync(xx, 0, (size_t)n * sizeof(double), s);
    if (bnorm == 0.0 || n == 0) {
        if (ordn) cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), s);
        loc.converged = 1;
        if (info) *info = loc;
        return check_err(h, s);
    }
    cudaMemcpyAsync(h->w, bb, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    double beta = bnorm;
    int it = 0, status = EDFA_ERR_NOT_CONVERGED;
    while (it < maxit) {
        rc = kry_scale_const(h->w, h->V, n, 1.0 / beta, s);
        if (rc) return rc;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jlast = -1;
        // Iteration j+1 is enqueued before the host waits for iteration j's
        // Hessenberg column, so the device does not idle through the host's
        // round trip; when iteration j ends the cycle, iteration j+1's work is
        // discarded (it writes only V_{j+2}, Z_{j+1} and scratch).
        auto enqueue = [&](int j) -> int {
            double* vj = h->V + (int64_t)j * n;
            double* zj = h->Z + (int64_t)j * n;
            int e;
            if ((e = prec(vj, zj))) return e;
            cudaEvent_t* pe = prof_begin(h, 7, s);
            if ((e = mv(zj, h->w))) return e;
            if (pe) cudaEventRecord(pe[1], s);
            // classical Gram-Schmidt, repeated when the reorthogonalisation test asks for it
            // (decided on the device: the second pass's kernels read the gate)
            const int nv = j + 1;
            pe = prof_begin(h, 5, s);
            if ((e = kry_multidot(h->V, n, nv, h->w, n, h->part, h1, nullptr, nullptr, 1, s))) return e;
            if (pe) {
                cudaEventRecord(pe[1], s);
                h->stats.kry_vecs += nv;
            }
            FillList fl;
            if (prefill && j + 1 < m) ordered_prefill_list(h, h->Z + (int64_t)(j + 1) * n, fl);
            pe = prof_begin(h, 6, s);
            if ((e = kry_update(h->V, n, nv, h1, h->w, n, h->part, misc, s, nullptr, &fl))) return e;
            if (pe) cudaEventRecord(pe[1], s);
            if ((e = kry_dgks(misc, h1 + nv, h->kgate, s))) return e;
            if ((e = kry_multidot(h->V, n, nv, h->w, n, h->part, h2, h1, hf, 0, s, h->kgate))) return e;
            if ((e = kry_update(h->V, n, nv, h2, h->w, n, h->part, misc, s, h->kgate))) return e;
            if ((e = kry_scale_from(h->w, h->V + (int64_t)(j + 1) * n, n, misc, hf + nv, s))) return e;
            // the column and the device error record into this iteration's host slot
            cudaMemcpyAsync(hh + (j & 1) * (m + 2), hf, sizeof(double) * (nv + 1), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(h->err_host + 1 + (j & 1), h->err, sizeof(DevErr), cudaMemcpyDeviceToHost, s);
            return cudaEventRecord(h->ev[12 + (j & 1)], s) == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
        };
        if (prefill) {
            FillList fl;
            ordered_prefill_list(h, h->Z, fl);
            if ((rc = kry_fill(fl, s))) return rc;
        }
        if ((rc = enqueue(0))) return rc;
        for (int j = 0; j < m && it < maxit; ++j) {
            if (j + 1 < m && it + 1 < maxit && (rc = enqueue(j + 1))) return rc;
            if (cudaEventSynchronize(h->ev[12 + (j & 1)]) != cudaSuccess) return check_err(h, s);
            if (h->err_host[1 + (j & 1)].code != 0) return check_err(h, s);
            const double* col = hh + (j & 1) * (m + 2);
            for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = col[i];
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            double den = std::sqrt(a * a + c * c);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? c / den : 0.0;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            jlast = j;
            const double est = std::fabs(g[j + 1]) / bnorm;
            h->hist.push_back(est);
            loc.est_rel = est;
            if (est <= rtol || col[j + 1] == 0.0) break;
        }
        const int k = jlast + 1;
        for (int i = k - 1; i >= 0; --i) {
            double v = g[i];
            for (int l = i + 1; l < k; ++l) v -= H[(size_t)i * m + l] * y[l];
            y[i] = H[(size_t)i * m + i] != 0.0 ? v / H[(size_t)i * m + i] : 0.0;
        }
        double* hy = hh + 2 * (m + 2);  // not a slot an iteration in flight writes
        memcpy(hy, y.data(), sizeof(double) * k);
        cudaMemcpyAsync(h1, hy, sizeof(double) * k, cudaMemcpyHostToDevice, s);
        if ((rc = kry_combine(h->Z, n, k, h1, xx, n, s))) return rc;
        if ((rc = mv(xx, h->w))) return rc;
        if ((rc = kry_residual(bb, h->w, n, h->part, misc, s))) return rc;
        cudaMemcpyAsync(hh, misc, sizeof(double), cudaMemcpyDeviceToHost, s);
        if ((rc = check_err(h, s))) return rc;
        beta = std::sqrt(hh[0]);
        loc.true_rel = beta / bnorm;
        if (loc.true_rel <= rtol) { status = EDFA_OK; break; }
        if (beta == 0.0) { status = EDFA_OK; break; }
        loc.restarts++;
    }
    if (ordn && (rc = order_vector(h, xx, x, 0, s))) return rc;
    cudaEventRecord(h->ev[1], s);
    cudaEventSynchronize(h->ev[1]);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->stats.ms_solve = ms;
    prof_collect(h);
    loc.iterations = it;
    loc.converged = status == EDFA_OK;
    if (info) *info = loc;
    return status;
}

// Right-preconditioned Bi-CGStab (van der Vorst 1992), the outer solver of the
// paper's experiments (Sec. 4): x0 = 0, stop at ||r_k|| / ||r_0|| <= rtol with
// the true residual confirmed; restart from the true residual when it is not met
// or on a breakdown.  Scalars are read back to the host four times per iteration.
int edfa_solve_bicgstab(edfa_handle h, const double* b, double* x, double rtol, int32_t maxit,
                        edfa_solve_info* info, edfa_stream stream)
{
    g_detail = -1;
    if (!h || !(rtol >= 0.0) || maxit < 0) return EDFA_ERR_INVALID;
    const int64_t n = (int64_t)h->Nf + h->Ne;
    if (n > 0 && (!b || !x)) return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->bcg) {
        if (dalloc_t(h, &h->bcg, (size_t)8 * (n > 0 ? n : 1)) ||
            dalloc_t(h, &h->bcg_part, (size_t)kry_part_size(n > 0 ? n : 1, 2)) || dalloc_t(h, &h->bcg_sc, 8))
            return EDFA_ERR_OOM;
        if (!h->hbuf_host) {
            if (cudaMallocHost((void**)&h->hbuf_host, sizeof(double) * 16) != cudaSuccess) return EDFA_ERR_OOM;
        }
    }
    double* r = h->bcg;
    double* rh = r + n;
    double* p = rh + n;
    double* v = p + n;
    double* ph = v + n;
    double* sv = ph + n;
    double* sh = sv + n;
    double* t = sh + n;
    double* sc = h->bcg_sc;  // device scalars
    double* hh = h->hbuf_host;
    edfa_solve_info loc{};
    h->hist.assign(1, 1.0);
    cudaEventRecord(h->ev[0], s);
    int rc;
    auto fetch = [&](int k) -> int {
        cudaMemcpyAsync(hh, sc, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
        return check_err(h, s);
    };
    cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), s);
    if ((rc = kry_multidot(nullptr, n, 0, b, n, h->bcg_part, sc, nullptr, nullptr, 1, s))) return rc;
    if ((rc = fetch(1))) return rc;
    const double bnorm = std::sqrt(hh[0]);
    if (bnorm == 0.0 || n == 0) {
        loc.converged = 1;
        if (info) *info = loc;
        return EDFA_OK;
    }
    cudaMemcpyAsync(r, b, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    int it = 0, status = EDFA_ERR_NOT_CONVERGED;
    for (;;) {
        cudaMemcpyAsync(rh, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(p, 0, (size_t)n * sizeof(double), s);
        cudaMemsetAsync(v, 0, (size_t)n * sizeof(double), s);
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        // rho = (r^, r)
        if ((rc = kry_multidot(rh, n, 1, r, n, h->bcg_part, sc, nullptr, nullptr, 0, s))) return rc;
        if ((rc = fetch(1))) return rc;
        double rho = hh[0];
        while (it < maxit) {
            if (rho == 0.0) break;  // restart
            const double beta = (rho / rho_old) * (alpha / omega);
            if ((rc = kry_bcg_p(r, p, v, beta, omega, n, s))) return rc;
            if ((rc = apply_prec(h, p, ph, s))) return rc;
            if ((rc = matvec(h, ph, v, s))) return rc;
            if ((rc = kry_multidot(rh, n, 1, v, n, h->bcg_part, sc, nullptr, nullptr, 0, s))) return rc;
            if ((rc = fetch(1))) return rc;
            const double rv = hh[0];
            if (rv == 0.0) break;  // restart
            alpha = rho / rv;
            if ((rc = kry_bcg_s(r, v, alpha, sv, n, h->bcg_part, sc, s))) return rc;
            if ((rc = fetch(1))) return rc;
            ++it;
            const double snorm = std::sqrt(hh[0]);
            if (snorm / bnorm <= rtol) {
                if ((rc = kry_axpy(x, ph, alpha, n, s))) return rc;
                cudaMemcpyAsync(r, sv, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
                h->hist.push_back(snorm / bnorm);
                loc.est_rel = snorm / bnorm;
                break;
            }
            if ((rc = apply_prec(h, sv, sh, s))) return rc;
            if ((rc = matvec(h, sh, t, s))) return rc;
            // (s, t) and (t, t)
            if ((rc = kry_multidot(sv, n, 1, t, n, h->bcg_part, sc, nullptr, nullptr, 1, s))) return rc;
            if ((rc = fetch(2))) return rc;
            omega = hh[1] != 0.0 ? hh[0] / hh[1] : 0.0;
            if ((rc = kry_bcg_xr(x, ph, sh, sv, t, alpha, omega, r, n, s))) return rc;
            rho_old = rho;
            // next rho = (r^, r) and ||r||^2
            if ((rc = kry_multidot(rh, n, 1, r, n, h->bcg_part, sc, nullptr, nullptr, 1, s))) return rc;
            if ((rc = fetch(2))) return rc;
            rho = hh[0];
            const double rn = std::sqrt(hh[1]);
            h->hist.push_back(rn / bnorm);
            loc.est_rel = rn / bnorm;
            if (rn / bnorm <= rtol) break;
            if (omega == 0.0) break;  // restart
        }
        // true residual
        if ((rc = matvec(h, x, t, s))) return rc;
        if ((rc = kry_residual(b, t, n, h->bcg_part, sc, s))) return rc;
        if ((rc = fetch(1))) return rc;
        loc.true_rel = std::sqrt(hh[0]) / bnorm;
        cudaMemcpyAsync(r, t, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (loc.true_rel <= rtol) { status = EDFA_OK; break; }
        if (it >= maxit) break;
        loc.restarts++;
    }
    cudaEventRecord(h->ev[1], s);
    cudaEventSynchronize(h->ev[1]);
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->stats.ms_solve = ms;
    prof_collect(h);
    loc.iterations = it;
    loc.converged = status == EDFA_OK;
    if (info) *info = loc;
    return status;
}

int32_t edfa_history(edfa_handle h, double* hist, int32_t cap)
{
    if (!h || !hist || cap <= 0) return 0;
    int32_t n = (int32_t)h->hist.size();
    if (n > cap) n = cap;
    memcpy(hist, h->hist.data(), sizeof(double) * n);
    return n;
}

int edfa_get_view(edfa_handle h, edfa_view* v)
{
    if (!h || !v) return EDFA_ERR_INVALID;
    v->Nf = h->Nf;
    v->Ne = h->Ne;
    v->qptr = h->qptr;
    v->qidx = h->qidx;
    v->xval = h->xval;
    v->gval = h->gval;
    v->xval_f32 = h->xval32;
    // the S~ the preconditioner factorises (after post-filtration of S~, if any)
    v->s_nnz = h->sf_nnz;
    v->s_rowptr = h->sf_ptr;
    v->s_col = h->sf_col;
    v->s_val = h->sf_val;
    v->s_val_f32 = h->sf_val32;
    v->a_ncolours = h->oa.on ? h->oa.ncolours : 0;
    v->s_ncolours = h->os.on ? h->os.ncolours : 0;
    v->a_perm = h->oa.on ? h->oa.perm : nullptr;
    v->s_perm = h->os.on ? h->os.perm : nullptr;
    v->fa_nnz = h->fa.nnz;
    v->fa_rowptr = h->fa.rowptr;
    v->fa_col = h->fa.col;
    v->fa_lu = h->fa.lu64;
    v->fa_lu_f32 = h->fa.lu32;
    v->fs_nnz = h->fs.nnz;
    v->fs_rowptr = h->fs.rowptr;
    v->fs_col = h->fs.col;
    v->fs_lu = h->fs.lu64;
    v->fs_lu_f32 = h->fs.lu32;
    return EDFA_OK;
}

int edfa_get_stats(edfa_handle h, edfa_stats* st)
{
    if (!h || !st) return EDFA_ERR_INVALID;
    if (h->prof_used) {
        cudaDeviceSynchronize();
        prof_collect(h);
    }
    *st = h->stats;
    return EDFA_OK;
}

int edfa_set_profiling(edfa_handle h, int32_t on) { return edfa_set_profiling_mask(h, on ? 0xFFu : 0u); }

int edfa_set_profiling_mask(edfa_handle h, uint32_t kinds)
{
    if (!h || (kinds >> 8) != 0) return EDFA_ERR_INVALID;
    h->profiling = kinds;
    h->prof_used = 0;
    for (int k = 0; k < 5; ++k) { h->stats.sweep_ms[k] = 0; h->stats.sweep_n[k] = 0; }
    for (int k = 0; k < 3; ++k) { h->stats.kry_ms[k] = 0; h->stats.kry_n[k] = 0; }
    h->stats.kry_vecs = 0;
    return EDFA_OK;
}

int64_t edfa_launch_count(void) { return g_launches.load(); }

int edfa_free(edfa_handle h)
{
    if (!h) return EDFA_ERR_INVALID;
    cudaDeviceSynchronize();
    free_all(h);
    return EDFA_OK;
}

}  // extern "C"
