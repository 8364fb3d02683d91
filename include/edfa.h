/*
 * edfa.h - C ABI of the GB300 (sm_103a) EDFA library.
 *
 * EDFA (Explicit Decoupling Factor Approximation) is the block preconditioner
 * of Nardean, Ferronato & Abushaikha, arXiv 2009.13916, for the block system
 * of the MHFE-FV flow model (Sec. 2.3, Eq. system):
 *
 *        [ A  B ] [ pi ]   [ f_pi ]      A = A_pipi  (N_f x N_f, faces)
 *        [ C  D ] [ p  ] = [ f_p  ]      B = A_pip   (N_f x N_e)
 *                                        C = A_ppi   (N_e x N_f)
 *                                        D = A_pp    (N_e x N_e, cells)
 *
 * Stage 1 (edfa_build, Algorithm 1): restriction sets Q^(m), one restricted
 * dense solve per cell (Eq. syst_MRHS_res, Eq. syst_MRHS_res-F) giving the
 * decoupling-factor approximations X~ = -F~ (and G~), the product H~ and the
 * ILU(0) factors standing for A~^{-1}.
 * Stage 2 (edfa_setup, Algorithm 2): S~ = D - H~ (Eq. sparse_S) and its ILU(0).
 * Application (edfa_apply): z = P^{-1} r with P^{-1} of Eq. (EDFA_prec).
 * Solve (edfa_solve): right-preconditioned flexible GMRES(m), x0 = 0, stopping
 * at ||b - A x||_2 / ||b||_2 <= rtol (the stopping rule of Sec. 4).
 *
 * Conventions shared by every entry point
 *  - Every pointer inside edfa_csr and every vector argument is DEVICE memory
 *    on the current CUDA device, owned by the caller.  The handle keeps
 *    non-owning references to A, B, C, D until edfa_free: keep them alive and
 *    unchanged (D may be replaced through edfa_setup).
 *  - The handle owns everything it computes (restriction sets, X~, G~, H~,
 *    S~, factors, Krylov workspace) and releases it in edfa_free.
 *  - CSR: int64 row pointers (nrows+1 entries, rowptr[0] = 0, non-decreasing),
 *    int32 column indices ascending and unique within a row, FP64 values.
 *    Sizes must fit int32 (N_f + N_e < 2^31).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  The calls synchronise `stream` where stated (sizing of ragged
 *    outputs in edfa_build, the convergence test of edfa_solve); edfa_apply
 *    never synchronises.
 *  - Every call returns EDFA_OK (0) or an error code; no C++ exception
 *    crosses the ABI.  edfa_strerror gives a static message;
 *    edfa_last_error_detail gives the offending row/cell of the last failure
 *    on the calling thread (or -1).
 */
#ifndef EDFA_H
#define EDFA_H

#include <stdint.h>

#if defined(__GNUC__)
#define EDFA_API __attribute__((visibility("default")))
#else
#define EDFA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* edfa_stream;

enum {
    EDFA_OK = 0,
    EDFA_ERR_INVALID = 1,       /* bad sizes, pattern, option or non-finite value */
    EDFA_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    EDFA_ERR_OOM = 3,           /* device allocation failed */
    EDFA_ERR_BREAKDOWN = 4,     /* zero/negative local pivot or zero ILU(0) pivot */
    EDFA_ERR_NOT_CONVERGED = 5, /* FGMRES reached maxit */
    EDFA_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
    EDFA_ERR_BOUNDS = 7,        /* a ragged set exceeded a fixed device capacity */
    EDFA_ERR_UNSUPPORTED = 8    /* combination of options not implemented */
};

typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;
    const int64_t* rowptr; /* device [nrows+1] */
    const int32_t* col;    /* device [nnz] */
    const double* val;     /* device [nnz] */
} edfa_csr;

/* Restriction-set builders (Sec. 3, static and dynamic techniques). */
enum {
    EDFA_Q_OWN = 0,     /* F_m: the faces of cell m (stored rows of column m of B) */
    EDFA_Q_NBR = 1,     /* F_m plus the faces of every cell sharing a face with m */
    EDFA_Q_CROW = 2,    /* stored columns of row m of C (the base pattern Q_{A_ppi}) */
    EDFA_Q_THRESH = 3,  /* F_m plus j with |A_ij| >= thresh |A_ii| for some i in F_m */
    EDFA_Q_DYNAMIC = 4, /* Algorithm 1 dynamic branch from Q_{A_ppi}: n_add, n_ent, it_max */
    EDFA_Q_GIVEN = 5    /* caller-supplied qptr/qidx (device, ascending per cell) */
};

typedef struct {
    int32_t qmode;
    double thresh;          /* EDFA_Q_THRESH */
    int32_t n_add, n_ent, it_max; /* EDFA_Q_DYNAMIC */
    const int64_t* qptr;    /* EDFA_Q_GIVEN: device [N_e+1] */
    const int32_t* qidx;    /* EDFA_Q_GIVEN: device [qptr[N_e]] */
    int32_t schur_form;     /* 0: S~ = D - C X~ ; 1: S~ = D - G~ A F~ (Eq. sparse_S) */
    int32_t variant;        /* 0: full block LDU of Eq. (EDFA_prec); 1: upper block triangular */
    int32_t precision;      /* 0: FP64 throughout; 1: FP32 local solves, S~, factors and
                               application, FP64 Krylov vectors, Arnoldi and true residual */
    int32_t warps_per_block;/* local-solve launch shape; 0 = default */
    int32_t sweep_warps_per_sm; /* resident warps per SM of the sync-free ILU(0) sweeps; 0 = default (16) */
    int32_t sweep_mode;     /* S~ triangular sweeps: 0 = automatic (one 16-CTA thread-block cluster
                               holding the solution in distributed shared memory, rows polling their
                               dependencies there, when N_e values fit and the cluster can be
                               scheduled; else sync-free all-SM sweeps); 1 = sync-free all-SM sweeps
                               only, also for A~ (no chain decomposition); 2 = the cluster with one
                               barrier per dependency level.  In modes 0 and 2 the A~ sweeps run as a
                               few phases of independent chains when their DAG allows it */
    int32_t filtration;     /* sparsification of S~ (Sec. 3, implementation details): one of
                               EDFA_FILT_*; an entry is discarded when its absolute value is below
                               tau_filt times the Euclidean norm of the vector it belongs to, and
                               diagonal entries of H~ and S~ are always kept */
    double tau_filt;        /* filtration tolerance (>= 0; 0 keeps every entry) */
    int32_t ordering;       /* ordering of the inner ILU(0) factorisations (the paper leaves the inner
                               preconditioners open, Sec. 3): 0 = natural (default); 1 = multicolour
                               ordering of S~; 2 = multicolour orderings of A~ and S~.  Colouring of the
                               graph of M + M^T by Jones & Plassmann with the SplitMix64 finaliser of
                               row + 1 as priority, rows sorted by (colour, row); every triangular sweep
                               of an ordered factor then has at most as many dependency levels as
                               colours.  With an ordering of S~ its sweeps always run on all SMs (the
                               single-cluster sweeps of sweep_mode 0 and 2 are for deep natural-order
                               factors); an ordered A~ is never chain-decomposed */
    int32_t s_block;        /* with an ordering of S~: 0 or 1 = the colouring above; 2..16 = block
                               multicolour ordering: blocks of s_block consecutive rows coloured as
                               units (SplitMix64 priority of block + 1), row r of block B taking colour
                               c(B) s_block + r - B s_block, so the rows of one block keep their
                               natural order.  The ILU(0) then stays closer to the natural one (fewer
                               FGMRES iterations) at s_block times the colours.  EDFA_ERR_BOUNDS when
                               the colours exceed 256 */
} edfa_options;

/* Filtration of the approximate Schur complement (Algorithms 1 and 2). */
enum {
    EDFA_FILT_NONE = 0,
    EDFA_FILT_PRE = 1,     /* pre-filtration: every local solution X~ column m (and G~ row m in the
                              two-sided form) before H~ is formed (Stage 1) */
    EDFA_FILT_POST_H = 2,  /* post-filtration of the rows of H~ (Stage 1; S~ = D - H~ keeps the
                              pattern of D) */
    EDFA_FILT_POST_S = 3   /* post-filtration of the rows of S~ = D - H~ (Stage 2: the pattern of S~,
                              its ILU(0) levels and sweep plans are rebuilt by every edfa_setup) */
};

typedef struct edfa_handle_s* edfa_handle;

typedef struct {
    int32_t iterations;   /* total inner FGMRES iterations */
    int32_t converged;    /* 1 if the true residual met rtol */
    int32_t restarts;
    double est_rel;       /* last Arnoldi estimate |g_{j+1}| / ||b|| */
    double true_rel;      /* ||b - A x|| / ||b|| at exit */
} edfa_solve_info;

/* Per-phase device times of the last build/setup/solve (CUDA events on the stream). */
typedef struct {
    float ms_qsets, ms_local, ms_schur, ms_ilu_a;  /* Stage 1 */
    float ms_stage2;                               /* S~ = D - H~ and ILU(0) of S~ */
    float ms_solve;                                /* last edfa_solve */
    int64_t n_local;                               /* number of local systems solved */
    int64_t q_total;                               /* sum of |Q^(m)| */
    int32_t q_max;                                 /* max |Q^(m)| */
    int64_t s_nnz;                                 /* nnz of S~ */
    int32_t levels_a, levels_s;                    /* dependency depth of the ILU(0) sweeps */
    /* with profiling on (edfa_set_profiling): accumulated device time and
       launch count of the triangular sweeps, kind 0..4 = A~ forward, A~
       backward, S~ forward, S~ backward (sync-free all-SM sweeps), both S~
       sweeps in one thread-block-cluster launch */
    double sweep_ms[5];
    int64_t sweep_n[5];
    /* launch shapes picked by the autotuner (lanes per local system, warps per
       block of the local-solve kernel, warps per block of the Schur kernel) */
    int32_t tuned_lanes, tuned_warps, tuned_schur_warps;
    /* 1 when both S~ sweeps run in one 16-CTA cluster (edfa_options.sweep_mode),
       with the bytes of their packed level chunks */
    int32_t s_cluster;
    int64_t s_cluster_bytes;
    /* Stage 2 split: S~ values; S~ pattern (post-filtration of S~), level
       plans and cluster-record layout (edfa_build, and every edfa_setup with
       post-filtration of S~); numeric ILU(0) of S~; writing of the cluster
       sweep records */
    float ms_s_values, ms_s_plan, ms_s_factor, ms_s_cluster;
    /* with profiling on: accumulated device time and launch count of the
       FGMRES kernels, kind 0 = first-pass multi-dot V^T w (with ||w||^2),
       1 = first-pass update w -= V h, 2 = block SpMV y = [A B; C D] x */
    double kry_ms[3];
    int64_t kry_n[3];
    int64_t kry_vecs;  /* basis vectors read by the timed multi-dot launches, summed */
} edfa_stats;

/* Read-only views of what the handle computed (device pointers, valid until
 * edfa_free; values FP64 unless precision = 1, where the *_f32 fields are set). */
typedef struct {
    int32_t Nf, Ne;
    const int64_t* qptr;  /* [Ne+1] */
    const int32_t* qidx;  /* [qptr[Ne]] ascending per cell */
    const double* xval;   /* X~ column m on Q^(m) (FP64 path) */
    const double* gval;   /* G~ row m on Q^(m) (two-sided form only) */
    const float* xval_f32;
    int64_t s_nnz;
    const int64_t* s_rowptr;
    const int32_t* s_col;
    const double* s_val;  /* S~ values (FP64 path) */
    const float* s_val_f32;
    /* orderings of the inner factorisations (edfa_options.ordering); perm[k] is
       the face / cell at ordered position k, NULL in the natural order */
    int32_t a_ncolours, s_ncolours;
    const int32_t* a_perm;   /* [N_f] */
    const int32_t* s_perm;   /* [N_e] */
    /* the ILU(0) factors as computed (of the ordered matrices when ordered):
       pattern and L\U values, L unit lower (its diagonal not stored) */
    int64_t fa_nnz, fs_nnz;
    const int64_t* fa_rowptr;
    const int32_t* fa_col;
    const double* fa_lu;
    const float* fa_lu_f32;
    const int64_t* fs_rowptr;
    const int32_t* fs_col;
    const double* fs_lu;
    const float* fs_lu_f32;
} edfa_view;

EDFA_API void edfa_default_options(edfa_options* opt);

/* Stage 1 (+ Stage 2 with the given D).  On success *h receives a new handle.
 * Synchronises `stream` to size the restriction sets and S~. */
EDFA_API int edfa_build(edfa_handle* h, const edfa_csr* A, const edfa_csr* B, const edfa_csr* C,
               const edfa_csr* D, const edfa_options* opt, edfa_stream stream);

/* Stage 2 only: new values of D with the SAME pattern as at build time.
 * Recomputes S~ = D - H~ and its ILU(0).  D must stay alive until the next
 * edfa_setup or edfa_free. */
EDFA_API int edfa_setup(edfa_handle h, const edfa_csr* D, edfa_stream stream);

/* z = P^{-1} r, both device vectors of length N_f + N_e (faces first). */
EDFA_API int edfa_apply(edfa_handle h, const double* r, double* z, edfa_stream stream);

/* y = [A B; C D] x (device vectors of length N_f + N_e). */
EDFA_API int edfa_matvec(edfa_handle h, const double* x, double* y, edfa_stream stream);

/* FGMRES(restart), x0 = 0; x receives the solution (device, N_f + N_e).
 * Returns EDFA_ERR_NOT_CONVERGED if maxit inner iterations do not reach rtol
 * (x then holds the last iterate).  info may be NULL.  With an ordering
 * (edfa_options.ordering >= 1) the iteration runs on the permuted system, in
 * the numbering of the ordered factors (b permuted in, x permuted out, 2 (N_f +
 * N_e) doubles of workspace allocated on the first such solve): the same
 * iteration as in the natural numbering up to the rounding of its sums. */
EDFA_API int edfa_solve(edfa_handle h, const double* b, double* x, int32_t restart, double rtol,
               int32_t maxit, edfa_solve_info* info, edfa_stream stream);

/* Right-preconditioned Bi-CGStab (van der Vorst 1992), the outer solver of the
 * paper's experiments (Sec. 4), with the preconditioner of the handle; x0 = 0,
 * stopping rule ||r_k||_2 / ||r_0||_2 <= rtol (r_0 = b), the true residual
 * ||b - A x|| confirmed at the end (the method restarts from the true residual
 * when the recursive one met rtol but the true one did not, or on a breakdown).
 * One iteration applies the preconditioner twice.  x receives the solution
 * (device, N_f + N_e); info->iterations counts iterations, info->restarts the
 * restarts.  Returns EDFA_ERR_NOT_CONVERGED if maxit iterations do not reach
 * rtol (x then holds the last iterate).  Synchronises `stream` four times per
 * iteration to read the scalars.  Workspace (8 (N_f + N_e) doubles) is kept by
 * the handle. */
EDFA_API int edfa_solve_bicgstab(edfa_handle h, const double* b, double* x, double rtol, int32_t maxit,
                                 edfa_solve_info* info, edfa_stream stream);

/* Batched solve of many independent systems held block-diagonally in one
 * handle (the caller concatenates the systems: system i owns faces
 * [face_off[i], face_off[i+1]) and cells [cell_off[i], cell_off[i+1]), with no
 * coupling between systems; build the handle once over the concatenation, so
 * the restriction sets, local solves, S~ and ILU(0) of all systems run in
 * single launches).  One FGMRES(restart) per system, x0 = 0, stopping rule
 * ||b_i - A_i x_i|| / ||b_i|| <= rtol per system; the systems advance in lock
 * step (a system stops iterating once it has converged), reductions are per
 * system and the Hessenberg/Givens updates run on the device.  One restart
 * cycle is captured as a CUDA graph and replayed until every system has
 * converged or reached maxit inner iterations.
 * face_off, cell_off: host arrays of nsys+1 entries (face_off[nsys] = N_f,
 * cell_off[nsys] = N_e).  iterations, true_rel: host arrays of nsys entries
 * (may be NULL); cycles: host (may be NULL).  Workspace ((2 restart + 2) (N_f +
 * N_e) doubles) is kept by the handle for further calls with the same layout.
 * Returns EDFA_ERR_NOT_CONVERGED when some system did not converge. */
EDFA_API int edfa_solve_batched(edfa_handle h, int32_t nsys, const int64_t* face_off, const int64_t* cell_off,
                                const double* b, double* x, int32_t restart, double rtol, int32_t maxit,
                                int32_t* iterations, double* true_rel, int32_t* cycles, edfa_stream stream);

/* Residual-estimate history of the last edfa_solve (host array of
 * iterations+1 entries, hist[0] = 1); returns the number written. */
EDFA_API int32_t edfa_history(edfa_handle h, double* hist, int32_t cap);

EDFA_API int edfa_get_view(edfa_handle h, edfa_view* v);
EDFA_API int edfa_get_stats(edfa_handle h, edfa_stats* s);

/* Turn per-launch device timing of the triangular sweeps and the first-pass
 * FGMRES kernels on (1) or off (0); turning it on clears the accumulated times
 * (edfa_stats.sweep_ms, kry_ms).  Timing adds one event pair per timed launch. */
EDFA_API int edfa_set_profiling(edfa_handle h, int32_t on);

/* The same for a subset of the timed kinds: bit k of `kinds` times the
 * launches of kind k, with k the index into edfa_stats.sweep_ms (0-4: A~
 * forward, A~ backward, S~ forward, S~ backward, S~ in one cluster) or 5 + the
 * index into edfa_stats.kry_ms (5: first-pass multi-dot, 6: first-pass update,
 * 7: block product).  edfa_set_profiling(h, 1) equals kinds = 0xFF.  Fewer
 * kinds record fewer events.  EDFA_ERR_INVALID for bits above 7. */
EDFA_API int edfa_set_profiling_mask(edfa_handle h, uint32_t kinds);

/* Preconditioner for the transposed system [A B; C D]^T = [A C^T; B^T D^T]
 * (adjoint solves), built from the forward handle `fwd`: the transposed blocks
 * C^T, B^T, D^T are formed on the device and owned by the new handle; the
 * forward restriction sets are reused, so every local system A^(m) is the
 * same and only the right-hand sides swap roles (the F~/G~ roles of
 * Eq. EDFA_systems_1/2 exchange).  With schur_form = 1 the new S~ is exactly
 * the transpose of the forward S~.  `fwd` must stay alive during the call
 * only.  Synchronises `stream` like edfa_build. */
EDFA_API int edfa_build_adjoint(edfa_handle* adj, edfa_handle fwd, edfa_stream stream);

/* Gradient of a scalar L(u) with respect to the per-cell log-conductivities
 * theta_E = log k_E of an isotropic brick-grid MHFE-FV system with strong-flux
 * cell rows (Eq. fluxes_MHFEM_STRONG, Appendix A) and prescribed pressures on
 * faces:  grad_E = lambda^T (d b / d theta_E - d A / d theta_E u), where
 * A^T lambda = dL/du (the adjoint solve) and A u = b.  All arrays are device
 * memory:  cell_faces [Ne*6] (local order x-,x+,y-,y+,z-,z+), face_cells
 * [Nf*2] (minus-side cell, plus-side cell, -1 = none), face_dir [Nf] (1 =
 * prescribed pressure), face_pbar [Nf], W [Ne*36] the inverse elemental
 * matrices (B^E)^{-1} row-major, u and lambda [Nf+Ne], grad [Ne] (output).
 * Asynchronous on `stream`. */
EDFA_API int edfa_grad_logk(int32_t Nf, int32_t Ne, const int32_t* cell_faces, const int32_t* face_cells,
                            const int8_t* face_dir, const double* face_pbar, const double* W,
                            const double* u, const double* lam, double* grad, edfa_stream stream);

/* Restriction sets Q^(m) without any device memory allocation.
 *
 * For callers that must not allocate device memory after start-up: host
 * programs that hand all device memory to their own pool or budget up front
 * (a simulator time loop with a fixed memory reservation, an embedding
 * application whose allocator owns the GPU), or code that cannot afford the
 * device-wide synchronisation and the possible failure of cudaMalloc in the
 * middle of a run.  It computes the same sets as edfa_build for the static
 * modes EDFA_Q_OWN, EDFA_Q_NBR, EDFA_Q_CROW and EDFA_Q_THRESH (thresh used by
 * the last one); the paper has no counterpart of this entry point.
 *
 * A, B, C: the blocks as for edfa_build (device CSR, validated here with
 *          the checks edfa_build makes; invalid blocks return
 *          EDFA_ERR_INVALID before any kernel reads through their indices).
 * qptr:    caller-owned device array of N_e + 1 int64, receives the offsets.
 * qidx:    caller-owned device array of qidx_capacity int32, receives the
 *          sets, ascending per cell.
 * qtot:    host pointer, receives the total size qptr[N_e].
 * Working memory comes from one fixed device array of
 * EDFA_NOALLOC_SCRATCH_BYTES inside the library (held by every GPU that
 * loads the library until the process exits); the call needs
 * 8 (N_e+1) x 2 + 4 nnz(B) + 8 (N_e/2048 + 2) + 512 bytes of it, rounded up to
 * 256-byte pieces.  A problem that needs more returns EDFA_ERR_BOUNDS before
 * touching the device, with the needed bytes in edfa_last_error_detail.  If
 * the sets do not fit in qidx_capacity the call returns EDFA_ERR_BOUNDS with
 * the needed capacity in *qtot and edfa_last_error_detail (qidx untouched).
 *
 * The library's kernels load lazily (CUDA's default module loading), and the
 * fixed array is reserved on a device when the module holding it is first
 * used there: by the first edfa_qsets_noalloc or edfa_build call on that
 * device.  Make one such call at start-up, before the caller's pool takes the
 * device memory (or run with CUDA_MODULE_LOADING=EAGER, which reserves it
 * when the library is loaded).  The first call on a device also looks up the
 * device address of the fixed array (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  Every call
 * reuses the same array and leaves its contents behind (the parts that must
 * start at zero are cleared on each call), so calls whose work overlaps on
 * the GPU (different streams or host threads at the same time) race and must
 * not be issued.  The call synchronises `stream` twice: after validating the
 * blocks, and to read the total size; the fill of qidx is then enqueued on
 * `stream`.  Calls no allocating CUDA or library routine. */
#define EDFA_NOALLOC_SCRATCH_BYTES (64ull << 20)
EDFA_API int edfa_qsets_noalloc(const edfa_csr* A, const edfa_csr* B, const edfa_csr* C, int32_t qmode,
                                double thresh, int64_t* qptr, int32_t* qidx, int64_t qidx_capacity,
                                int64_t* qtot, edfa_stream stream);

/* Diagnostic of the library's failure detection (no counterpart in the paper).
 * Every device-side wait of the library (a row waiting for a value another
 * warp computes, a warp waiting on a flag or an mbarrier) is bounded: when its
 * poll budget runs out it records EDFA_ERR_TIMEOUT with the waiting row in the
 * detail, every other wait of that kernel gives up, and the kernel returns, so
 * a lost dependency never hangs the GPU and the CUDA context stays usable.
 * This call makes such a wait run out on purpose: it runs the sync-free
 * forward-sweep kernel on a 2 x 2 unit lower-triangular system with a level
 * plan that omits row 0, so row 1 waits for a value nothing writes.  Returns
 * EDFA_ERR_TIMEOUT (edfa_last_error_detail() = 1) when the budget ran out as
 * designed; *ms (may be NULL) receives the kernel's duration.  Synchronises
 * `stream`; allocates and frees a few hundred bytes of device memory; must not
 * run concurrently with other work of this library on the device. */
EDFA_API int edfa_selftest_wait_timeout(float* ms, edfa_stream stream);

/* Measurement utility (no counterpart in the paper): the device's fused
 * multiply-add rate, precision 0 = FP64, 1 = FP32, in FMA per second, from one
 * timed launch of a kernel running eight independent FMA chains per thread on
 * every SM (about 30 ms).  It is the ALU denominator for kernels bound by
 * arithmetic rather than memory, such as the dense per-cell factorisations of
 * the local solves.  Synchronises `stream`; allocates and frees 8 bytes of
 * device memory. */
EDFA_API int edfa_probe_fma_rate(int32_t precision, double* fma_per_s, edfa_stream stream);

/* Number of CUDA kernels this library has launched in this process. */
EDFA_API int64_t edfa_launch_count(void);

EDFA_API int edfa_free(edfa_handle h);

EDFA_API const char* edfa_strerror(int code);
EDFA_API int64_t edfa_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* EDFA_H */
