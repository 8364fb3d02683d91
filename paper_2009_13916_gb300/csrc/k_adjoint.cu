// Adjoint of the EDFA-preconditioned solve.
//
//  * edfa_build_adjoint: the preconditioner for the transposed system
//      [A B; C D]^T = [A C^T; B^T D^T]        (A is symmetric)
//    built from a forward handle: the transposed blocks are formed on the
//    device, and the forward restriction sets are reused, so every local
//    system A^(m) is the same and only the right-hand sides swap roles
//    (the new X~ approximates A^{-1} C^T, i.e. -G~^T of the forward system).
//  * edfa_grad_logk: for isotropic cell conductivities k_E = exp(theta_E) on
//    a brick grid with the strong-flux cell rows (Eq. fluxes_MHFEM_STRONG,
//    Appendix A), the gradient of L(u(theta)), A(theta) u = b(theta),
//        dL/dtheta_E = lambda^T (db/dtheta_E - dA/dtheta_E u),  A^T lambda = dL/du.
//    With pi_j = pbar_j on prescribed faces, this is minus the sum over
//    non-prescribed rows r of lambda_r times the theta_E-derivative of row r
//    of the un-eliminated system applied to u.  Since W^E = k_E W^E_1, the
//    derivative of W^E is W^E itself; the rows that depend on k_E are
//      - face rows i in F_E: derivative q_i^E = sum_j W^E_ij (p_E - pi_j);
//      - cell row E and the row of the neighbour E' across each interior face
//        i: the strong flux q = w Lambda^E - (1-w) Lambda^E' with
//        w = W^E'_ii / (W^E_ii + W^E'_ii) has derivative
//        dq = w Lambda^E - w (1-w) (Lambda^E + Lambda^E') in row E and -dq in
//        row E' (flux antisymmetry);
//      - cell row E at a prescribed face: the weak flux q_i^E itself.
#include "internal.cuh"

namespace edfa {

// ------------------------------------------------------------ CSR transpose
__global__ void k_tr_count(Csr<double> M, unsigned long long* cnt)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < M.nnz) atomicAdd(&cnt[M.col[p]], 1ull);
}

__global__ void k_tr_fill(Csr<double> M, unsigned long long* cursor, int32_t* tcol, double* tval)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= M.nrows) return;
    for (int64_t p = M.rowptr[r]; p < M.rowptr[r + 1]; ++p) {
        unsigned long long pos = atomicAdd(&cursor[M.col[p]], 1ull);
        tcol[pos] = (int32_t)r;
        tval[pos] = M.val[p];
    }
}

__global__ void k_tr_sort(int64_t n, const int64_t* ptr, int32_t* col, double* val)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t b = ptr[r], e = ptr[r + 1];
    for (int64_t p = b + 1; p < e; ++p) {
        int32_t c = col[p];
        double v = val[p];
        int64_t q = p - 1;
        while (q >= b && col[q] > c) { col[q + 1] = col[q]; val[q + 1] = val[q]; --q; }
        col[q + 1] = c;
        val[q + 1] = v;
    }
}

// transpose M (device) into freshly allocated arrays appended to `bufs`
static int transpose_csr(const edfa_csr& M, edfa_csr* T, std::vector<DBuf>& bufs, cudaStream_t s)
{
    const int32_t nr = M.ncols, nc = M.nrows;
    int64_t* rp = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    size_t nz = (size_t)(M.nnz > 0 ? M.nnz : 1);
    if (cudaMalloc((void**)&rp, ((size_t)nr + 1) * sizeof(int64_t)) != cudaSuccess) return EDFA_ERR_OOM;
    bufs.push_back(DBuf{rp, 0});
    if (cudaMalloc((void**)&col, nz * sizeof(int32_t)) != cudaSuccess) return EDFA_ERR_OOM;
    bufs.push_back(DBuf{col, 0});
    if (cudaMalloc((void**)&val, nz * sizeof(double)) != cudaSuccess) return EDFA_ERR_OOM;
    bufs.push_back(DBuf{val, 0});
    cudaMemsetAsync(rp, 0, ((size_t)nr + 1) * sizeof(int64_t), s);
    Csr<double> m = csr_of(M);
    if (M.nnz > 0) (edfa::count_launch(), k_tr_count<<<(unsigned)((M.nnz + 255) / 256), 256, 0, s>>>(m, (unsigned long long*)rp));
    int rc = scan_i64(nullptr, rp, nr, s);
    if (rc) return rc;
    unsigned long long* cursor = nullptr;
    if (cudaMallocAsync((void**)&cursor, ((size_t)nr + 1) * sizeof(int64_t), s) != cudaSuccess) return EDFA_ERR_OOM;
    cudaMemcpyAsync(cursor, rp, ((size_t)nr + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (M.nrows > 0) (edfa::count_launch(), k_tr_fill<<<(unsigned)((M.nrows + 255) / 256), 256, 0, s>>>(m, cursor, col, val));
    if (nr > 0) (edfa::count_launch(), k_tr_sort<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(nr, rp, col, val));
    cudaFreeAsync(cursor, s);
    T->nrows = nr;
    T->ncols = nc;
    T->nnz = M.nnz;
    T->rowptr = rp;
    T->col = col;
    T->val = val;
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}

// ------------------------------------------------------------ gradient
__device__ __forceinline__ double face_p(int f, const int8_t* fdir, const double* pbar, const double* u)
{
    return fdir[f] ? pbar[f] : u[f];
}

__global__ void __launch_bounds__(128)
k_grad_logk(int32_t Nf, int32_t Ne, const int32_t* __restrict__ cf, const int32_t* __restrict__ fc,
            const int8_t* __restrict__ fdir, const double* __restrict__ pbar, const double* __restrict__ W,
            const double* __restrict__ u, const double* __restrict__ lam, double* __restrict__ grad)
{
    int64_t E = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (E >= Ne) return;
    const double* We = W + 36 * E;
    int f[6];
    double pi[6];
    for (int l = 0; l < 6; ++l) {
        f[l] = cf[6 * E + l];
        pi[l] = face_p(f[l], fdir, pbar, u);
    }
    const double pE = u[Nf + E];
    const double lamE = lam[Nf + E];
    double g = 0.0;
    for (int l = 0; l < 6; ++l) {
        const int i = f[l];
        double qE = 0.0, Ll = 0.0, sE = 0.0;
        for (int j = 0; j < 6; ++j) {
            const double w = We[l * 6 + j];
            qE += w * (pE - pi[j]);
            Ll += w;
            if (j != l) sE += w * pi[j];
        }
        if (!fdir[i]) g -= lam[i] * qE;
        const int side = (l & 1) ? 0 : 1;
        const int E2 = fc[2 * (int64_t)i + (1 - side)];
        if (E2 >= 0) {
            const double* W2 = W + 36 * (int64_t)E2;
            int l2 = 0;
            while (l2 < 6 && cf[6 * (int64_t)E2 + l2] != i) ++l2;
            double L2 = 0.0, s2 = 0.0;
            for (int j = 0; j < 6; ++j) {
                const double w = W2[l2 * 6 + j];
                L2 += w;
                if (j != l2) s2 += w * face_p(cf[6 * (int64_t)E2 + j], fdir, pbar, u);
            }
            const double lamE_ = Ll * pE - sE;
            const double lamE2_ = L2 * u[Nf + E2] - s2;
            const double wgt = W2[l2 * 6 + l2] / (We[l * 6 + l] + W2[l2 * 6 + l2]);
            const double dq = wgt * lamE_ - wgt * (1.0 - wgt) * (lamE_ + lamE2_);
            g -= (lamE - lam[Nf + E2]) * dq;
        } else if (fdir[i]) {
            g -= lamE * qE;
        }
    }
    grad[E] = g;
}

}  // namespace edfa

using namespace edfa;

extern "C" int edfa_build_adjoint(edfa_handle* out, edfa_handle fwd, edfa_stream stream)
{
    if (!out || !fwd) return EDFA_ERR_INVALID;
    *out = nullptr;
    if (fwd->opt.qmode == EDFA_Q_GIVEN && !fwd->qidx) return EDFA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<DBuf> bufs;
    edfa_csr Bt{}, Ct{}, Dt{};
    int rc = transpose_csr(fwd->C, &Bt, bufs, s);       // new B = C^T (faces x cells)
    if (!rc) rc = transpose_csr(fwd->B, &Ct, bufs, s);  // new C = B^T (cells x faces)
    if (!rc) rc = transpose_csr(fwd->D, &Dt, bufs, s);  // new D = D^T
    if (!rc) {
        edfa_options o = fwd->opt;
        o.qmode = EDFA_Q_GIVEN;
        o.qptr = fwd->qptr;
        o.qidx = fwd->qidx;
        edfa_handle h = nullptr;
        rc = edfa_build(&h, &fwd->A, &Bt, &Ct, &Dt, &o, stream);
        if (!rc) {
            for (auto& b : bufs) h->owned.push_back(b);
            h->opt.qptr = nullptr;
            h->opt.qidx = nullptr;
            *out = h;
            return EDFA_OK;
        }
    }
    cudaStreamSynchronize(s);
    for (auto& b : bufs) cudaFree(b.p);
    return rc;
}

extern "C" int edfa_grad_logk(int32_t Nf, int32_t Ne, const int32_t* cell_faces, const int32_t* face_cells,
                              const int8_t* face_dir, const double* face_pbar, const double* W, const double* u,
                              const double* lam, double* grad, edfa_stream stream)
{
    if (Nf < 0 || Ne < 0) return EDFA_ERR_INVALID;
    if (Ne == 0) return EDFA_OK;
    if (!cell_faces || !face_cells || !face_dir || !face_pbar || !W || !u || !lam || !grad) return EDFA_ERR_INVALID;
    (edfa::count_launch(), k_grad_logk<<<(unsigned)((Ne + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        Nf, Ne, cell_faces, face_cells, face_dir, face_pbar, W, u, lam, grad));
    return cudaGetLastError() == cudaSuccess ? EDFA_OK : EDFA_ERR_CUDA;
}
