// CSR transpose and the pattern-restricted outer product used by the adjoint.
//
// The adjoint of x = A^{-1} b with loss l(x) solves A^T lambda = dl/dx; its
// preconditioner is the transposed SAIT apply (M_U M_L)^T = M_L^T M_U^T, so
// the library stores transposed copies of A, M_L and M_U.  The gradient with
// respect to A's stored entries is dl/dA_ij = -lambda_i x_j (the outer product
// restricted to A's pattern).
#include <algorithm>

#include "internal.cuh"

namespace {

__global__ void k_col_count(int64_t nnz, const int32_t *__restrict__ ci, int32_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + ci[e], 1);
}

__global__ void k_tr_fill(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ va, const int64_t *__restrict__ trp, int32_t *cursor,
                          int32_t *tci, double *tva) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        const int64_t dst = trp[j] + atomicAdd(cursor + j, 1);
        tci[dst] = (int32_t)i;
        tva[dst] = va[k];
    }
}

// the atomic fill leaves each transposed row in arbitrary order: sort it
// (insertion sort per row; transposed rows of the matrices here are short)
__global__ void k_row_sort(int64_t n, const int64_t *__restrict__ trp, int32_t *tci, double *tva,
                           int32_t *rp32) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    rp32[r] = (int32_t)trp[r];
    if (r == n) return;
    const int64_t b = trp[r], e = trp[r + 1];
    for (int64_t p = b + 1; p < e; p++) {
        const int32_t c = tci[p];
        const double v = tva[p];
        int64_t q = p - 1;
        while (q >= b && tci[q] > c) {
            tci[q + 1] = tci[q];
            tva[q + 1] = tva[q];
            q--;
        }
        tci[q + 1] = c;
        tva[q + 1] = v;
    }
}

__global__ void k_outer_pattern(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ u, const double *__restrict__ v, double alpha,
                                double *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ui = alpha * u[i];
    for (int k = rp[i]; k < rp[i + 1]; k++) out[k] = ui * v[ci[k]];
}

}  // namespace

extern "C" sait_status sait_mat_transpose(sait_ctx ctx, sait_mat M, sait_mat *out) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!M || !out) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_mat_transpose: null argument");
    *out = nullptr;
    const int64_t n = M->n, nnz = M->nnz;
    cudaStream_t s = ctx->stream;
    sait_mat T = nullptr;
    SAIT_TRY(mat_alloc(ctx, n, nnz, &T));
    DTemp<int32_t> cnt;
    DTemp<int64_t> trp;
    cudaError_t e = cnt.alloc(n, s);
    if (e == cudaSuccess) e = trp.alloc(n + 1, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, std::max<int64_t>(n, 1) * sizeof(int32_t), s);
    if (e == cudaSuccess && nnz > 0)
        launch_k(k_col_count, (unsigned)std::min<int64_t>(cdiv(nnz, 256), 152LL * 16), 256, 0, s, nnz,
                 (const int32_t *)M->ci, cnt.p);
    if (e == cudaSuccess) e = scan_i32(cnt.p, trp.p, n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, std::max<int64_t>(n, 1) * sizeof(int32_t), s);
    if (e == cudaSuccess && n > 0)
        launch_k(k_tr_fill, (unsigned)cdiv(n, 256), 256, 0, s, n, (const int32_t *)M->rp, (const int32_t *)M->ci,
                 (const double *)M->va, (const int64_t *)trp.p, cnt.p, T->ci, T->va);
    if (e == cudaSuccess)
        launch_k(k_row_sort, (unsigned)cdiv(n + 1, 256), 256, 0, s, n, (const int64_t *)trp.p, T->ci, T->va,
                 T->rp);
    if (e == cudaSuccess) e = cudaGetLastError();
    sait_status st = SAIT_OK;
    if (e != cudaSuccess) st = ctx_cuda(ctx, e, "sait_mat_transpose", __FILE__, __LINE__);
    if (st == SAIT_OK) st = mat_prepare_store(ctx, T, M->store);
    if (st == SAIT_OK && cudaStreamSynchronize(s) != cudaSuccess)
        st = ctx_cuda(ctx, cudaGetLastError(), "sait_mat_transpose", __FILE__, __LINE__);
    if (st != SAIT_OK) {
        sait_mat_destroy(T);
        return st;
    }
    T->lanes = choose_lanes(n, nnz);
    *out = T;
    return SAIT_OK;
}

extern "C" sait_status sait_outer_on_pattern(sait_ctx ctx, sait_mat A, double alpha, const double *u,
                                             const double *v, double *out) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || (A->n > 0 && (!u || !v)) || (A->nnz > 0 && !out))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_outer_on_pattern: bad argument");
    if (A->n > 0)
        launch_k(k_outer_pattern, (unsigned)cdiv(A->n, 256), 256, 0, ctx->stream, A->n, (const int32_t *)A->rp,
                 (const int32_t *)A->ci, u, v, alpha, out);
    SAIT_CK(cudaGetLastError());
    return SAIT_OK;
}
