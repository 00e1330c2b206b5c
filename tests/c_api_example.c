/* Using the library from C through include/sait.h alone.
 *
 * Solves the 5-point Poisson problem on a g x g grid with GMRES(30)
 * preconditioned by SAIT (Section 3.1: z = M_U (M_L r)), the factors L, U
 * coming from ILU(0) on the GPU and M_L, M_U from m_terms = 3 series terms
 * with the row-relative drop 1e-3.  All matrices and vectors live in device
 * memory owned by the caller; the library owns the sait_* handles.
 *
 *   cc -std=c11 -I include c_api_example.c -L <dir of libsait.so> -lsait \
 *      -L <CUDA>/lib64 -lcudart -I <CUDA>/include -o c_api_example
 *   ./c_api_example [g]
 *
 * Exit status 0 when the true relative residual is at most 1e-8. */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "sait.h"

#define CUDA_OK(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));            \
            return 2;                                                              \
        }                                                                          \
    } while (0)

#define SAIT_OK_OR_FAIL(ctx, call)                                                 \
    do {                                                                           \
        sait_status s_ = (call);                                                   \
        if (s_ != SAIT_OK) {                                                       \
            fprintf(stderr, "%s: %s (%s)\n", #call, sait_status_string(s_),        \
                    sait_ctx_last_error(ctx));                                     \
            return 3;                                                              \
        }                                                                          \
    } while (0)

int main(int argc, char **argv) {
    const int g = argc > 1 ? atoi(argv[1]) : 64;
    const int64_t n = (int64_t)g * g;
    /* host CSR of the 5-point Laplacian (4 on the diagonal, -1 to neighbours) */
    int32_t *rp = malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *ci = malloc((size_t)(5 * n) * sizeof(int32_t));
    double *va = malloc((size_t)(5 * n) * sizeof(double));
    double *b = malloc((size_t)n * sizeof(double));
    double *x = malloc((size_t)n * sizeof(double));
    if (!rp || !ci || !va || !b || !x) return 2;
    int64_t e = 0;
    rp[0] = 0;
    for (int i = 0; i < g; i++)
        for (int j = 0; j < g; j++) {
            const int64_t r = (int64_t)i * g + j;
            if (i > 0) { ci[e] = (int32_t)(r - g); va[e++] = -1.0; }
            if (j > 0) { ci[e] = (int32_t)(r - 1); va[e++] = -1.0; }
            ci[e] = (int32_t)r; va[e++] = 4.0;
            if (j < g - 1) { ci[e] = (int32_t)(r + 1); va[e++] = -1.0; }
            if (i < g - 1) { ci[e] = (int32_t)(r + g); va[e++] = -1.0; }
            rp[r + 1] = (int32_t)e;
            b[r] = 1.0;
        }
    const int64_t nnz = e;

    int32_t *d_rp, *d_ci;
    double *d_va, *d_b, *d_x;
    CUDA_OK(cudaMalloc((void **)&d_rp, (size_t)(n + 1) * sizeof(int32_t)));
    CUDA_OK(cudaMalloc((void **)&d_ci, (size_t)nnz * sizeof(int32_t)));
    CUDA_OK(cudaMalloc((void **)&d_va, (size_t)nnz * sizeof(double)));
    CUDA_OK(cudaMalloc((void **)&d_b, (size_t)n * sizeof(double)));
    CUDA_OK(cudaMalloc((void **)&d_x, (size_t)n * sizeof(double)));
    CUDA_OK(cudaMemcpy(d_rp, rp, (size_t)(n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(d_ci, ci, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(d_va, va, (size_t)nnz * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(d_b, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemset(d_x, 0, (size_t)n * sizeof(double)));

    sait_ctx ctx = NULL;
    sait_status st = sait_ctx_create(&ctx, NULL);
    if (st != SAIT_OK) {
        fprintf(stderr, "sait_ctx_create: %s\n", sait_status_string(st));
        return 3;
    }
    const sait_csr A = {n, nnz, d_rp, d_ci, d_va};
    sait_mat Am = NULL, L = NULL, U = NULL, ML = NULL, MU = NULL;
    sait_prec P = NULL;
    const sait_drop drop = {SAIT_DROP_ROWREL, 0, 1e-3};
    SAIT_OK_OR_FAIL(ctx, sait_mat_create_csr(ctx, &A, &Am));
    SAIT_OK_OR_FAIL(ctx, sait_ilu0(ctx, &A, &L, &U));
    SAIT_OK_OR_FAIL(ctx, sait_build(ctx, L, SAIT_LOWER, 3, drop, SAIT_F64, &ML));
    SAIT_OK_OR_FAIL(ctx, sait_build(ctx, U, SAIT_UPPER, 3, drop, SAIT_F64, &MU));
    SAIT_OK_OR_FAIL(ctx, sait_prec_create_sait(ctx, ML, MU, &P));
    sait_info info;
    SAIT_OK_OR_FAIL(ctx, sait_gmres(ctx, Am, P, d_b, d_x, 30, 1e-8, 10000, &info));
    CUDA_OK(cudaMemcpy(x, d_x, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));

    /* true residual on the host */
    double rr = 0.0, bb = 0.0;
    for (int64_t r = 0; r < n; r++) {
        double ax = 0.0;
        for (int32_t k = rp[r]; k < rp[r + 1]; k++) ax += va[k] * x[ci[k]];
        rr += (b[r] - ax) * (b[r] - ax);
        bb += b[r] * b[r];
    }
    const double rel = sqrt(rr / bb);
    int64_t nnz_ml = 0, n_ml = 0;
    SAIT_OK_OR_FAIL(ctx, sait_mat_info(ML, &n_ml, &nnz_ml));
    printf("n = %lld, nnz(M_L) = %lld, GMRES steps %d, relative residual %.3e\n", (long long)n,
           (long long)nnz_ml, info.iters, rel);

    sait_prec_destroy(P);
    sait_mat_destroy(MU);
    sait_mat_destroy(ML);
    sait_mat_destroy(U);
    sait_mat_destroy(L);
    sait_mat_destroy(Am);
    sait_ctx_destroy(ctx);
    cudaFree(d_rp);
    cudaFree(d_ci);
    cudaFree(d_va);
    cudaFree(d_b);
    cudaFree(d_x);
    free(rp);
    free(ci);
    free(va);
    free(b);
    free(x);
    return rel <= 1e-8 ? 0 : 1;
}
