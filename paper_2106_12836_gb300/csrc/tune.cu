// Product autotuning: for one matrix in its current storage precision, time
// every product kernel that can serve it (SELL-32 when its padding allows,
// CSR with 2, 4, 8, 16 or 32 lanes per row) with CUDA events on the context
// stream, and keep the fastest for every later product with that matrix
// (sait_spmv, the SAIT apply, the solvers' products and residuals).
#include <algorithm>

#include "internal.cuh"

extern "C" sait_status sait_mat_autotune(sait_ctx ctx, sait_mat M, sait_tune_report *report) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!M || !report) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_mat_autotune: null argument");
    *report = sait_tune_report{};
    const int64_t n = M->n;
    if (n == 0) return SAIT_OK;
    cudaStream_t s = ctx->stream;
    SAIT_TRY(mat_prepare_store(ctx, M, M->store));
    DTemp<double> x, y;
    SAIT_CK(x.alloc(n, s));
    SAIT_CK(y.alloc(n, s));
    SAIT_CK(cudaMemsetAsync(x.p, 0, n * sizeof(double), s));
    cudaEvent_t e0, e1;
    SAIT_CK(cudaEventCreate(&e0));
    SAIT_CK(cudaEventCreate(&e1));
    constexpr int kReps = 10;
    auto time_one = [&](float *us) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int w = 0; w < 3 && e == cudaSuccess; w++)
            e = launch_spmv(M, M->store, x.p, false, y.p, false, nullptr, s, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < kReps && e == cudaSuccess; r++)
            e = launch_spmv(M, M->store, x.p, false, y.p, false, nullptr, s, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        *us = ms * 1e3f / kReps;
        return e;
    };
    cudaError_t e = cudaSuccess;
    int c = 0;
    if (sell_ready(M, M->store)) {
        M->force_csr = false;
        report->format[c] = 1;
        report->lanes[c] = 32;
        e = time_one(&report->us[c]);
        c++;
    }
    for (int G = 2; G <= 32 && e == cudaSuccess; G *= 2, c++) {
        M->force_csr = true;
        M->lanes = G;
        report->format[c] = 0;
        report->lanes[c] = G;
        e = time_one(&report->us[c]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        M->force_csr = false;
        M->lanes = choose_lanes(M->n, M->nnz);
        return ctx_cuda(ctx, e, "sait_mat_autotune", __FILE__, __LINE__);
    }
    report->ncand = c;
    int best = 0, best_csr = -1;
    for (int t = 0; t < c; t++) {
        if (report->us[t] < report->us[best]) best = t;
        if (report->format[t] == 0 && (best_csr < 0 || report->us[t] < report->us[best_csr])) best_csr = t;
    }
    report->chosen = best;
    M->force_csr = report->format[best] == 0;
    M->lanes = report->lanes[best_csr];  // also the lanes of CSR residuals and fallbacks
    return SAIT_OK;
}
