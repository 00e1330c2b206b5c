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

// Optimal parameters (Section 3): the runtime of a preconditioned solve is
// iter(M_L, M_U) x (comp(M_L, M_U) + othercomp), and the parameters that
// minimise it depend on the problem, the solver and the machine, so each
// candidate is built and solved here and timed with CUDA events on the
// context stream.  Builds and solves are the library's own entry points.
extern "C" sait_status sait_tune_params(sait_ctx ctx, sait_mat A, sait_mat L, sait_mat U, const double *b,
                                        double *x, sait_solver solver, int32_t restart, double tol, int32_t maxit,
                                        int32_t ncand, const sait_param *cand, sait_dtype store,
                                        int32_t count_build, sait_param_report *report) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || !L || !U || !b || !x || !cand || !report)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_tune_params: null argument");
    if (ncand < 1 || ncand > SAIT_PARAM_MAX)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_tune_params: ncand must be 1..SAIT_PARAM_MAX");
    if (solver != SAIT_SOLVER_GMRES && solver != SAIT_SOLVER_BICGSTAB && solver != SAIT_SOLVER_PCG)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_tune_params: unknown solver");
    if (L->n != A->n || U->n != A->n)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_tune_params: L, U and A differ in size");
    *report = sait_param_report{};
    report->ncand = ncand;
    report->chosen = -1;
    const int64_t n = A->n;
    cudaStream_t s = ctx->stream;
    DTemp<double> best;
    SAIT_CK(best.alloc(std::max<int64_t>(n, 1), s));
    cudaEvent_t ev[3];
    for (int k = 0; k < 3; k++) SAIT_CK(cudaEventCreate(&ev[k]));
    auto destroy_events = [&]() {
        for (int k = 0; k < 3; k++) cudaEventDestroy(ev[k]);
    };
    double best_ms = 0.0;
    for (int c = 0; c < ncand; c++) {
        sait_mat ML = nullptr, MU = nullptr;
        sait_prec P = nullptr;
        sait_info info{};
        cudaError_t e = cudaMemsetAsync(x, 0, n * sizeof(double), s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
        if (e != cudaSuccess) {
            destroy_events();
            return ctx_cuda(ctx, e, "sait_tune_params", __FILE__, __LINE__);
        }
        sait_status st = sait_build(ctx, L, SAIT_LOWER, cand[c].m_terms, cand[c].drop, store, &ML);
        if (st == SAIT_OK) st = sait_build(ctx, U, SAIT_UPPER, cand[c].m_terms, cand[c].drop, store, &MU);
        if (st == SAIT_OK) st = sait_prec_create_sait(ctx, ML, MU, &P);
        if (st == SAIT_OK) {
            e = cudaEventRecord(ev[1], s);
            if (e != cudaSuccess) st = ctx_cuda(ctx, e, "sait_tune_params", __FILE__, __LINE__);
        }
        if (st == SAIT_OK) {
            if (solver == SAIT_SOLVER_GMRES) st = sait_gmres(ctx, A, P, b, x, restart, tol, maxit, &info);
            else if (solver == SAIT_SOLVER_BICGSTAB) st = sait_bicgstab(ctx, A, P, b, x, tol, maxit, &info);
            else st = sait_pcg(ctx, A, P, b, x, tol, maxit, &info);
            const bool ran = st == SAIT_OK || st == SAIT_ERR_NOT_CONVERGED || st == SAIT_ERR_BREAKDOWN ||
                             st == SAIT_ERR_NONFINITE;
            e = cudaEventRecord(ev[2], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
            float b_ms = 0.0f, s_ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&b_ms, ev[0], ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&s_ms, ev[1], ev[2]);
            if (e != cudaSuccess) st = ctx_cuda(ctx, e, "sait_tune_params", __FILE__, __LINE__);
            else if (ran) {
                report->build_ms[c] = b_ms;
                report->solve_ms[c] = s_ms;
                report->iters[c] = info.iters;
                report->rel_resid[c] = info.rel_resid;
            }
        }
        if (ML && MU) report->nnz[c] = ML->nnz + MU->nnz;
        report->status[c] = st;
        if (P) sait_prec_destroy(P);
        if (ML) sait_mat_destroy(ML);
        if (MU) sait_mat_destroy(MU);
        if (st == SAIT_OK) {
            const double ms = report->solve_ms[c] + (count_build ? report->build_ms[c] : 0.0);
            if (report->chosen < 0 || ms < best_ms) {
                report->chosen = c;
                best_ms = ms;
                e = cudaMemcpyAsync(best.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) {
                    destroy_events();
                    return ctx_cuda(ctx, e, "sait_tune_params", __FILE__, __LINE__);
                }
            }
        } else if (st != SAIT_ERR_OOM && st != SAIT_ERR_NOT_CONVERGED && st != SAIT_ERR_BREAKDOWN &&
                   st != SAIT_ERR_NONFINITE) {
            destroy_events();
            return st;  // invalid input or a CUDA failure: stop (the message is in ctx)
        }
    }
    destroy_events();
    if (report->chosen < 0) return ctx_fail(ctx, SAIT_ERR_NOT_CONVERGED, "sait_tune_params: no candidate converged");
    SAIT_CK(cudaMemcpyAsync(x, best.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SAIT_CK(cudaStreamSynchronize(s));
    return SAIT_OK;
}
