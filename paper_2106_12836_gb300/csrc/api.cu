// C ABI: contexts, matrices, products and preconditioner objects.
#include <climits>
#include <cstdio>

#include "internal.cuh"

sait_status ctx_fail(sait_ctx ctx, sait_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

sait_status ctx_cuda(sait_ctx ctx, cudaError_t e, const char *what, const char *file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    cudaGetLastError();  // clear a non-sticky error
    return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? SAIT_ERR_OOM : SAIT_ERR_CUDA, buf);
}

thread_local int64_t g_sait_launches = 0;

// ---- timing ---------------------------------------------------------------------
static cudaEvent_t get_event(sait_ctx ctx) {
    if (!ctx->spare.empty()) {
        cudaEvent_t e = ctx->spare.back();
        ctx->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

ScopedTimer::ScopedTimer(sait_ctx c, int g) : ctx(c), group(g) {
    if (!ctx || !ctx->timing || !(ctx->timing_groups >> g & 1u)) return;
    if (ctx->group_seen[g]++ % ctx->timing_every != 0) return;  // one call in timing_every
    a = get_event(ctx);
    if (!a) return;
    cudaEventRecord(a, ctx->stream);
    ctx->group_live[g] = true;
}

ScopedTimer::~ScopedTimer() {
    if (!a) return;
    ctx->group_live[group] = false;
    cudaEvent_t b = get_event(ctx);
    if (!b) { ctx->spare.push_back(a); return; }
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back(TimerRec{group, a, b});
    ctx->host_calls[group]++;
}

int *group_counter(sait_ctx ctx, int group) {
    return ctx && ctx->timing && ctx->group_live[group] ? ctx->d_word + kCounterBase + group : nullptr;
}

extern "C" sait_status sait_ctx_set_timing(sait_ctx ctx, int enable) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (enable && !ctx->timing)
        SAIT_CK(cudaMemsetAsync(ctx->d_word + kCounterBase, 0, SAIT_TIMER_COUNT * sizeof(int), ctx->stream));
    ctx->timing = enable != 0;
    return SAIT_OK;
}

extern "C" sait_status sait_ctx_set_timing_groups(sait_ctx ctx, uint32_t groups, int32_t every) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (every < 1) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_ctx_set_timing_groups: every < 1");
    ctx->timing_groups = groups;
    ctx->timing_every = every;
    for (int g = 0; g < SAIT_TIMER_COUNT; g++) ctx->group_seen[g] = 0;
    return SAIT_OK;
}

extern "C" sait_status sait_ctx_set_wait_limit(sait_ctx ctx, int64_t polls) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    ctx->wait_limit = polls > 0 ? polls : 0;
    return SAIT_OK;
}

extern "C" sait_status sait_ctx_set_device_loop(sait_ctx ctx, int32_t on) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    ctx->device_loop = on ? 1 : 0;
    return SAIT_OK;
}

extern "C" sait_status sait_ctx_stats(sait_ctx ctx, sait_stats *out, int reset) {
    if (!ctx || !out) return SAIT_ERR_INVALID_ARG;
    SAIT_CK(cudaStreamSynchronize(ctx->stream));
    for (const TimerRec &r : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->ms[r.group] += ms;
        ctx->spare.push_back(r.a);
        ctx->spare.push_back(r.b);
    }
    ctx->pending.clear();
    int dev_calls[SAIT_TIMER_COUNT];
    SAIT_CK(cudaMemcpy(dev_calls, ctx->d_word + kCounterBase, sizeof(dev_calls), cudaMemcpyDeviceToHost));
    out->launches = g_sait_launches - ctx->launch_base;
    for (int g = 0; g < SAIT_TIMER_COUNT; g++) {
        out->ms[g] = ctx->ms[g];
        // groups whose kernels may be skipped after convergence are counted on the device
        const bool device_counted = g == SAIT_TIMER_APPLY || g == SAIT_TIMER_SPMV || g == SAIT_TIMER_ORTHO;
        out->calls[g] = device_counted ? dev_calls[g] : ctx->host_calls[g];
    }
    if (reset) {
        for (int g = 0; g < SAIT_TIMER_COUNT; g++) { ctx->ms[g] = 0.0; ctx->host_calls[g] = 0; }
        ctx->launch_base = g_sait_launches;
        SAIT_CK(cudaMemsetAsync(ctx->d_word + kCounterBase, 0, SAIT_TIMER_COUNT * sizeof(int), ctx->stream));
        SAIT_CK(cudaStreamSynchronize(ctx->stream));
    }
    return SAIT_OK;
}

namespace {

enum { V_ROWPTR = 1, V_RANGE = 2, V_UNSORTED = 4 };

__global__ void k_validate(int64_t n, int64_t nnz, const int32_t *__restrict__ rp,
                           const int32_t *__restrict__ ci, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int bits = 0;
    if (i == 0 && rp[0] != 0) bits |= V_ROWPTR;
    if (i == n) {
        if (rp[n] != nnz) bits |= V_ROWPTR;
    } else {
        const int b = rp[i], e = rp[i + 1];
        if (e < b || b < 0 || e > nnz) {
            bits |= V_ROWPTR;
        } else {
            for (int k = b; k < e; k++) {
                if (ci[k] < 0 || ci[k] >= n) bits |= V_RANGE;
                if (k > b && ci[k] <= ci[k - 1]) bits |= V_UNSORTED;
            }
        }
    }
    if (bits) atomicOr(err, bits);
}

}  // namespace

// ---- context ------------------------------------------------------------------
extern "C" sait_status sait_ctx_create(sait_ctx *ctx, void *stream) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    *ctx = nullptr;
    sait_ctx c = new (std::nothrow) sait_ctx_s();
    if (!c) return SAIT_ERR_OOM;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_word, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_word, 0, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, 4096);
    if (e == cudaSuccess) {
        // keep freed temporaries in the stream-ordered pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->d_word) cudaFree(c->d_word);
        if (c->h_pinned) cudaFreeHost(c->h_pinned);
        delete c;
        return e == cudaErrorMemoryAllocation ? SAIT_ERR_OOM : SAIT_ERR_CUDA;
    }
    c->launch_base = g_sait_launches;
    static_apply_forget(c->device);
    *ctx = c;
    return SAIT_OK;
}

extern "C" sait_status sait_ctx_destroy(sait_ctx ctx) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (const TimerRec &r : ctx->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : ctx->spare) cudaEventDestroy(e);
    cudaFree(ctx->d_word);
    cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return SAIT_OK;
}

extern "C" const char *sait_status_string(sait_status st) {
    switch (st) {
        case SAIT_OK: return "ok";
        case SAIT_ERR_INVALID_ARG: return "invalid argument";
        case SAIT_ERR_NOT_TRIANGULAR: return "matrix is not triangular";
        case SAIT_ERR_ZERO_PIVOT: return "zero, missing or non-finite pivot";
        case SAIT_ERR_OOM: return "out of device memory";
        case SAIT_ERR_CUDA: return "CUDA error";
        case SAIT_ERR_NOT_CONVERGED: return "not converged";
        case SAIT_ERR_BREAKDOWN: return "Krylov breakdown";
        case SAIT_ERR_TIMEOUT: return "device wait timed out";
        case SAIT_ERR_NONFINITE: return "non-finite value";
        case SAIT_ERR_UNSUPPORTED: return "size beyond a supported limit";
    }
    return "unknown status";
}

extern "C" const char *sait_ctx_last_error(sait_ctx ctx) {
    return ctx ? ctx->last_error.c_str() : "null context";
}

// ---- matrices -----------------------------------------------------------------
cudaError_t mat_array(sait_ctx ctx, sait_mat M, void **p, size_t bytes) {
    M->pooled = true;
    return cudaMallocAsync(p, bytes ? bytes : 1, ctx->stream);
}

sait_status mat_alloc(sait_ctx ctx, int64_t n, int64_t nnz, sait_mat *out) {
    sait_mat M = new (std::nothrow) sait_mat_s();
    if (!M) return ctx_fail(ctx, SAIT_ERR_OOM, "host allocation failed");
    M->n = n;
    M->nnz = nnz;
    M->device = ctx->device;
    cudaError_t e = mat_array(ctx, M, (void **)&M->rp, (n + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = mat_array(ctx, M, (void **)&M->ci, (nnz ? nnz : 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = mat_array(ctx, M, (void **)&M->va, (nnz ? nnz : 1) * sizeof(double));
    if (e != cudaSuccess) {
        sait_mat_destroy(M);
        return ctx_cuda(ctx, e, "mat_alloc", __FILE__, __LINE__);
    }
    M->lanes = choose_lanes(n, nnz);
    *out = M;
    return SAIT_OK;
}

sait_status mat_prepare_store(sait_ctx ctx, sait_mat M, sait_dtype store_mode) {
    SAIT_TRY(mat_prepare_sell(ctx, M, store_mode));
    const sait_dtype store = store_base(store_mode);
    if (store == SAIT_F32 && !M->va32) {
        SAIT_CK(mat_array(ctx, M, (void **)&M->va32, (M->nnz ? M->nnz : 1) * sizeof(float)));
        SAIT_CK(cast_values(M->va, M->va32, nullptr, M->nnz, ctx->stream));
    } else if (store == SAIT_BF16 && !M->va16) {
        SAIT_CK(mat_array(ctx, M, (void **)&M->va16, (M->nnz ? M->nnz : 1) * sizeof(__nv_bfloat16)));
        SAIT_CK(cast_values(M->va, nullptr, M->va16, M->nnz, ctx->stream));
    }
    M->store = store_mode;
    return SAIT_OK;
}

sait_status mat_copy_csr(sait_ctx ctx, const sait_csr *A, sait_mat *out) {
    if (!A || !out) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_mat_create_csr: null argument");
    *out = nullptr;
    if (A->n < 0 || A->nnz < 0 || A->nnz >= INT_MAX || A->n >= INT_MAX || !A->row_ptr ||
        (A->nnz > 0 && (!A->col || !A->val)))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_mat_create_csr: bad sizes or pointers");
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), s));
    launch_k(k_validate, (unsigned)cdiv(A->n + 1, 256), 256, 0, s, A->n, A->nnz, A->row_ptr, A->col, ctx->d_word);
    SAIT_CK(cudaGetLastError());
    SAIT_CK(cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    if (h[0] & V_ROWPTR) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "row pointers are not a valid CSR");
    if (h[0] & V_RANGE) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "column index out of range");
    if (h[0] & V_UNSORTED) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "columns not strictly ascending in a row");
    sait_mat M = nullptr;
    SAIT_TRY(mat_alloc(ctx, A->n, A->nnz, &M));
    cudaError_t e = cudaMemcpyAsync(M->rp, A->row_ptr, (A->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && A->nnz)
        e = cudaMemcpyAsync(M->ci, A->col, A->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && A->nnz)
        e = cudaMemcpyAsync(M->va, A->val, A->nnz * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        sait_mat_destroy(M);
        return ctx_cuda(ctx, e, "sait_mat_create_csr", __FILE__, __LINE__);
    }
    *out = M;
    return SAIT_OK;
}

extern "C" sait_status sait_mat_create_csr(sait_ctx ctx, const sait_csr *A, sait_mat *out) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    sait_mat M = nullptr;
    SAIT_TRY(mat_copy_csr(ctx, A, &M));
    cudaStream_t s = ctx->stream;
    sait_status st = mat_prepare_store(ctx, M, SAIT_F64);
    if (st == SAIT_OK && cudaStreamSynchronize(s) != cudaSuccess)
        st = ctx_cuda(ctx, cudaGetLastError(), "sait_mat_create_csr", __FILE__, __LINE__);
    if (st != SAIT_OK) {
        sait_mat_destroy(M);
        return st;
    }
    *out = M;
    return SAIT_OK;
}

extern "C" sait_status sait_mat_destroy(sait_mat M) {
    if (!M) return SAIT_ERR_INVALID_ARG;
    if (M->pooled) {  // cudaFree does not wait for work still reading pool memory
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != M->device) cudaSetDevice(M->device);
        cudaDeviceSynchronize();
        if (cur >= 0 && cur != M->device) cudaSetDevice(cur);
    }
    if (M->rp) cudaFree(M->rp);
    if (M->ci) cudaFree(M->ci);
    if (M->va) cudaFree(M->va);
    if (M->va32) cudaFree(M->va32);
    if (M->va16) cudaFree(M->va16);
    if (M->soff) cudaFree(M->soff);
    if (M->sperm) cudaFree(M->sperm);
    if (M->sci) cudaFree(M->sci);
    if (M->sva64) cudaFree(M->sva64);
    if (M->sva32) cudaFree(M->sva32);
    if (M->sva16) cudaFree(M->sva16);
    delete M;
    return SAIT_OK;
}

extern "C" sait_status sait_mat_info(sait_mat M, int64_t *n, int64_t *nnz) {
    if (!M) return SAIT_ERR_INVALID_ARG;
    if (n) *n = M->n;
    if (nnz) *nnz = M->nnz;
    return SAIT_OK;
}

extern "C" sait_status sait_mat_export_csr(sait_ctx ctx, sait_mat M, int32_t *row_ptr, int32_t *col,
                                           double *val) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!M) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_mat_export_csr: null matrix");
    cudaStream_t s = ctx->stream;
    if (row_ptr) SAIT_CK(cudaMemcpyAsync(row_ptr, M->rp, (M->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (col && M->nnz) SAIT_CK(cudaMemcpyAsync(col, M->ci, M->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (val && M->nnz) SAIT_CK(cudaMemcpyAsync(val, M->va, M->nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return SAIT_OK;
}

extern "C" sait_status sait_mat_set_store(sait_ctx ctx, sait_mat M, sait_dtype store) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!M || !store_valid(store))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_mat_set_store: bad argument");
    SAIT_TRY(mat_prepare_store(ctx, M, store));
    SAIT_CK(cudaStreamSynchronize(ctx->stream));
    return SAIT_OK;
}

// ---- products -----------------------------------------------------------------
extern "C" sait_status sait_spmv(sait_ctx ctx, sait_mat A, const double *x, double *y) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || (A->n > 0 && (!x || !y))) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_spmv: null argument");
    ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
    SAIT_CK(launch_spmv(A, A->store, x, false, y, false, nullptr, ctx->stream,
                        group_counter(ctx, SAIT_TIMER_SPMV)));
    return SAIT_OK;
}

static sait_status apply_pair(sait_ctx ctx, sait_mat ML, sait_mat MU, const double *r, double *z,
                              void *w, const int *active) {
    const bool f64 = store_x64(ML->store) && store_x64(MU->store);
    ScopedTimer tm(ctx, SAIT_TIMER_APPLY);
    if (!f64 && !store_x64(ML->store)) {
        // FP32 products round every gathered entry of r to FP32: round r once
        // into the second half of the n-double scratch and gather 4-byte values
        float *r32 = (float *)w + ML->n;
        SAIT_CK(launch_narrow(ML->n, r, r32, active, ctx->stream, ctx->num_sms));
        SAIT_CK(launch_spmv(ML, ML->store, r32, true, w, true, active, ctx->stream,
                            group_counter(ctx, SAIT_TIMER_APPLY), true));
    } else {
        SAIT_CK(launch_spmv(ML, ML->store, r, false, w, !f64, active, ctx->stream,
                            group_counter(ctx, SAIT_TIMER_APPLY), true));
    }
    // M_U's product may start while M_L's drains (its SELL kernel waits for it first)
    SAIT_CK(launch_spmv(MU, MU->store, w, !f64, z, false, active, ctx->stream, nullptr, true));
    return SAIT_OK;
}

extern "C" sait_status sait_apply(sait_ctx ctx, sait_mat ML, sait_mat MU, const double *r, double *z) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!ML || !MU || ML->n != MU->n || (ML->n > 0 && (!r || !z)))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_apply: bad argument");
    DTemp<double> w;
    SAIT_CK(w.alloc(ML->n, ctx->stream));
    return apply_pair(ctx, ML, MU, r, z, w.p, nullptr);
}

// ---- preconditioners ------------------------------------------------------------
extern "C" sait_status sait_prec_create_sait(sait_ctx ctx, sait_mat ML, sait_mat MU, sait_prec *P) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!ML || !MU || !P || ML->n != MU->n)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_prec_create_sait: bad argument");
    sait_prec p = new (std::nothrow) sait_prec_s();
    if (!p) return ctx_fail(ctx, SAIT_ERR_OOM, "host allocation failed");
    p->kind = 1;
    p->lo = ML;
    p->up = MU;
    p->n = ML->n;
    p->device = ctx->device;
    p->pooled = true;
    cudaError_t e = cudaMallocAsync((void **)&p->tmp, (p->n ? p->n : 1) * sizeof(double), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // usable from any stream on return
    if (e != cudaSuccess) {
        if (p->tmp) cudaFreeAsync(p->tmp, ctx->stream);
        delete p;
        return ctx_cuda(ctx, e, "sait_prec_create_sait", __FILE__, __LINE__);
    }
    *P = p;
    return SAIT_OK;
}

static sait_status capture_trisolve_graph(sait_ctx ctx, sait_prec p) {
    // The substitution is one launch per level set; capture both sweeps once so
    // that a replay costs one graph launch instead of 2 x levels launches.
    cudaStream_t cs;
    SAIT_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const int64_t launches0 = g_sait_launches;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = launch_trisolve(p->lo, p->lev_lo, true, p->gin, p->tmp, cs);
        cudaError_t e2 = launch_trisolve(p->up, p->lev_up, false, p->tmp, p->gout, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
        if (e == cudaSuccess && e2 != cudaSuccess) e = e2;
    }
    p->graph_kernels = g_sait_launches - launches0;  // captured, not executed
    g_sait_launches = launches0;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "capture_trisolve_graph", __FILE__, __LINE__);
    return SAIT_OK;
}

extern "C" sait_status sait_prec_create_ilu(sait_ctx ctx, sait_mat L, sait_mat U, sait_prec *P) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!L || !U || !P || L->n != U->n)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_prec_create_ilu: bad argument");
    *P = nullptr;
    sait_prec p = new (std::nothrow) sait_prec_s();
    if (!p) return ctx_fail(ctx, SAIT_ERR_OOM, "host allocation failed");
    p->kind = 2;
    p->lo = L;
    p->up = U;
    p->n = L->n;
    p->device = ctx->device;
    sait_status st = build_levels(ctx, L->rp, L->ci, L->n, true, &p->lev_lo);
    if (st == SAIT_OK) st = build_levels(ctx, U->rp, U->ci, U->n, false, &p->lev_up);
    cudaError_t e = cudaSuccess;
    if (st == SAIT_OK) e = cudaMalloc((void **)&p->tmp, (p->n ? p->n : 1) * sizeof(double));
    if (e == cudaSuccess && st == SAIT_OK) e = cudaMalloc((void **)&p->gin, (p->n ? p->n : 1) * sizeof(double));
    if (e == cudaSuccess && st == SAIT_OK) e = cudaMalloc((void **)&p->gout, (p->n ? p->n : 1) * sizeof(double));
    if (e != cudaSuccess) st = ctx_cuda(ctx, e, "sait_prec_create_ilu", __FILE__, __LINE__);
    if (st == SAIT_OK) st = capture_trisolve_graph(ctx, p);
    if (st != SAIT_OK) {
        sait_prec_destroy(p);
        return st;
    }
    *P = p;
    return SAIT_OK;
}

extern "C" sait_status sait_prec_levels(sait_prec P, int32_t *levels_lower, int32_t *levels_upper) {
    if (!P) return SAIT_ERR_INVALID_ARG;
    if (levels_lower) *levels_lower = P->lev_lo.nlev;
    if (levels_upper) *levels_upper = P->lev_up.nlev;
    return SAIT_OK;
}

__global__ void k_copy_if(int64_t n, const double *__restrict__ x, double *__restrict__ y,
                          const int *__restrict__ active) {
    if (active && *active == 0) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}

sait_status prec_apply_impl(sait_ctx ctx, sait_prec P, const double *r, double *z, const int *active) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P ? P->n : 0;
    if (!P) return SAIT_OK;
    if (P->kind == 1) return apply_pair(ctx, P->lo, P->up, r, z, P->tmp, active);
    if (P->kind == 2) {
        if (n == 0) return SAIT_OK;
        ScopedTimer tm(ctx, SAIT_TIMER_TRISOLVE);
        launch_k(k_copy_if, (unsigned)cdiv(n, 256), 256, 0, s, n, r, P->gin, active);
        SAIT_CK(cudaGetLastError());
        SAIT_CK(cudaGraphLaunch(P->graph, s));
        g_sait_launches += P->graph_kernels;
        launch_k(k_copy_if, (unsigned)cdiv(n, 256), 256, 0, s, n, P->gout, z, active);
        SAIT_CK(cudaGetLastError());
        return SAIT_OK;
    }
    if (P->kind == 3) return jacobi_apply(ctx, P, r, z, active);
    return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "unknown preconditioner kind");
}

extern "C" sait_status sait_prec_apply(sait_ctx ctx, sait_prec P, const double *r, double *z) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!P || (P->n > 0 && (!r || !z))) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_prec_apply: bad argument");
    return prec_apply_impl(ctx, P, r, z, nullptr);
}

extern "C" sait_status sait_prec_destroy(sait_prec P) {
    if (!P) return SAIT_ERR_INVALID_ARG;
    if (P->pooled) {  // cudaFree does not wait for work still reading pool memory
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != P->device) cudaSetDevice(P->device);
        cudaDeviceSynchronize();
        if (cur >= 0 && cur != P->device) cudaSetDevice(cur);
    }
    if (P->graph) cudaGraphExecDestroy(P->graph);
    free_levels(&P->lev_lo);
    free_levels(&P->lev_up);
    if (P->tmp) cudaFree(P->tmp);
    if (P->gin) cudaFree(P->gin);
    if (P->gout) cudaFree(P->gout);
    if (P->dinv) cudaFree(P->dinv);
    delete P;
    return SAIT_OK;
}
