// Jacobi sweeps as the triangular-solve replacement (Section 4, comparison
// with Jacobi iteration): k iterations of x^j = T~ x^{j-1} + D^-1 b from
// x^0 = 0 on L y = r, then on U z = y.  k sweeps apply exactly the undropped
// series M_k = sum_{j<k} T~^j D^-1 (Section 2), without storing it.
//
// One launch per sweep: a group of G lanes owns a row, accumulates
// sum_{j != i} t_ij x_j and writes x_i = d_i^-1 (b_i - sum).  The first sweep
// (x^1 = D^-1 b) is folded into the second, which reads d_j^-1 b_j in place of
// x_j, so k sweeps cost k - 1 passes over T (one scaled copy when k = 1).
#include "internal.cuh"

namespace {

template <int G, bool FIRST>
__global__ void __launch_bounds__(256)
k_jacobi_sweep(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
               const double *__restrict__ va, const double *__restrict__ dinv, const double *__restrict__ b,
               const double *__restrict__ xin, double *__restrict__ xout, const int *__restrict__ active,
               int *calls) {
    if (active && *active == 0) return;
    if (calls && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(calls, 1);
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x & (G - 1);
    double s = 0.0;
    if (row < n) {
        const int e0 = rp[row], e1 = rp[row + 1];
        for (int e = e0 + lane; e < e1; e += G) {
            const int c = ci[e];
            if (c == row) continue;
            const double xc = FIRST ? __ldg(dinv + c) * __ldg(b + c) : __ldg(xin + c);
            s = fma(va[e], xc, s);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && lane == 0) xout[row] = dinv[row] * (b[row] - s);
}

__global__ void k_jacobi_scale(int64_t n, const double *__restrict__ dinv, const double *__restrict__ b,
                               double *__restrict__ x, const int *__restrict__ active) {
    if (active && *active == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = dinv[i] * b[i];
}

// dinv_i = 1 / t_ii; bad[0] = 1 when a row has no finite nonzero diagonal
__global__ void k_jacobi_dinv(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ va, double *__restrict__ dinv, int *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] == i) d = va[e];
        if (d == 0.0 || !isfinite(d)) {
            *bad = 1;
            dinv[i] = 0.0;
        } else {
            dinv[i] = 1.0 / d;
        }
    }
}

template <bool FIRST>
void launch_sweep(const sait_mat_s *T, const double *dinv, const double *b, const double *xin, double *xout,
                  const int *active, cudaStream_t s, int *calls) {
    const int G = T->lanes;
    const unsigned blocks = (unsigned)cdiv(T->n * G, 256);
#define SAIT_JSWEEP(g)                                                                                      \
    launch_k(k_jacobi_sweep<g, FIRST>, blocks, 256, 0, s, T->n, (const int32_t *)T->rp, (const int32_t *)T->ci, \
             (const double *)T->va, dinv, b, xin, xout, active, calls)
    switch (G) {
        case 2: SAIT_JSWEEP(2); break;
        case 4: SAIT_JSWEEP(4); break;
        case 8: SAIT_JSWEEP(8); break;
        case 16: SAIT_JSWEEP(16); break;
        default: SAIT_JSWEEP(32); break;
    }
#undef SAIT_JSWEEP
}

// x = (k sweeps on T x = b); buf is an n-vector scratch distinct from b and x
cudaError_t jacobi_triangle(const sait_mat_s *T, const double *dinv, int k, const double *b, double *x,
                            double *buf, const int *active, cudaStream_t s, int *calls) {
    const int64_t n = T->n;
    if (k == 1) {
        launch_k(k_jacobi_scale, (unsigned)std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, s, n, dinv, b, x, active);
        return cudaGetLastError();
    }
    // sweeps 2..k alternate between buf and x and must end in x
    double *dst = ((k - 2) % 2 == 0) ? x : buf;
    launch_sweep<true>(T, dinv, b, nullptr, dst, active, s, calls);
    for (int j = 3; j <= k; j++) {
        double *src = dst;
        dst = (src == x) ? buf : x;
        launch_sweep<false>(T, dinv, b, src, dst, active, s, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace

sait_status jacobi_apply(sait_ctx ctx, sait_prec P, const double *r, double *z, const int *active) {
    if (P->n == 0) return SAIT_OK;
    ScopedTimer tm(ctx, SAIT_TIMER_APPLY);
    const int64_t n = P->n;
    double *y = P->tmp, *buf = P->gin;
    int *calls = group_counter(ctx, SAIT_TIMER_APPLY);
    SAIT_CK(jacobi_triangle(P->lo, P->dinv, P->sweeps, r, y, buf, active, ctx->stream, calls));
    SAIT_CK(jacobi_triangle(P->up, P->dinv + n, P->sweeps, y, z, buf, active, ctx->stream, nullptr));
    return SAIT_OK;
}

extern "C" sait_status sait_prec_create_jacobi(sait_ctx ctx, sait_mat L, sait_mat U, int32_t sweeps,
                                               sait_prec *P) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!L || !U || !P || L->n != U->n || sweeps < 1)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_prec_create_jacobi: bad argument");
    *P = nullptr;
    sait_prec p = new (std::nothrow) sait_prec_s();
    if (!p) return ctx_fail(ctx, SAIT_ERR_OOM, "host allocation failed");
    p->kind = 3;
    p->lo = L;
    p->up = U;
    p->n = L->n;
    p->sweeps = sweeps;
    p->device = ctx->device;
    const size_t n1 = p->n ? (size_t)p->n : 1;
    cudaError_t e = cudaMalloc((void **)&p->tmp, n1 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->gin, n1 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->dinv, 2 * n1 * sizeof(double));
    sait_status st = SAIT_OK;
    if (e != cudaSuccess) st = ctx_cuda(ctx, e, "sait_prec_create_jacobi", __FILE__, __LINE__);
    if (st == SAIT_OK && p->n > 0) {
        int *bad = (int *)ctx->h_pinned;
        DTemp<int> dbad;
        cudaStream_t s = ctx->stream;
        e = dbad.alloc(1, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dbad.p, 0, sizeof(int), s);
        const unsigned g = (unsigned)std::min<int64_t>(cdiv(p->n, 256), 4096);
        if (e == cudaSuccess) {
            launch_k(k_jacobi_dinv, g, 256, 0, s, p->n, (const int32_t *)L->rp, (const int32_t *)L->ci,
                     (const double *)L->va, p->dinv, dbad.p);
            launch_k(k_jacobi_dinv, g, 256, 0, s, p->n, (const int32_t *)U->rp, (const int32_t *)U->ci,
                     (const double *)U->va, p->dinv + p->n, dbad.p);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(bad, dbad.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = ctx_cuda(ctx, e, "sait_prec_create_jacobi", __FILE__, __LINE__);
        else if (*bad) st = ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_prec_create_jacobi: zero or missing diagonal");
    }
    if (st != SAIT_OK) {
        sait_prec_destroy(p);
        return st;
    }
    *P = p;
    return SAIT_OK;
}
