// Krylov solvers with a SAIT (or exact-ILU) preconditioner, all state on the
// device.  The SAIT apply z = M_U (M_L r) is the preconditioning step of every
// iteration (Section 3.1); the runtime model of the paper (equation runtime)
// splits an iteration into that apply and the "other computation", which here
// is one FP64 product with A and the orthogonalisation / vector updates.
//
// Every kernel of an iteration reads a device flag `active` and returns at
// once when it is 0, so the host can enqueue several iterations ahead and
// read the status word only every kPoll iterations.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPoll = 8;       // iterations enqueued between status reads
constexpr int kMaxRestart = 512;

struct Scal {        // device-resident solver scalars
    int active;      // 1 while the current cycle / iteration runs
    int jdone;       // GMRES: Arnoldi steps done in this cycle; BiCGSTAB: iterations done
    int state;       // 0 running, 1 converged, 2 breakdown, 3 non-finite, 4 x updated (half step)
    int pad;
    double bnorm, beta, tolb, inv;
    double rho, rho_old, alpha, omega, beta_b;
    double r0, r1, r2, r3;    // reduction results
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; w++) r += ws[w];
    __syncthreads();
    return r;  // valid in thread 0
}

// partial[b*3 + q] = sum over this block's rows of x_q * y_q, q < nd (nd <= 3)
__global__ void __launch_bounds__(kThreads)
k_dots(int64_t n, int nd, const double *__restrict__ x0, const double *__restrict__ y0,
       const double *__restrict__ x1, const double *__restrict__ y1, const double *__restrict__ x2,
       const double *__restrict__ y2, double *partial, const int *active) {
    if (active && *active == 0) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        s0 = fma(x0[i], y0[i], s0);
        if (nd > 1) s1 = fma(x1[i], y1[i], s1);
        if (nd > 2) s2 = fma(x2[i], y2[i], s2);
    }
    double t0 = block_sum(s0);
    double t1 = nd > 1 ? block_sum(s1) : 0.0;
    double t2 = nd > 2 ? block_sum(s2) : 0.0;
    if (threadIdx.x == 0) {
        partial[blockIdx.x * 3 + 0] = t0;
        partial[blockIdx.x * 3 + 1] = t1;
        partial[blockIdx.x * 3 + 2] = t2;
    }
}

// out[q] = sum_b partial[b*stride + q]   (one block per q, fixed order);
// with Hj given, also Hj[q] = out[q] (first) or Hj[q] += out[q]
__global__ void __launch_bounds__(kThreads)
k_reduce(const double *__restrict__ partial, int nb, int stride, double *out, const int *active, double *Hj,
         int first) {
    if (active && *active == 0) return;
    const int q = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) s += partial[(int64_t)b * stride + q];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        out[q] = s;
        if (Hj) Hj[q] = first ? s : Hj[q] + s;
    }
}

// Classical Gram-Schmidt with two passes, split by precision.  GB300's FP64
// pipe (1.2 TFLOP/s measured, against 63.5 TFLOP/s FP32) would bound FP64
// passes far below HBM speed, so no pass runs per-entry FP64 products.  The
// basis is kept as V (FP64, the vectors the products read), and as the pair
// (V_hi, V_lo) of FP32 arrays carrying V to ~2^-46 (split_pair):
//   pass 1 dots   h1 = V^T w   FP32 products on V_hi;
//   pass 1 update w -= V h1    double-float products on (V_hi, V_lo) and
//                              (h_hi, h_lo), error-free two-sum accumulation
//                              on the FP32 pipe, one FP64 subtraction per
//                              entry (this subtraction cancels, so its error
//                              must stay near FP64 level);
//   pass 2 dots   h2 = V^T w   FP32 products on V_hi and fl32(w);
//   pass 2 update w -= V h2    FP32 products on V_hi (h2 is ~1e-7 |w|),
// and H(:, j) = h1 + h2 in FP64.  The updates keep the Arnoldi relation
// A Z = V H at ~1e-14 relative; the FP32 dots leave the basis orthogonal to
// ~1e-7, which does not move GMRES's residual estimate at the 1e-8 target.
//
// Layout: the basis columns have a leading dimension ldv = n rounded up to a
// multiple of 4 with zero padding, so every kernel below moves 16-byte
// vectors (four rows per thread) and never needs a ragged tail.
//
// Dots: partial[b*ldp + q] = sum over block b's rows of V_q . w (q < nvec).
// One register accumulator per vector of a chunk; the last chunk is
// instantiated for its exact size so no FMA slot is wasted.
constexpr int kCH = 16;

__device__ __forceinline__ float4 load_w4(const float4 *w, int64_t i4) { return w[i4]; }
__device__ __forceinline__ float4 load_w4(const double2 *w, int64_t i4) {
    const double2 a = w[2 * i4], b = w[2 * i4 + 1];
    return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

template <typename TW, int CH>
__device__ __forceinline__ void dot_chunk(int64_t n4, const float4 *__restrict__ V, int64_t ldv4, int q0,
                                          const TW *__restrict__ w, double *partial, int ldp,
                                          double (*red)[kCH]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[CH > 0 ? CH : 1];
#pragma unroll
    for (int t = 0; t < (CH > 0 ? CH : 1); t++) acc[t] = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kThreads) {
        const float4 wv = load_w4(w, i);
        float4 vv[CH > 0 ? CH : 1];
#pragma unroll
        for (int t = 0; t < CH; t++) vv[t] = __ldg(V + (int64_t)(q0 + t) * ldv4 + i);
#pragma unroll
        for (int t = 0; t < CH; t++) {
            float a = fmaf(vv[t].x, wv.x, acc[t]);
            a = fmaf(vv[t].y, wv.y, a);
            a = fmaf(vv[t].z, wv.z, a);
            acc[t] = fmaf(vv[t].w, wv.w, a);
        }
    }
    // warp sums in FP32 (the products are FP32 anyway; FP64 adds here would
    // cost more than the whole sweep on GB300), then FP64 across warps/blocks
#pragma unroll
    for (int t = 0; t < CH; t++) {
        float v = acc[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][t] = (double)v;
    }
    __syncthreads();
    if ((int)threadIdx.x < CH) {
        double sum = 0.0;
        for (int w2 = 0; w2 < kThreads / 32; w2++) sum += red[w2][threadIdx.x];
        partial[(int64_t)blockIdx.x * ldp + q0 + (int)threadIdx.x] = sum;
    }
    __syncthreads();
}

template <typename TW>
__device__ __forceinline__ void dot_tail(int rem, int64_t n4, const float4 *V, int64_t ldv4, int q0, const TW *w,
                                         double *partial, int ldp, double (*red)[kCH]) {
    switch (rem) {
#define SAIT_TAIL(k) case k: dot_chunk<TW, k>(n4, V, ldv4, q0, w, partial, ldp, red); break;
        SAIT_TAIL(1) SAIT_TAIL(2) SAIT_TAIL(3) SAIT_TAIL(4) SAIT_TAIL(5) SAIT_TAIL(6) SAIT_TAIL(7)
        SAIT_TAIL(8) SAIT_TAIL(9) SAIT_TAIL(10) SAIT_TAIL(11) SAIT_TAIL(12) SAIT_TAIL(13) SAIT_TAIL(14)
        SAIT_TAIL(15)
#undef SAIT_TAIL
        default: break;
    }
}

// h = V^T w with FP32 products: TW = double2 (w in FP64, rounded on load) or float4
template <typename TW>
__global__ void __launch_bounds__(kThreads)
k_cgs_dot(int64_t n4, const float4 *__restrict__ V, int64_t ldv4, int nvec, const TW *__restrict__ w,
          double *partial, int ldp, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ double red[kThreads / 32][kCH];
    int q0 = 0;
    for (; nvec - q0 >= kCH; q0 += kCH) dot_chunk<TW, kCH>(n4, V, ldv4, q0, w, partial, ldp, red);
    dot_tail<TW>(nvec - q0, n4, V, ldv4, q0, w, partial, ldp, red);
}

// Pass-1 update: w -= V h in double-float (see above), four rows per thread.
// Writes w (FP64) and its FP32 rounding for the pass-2 dots.
__global__ void __launch_bounds__(kThreads, 6)
k_cgs_update_df(int64_t n4, const float4 *__restrict__ Vh, const float4 *__restrict__ Vl, int64_t ldv4, int nvec,
                const double *__restrict__ h, double2 *w, float4 *w32, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ float hh[kMaxRestart + 1], hl[kMaxRestart + 1];
    for (int q = threadIdx.x; q < nvec; q += kThreads) {
        const double hd = h[q];
        const float a = (float)hd;
        hh[q] = a;
        hl[q] = (float)(hd - (double)a);
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kThreads) {
        float S[4] = {0.0f, 0.0f, 0.0f, 0.0f}, E[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int q = 0;
        for (; q + 2 <= nvec; q += 2) {
            const float4 h0 = __ldg(Vh + (int64_t)q * ldv4 + i), l0 = __ldg(Vl + (int64_t)q * ldv4 + i);
            const float4 h1 = __ldg(Vh + (int64_t)(q + 1) * ldv4 + i), l1 = __ldg(Vl + (int64_t)(q + 1) * ldv4 + i);
            const float a0 = hh[q], b0 = hl[q], a1 = hh[q + 1], b1 = hl[q + 1];
            df_term(S[0], E[0], h0.x, l0.x, a0, b0);
            df_term(S[1], E[1], h0.y, l0.y, a0, b0);
            df_term(S[2], E[2], h0.z, l0.z, a0, b0);
            df_term(S[3], E[3], h0.w, l0.w, a0, b0);
            df_term(S[0], E[0], h1.x, l1.x, a1, b1);
            df_term(S[1], E[1], h1.y, l1.y, a1, b1);
            df_term(S[2], E[2], h1.z, l1.z, a1, b1);
            df_term(S[3], E[3], h1.w, l1.w, a1, b1);
        }
        if (q < nvec) {
            const float4 h0 = __ldg(Vh + (int64_t)q * ldv4 + i), l0 = __ldg(Vl + (int64_t)q * ldv4 + i);
            const float a0 = hh[q], b0 = hl[q];
            df_term(S[0], E[0], h0.x, l0.x, a0, b0);
            df_term(S[1], E[1], h0.y, l0.y, a0, b0);
            df_term(S[2], E[2], h0.z, l0.z, a0, b0);
            df_term(S[3], E[3], h0.w, l0.w, a0, b0);
        }
        double2 wa = w[2 * i], wb = w[2 * i + 1];
        wa.x -= (double)S[0] + (double)E[0];
        wa.y -= (double)S[1] + (double)E[1];
        wb.x -= (double)S[2] + (double)E[2];
        wb.y -= (double)S[3] + (double)E[3];
        w[2 * i] = wa;
        w[2 * i + 1] = wb;
        w32[i] = make_float4((float)wa.x, (float)wa.y, (float)wb.x, (float)wb.y);
    }
}

// Pass-2 update: w -= V h with FP32 products on V_hi, four rows per thread;
// partial[b] = ||w||^2 (FP64) of block b's rows.
__global__ void __launch_bounds__(kThreads)
k_cgs_update32(int64_t n4, const float4 *__restrict__ V, int64_t ldv4, int nvec, const double *__restrict__ h,
               double2 *w, double *partial, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ float hs[kMaxRestart + 1];
    for (int q = threadIdx.x; q < nvec; q += kThreads) hs[q] = (float)h[q];
    __syncthreads();
    double nrm = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kThreads) {
        float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;  // two chains per row
        int q = 0;
        for (; q + 2 <= nvec; q += 2) {
            const float4 v0 = __ldg(V + (int64_t)q * ldv4 + i), v1 = __ldg(V + (int64_t)(q + 1) * ldv4 + i);
            const float a0 = hs[q], a1 = hs[q + 1];
            s0.x = fmaf(v0.x, a0, s0.x); s0.y = fmaf(v0.y, a0, s0.y);
            s0.z = fmaf(v0.z, a0, s0.z); s0.w = fmaf(v0.w, a0, s0.w);
            s1.x = fmaf(v1.x, a1, s1.x); s1.y = fmaf(v1.y, a1, s1.y);
            s1.z = fmaf(v1.z, a1, s1.z); s1.w = fmaf(v1.w, a1, s1.w);
        }
        if (q < nvec) {
            const float4 v0 = __ldg(V + (int64_t)q * ldv4 + i);
            const float a0 = hs[q];
            s0.x = fmaf(v0.x, a0, s0.x); s0.y = fmaf(v0.y, a0, s0.y);
            s0.z = fmaf(v0.z, a0, s0.z); s0.w = fmaf(v0.w, a0, s0.w);
        }
        double2 wa = w[2 * i], wb = w[2 * i + 1];
        wa.x -= (double)(s0.x + s1.x);
        wa.y -= (double)(s0.y + s1.y);
        wb.x -= (double)(s0.z + s1.z);
        wb.y -= (double)(s0.w + s1.w);
        w[2 * i] = wa;
        w[2 * i + 1] = wb;
        nrm = fma(wa.x, wa.x, nrm);
        nrm = fma(wa.y, wa.y, nrm);
        nrm = fma(wb.x, wb.x, nrm);
        nrm = fma(wb.y, wb.y, nrm);
    }
    nrm = block_sum(nrm);
    if (threadIdx.x == 0) partial[blockIdx.x] = nrm;
}

// v = w / ||w|| in FP64 (rows < n), plus its FP32 pair (hi, lo)
__global__ void k_scale3(int64_t n, const double *__restrict__ x, double *y, float *yh, float *yl, const Scal *sc,
                         const int *active) {
    if (active && *active == 0) return;
    const double a = sc->inv;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const double v = x[i] * a;
        float hi, lo;
        split_pair(v, hi, lo);
        y[i] = v;
        yh[i] = hi;
        yl[i] = lo;
    }
}

// w -= V h (sub = true) or w = V h (sub = false); nvec from *nvec_dev if given.
__global__ void __launch_bounds__(kThreads)
k_gemv(int64_t n, const double *__restrict__ V, int64_t ldv, int nvec, const int *nvec_dev,
       const double *__restrict__ h, double *w, int sub, const int *active) {
    if (active && *active == 0) return;
    __shared__ double hs[kMaxRestart + 1];
    const int nv = nvec_dev ? *nvec_dev : nvec;
    for (int q = threadIdx.x; q < nv; q += kThreads) hs[q] = h[q];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double s = 0.0;
        for (int q = 0; q < nv; q++) s = fma(V[(int64_t)q * ldv + i], hs[q], s);
        w[i] = sub ? w[i] - s : s;
    }
}

// r = b - A x, FP64, G lanes per row
template <int G>
__global__ void __launch_bounds__(kThreads)
k_residual(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
           const double *__restrict__ va, const double *__restrict__ x, const double *__restrict__ b,
           double *__restrict__ r) {
    const int64_t row = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / G;
    const int lane = threadIdx.x & (G - 1);
    double s = 0.0;
    if (row < n)
        for (int k = rp[row] + lane; k < rp[row + 1]; k += G) s = fma(va[k], x[ci[k]], s);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && lane == 0) r[row] = b[row] - s;
}

__global__ void k_axpy1(int64_t n, const double *__restrict__ x, double *y) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        y[i] += x[i];
}

// ---- GMRES scalar kernels (one thread) -------------------------------------
__global__ void k_gmres_start(Scal *sc, double *g, int m) {
    const double beta = sqrt(sc->r0);
    sc->beta = beta;
    sc->inv = beta > 0.0 ? 1.0 / beta : 0.0;
    sc->active = 1;
    sc->jdone = 0;
    sc->state = 0;
    g[0] = beta;
    for (int i = 1; i <= m; i++) g[i] = 0.0;
}

// sc->r0 = ||w||^2 from the update's per-block partials (fixed order), then
// one thread applies the previous rotations to column j of H and forms the
// new one.  The column and the rotations are staged in shared memory first:
// the rotation chain is sequential, and global loads inside it would each
// cost a full memory latency.
__global__ void __launch_bounds__(kThreads)
k_givens(int j, int m, int remaining, double *H, double *cs, double *sn, double *g, Scal *sc,
         const double *__restrict__ partial, int nb, int *calls) {
    if (sc->active == 0) return;
    __shared__ double hc[kMaxRestart + 2], cc[kMaxRestart], ss[kMaxRestart];
    double *Hj = H + (int64_t)j * (m + 1);
    for (int i = threadIdx.x; i <= j; i += kThreads) hc[i] = Hj[i];
    for (int i = threadIdx.x; i < j; i += kThreads) {
        cc[i] = cs[i];
        ss[i] = sn[i];
    }
    double t0 = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) t0 += partial[b];
    t0 = block_sum(t0);  // synchronizes the block
    if (threadIdx.x != 0) return;
    sc->r0 = t0;
    if (calls) atomicAdd(calls, 1);
    const double hn = sqrt(t0);
    hc[j + 1] = hn;
    for (int i = 0; i < j; i++) {
        const double t = cc[i] * hc[i] + ss[i] * hc[i + 1];
        hc[i + 1] = -ss[i] * hc[i] + cc[i] * hc[i + 1];
        hc[i] = t;
    }
    const double a = hc[j], b = hn;
    double c = 1.0, s = 0.0;
    if (b != 0.0) {
        const double t = hypot(a, b);
        c = a / t;
        s = b / t;
    }
    cs[j] = c;
    sn[j] = s;
    hc[j] = c * a + s * b;
    hc[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; i++) Hj[i] = hc[i];
    const double gj = g[j];
    g[j + 1] = -s * gj;
    g[j] = c * gj;
    sc->jdone = j + 1;
    sc->inv = hn != 0.0 ? 1.0 / hn : 0.0;
    const double est = fabs(s * gj);
    if (!isfinite(est) || !isfinite(hn)) {
        sc->state = 3;
        sc->active = 0;
    } else if (est <= sc->tolb || hn == 0.0 || j + 1 >= remaining || j + 1 >= m) {
        sc->active = 0;
    }
}

// back substitution H y = g on the first jdone rows, column-oriented: once
// y_i is known every thread removes its multiple from the rows above
__global__ void __launch_bounds__(kThreads) k_hsolve(const double *H, const double *g, double *y, int m, Scal *sc) {
    __shared__ double sv[kMaxRestart + 1], yv[kMaxRestart + 1];
    const int jd = sc->jdone;
    for (int k = threadIdx.x; k < jd; k += kThreads) sv[k] = g[k];
    __syncthreads();
    for (int i = jd - 1; i >= 0; i--) {
        const double *Hi = H + (int64_t)i * (m + 1);  // column i: Hi[k] = H(k, i)
        if (threadIdx.x == 0) {
            const double d = Hi[i];
            if (d == 0.0) {
                sc->state = 2;
                yv[i] = 0.0;
            } else {
                yv[i] = sv[i] / d;
            }
        }
        __syncthreads();
        const double yi = yv[i];
        for (int k = threadIdx.x; k < i; k += kThreads) sv[k] -= Hi[k] * yi;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < jd; k += kThreads) y[k] = yv[k];
}

// ---- BiCGSTAB kernels ---------------------------------------------------------
__global__ void k_bicg_init(Scal *sc) {  // r0 holds ||r||^2 of the (re)start residual
    sc->rho_old = sc->alpha = sc->omega = 1.0;
    sc->active = 1;
    sc->state = 0;
    sc->r3 = sqrt(sc->r0);  // smallest residual norm of this recurrence
}

__global__ void k_bicg_beta(Scal *sc) {  // after rho = (rh, r) in r0
    if (sc->active == 0) return;
    const double rho = sc->r0;
    sc->rho = rho;
    if (rho == 0.0 || sc->omega == 0.0 || !isfinite(rho)) {
        sc->state = !isfinite(rho) ? 3 : 2;
        sc->active = 0;
        return;
    }
    sc->beta_b = (rho / sc->rho_old) * (sc->alpha / sc->omega);
}

__global__ void k_bicg_p(int64_t n, const double *__restrict__ r, const double *__restrict__ v, double *p,
                         const Scal *sc) {
    if (sc->active == 0) return;
    const double beta = sc->beta_b, omega = sc->omega;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

__global__ void k_bicg_alpha(Scal *sc) {  // after (rh, v) in r0
    if (sc->active == 0) return;
    const double rv = sc->r0;
    if (rv == 0.0 || !isfinite(rv)) {
        sc->state = !isfinite(rv) ? 3 : 2;
        sc->active = 0;
        return;
    }
    sc->alpha = sc->rho / rv;
}

// s = r - alpha v
__global__ void k_bicg_s(int64_t n, const double *__restrict__ r, const double *__restrict__ v, double *s,
                         const Scal *sc) {
    if (sc->active == 0) return;
    const double alpha = sc->alpha;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        s[i] = r[i] - alpha * v[i];
}

__global__ void k_bicg_check_s(Scal *sc) {  // after (s, s) in r0
    if (sc->active == 0) return;
    sc->jdone += 1;
    const double sn = sqrt(sc->r0);
    if (!isfinite(sn)) { sc->state = 3; sc->active = 0; return; }
    if (sn <= sc->tolb) { sc->state = 4; sc->active = 0; }
}

// half step converged: x += alpha ph (runs once, when state == 4)
__global__ void k_bicg_xhalf(int64_t n, double *x, const double *__restrict__ ph, Scal *sc) {
    if (sc->state != 4) return;
    const double alpha = sc->alpha;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        x[i] += alpha * ph[i];
}

__global__ void k_bicg_xhalf_done(Scal *sc) {
    if (sc->state == 4) sc->state = 1;
}

__global__ void k_bicg_omega(Scal *sc) {  // after (t,t) in r0, (t,s) in r1
    if (sc->active == 0) return;
    const double tt = sc->r0;
    sc->omega = tt == 0.0 ? 0.0 : sc->r1 / tt;
}

// x += alpha ph + omega sh;  r = s - omega t
__global__ void k_bicg_xr(int64_t n, double *x, double *r, const double *__restrict__ ph,
                          const double *__restrict__ sh, const double *__restrict__ s,
                          const double *__restrict__ t, const Scal *sc) {
    if (sc->active == 0) return;
    const double alpha = sc->alpha, omega = sc->omega;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        x[i] += alpha * ph[i] + omega * sh[i];
        r[i] = s[i] - omega * t[i];
    }
}

__global__ void k_bicg_check_r(Scal *sc, int remaining) {  // after (r, r) in r0
    if (sc->active == 0) return;
    sc->rho_old = sc->rho;
    const double rn = sqrt(sc->r0);
    if (!isfinite(rn)) { sc->state = 3; sc->active = 0; return; }
    if (rn <= sc->tolb) { sc->state = 1; sc->active = 0; return; }
    if (sc->jdone >= remaining) { sc->active = 0; return; }
    // divergence guard: restart the recurrence from the current iterate once
    // the residual has grown four orders of magnitude above its minimum
    if (rn > 1e4 * sc->r3) { sc->state = 5; sc->active = 0; return; }
    sc->r3 = fmin(sc->r3, rn);
}


// ---- PCG kernels (Saad, Algorithm 9.1) ----------------------------------------------
__global__ void k_pcg_alpha(Scal *sc) {  // after (p, q) in r0
    if (sc->active == 0) return;
    const double pq = sc->r0;
    if (pq == 0.0 || !isfinite(pq)) {
        sc->state = isfinite(pq) ? 2 : 3;
        sc->active = 0;
        return;
    }
    sc->alpha = sc->rho / pq;
}

// x += alpha p; r -= alpha q; partial ||r||^2
__global__ void __launch_bounds__(kThreads)
k_pcg_xr(int64_t n, double *x, double *r, const double *__restrict__ p, const double *__restrict__ q,
         const Scal *sc, double *partial) {
    if (sc->active == 0) return;
    const double alpha = sc->alpha;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        s = fma(ri, ri, s);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x * 3] = s;
}

__global__ void k_pcg_check(Scal *sc, int remaining) {  // after ||r||^2 in r0
    if (sc->active == 0) return;
    sc->jdone += 1;
    const double rn = sqrt(sc->r0);
    if (!isfinite(rn)) { sc->state = 3; sc->active = 0; return; }
    if (rn <= sc->tolb) { sc->state = 1; sc->active = 0; return; }
    if (sc->jdone >= remaining) sc->active = 0;
}

__global__ void k_pcg_beta(Scal *sc) {  // after (r, z) in r0
    if (sc->active == 0) return;
    const double rho = sc->r0;
    sc->beta_b = rho / sc->rho;
    sc->rho = rho;
}

__global__ void k_pcg_p(int64_t n, const double *__restrict__ z, double *p, const Scal *sc) {
    if (sc->active == 0) return;
    const double beta = sc->beta_b;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        p[i] = z[i] + beta * p[i];
}

__global__ void k_pcg_start(Scal *sc) {  // after (r, z) in r0
    sc->rho = sc->r0;
    sc->active = 1;
    sc->state = 0;
}

// ---- host helpers ---------------------------------------------------------------
struct Work {
    int nb = 1;
    double *partial = nullptr;   // nb x ldp
    double *partial2 = nullptr;  // nb
};

cudaError_t dots(sait_ctx ctx, const Work &W, int64_t n, int nd, const double *x0, const double *y0,
                 const double *x1, const double *y1, const double *x2, const double *y2, double *out,
                 const int *active) {
    launch_k(k_dots, W.nb, kThreads, 0, ctx->stream, n, nd, x0, y0, x1, y1, x2, y2, W.partial, active);
    launch_k(k_reduce, nd, kThreads, 0, ctx->stream, W.partial, W.nb, 3, out, active, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t residual(sait_ctx ctx, sait_mat A, const double *x, const double *b, double *r) {
    const int G = A->lanes;
    const unsigned grid = (unsigned)cdiv(A->n * G, kThreads);
    cudaStream_t s = ctx->stream;
    if (A->n == 0) return cudaSuccess;
    switch (G) {
        case 2: launch_k(k_residual<2>, grid, kThreads, 0, s, A->n, A->rp, A->ci, A->va, x, b, r); break;
        case 4: launch_k(k_residual<4>, grid, kThreads, 0, s, A->n, A->rp, A->ci, A->va, x, b, r); break;
        case 8: launch_k(k_residual<8>, grid, kThreads, 0, s, A->n, A->rp, A->ci, A->va, x, b, r); break;
        case 16: launch_k(k_residual<16>, grid, kThreads, 0, s, A->n, A->rp, A->ci, A->va, x, b, r); break;
        default: launch_k(k_residual<32>, grid, kThreads, 0, s, A->n, A->rp, A->ci, A->va, x, b, r); break;
    }
    return cudaGetLastError();
}

sait_status read_scal(sait_ctx ctx, const Scal *d, Scal *h) {
    SAIT_CK(cudaMemcpyAsync(ctx->h_pinned, d, sizeof(Scal), cudaMemcpyDeviceToHost, ctx->stream));
    SAIT_CK(cudaStreamSynchronize(ctx->stream));
    *h = *(const Scal *)ctx->h_pinned;
    return SAIT_OK;
}

// preconditioned vector z = P v (copy when P is null); `active` gates the kernels
sait_status precondition(sait_ctx ctx, sait_prec P, const double *v, double *z, int64_t n, const int *active) {
    if (P) return prec_apply_impl(ctx, P, v, z, active);
    SAIT_CK(cudaMemcpyAsync(z, v, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    return SAIT_OK;
}

sait_status check_solver_args(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x,
                              double tol, int32_t maxit, const char *who) {
    if (!A || (A->n > 0 && (!b || !x)) || !(tol >= 0.0) || maxit < 0)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, std::string(who) + ": bad argument");
    if (P && P->n != A->n) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, std::string(who) + ": size mismatch");
    return SAIT_OK;
}

}  // namespace

extern "C" sait_status sait_gmres(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x,
                                  int32_t restart, double tol, int32_t maxit, sait_info *info) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    SAIT_TRY(check_solver_args(ctx, A, P, b, x, tol, maxit, "sait_gmres"));
    if (restart < 1 || restart > kMaxRestart)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_gmres: restart must lie in [1, 512]");
    const int64_t n = A->n;
    const int m = restart;
    cudaStream_t s = ctx->stream;
    sait_info inf{0, 0, 0, 0, 0.0};
    if (info) *info = inf;
    if (n == 0) return SAIT_OK;

    Work W;
    W.nb = (int)std::min<int64_t>(cdiv(n, kThreads), 4LL * ctx->num_sms);
    const int ldp = m + 2;
    DTemp<double> V, H, cs, sn, g, y, z, u, part, part2;
    DTemp<float> V32, VL, w32;  // the basis as FP32 (hi, lo) pairs; fl32(w) after pass 1
    DTemp<Scal> scd;
    const int64_t ldv = (n + 3) / 4 * 4, n4 = ldv / 4;  // columns padded to 16-byte vectors
    SAIT_CK(V.alloc((size_t)(m + 1) * ldv, s));
    SAIT_CK(V32.alloc((size_t)(m + 1) * ldv, s));
    SAIT_CK(VL.alloc((size_t)(m + 1) * ldv, s));
    SAIT_CK(w32.alloc((size_t)ldv, s));
    if (ldv > n) {  // the padding rows stay zero for the whole solve
        SAIT_CK(cudaMemset2DAsync(V.p + n, ldv * sizeof(double), 0, (ldv - n) * sizeof(double), m + 1, s));
        SAIT_CK(cudaMemset2DAsync(V32.p + n, ldv * sizeof(float), 0, (ldv - n) * sizeof(float), m + 1, s));
        SAIT_CK(cudaMemset2DAsync(VL.p + n, ldv * sizeof(float), 0, (ldv - n) * sizeof(float), m + 1, s));
        SAIT_CK(cudaMemsetAsync(w32.p + n, 0, (ldv - n) * sizeof(float), s));
    }
    SAIT_CK(H.alloc((size_t)(m + 1) * m, s));
    SAIT_CK(cs.alloc(m, s));
    SAIT_CK(sn.alloc(m, s));
    SAIT_CK(g.alloc(m + 1, s));
    SAIT_CK(y.alloc(m + 2, s));
    SAIT_CK(z.alloc(n, s));
    SAIT_CK(u.alloc(n, s));
    SAIT_CK(part.alloc((size_t)W.nb * std::max(ldp, 3), s));
    const int nb_upd = (int)std::min<int64_t>(cdiv(n4, kThreads), 16LL * ctx->num_sms);
    const int nb_dot = (int)std::min<int64_t>(cdiv(n4, kThreads), (int64_t)W.nb);
    SAIT_CK(part2.alloc((size_t)std::max(W.nb, nb_upd), s));
    SAIT_CK(scd.alloc(1, s));
    SAIT_CK(cudaMemsetAsync(scd.p, 0, sizeof(Scal), s));
    W.partial = part.p;
    W.partial2 = part2.p;
    Scal *sc = scd.p;
    const int *act = &sc->active;
    double *r0 = &sc->r0;

    // ||b||
    SAIT_CK(dots(ctx, W, n, 1, b, b, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
    Scal hs;
    SAIT_TRY(read_scal(ctx, sc, &hs));
    const double bnorm = sqrt(hs.r0);
    if (!std::isfinite(bnorm)) return ctx_fail(ctx, SAIT_ERR_NONFINITE, "sait_gmres: non-finite b");
    if (bnorm == 0.0) {
        SAIT_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        SAIT_CK(cudaStreamSynchronize(s));
        return SAIT_OK;
    }
    const double tolb = tol * bnorm;
    {
        Scal init{};
        init.bnorm = bnorm;
        init.tolb = tolb;
        SAIT_CK(cudaMemcpyAsync(&sc->bnorm, &init.bnorm, sizeof(double), cudaMemcpyHostToDevice, s));
        SAIT_CK(cudaMemcpyAsync(&sc->tolb, &init.tolb, sizeof(double), cudaMemcpyHostToDevice, s));
        SAIT_CK(cudaStreamSynchronize(s));
    }
    const unsigned egrid = (unsigned)std::min<int64_t>(cdiv(n, kThreads), 8LL * ctx->num_sms);
    int iters = 0, cycles = 0;
    // The level-scheduled substitution cannot skip its launches once the
    // cycle has converged, so with an exact-ILU preconditioner poll every step.
    const int poll = (P && P->kind == 2) ? 1 : kPoll;
    sait_status result = SAIT_ERR_NOT_CONVERGED;
    for (;;) {
        // r = b - A x  -> V_0, beta = ||r||
        SAIT_CK(residual(ctx, A, x, b, V.p));
        SAIT_CK(dots(ctx, W, n, 1, V.p, V.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        launch_k(k_gmres_start, 1, 1, 0, s, sc, g.p, m);
        SAIT_CK(cudaGetLastError());
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.rel_resid = hs.beta / bnorm;
        if (!std::isfinite(hs.beta)) { result = SAIT_ERR_NONFINITE; break; }
        if (inf.rel_resid <= tol) { result = SAIT_OK; break; }
        if (iters >= maxit) break;
        launch_k(k_scale3, egrid, kThreads, 0, s, n, (const double *)V.p, V.p, V32.p, VL.p, (const Scal *)sc,
                 nullptr);
        const int remaining = maxit - iters;
        for (int j = 0; j < m; j++) {
            double *vj = V.p + (size_t)j * ldv, *w = V.p + (size_t)(j + 1) * ldv;
            SAIT_TRY(precondition(ctx, P, vj, z.p, n, act));
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, z.p, false, w, false, act, s,
                                    group_counter(ctx, SAIT_TIMER_SPMV)));
            }
            {
                ScopedTimer tm(ctx, SAIT_TIMER_ORTHO);
                double *Hj = H.p + (size_t)j * (m + 1);
                const int nv = j + 1;
                const float4 *Vh4 = (const float4 *)V32.p, *Vl4 = (const float4 *)VL.p;
                // pass 1: FP32 dots, double-float update
                launch_k(k_cgs_dot<double2>, nb_dot, kThreads, 0, s, n4, Vh4, n4, nv, (const double2 *)w,
                         W.partial, ldp, act);
                launch_k(k_reduce, nv, kThreads, 0, s, (const double *)W.partial, nb_dot, ldp, y.p, act, Hj, 1);
                launch_k(k_cgs_update_df, nb_upd, kThreads, 0, s, n4, Vh4, Vl4, n4, nv, (const double *)y.p,
                         (double2 *)w, (float4 *)w32.p, act);
                // pass 2: FP32 dots and update, ||w||^2
                launch_k(k_cgs_dot<float4>, nb_dot, kThreads, 0, s, n4, Vh4, n4, nv, (const float4 *)w32.p,
                         W.partial, ldp, act);
                launch_k(k_reduce, nv, kThreads, 0, s, (const double *)W.partial, nb_dot, ldp, y.p, act, Hj, 0);
                launch_k(k_cgs_update32, nb_upd, kThreads, 0, s, n4, Vh4, n4, nv, (const double *)y.p,
                         (double2 *)w, W.partial2, act);
                launch_k(k_givens, 1, kThreads, 0, s, j, m, remaining, H.p, cs.p, sn.p, g.p, sc,
                         (const double *)W.partial2, nb_upd, group_counter(ctx, SAIT_TIMER_ORTHO));
                launch_k(k_scale3, egrid, kThreads, 0, s, n, (const double *)w, w, V32.p + (size_t)(j + 1) * ldv,
                         VL.p + (size_t)(j + 1) * ldv, (const Scal *)sc, act);
            }
            SAIT_CK(cudaGetLastError());
            if ((j + 1) % poll == 0 || j + 1 == m) {
                SAIT_TRY(read_scal(ctx, sc, &hs));
                if (!hs.active) break;
            }
        }
        SAIT_TRY(read_scal(ctx, sc, &hs));
        iters += hs.jdone;
        cycles++;
        if (hs.state == 3) { result = SAIT_ERR_NONFINITE; break; }
        launch_k(k_hsolve, 1, kThreads, 0, s, H.p, g.p, y.p, m, sc);
        launch_k(k_gemv, egrid, kThreads, 0, s, n, V.p, ldv, 0, &sc->jdone, y.p, u.p, 0, nullptr);
        SAIT_CK(cudaGetLastError());
        SAIT_TRY(precondition(ctx, P, u.p, z.p, n, nullptr));
        launch_k(k_axpy1, egrid, kThreads, 0, s, n, z.p, x);
        SAIT_CK(cudaGetLastError());
        SAIT_TRY(read_scal(ctx, sc, &hs));
        if (hs.state == 2) { result = SAIT_ERR_BREAKDOWN; break; }
    }
    if (result == SAIT_ERR_NOT_CONVERGED || result == SAIT_ERR_BREAKDOWN) {
        SAIT_CK(residual(ctx, A, x, b, z.p));
        SAIT_CK(dots(ctx, W, n, 1, z.p, z.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.rel_resid = sqrt(hs.r0) / bnorm;
    }
    inf.iters = iters;
    inf.cycles = cycles;
    inf.reorth_steps = iters;  // every Arnoldi step takes the two Gram-Schmidt passes
    if (info) *info = inf;
    SAIT_CK(cudaStreamSynchronize(s));
    if (result != SAIT_OK) {
        char buf[160];
        snprintf(buf, sizeof(buf), "sait_gmres: %s after %d steps, relres %.3e", sait_status_string(result),
                 iters, inf.rel_resid);
        return ctx_fail(ctx, result, buf);
    }
    return SAIT_OK;
}

extern "C" sait_status sait_bicgstab(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x,
                                     double tol, int32_t maxit, sait_info *info) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    SAIT_TRY(check_solver_args(ctx, A, P, b, x, tol, maxit, "sait_bicgstab"));
    const int64_t n = A->n;
    cudaStream_t s = ctx->stream;
    sait_info inf{0, 0, 0, 0, 0.0};
    if (info) *info = inf;
    if (n == 0) return SAIT_OK;
    Work W;
    W.nb = (int)std::min<int64_t>(cdiv(n, kThreads), 2LL * ctx->num_sms);
    DTemp<double> r, rh, p, v, ph, sv, sh, t, part;
    DTemp<Scal> scd;
    for (DTemp<double> *d : {&r, &rh, &p, &v, &ph, &sv, &sh, &t}) SAIT_CK(d->alloc(n, s));
    SAIT_CK(part.alloc((size_t)W.nb * 3, s));
    SAIT_CK(scd.alloc(1, s));
    SAIT_CK(cudaMemsetAsync(scd.p, 0, sizeof(Scal), s));
    W.partial = part.p;
    Scal *sc = scd.p;
    const int *act = &sc->active;
    double *r0 = &sc->r0;
    const unsigned egrid = (unsigned)std::min<int64_t>(cdiv(n, kThreads), 8LL * ctx->num_sms);

    SAIT_CK(dots(ctx, W, n, 1, b, b, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
    Scal hs;
    SAIT_TRY(read_scal(ctx, sc, &hs));
    const double bnorm = sqrt(hs.r0);
    if (!std::isfinite(bnorm)) return ctx_fail(ctx, SAIT_ERR_NONFINITE, "sait_bicgstab: non-finite b");
    if (bnorm == 0.0) {
        SAIT_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        SAIT_CK(cudaStreamSynchronize(s));
        return SAIT_OK;
    }
    {
        double tb = tol * bnorm;
        SAIT_CK(cudaMemcpyAsync(&sc->tolb, &tb, sizeof(double), cudaMemcpyHostToDevice, s));
        SAIT_CK(cudaMemcpyAsync(&sc->bnorm, &bnorm, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    int iters = 0, cycles = 0;
    const int poll = (P && P->kind == 2) ? 1 : kPoll;
    sait_status result = SAIT_ERR_NOT_CONVERGED;
    for (;;) {
        // (re)start: r = b - A x, rh = r
        SAIT_CK(residual(ctx, A, x, b, r.p));
        SAIT_CK(dots(ctx, W, n, 1, r.p, r.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.rel_resid = sqrt(hs.r0) / bnorm;
        if (!std::isfinite(inf.rel_resid)) { result = SAIT_ERR_NONFINITE; break; }
        if (inf.rel_resid <= tol) { result = SAIT_OK; break; }
        if (iters >= maxit) break;
        if (cycles > 0 && hs.state == 2) { result = SAIT_ERR_BREAKDOWN; break; }
        SAIT_CK(cudaMemcpyAsync(rh.p, r.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SAIT_CK(cudaMemsetAsync(p.p, 0, n * sizeof(double), s));
        SAIT_CK(cudaMemsetAsync(v.p, 0, n * sizeof(double), s));
        SAIT_CK(cudaMemsetAsync(&sc->jdone, 0, sizeof(int), s));
        launch_k(k_bicg_init, 1, 1, 0, s, sc);
        const int remaining = maxit - iters;
        for (int it = 0; it < remaining; it++) {
            SAIT_CK(dots(ctx, W, n, 1, rh.p, r.p, nullptr, nullptr, nullptr, nullptr, r0, act));
            launch_k(k_bicg_beta, 1, 1, 0, s, sc);
            launch_k(k_bicg_p, egrid, kThreads, 0, s, n, r.p, v.p, p.p, sc);
            SAIT_TRY(precondition(ctx, P, p.p, ph.p, n, act));
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, ph.p, false, v.p, false, act, s,
                                    group_counter(ctx, SAIT_TIMER_SPMV)));
            }
            SAIT_CK(dots(ctx, W, n, 1, rh.p, v.p, nullptr, nullptr, nullptr, nullptr, r0, act));
            launch_k(k_bicg_alpha, 1, 1, 0, s, sc);
            launch_k(k_bicg_s, egrid, kThreads, 0, s, n, r.p, v.p, sv.p, sc);
            SAIT_CK(dots(ctx, W, n, 1, sv.p, sv.p, nullptr, nullptr, nullptr, nullptr, r0, act));
            launch_k(k_bicg_check_s, 1, 1, 0, s, sc);
            launch_k(k_bicg_xhalf, egrid, kThreads, 0, s, n, x, ph.p, sc);
            launch_k(k_bicg_xhalf_done, 1, 1, 0, s, sc);
            SAIT_TRY(precondition(ctx, P, sv.p, sh.p, n, act));
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, sh.p, false, t.p, false, act, s,
                                    group_counter(ctx, SAIT_TIMER_SPMV)));
            }
            SAIT_CK(dots(ctx, W, n, 2, t.p, t.p, t.p, sv.p, nullptr, nullptr, r0, act));
            launch_k(k_bicg_omega, 1, 1, 0, s, sc);
            launch_k(k_bicg_xr, egrid, kThreads, 0, s, n, x, r.p, ph.p, sh.p, sv.p, t.p, sc);
            SAIT_CK(dots(ctx, W, n, 1, r.p, r.p, nullptr, nullptr, nullptr, nullptr, r0, act));
            launch_k(k_bicg_check_r, 1, 1, 0, s, sc, remaining);
            SAIT_CK(cudaGetLastError());
            if ((it + 1) % poll == 0 || it + 1 == remaining) {
                SAIT_TRY(read_scal(ctx, sc, &hs));
                if (!hs.active) break;
            }
        }
        SAIT_TRY(read_scal(ctx, sc, &hs));
        iters += hs.jdone;
        cycles++;
        if (hs.state == 3) { result = SAIT_ERR_NONFINITE; break; }
    }
    if (result != SAIT_OK) {
        SAIT_CK(residual(ctx, A, x, b, r.p));
        SAIT_CK(dots(ctx, W, n, 1, r.p, r.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.rel_resid = sqrt(hs.r0) / bnorm;
    }
    inf.iters = iters;
    inf.cycles = cycles;
    if (info) *info = inf;
    SAIT_CK(cudaStreamSynchronize(s));
    if (result != SAIT_OK) {
        char buf[160];
        snprintf(buf, sizeof(buf), "sait_bicgstab: %s after %d iterations, relres %.3e",
                 sait_status_string(result), iters, inf.rel_resid);
        return ctx_fail(ctx, result, buf);
    }
    return SAIT_OK;
}

extern "C" sait_status sait_pcg(sait_ctx ctx, sait_mat A, sait_prec P, const double *b, double *x, double tol,
                                int32_t maxit, sait_info *info) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    SAIT_TRY(check_solver_args(ctx, A, P, b, x, tol, maxit, "sait_pcg"));
    const int64_t n = A->n;
    cudaStream_t s = ctx->stream;
    sait_info inf{0, 0, 0, 0, 0.0};
    if (info) *info = inf;
    if (n == 0) return SAIT_OK;
    Work W;
    W.nb = (int)std::min<int64_t>(cdiv(n, kThreads), 2LL * ctx->num_sms);
    DTemp<double> r, z, p, q, part;
    DTemp<Scal> scd;
    for (DTemp<double> *d : {&r, &z, &p, &q}) SAIT_CK(d->alloc(n, s));
    SAIT_CK(part.alloc((size_t)W.nb * 3, s));
    SAIT_CK(scd.alloc(1, s));
    SAIT_CK(cudaMemsetAsync(scd.p, 0, sizeof(Scal), s));
    W.partial = part.p;
    Scal *sc = scd.p;
    const int *act = &sc->active;
    double *r0 = &sc->r0;
    const unsigned egrid = (unsigned)std::min<int64_t>(cdiv(n, kThreads), 8LL * ctx->num_sms);
    SAIT_CK(dots(ctx, W, n, 1, b, b, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
    Scal hs;
    SAIT_TRY(read_scal(ctx, sc, &hs));
    const double bnorm = sqrt(hs.r0);
    if (!std::isfinite(bnorm)) return ctx_fail(ctx, SAIT_ERR_NONFINITE, "sait_pcg: non-finite b");
    if (bnorm == 0.0) {
        SAIT_CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        SAIT_CK(cudaStreamSynchronize(s));
        return SAIT_OK;
    }
    const double tb = tol * bnorm;
    SAIT_CK(cudaMemcpyAsync(&sc->tolb, &tb, sizeof(double), cudaMemcpyHostToDevice, s));
    SAIT_CK(residual(ctx, A, x, b, r.p));
    SAIT_CK(dots(ctx, W, n, 1, r.p, r.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
    SAIT_TRY(read_scal(ctx, sc, &hs));
    inf.rel_resid = sqrt(hs.r0) / bnorm;
    sait_status result = SAIT_ERR_NOT_CONVERGED;
    if (inf.rel_resid <= tol) {
        result = SAIT_OK;
    } else {
        SAIT_TRY(precondition(ctx, P, r.p, z.p, n, nullptr));
        SAIT_CK(cudaMemcpyAsync(p.p, z.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SAIT_CK(dots(ctx, W, n, 1, r.p, z.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        launch_k(k_pcg_start, 1, 1, 0, s, sc);
        const int poll = (P && P->kind == 2) ? 1 : kPoll;
        for (int it = 0; it < maxit; it++) {
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, p.p, false, q.p, false, act, s, group_counter(ctx, SAIT_TIMER_SPMV)));
            }
            SAIT_CK(dots(ctx, W, n, 1, p.p, q.p, nullptr, nullptr, nullptr, nullptr, r0, act));
            launch_k(k_pcg_alpha, 1, 1, 0, s, sc);
            launch_k(k_pcg_xr, (unsigned)W.nb, kThreads, 0, s, n, x, r.p, (const double *)p.p, (const double *)q.p,
                     (const Scal *)sc, W.partial);
            launch_k(k_reduce, 1, kThreads, 0, s, (const double *)W.partial, W.nb, 3, r0, act, nullptr, 0);
            launch_k(k_pcg_check, 1, 1, 0, s, sc, (int)maxit);
            SAIT_TRY(precondition(ctx, P, r.p, z.p, n, act));
            SAIT_CK(dots(ctx, W, n, 1, r.p, z.p, nullptr, nullptr, nullptr, nullptr, r0, act));
            launch_k(k_pcg_beta, 1, 1, 0, s, sc);
            launch_k(k_pcg_p, egrid, kThreads, 0, s, n, (const double *)z.p, p.p, (const Scal *)sc);
            SAIT_CK(cudaGetLastError());
            if ((it + 1) % poll == 0 || it + 1 == maxit) {
                SAIT_TRY(read_scal(ctx, sc, &hs));
                if (!hs.active) break;
            }
        }
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.iters = hs.jdone;
        if (hs.state == 1) result = SAIT_OK;
        else if (hs.state == 2) result = SAIT_ERR_BREAKDOWN;
        else if (hs.state == 3) result = SAIT_ERR_NONFINITE;
        // true residual at exit
        SAIT_CK(residual(ctx, A, x, b, r.p));
        SAIT_CK(dots(ctx, W, n, 1, r.p, r.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.rel_resid = sqrt(hs.r0) / bnorm;
    }
    inf.cycles = 1;
    if (info) *info = inf;
    SAIT_CK(cudaStreamSynchronize(s));
    if (result != SAIT_OK) {
        char buf[160];
        snprintf(buf, sizeof(buf), "sait_pcg: %s after %d iterations, relres %.3e", sait_status_string(result),
                 inf.iters, inf.rel_resid);
        return ctx_fail(ctx, result, buf);
    }
    return SAIT_OK;
}
