// Batched SAIT-preconditioned BiCGSTAB.
//
// (1) Many independent systems, given as one block-diagonal matrix whose
//     block s spans rows sys_ptr[s] .. sys_ptr[s+1].  ILU(0), SAIT and the
//     apply of a block-diagonal matrix are block-diagonal, so the factors,
//     the SAIT matrices and every product are single launches over all
//     systems.  Each system has its own BiCGSTAB scalars, convergence test
//     and iteration count; reductions run over a tile schedule whose tiles
//     never cross a system boundary, so every per-system sum has a fixed
//     order.  Converged systems freeze (their updates are masked).
// (2) Many right-hand sides of one matrix (X, B row-major n x k): the same
//     recurrences with per-column scalars; the products are block products,
//     so every matrix entry is read once per iteration for all k columns.
//
// kPollB iterations of either solver, with the count of the systems still
// active, are captured once as the body of a WHILE conditional graph node:
// one graph launch per restart round runs the iterations on the device until
// the count is zero (or the iteration limit is reached).  Where conditional
// nodes are unavailable the body is captured as a plain graph and replayed
// from the host until the count, read after each replay, is zero.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int kT = 256;        // threads per block
constexpr int kPollB = 8;      // iterations replayed between status reads

// per-system state (structure of arrays)
struct BState {
    double *rho, *rho_old, *alpha, *omega, *beta, *tolb, *bnorm, *rmin;  // rmin: smallest ||r|| so far
    double *red;                                                          // nsys x 3 reduction results
    int *active, *state, *iters;  // state: 0 run, 1 converged, 2 breakdown, 3 non-finite, 4 half step,
                                  // 5 residual grew 1e4 x above its minimum: restart the recurrence
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; w++) r += ws[w];
    __syncthreads();
    return r;
}

// ---- tile schedule ------------------------------------------------------------
__global__ void k_tile_count(int nsys, const int64_t *__restrict__ sys_ptr, int64_t tile, int32_t *cnt, int *err) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const int64_t len = sys_ptr[s + 1] - sys_ptr[s];
    if (len < 0) atomicOr(err, 1);
    cnt[s] = len > 0 ? (int32_t)cdiv(len, tile) : 0;
}

// tiles[t] = (system, first row, end row)
__global__ void k_tile_fill(int nsys, const int64_t *__restrict__ sys_ptr, int64_t tile,
                            const int64_t *__restrict__ tptr, int32_t *tsys, int64_t *tbeg, int64_t *tend) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    int64_t t = tptr[s];
    for (int64_t r = sys_ptr[s]; r < sys_ptr[s + 1]; r += tile, t++) {
        tsys[t] = s;
        tbeg[t] = r;
        tend[t] = min(r + tile, sys_ptr[s + 1]);
    }
}

// partial[t*3 + q] = sum over tile t of xq . yq (q < nd), for active systems
__global__ void __launch_bounds__(kT)
k_bt_dots(const int32_t *__restrict__ tsys, const int64_t *__restrict__ tbeg, const int64_t *__restrict__ tend,
          const int *__restrict__ active, int nd, const double *x0, const double *y0, const double *x1,
          const double *y1, const double *x2, const double *y2, double *partial) {
    const int t = blockIdx.x;
    if (active && !active[tsys[t]]) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t i = tbeg[t] + threadIdx.x; i < tend[t]; i += kT) {
        s0 = fma(x0[i], y0[i], s0);
        if (nd > 1) s1 = fma(x1[i], y1[i], s1);
        if (nd > 2) s2 = fma(x2[i], y2[i], s2);
    }
    s0 = block_sum(s0);
    if (nd > 1) s1 = block_sum(s1);
    if (nd > 2) s2 = block_sum(s2);
    if (threadIdx.x == 0) {
        partial[t * 3 + 0] = s0;
        partial[t * 3 + 1] = s1;
        partial[t * 3 + 2] = s2;
    }
}

// red[s*3 + q] = sum of the tile partials of system s, in tile order
__global__ void k_bt_reduce(int nsys, const int64_t *__restrict__ tptr, const int *__restrict__ active, int nd,
                            const double *__restrict__ partial, double *red) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || (active && !active[s])) return;
    for (int q = 0; q < nd; q++) {
        double acc = 0.0;
        for (int64_t t = tptr[s]; t < tptr[s + 1]; t++) acc += partial[t * 3 + q];
        red[s * 3 + q] = acc;
    }
}

// ---- per-system scalar steps (one thread per system) --------------------------
__global__ void k_b_start(int nsys, BState st, double tol) {  // red[.,0] = ||b||^2, red[.,1] = ||r||^2
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double bn = sqrt(st.red[s * 3]), rn = sqrt(st.red[s * 3 + 1]);
    st.bnorm[s] = bn;
    st.tolb[s] = tol * bn;
    st.rmin[s] = rn;
    st.rho_old[s] = st.alpha[s] = st.omega[s] = 1.0;
    st.iters[s] = 0;
    const bool done = bn == 0.0 || rn <= tol * bn;
    st.state[s] = done ? 1 : (isfinite(rn) ? 0 : 3);
    st.active[s] = (!done && isfinite(rn)) ? 1 : 0;
}

__global__ void k_b_beta(int nsys, BState st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !st.active[s]) return;
    const double rho = st.red[s * 3];
    st.rho[s] = rho;
    if (rho == 0.0 || st.omega[s] == 0.0 || !isfinite(rho)) {
        st.state[s] = isfinite(rho) ? 2 : 3;
        st.active[s] = 0;
        return;
    }
    st.beta[s] = (rho / st.rho_old[s]) * (st.alpha[s] / st.omega[s]);
}

__global__ void k_b_alpha(int nsys, BState st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !st.active[s]) return;
    const double rv = st.red[s * 3];
    if (rv == 0.0 || !isfinite(rv)) {
        st.state[s] = isfinite(rv) ? 2 : 3;
        st.active[s] = 0;
        return;
    }
    st.alpha[s] = st.rho[s] / rv;
}

__global__ void k_b_check_s(int nsys, BState st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !st.active[s]) return;
    st.iters[s] += 1;
    const double sn = sqrt(st.red[s * 3]);
    if (!isfinite(sn)) { st.state[s] = 3; st.active[s] = 0; return; }
    if (sn <= st.tolb[s]) { st.state[s] = 4; st.active[s] = 0; }
}

__global__ void k_b_half_done(int nsys, BState st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys && st.state[s] == 4) st.state[s] = 1;
}

__global__ void k_b_omega(int nsys, BState st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !st.active[s]) return;
    const double tt = st.red[s * 3];
    st.omega[s] = tt == 0.0 ? 0.0 : st.red[s * 3 + 1] / tt;
}

__global__ void k_b_check_r(int nsys, BState st, int maxit) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !st.active[s]) return;
    st.rho_old[s] = st.rho[s];
    const double rn = sqrt(st.red[s * 3]);
    if (!isfinite(rn)) { st.state[s] = 3; st.active[s] = 0; return; }
    if (rn <= st.tolb[s]) { st.state[s] = 1; st.active[s] = 0; return; }
    if (st.iters[s] >= maxit) { st.active[s] = 0; return; }
    // divergence guard: restart from the current iterate once the residual has
    // grown four orders of magnitude above the best seen in this recurrence
    if (rn > 1e4 * st.rmin[s]) { st.state[s] = 5; st.active[s] = 0; return; }
    st.rmin[s] = fmin(st.rmin[s], rn);
}

__global__ void k_b_count(int nsys, const int *__restrict__ active, int *count) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int a = s < nsys ? active[s] : 0;
    a = __reduce_add_sync(0xffffffffu, a);
    if ((threadIdx.x & 31) == 0 && a) atomicAdd(count, a);
}

// ---- per-tile vector updates ---------------------------------------------------
__global__ void k_bt_p(const int32_t *__restrict__ tsys, const int64_t *__restrict__ tbeg,
                       const int64_t *__restrict__ tend, BState st, const double *__restrict__ r,
                       const double *__restrict__ v, double *p) {
    const int t = blockIdx.x, s = tsys[t];
    if (!st.active[s]) return;
    const double beta = st.beta[s], omega = st.omega[s];
    for (int64_t i = tbeg[t] + threadIdx.x; i < tend[t]; i += kT) p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

__global__ void k_bt_s(const int32_t *__restrict__ tsys, const int64_t *__restrict__ tbeg,
                       const int64_t *__restrict__ tend, BState st, const double *__restrict__ r,
                       const double *__restrict__ v, double *sv) {
    const int t = blockIdx.x, s = tsys[t];
    if (!st.active[s]) return;
    const double alpha = st.alpha[s];
    for (int64_t i = tbeg[t] + threadIdx.x; i < tend[t]; i += kT) sv[i] = r[i] - alpha * v[i];
}

__global__ void k_bt_xhalf(const int32_t *__restrict__ tsys, const int64_t *__restrict__ tbeg,
                           const int64_t *__restrict__ tend, BState st, const double *__restrict__ ph, double *x) {
    const int t = blockIdx.x, s = tsys[t];
    if (st.state[s] != 4) return;
    const double alpha = st.alpha[s];
    for (int64_t i = tbeg[t] + threadIdx.x; i < tend[t]; i += kT) x[i] += alpha * ph[i];
}

__global__ void k_bt_xr(const int32_t *__restrict__ tsys, const int64_t *__restrict__ tbeg,
                        const int64_t *__restrict__ tend, BState st, const double *__restrict__ ph,
                        const double *__restrict__ sh, const double *__restrict__ sv, const double *__restrict__ tv,
                        double *x, double *r) {
    const int t = blockIdx.x, s = tsys[t];
    if (!st.active[s]) return;
    const double alpha = st.alpha[s], omega = st.omega[s];
    for (int64_t i = tbeg[t] + threadIdx.x; i < tend[t]; i += kT) {
        x[i] += alpha * ph[i] + omega * sh[i];
        r[i] = sv[i] - omega * tv[i];
    }
}

// r = b - A x over all rows (block-diagonal A), FP64
__global__ void k_b_residual(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ va, const double *__restrict__ x,
                             const double *__restrict__ b, double *r) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int lane = threadIdx.x & 7;
    double s = 0.0;
    if (row < n)
        for (int k = rp[row] + lane; k < rp[row + 1]; k += 8) s = fma(va[k], x[ci[k]], s);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && lane == 0) r[row] = b[row] - s;
}

__global__ void k_b_relres(int nsys, const double *__restrict__ red, const double *__restrict__ bnorm, double *out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double bn = bnorm[s];
    out[s] = bn > 0.0 ? sqrt(red[s * 3]) / bn : 0.0;
}

// reactivate systems whose true residual is above the tolerance (recurrence restart)
__global__ void k_b_restart(int nsys, BState st, const double *__restrict__ relres, double tol, int maxit) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    if ((st.state[s] == 5 || (st.state[s] == 1 && relres[s] > tol)) && st.iters[s] < maxit) {
        st.state[s] = 0;
        st.active[s] = 1;
        st.rho_old[s] = st.alpha[s] = st.omega[s] = 1.0;
        st.rmin[s] = relres[s] * st.bnorm[s];
    } else {
        st.active[s] = 0;
    }
}

// copy r -> rh and zero p, v for active (restarted) systems
__global__ void k_bt_reset(const int32_t *__restrict__ tsys, const int64_t *__restrict__ tbeg,
                           const int64_t *__restrict__ tend, const int *__restrict__ active,
                           const double *__restrict__ r, double *rh, double *p, double *v) {
    const int t = blockIdx.x;
    if (!active[tsys[t]]) return;
    for (int64_t i = tbeg[t] + threadIdx.x; i < tend[t]; i += kT) {
        rh[i] = r[i];
        p[i] = 0.0;
        v[i] = 0.0;
    }
}

// ---- multi right-hand sides: per-column reductions over a row-major block ------
// partial[b*k*3 + q*k + c] = sum over this block's rows of Xq[i, c] Yq[i, c]
__global__ void __launch_bounds__(kT)
k_mc_dots(int64_t n, int k, int nd, const int *__restrict__ active, const double *x0, const double *y0,
          const double *x1, const double *y1, double *partial) {
    // thread (c = tid % k) accumulates column c over rows tid / k, stepping by the block's row count
    __shared__ double red[2][kT];
    const int c = threadIdx.x % k;
    const int rows_per_pass = kT / k;
    const int r0 = threadIdx.x / k;
    double s0 = 0.0, s1 = 0.0;
    const bool on = (int)threadIdx.x < rows_per_pass * k && (!active || active[c]);
    if (on) {
        // four rows per trip, all loads issued before the multiply-adds
        const int64_t step = (int64_t)gridDim.x * rows_per_pass;
        int64_t i = (int64_t)blockIdx.x * rows_per_pass + r0;
        for (; i + 3 * step < n; i += 4 * step) {
            double a[4], b[4], u[4], v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int64_t e = (i + q * step) * k + c;
                a[q] = x0[e];
                b[q] = y0[e];
                if (nd > 1) {
                    u[q] = x1[e];
                    v[q] = y1[e];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                s0 = fma(a[q], b[q], s0);
                if (nd > 1) s1 = fma(u[q], v[q], s1);
            }
        }
        for (; i < n; i += step) {
            const int64_t e = i * k + c;
            s0 = fma(x0[e], y0[e], s0);
            if (nd > 1) s1 = fma(x1[e], y1[e], s1);
        }
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    if ((int)threadIdx.x < k) {
        for (int q = 0; q < nd; q++) {
            double acc = 0.0;
            for (int rr = 0; rr < rows_per_pass; rr++) acc += red[q][rr * k + threadIdx.x];
            partial[(int64_t)blockIdx.x * k * 3 + q * k + threadIdx.x] = acc;
        }
    }
}

// red[c*3 + q] = sum_b partial[b*k*3 + q*k + c]: one block per column c, the
// block's threads each add a stride of the partials, then a tree (fixed
// order; a serial FP64 sum over the blocks would cost 64 cycles per partial).
__global__ void __launch_bounds__(kT)
k_mc_reduce(int k, int nb, int nd, const int *__restrict__ active, const double *__restrict__ partial,
            double *red) {
    const int c = blockIdx.x;
    if (active && !active[c]) return;
    for (int q = 0; q < nd; q++) {
        double a0 = 0.0, a1 = 0.0;
        int b = threadIdx.x;
        for (; b + kT < nb; b += 2 * kT) {
            a0 += partial[(int64_t)b * k * 3 + q * k + c];
            a1 += partial[(int64_t)(b + kT) * k * 3 + q * k + c];
        }
        if (b < nb) a0 += partial[(int64_t)b * k * 3 + q * k + c];
        const double t = block_sum(a0 + a1);
        if (threadIdx.x == 0) red[c * 3 + q] = t;
    }
}

// Vector updates of the many-right-hand-side recurrences, n x k row-major:
// thread (c = tid % k) handles column c over rows tid / k, stepping by the
// grid's row count, so its column's scalars are read once.
template <int OP>
__global__ void __launch_bounds__(kT)
k_mc_update(int64_t n, int k, BState st, const double *__restrict__ a, const double *__restrict__ b,
            const double *__restrict__ c2, const double *__restrict__ d, double *o1, double *o2) {
    const int c = threadIdx.x % k;
    const int rows_per_pass = kT / k;
    if ((int)threadIdx.x >= rows_per_pass * k) return;
    if (OP == 3 ? st.state[c] != 4 : !st.active[c]) return;
    const double alpha = st.alpha[c], beta = st.beta[c], omega = st.omega[c];
    for (int64_t i = (int64_t)blockIdx.x * rows_per_pass + threadIdx.x / k; i < n;
         i += (int64_t)gridDim.x * rows_per_pass) {
        const int64_t e = i * k + c;
        if (OP == 0) o1[e] = a[e] + beta * (o1[e] - omega * b[e]);       // p = r + beta (p - omega v)
        else if (OP == 1) o1[e] = a[e] - alpha * b[e];                    // s = r - alpha v
        else if (OP == 2) {                                               // x, r update
            o1[e] += alpha * a[e] + omega * b[e];
            o2[e] = c2[e] - omega * d[e];
        } else if (OP == 3) {                                             // half step: x += alpha ph
            o1[e] += alpha * a[e];
        } else if (OP == 4) {                                             // reset rh, p, v
            o1[e] = a[e];
            o2[e] = 0.0;
            ((double *)c2)[e] = 0.0;
        }
    }
}

// R = B - A X for a row-major block
__global__ void k_mc_residual(int64_t n, int k, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ va, const double *__restrict__ X, const double *__restrict__ B,
                              double *R) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e % k);
        double s = 0.0;
        for (int q = rp[i]; q < rp[i + 1]; q++) s = fma(va[q], X[(int64_t)ci[q] * k + c], s);
        R[e] = B[e] - s;
    }
}

struct Buffers {
    DTemp<double> r, rh, p, v, ph, sv, sh, t, partial, red, relres;
    DTemp<double> sc;  // 8 arrays of nsys doubles
    DTemp<int> si;     // 3 arrays of nsys ints
};

BState make_state(Buffers &B, int nsys) {
    BState st;
    double *d = B.sc.p;
    st.rho = d; st.rho_old = d + nsys; st.alpha = d + 2 * nsys; st.omega = d + 3 * nsys;
    st.beta = d + 4 * nsys; st.tolb = d + 5 * nsys; st.bnorm = d + 6 * nsys; st.rmin = d + 7 * nsys;
    st.red = B.red.p;
    st.active = B.si.p; st.state = B.si.p + nsys; st.iters = B.si.p + 2 * nsys;
    return st;
}

// launch an iteration's kernel sequence once under stream capture and return the
// executable graph; the number of kernels it holds goes to *kernels
template <class F>
sait_status capture(sait_ctx ctx, cudaStream_t cs, F body, cudaGraphExec_t *exec, int64_t *kernels) {
    const bool timing = ctx->timing;
    ctx->timing = false;  // no event records inside the graph
    const int64_t l0 = g_sait_launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sait_status st = SAIT_OK;
    if (e == cudaSuccess) {
        st = body(cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e2 != cudaSuccess && e == cudaSuccess) e = e2;
    }
    ctx->timing = timing;
    *kernels = g_sait_launches - l0;
    g_sait_launches = l0;
    if (e == cudaSuccess && st == SAIT_OK) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != SAIT_OK) return st;
    if (e != cudaSuccess) return ctx_cuda(ctx, e, "batched BiCGSTAB graph capture", __FILE__, __LINE__);
    return SAIT_OK;
}

// Ends one pass of the loop body: counts the pass and lets the loop go on
// while some system is active and fewer than max_bodies passes have run, so
// the device loop ends after at most max_bodies passes whatever the flags say.
__global__ void k_b_continue(cudaGraphConditionalHandle h, const int *__restrict__ count, int *bodies,
                             int max_bodies) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int b = *bodies + 1;
        *bodies = b;
        cudaGraphSetConditional(h, (*count > 0 && b < max_bodies) ? 1u : 0u);
    }
}

// The same body (kPollB iterations and the count of active systems) as the
// inside of a WHILE conditional node, followed by k_b_continue: one launch of
// the executable graph runs the iterations on the device until the systems
// stop or max_bodies passes have run, with no host round trip per pass.  Any
// failure (no conditional nodes) leaves *exec null so that the caller falls
// back to replaying the body graph from the host.
template <class F>
sait_status capture_loop(sait_ctx ctx, cudaStream_t cs, F body, const int *count, int *bodies, int max_bodies,
                         cudaGraphExec_t *exec, int64_t *kernels) {
    *exec = nullptr;
    const bool timing = ctx->timing;
    ctx->timing = false;
    const int64_t l0 = g_sait_launches;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    sait_status st = SAIT_OK;
    if (e == cudaSuccess) {
        cudaGraph_t inner = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = body(cs);
            launch_k(k_b_continue, 1, 32, 0, cs, h, count, bodies, max_bodies);
            cudaError_t e2 = cudaStreamEndCapture(cs, &inner);
            if (e == cudaSuccess) e = e2;
        }
    }
    ctx->timing = timing;
    *kernels = g_sait_launches - l0;
    g_sait_launches = l0;
    if (e == cudaSuccess && st == SAIT_OK) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != SAIT_OK) return st;
    if (e != cudaSuccess) {
        *exec = nullptr;
        cudaGetLastError();  // fall back to host replays
    }
    return SAIT_OK;
}

// Runs the iterations of one restart round: the device loop when there is
// one, else the body graph replayed from the host with a status read after
// each replay.  *iterations grows by kPollB per pass of the body.
sait_status run_iterations(sait_ctx ctx, cudaStream_t cs, cudaGraphExec_t loop, cudaGraphExec_t poll,
                           int64_t loop_kernels, int64_t poll_kernels, int maxit, int *count, int *bodies,
                           int *h, int *iterations, int *launches) {
    if (maxit <= 0) return SAIT_OK;
    if (loop) {
        SAIT_CK(cudaMemsetAsync(bodies, 0, sizeof(int), cs));
        SAIT_CK(cudaGraphLaunch(loop, cs));
        ++*launches;
        SAIT_CK(cudaMemcpyAsync(h, bodies, sizeof(int), cudaMemcpyDeviceToHost, cs));
        SAIT_CK(cudaStreamSynchronize(cs));
        g_sait_launches += loop_kernels * h[0];
        *iterations += kPollB * h[0];
        return SAIT_OK;
    }
    for (int it = 0; it < maxit; it += kPollB) {
        SAIT_CK(cudaGraphLaunch(poll, cs));
        ++*launches;
        g_sait_launches += poll_kernels;
        SAIT_CK(cudaMemcpyAsync(h, count, sizeof(int), cudaMemcpyDeviceToHost, cs));
        SAIT_CK(cudaStreamSynchronize(cs));
        *iterations += kPollB;
        if (h[0] == 0) break;
    }
    return SAIT_OK;
}

sait_status sync_streams(sait_ctx ctx, cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
    SAIT_CK(cudaEventRecord(ev, from));
    SAIT_CK(cudaStreamWaitEvent(to, ev, 0));
    return SAIT_OK;
}

}  // namespace

extern "C" sait_status sait_bicgstab_batched(sait_ctx ctx, sait_mat A, sait_prec P, int32_t nsys,
                                             const int64_t *sys_ptr, const double *b, double *x, double tol,
                                             int32_t maxit, sait_batch_info *info, double *rel_resid,
                                             int32_t *iters) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || nsys < 1 || !sys_ptr || !b || !x || !(tol >= 0.0) || maxit < 0 || (P && P->kind != 1) ||
        (P && P->n != A->n))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_bicgstab_batched: bad argument (P must be a SAIT pair)");
    const int64_t n = A->n;
    cudaStream_t s0 = ctx->stream;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    SAIT_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    SAIT_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    struct Cleanup {
        cudaStream_t cs;
        cudaEvent_t ev;
        cudaGraphExec_t g = nullptr, loop = nullptr;
        ~Cleanup() {
            cudaStreamSynchronize(cs);
            if (g) cudaGraphExecDestroy(g);
            if (loop) cudaGraphExecDestroy(loop);
            cudaEventDestroy(ev);
            cudaStreamDestroy(cs);
        }
    } cleanup{cs, ev};
    int *h = (int *)ctx->h_pinned;
    // tile schedule
    DTemp<int32_t> tcnt, tsys;
    DTemp<int64_t> tptr, tbeg, tend;
    SAIT_CK(tcnt.alloc(nsys, s0));
    SAIT_CK(tptr.alloc(nsys + 1, s0));
    SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), s0));
    const int64_t tile = ctx->batch_tile;
    launch_k(k_tile_count, (unsigned)cdiv(nsys, 256), 256, 0, s0, (int)nsys, sys_ptr, tile, tcnt.p, ctx->d_word);
    SAIT_CK(scan_i32(tcnt.p, tptr.p, nsys, s0));
    int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
    SAIT_CK(cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s0));
    SAIT_CK(cudaMemcpyAsync(h64, tptr.p + nsys, sizeof(int64_t), cudaMemcpyDeviceToHost, s0));
    SAIT_CK(cudaMemcpyAsync(h64 + 1, sys_ptr + nsys, sizeof(int64_t), cudaMemcpyDeviceToHost, s0));
    SAIT_CK(cudaMemcpyAsync(h64 + 2, sys_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s0));
    SAIT_CK(cudaStreamSynchronize(s0));
    const int64_t ntiles = h64[0];
    if (h64[1] != n || h64[2] != 0 || h[0] != 0)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG,
                        "sait_bicgstab_batched: sys_ptr must be non-decreasing from 0 to n");
    SAIT_CK(tsys.alloc(ntiles, s0));
    SAIT_CK(tbeg.alloc(ntiles, s0));
    SAIT_CK(tend.alloc(ntiles, s0));
    launch_k(k_tile_fill, (unsigned)cdiv(nsys, 256), 256, 0, s0, (int)nsys, sys_ptr, tile, (const int64_t *)tptr.p,
             tsys.p, tbeg.p, tend.p);
    Buffers B;
    for (DTemp<double> *d : {&B.r, &B.rh, &B.p, &B.v, &B.ph, &B.sv, &B.sh, &B.t}) SAIT_CK(d->alloc(n, s0));
    SAIT_CK(B.partial.alloc((size_t)ntiles * 3, s0));
    SAIT_CK(B.red.alloc((size_t)nsys * 3, s0));
    SAIT_CK(B.relres.alloc(nsys, s0));
    SAIT_CK(B.sc.alloc((size_t)nsys * 8, s0));
    SAIT_CK(B.si.alloc((size_t)nsys * 3, s0));
    SAIT_CK(cudaMemsetAsync(B.p.p, 0, n * sizeof(double), s0));
    SAIT_CK(cudaMemsetAsync(B.v.p, 0, n * sizeof(double), s0));
    BState st = make_state(B, nsys);
    const unsigned gt = (unsigned)ntiles, gs = (unsigned)cdiv(nsys, 256);
    const int32_t *TS = tsys.p;
    const int64_t *TB = tbeg.p, *TE = tend.p, *TP = tptr.p;
    // start: ||b||, r = b - A x, ||r||
    launch_k(k_b_residual, (unsigned)cdiv(n * 8, 256), 256, 0, s0, n, (const int32_t *)A->rp,
             (const int32_t *)A->ci, (const double *)A->va, (const double *)x, b, B.r.p);
    launch_k(k_bt_dots, gt, kT, 0, s0, TS, TB, TE, (const int *)nullptr, 2, b, b, (const double *)B.r.p,
             (const double *)B.r.p, (const double *)nullptr, (const double *)nullptr, B.partial.p);
    launch_k(k_bt_reduce, gs, 256, 0, s0, (int)nsys, TP, (const int *)nullptr, 2, (const double *)B.partial.p, B.red.p);
    launch_k(k_b_start, gs, 256, 0, s0, (int)nsys, st, tol);
    launch_k(k_bt_reset, gt, kT, 0, s0, TS, TB, TE, (const int *)st.active, (const double *)B.r.p, B.rh.p, B.p.p,
             B.v.p);
    SAIT_CK(cudaGetLastError());

    auto iteration = [&](cudaStream_t q) -> sait_status {
        const int *act = st.active;
        launch_k(k_bt_dots, gt, kT, 0, q, TS, TB, TE, act, 1, (const double *)B.rh.p, (const double *)B.r.p,
                 (const double *)nullptr, (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                 B.partial.p);
        launch_k(k_bt_reduce, gs, 256, 0, q, (int)nsys, TP, act, 1, (const double *)B.partial.p, B.red.p);
        launch_k(k_b_beta, gs, 256, 0, q, (int)nsys, st);
        launch_k(k_bt_p, gt, kT, 0, q, TS, TB, TE, st, (const double *)B.r.p, (const double *)B.v.p, B.p.p);
        cudaStream_t keep = ctx->stream;
        ctx->stream = q;
        sait_status s1 = P ? prec_apply_impl(ctx, P, B.p.p, B.ph.p, nullptr) : SAIT_OK;
        if (!P) cudaMemcpyAsync(B.ph.p, B.p.p, n * sizeof(double), cudaMemcpyDeviceToDevice, q);
        ctx->stream = keep;
        if (s1 != SAIT_OK) return s1;
        SAIT_CK(launch_spmv(A, SAIT_F64, B.ph.p, false, B.v.p, false, nullptr, q));
        launch_k(k_bt_dots, gt, kT, 0, q, TS, TB, TE, act, 1, (const double *)B.rh.p, (const double *)B.v.p,
                 (const double *)nullptr, (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                 B.partial.p);
        launch_k(k_bt_reduce, gs, 256, 0, q, (int)nsys, TP, act, 1, (const double *)B.partial.p, B.red.p);
        launch_k(k_b_alpha, gs, 256, 0, q, (int)nsys, st);
        launch_k(k_bt_s, gt, kT, 0, q, TS, TB, TE, st, (const double *)B.r.p, (const double *)B.v.p, B.sv.p);
        launch_k(k_bt_dots, gt, kT, 0, q, TS, TB, TE, act, 1, (const double *)B.sv.p, (const double *)B.sv.p,
                 (const double *)nullptr, (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                 B.partial.p);
        launch_k(k_bt_reduce, gs, 256, 0, q, (int)nsys, TP, act, 1, (const double *)B.partial.p, B.red.p);
        launch_k(k_b_check_s, gs, 256, 0, q, (int)nsys, st);
        launch_k(k_bt_xhalf, gt, kT, 0, q, TS, TB, TE, st, (const double *)B.ph.p, x);
        launch_k(k_b_half_done, gs, 256, 0, q, (int)nsys, st);
        ctx->stream = q;
        s1 = P ? prec_apply_impl(ctx, P, B.sv.p, B.sh.p, nullptr) : SAIT_OK;
        if (!P) cudaMemcpyAsync(B.sh.p, B.sv.p, n * sizeof(double), cudaMemcpyDeviceToDevice, q);
        ctx->stream = keep;
        if (s1 != SAIT_OK) return s1;
        SAIT_CK(launch_spmv(A, SAIT_F64, B.sh.p, false, B.t.p, false, nullptr, q));
        launch_k(k_bt_dots, gt, kT, 0, q, TS, TB, TE, act, 2, (const double *)B.t.p, (const double *)B.t.p,
                 (const double *)B.t.p, (const double *)B.sv.p, (const double *)nullptr, (const double *)nullptr,
                 B.partial.p);
        launch_k(k_bt_reduce, gs, 256, 0, q, (int)nsys, TP, act, 2, (const double *)B.partial.p, B.red.p);
        launch_k(k_b_omega, gs, 256, 0, q, (int)nsys, st);
        launch_k(k_bt_xr, gt, kT, 0, q, TS, TB, TE, st, (const double *)B.ph.p, (const double *)B.sh.p,
                 (const double *)B.sv.p, (const double *)B.t.p, x, B.r.p);
        launch_k(k_bt_dots, gt, kT, 0, q, TS, TB, TE, act, 1, (const double *)B.r.p, (const double *)B.r.p,
                 (const double *)nullptr, (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                 B.partial.p);
        launch_k(k_bt_reduce, gs, 256, 0, q, (int)nsys, TP, act, 1, (const double *)B.partial.p, B.red.p);
        launch_k(k_b_check_r, gs, 256, 0, q, (int)nsys, st, (int)maxit);
        SAIT_CK(cudaGetLastError());
        return SAIT_OK;
    };
    int64_t graph_kernels = 0;
    // kPollB iterations and the count of active systems, captured as one graph
    auto poll_block = [&](cudaStream_t q) -> sait_status {
        for (int k2 = 0; k2 < kPollB; k2++) SAIT_TRY(iteration(q));
        SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), q));
        launch_k(k_b_count, gs, 256, 0, q, (int)nsys, (const int *)st.active, ctx->d_word);
        SAIT_CK(cudaGetLastError());
        return SAIT_OK;
    };
    DTemp<int> bodies;
    SAIT_CK(bodies.alloc(1, s0));
    int64_t loop_kernels = 0;
    if (ctx->device_loop)
        SAIT_TRY(capture_loop(ctx, cs, poll_block, ctx->d_word, bodies.p, (int)cdiv(maxit, kPollB), &cleanup.loop,
                              &loop_kernels));
    if (!cleanup.loop) SAIT_TRY(capture(ctx, cs, poll_block, &cleanup.g, &graph_kernels));
    SAIT_TRY(sync_streams(ctx, s0, cs, ev));
    int total_iters = 0, graph_launches = 0;
    sait_status result = SAIT_OK;
    for (int round = 0;; round++) {
        // run until no system is active
        SAIT_TRY(run_iterations(ctx, cs, cleanup.loop, cleanup.g, loop_kernels, graph_kernels, maxit, ctx->d_word,
                                bodies.p, h, &total_iters, &graph_launches));
        // true residuals per system
        launch_k(k_b_residual, (unsigned)cdiv(n * 8, 256), 256, 0, cs, n, (const int32_t *)A->rp,
                 (const int32_t *)A->ci, (const double *)A->va, (const double *)x, b, B.r.p);
        launch_k(k_bt_dots, gt, kT, 0, cs, TS, TB, TE, (const int *)nullptr, 1, (const double *)B.r.p,
                 (const double *)B.r.p, (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                 (const double *)nullptr, B.partial.p);
        launch_k(k_bt_reduce, gs, 256, 0, cs, (int)nsys, TP, (const int *)nullptr, 1, (const double *)B.partial.p,
                 B.red.p);
        launch_k(k_b_relres, gs, 256, 0, cs, (int)nsys, (const double *)B.red.p, (const double *)st.bnorm, B.relres.p);
        launch_k(k_b_restart, gs, 256, 0, cs, (int)nsys, st, (const double *)B.relres.p, tol, (int)maxit);
        SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), cs));
        launch_k(k_b_count, gs, 256, 0, cs, (int)nsys, (const int *)st.active, ctx->d_word);
        SAIT_CK(cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, cs));
        SAIT_CK(cudaStreamSynchronize(cs));
        if (h[0] == 0 || round >= 64) break;
        launch_k(k_bt_reset, gt, kT, 0, cs, TS, TB, TE, (const int *)st.active, (const double *)B.r.p, B.rh.p, B.p.p,
                 B.v.p);
    }
    // results
    std::vector<double> rr(nsys);
    std::vector<int32_t> its(nsys), sts(nsys);
    SAIT_CK(cudaMemcpyAsync(rr.data(), B.relres.p, nsys * sizeof(double), cudaMemcpyDeviceToHost, cs));
    SAIT_CK(cudaMemcpyAsync(its.data(), st.iters, nsys * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    SAIT_CK(cudaMemcpyAsync(sts.data(), st.state, nsys * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    if (rel_resid) SAIT_CK(cudaMemcpyAsync(rel_resid, B.relres.p, nsys * sizeof(double), cudaMemcpyDeviceToDevice, cs));
    if (iters) SAIT_CK(cudaMemcpyAsync(iters, st.iters, nsys * sizeof(int32_t), cudaMemcpyDeviceToDevice, cs));
    SAIT_CK(cudaStreamSynchronize(cs));
    sait_batch_info bi{};
    bi.nsys = nsys;
    for (int q = 0; q < nsys; q++) {
        bi.max_rel_resid = std::max(bi.max_rel_resid, rr[q]);
        bi.max_iters = std::max(bi.max_iters, its[q]);
        bi.converged += rr[q] <= tol ? 1 : 0;
        if (sts[q] == 3) result = SAIT_ERR_NONFINITE;
        else if (sts[q] == 2 && result == SAIT_OK && rr[q] > tol) result = SAIT_ERR_BREAKDOWN;
    }
    bi.graph_replays = total_iters;
    bi.device_loop = cleanup.loop ? 1 : 0;
    bi.graph_launches = graph_launches;
    if (info) *info = bi;
    if (result == SAIT_OK && bi.converged < nsys) result = SAIT_ERR_NOT_CONVERGED;
    SAIT_TRY(sync_streams(ctx, cs, s0, ev));
    if (result != SAIT_OK) {
        char buf[160];
        snprintf(buf, sizeof(buf), "sait_bicgstab_batched: %s, %d of %d systems converged, max relres %.3e",
                 sait_status_string(result), bi.converged, nsys, bi.max_rel_resid);
        return ctx_fail(ctx, result, buf);
    }
    return SAIT_OK;
}

extern "C" sait_status sait_bicgstab_multi(sait_ctx ctx, sait_mat A, sait_prec P, int32_t k, const double *B,
                                           double *X, double tol, int32_t maxit, sait_batch_info *info,
                                           double *rel_resid, int32_t *iters) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || k < 1 || k > 256 || (256 % k != 0 && k > 32) || !B || !X || !(tol >= 0.0) || maxit < 0 ||
        (P && P->kind != 1) || (P && P->n != A->n))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG,
                        "sait_bicgstab_multi: bad argument (k in 1..32 or a divisor of 256; P a SAIT pair)");
    const int64_t n = A->n;
    const int64_t nk = n * k;
    cudaStream_t s0 = ctx->stream;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    SAIT_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    SAIT_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    struct Cleanup {
        cudaStream_t cs;
        cudaEvent_t ev;
        cudaGraphExec_t g = nullptr, loop = nullptr;
        ~Cleanup() {
            cudaStreamSynchronize(cs);
            if (g) cudaGraphExecDestroy(g);
            if (loop) cudaGraphExecDestroy(loop);
            cudaEventDestroy(ev);
            cudaStreamDestroy(cs);
        }
    } cleanup{cs, ev};
    int *h = (int *)ctx->h_pinned;
    const int rows_per_pass = kT / k;
    const int nb = (int)std::min<int64_t>(cdiv(n, rows_per_pass), 8LL * ctx->num_sms);
    Buffers Bf;
    for (DTemp<double> *d : {&Bf.r, &Bf.rh, &Bf.p, &Bf.v, &Bf.ph, &Bf.sv, &Bf.sh, &Bf.t}) SAIT_CK(d->alloc(nk, s0));
    DTemp<double> W;  // intermediate block of the SAIT apply
    SAIT_CK(W.alloc(nk, s0));
    SAIT_CK(Bf.partial.alloc((size_t)nb * k * 3, s0));
    SAIT_CK(Bf.red.alloc((size_t)k * 3, s0));
    SAIT_CK(Bf.relres.alloc(k, s0));
    SAIT_CK(Bf.sc.alloc((size_t)k * 8, s0));
    SAIT_CK(Bf.si.alloc((size_t)k * 3, s0));
    SAIT_CK(cudaMemsetAsync(Bf.p.p, 0, nk * sizeof(double), s0));
    SAIT_CK(cudaMemsetAsync(Bf.v.p, 0, nk * sizeof(double), s0));
    BState st = make_state(Bf, k);
    const unsigned gs = 1, ge = (unsigned)std::min<int64_t>(cdiv(nk, 256), 16LL * ctx->num_sms);
    auto dots = [&](cudaStream_t q, const int *act, int nd, const double *x0, const double *y0, const double *x1,
                    const double *y1) {
        launch_k(k_mc_dots, (unsigned)nb, kT, 0, q, n, (int)k, nd, act, x0, y0, x1, y1, Bf.partial.p);
        launch_k(k_mc_reduce, (unsigned)k, kT, 0, q, (int)k, nb, nd, act, (const double *)Bf.partial.p, Bf.red.p);
    };
    launch_k(k_mc_residual, ge, 256, 0, s0, n, (int)k, (const int32_t *)A->rp, (const int32_t *)A->ci,
             (const double *)A->va, (const double *)X, B, Bf.r.p);
    dots(s0, nullptr, 2, B, B, Bf.r.p, Bf.r.p);
    launch_k(k_b_start, gs, 256, 0, s0, (int)k, st, tol);
    launch_k(k_mc_update<4>, ge, 256, 0, s0, n, (int)k, st, (const double *)Bf.r.p, (const double *)nullptr,
             (const double *)Bf.v.p, (const double *)nullptr, Bf.rh.p, Bf.p.p);
    SAIT_CK(cudaGetLastError());
    auto apply = [&](cudaStream_t q, const double *in, double *out) -> sait_status {
        if (!P) {
            SAIT_CK(cudaMemcpyAsync(out, in, nk * sizeof(double), cudaMemcpyDeviceToDevice, q));
            return SAIT_OK;
        }
        cudaStream_t keep = ctx->stream;
        ctx->stream = q;
        sait_status r = apply_multi_impl(ctx, P->lo, P->up, (int)k, in, k, out, k, W.p);
        ctx->stream = keep;
        return r;
    };
    auto iteration = [&](cudaStream_t q) -> sait_status {
        const int *act = st.active;
        dots(q, act, 1, Bf.rh.p, Bf.r.p, nullptr, nullptr);
        launch_k(k_b_beta, gs, 256, 0, q, (int)k, st);
        launch_k(k_mc_update<0>, ge, 256, 0, q, n, (int)k, st, (const double *)Bf.r.p, (const double *)Bf.v.p,
                 (const double *)nullptr, (const double *)nullptr, Bf.p.p, (double *)nullptr);
        SAIT_TRY(apply(q, Bf.p.p, Bf.ph.p));
        SAIT_CK(launch_spmm(A, SAIT_F64, (int)k, k, k, Bf.ph.p, false, Bf.v.p, false, q, nullptr));
        dots(q, act, 1, Bf.rh.p, Bf.v.p, nullptr, nullptr);
        launch_k(k_b_alpha, gs, 256, 0, q, (int)k, st);
        launch_k(k_mc_update<1>, ge, 256, 0, q, n, (int)k, st, (const double *)Bf.r.p, (const double *)Bf.v.p,
                 (const double *)nullptr, (const double *)nullptr, Bf.sv.p, (double *)nullptr);
        dots(q, act, 1, Bf.sv.p, Bf.sv.p, nullptr, nullptr);
        launch_k(k_b_check_s, gs, 256, 0, q, (int)k, st);
        launch_k(k_mc_update<3>, ge, 256, 0, q, n, (int)k, st, (const double *)Bf.ph.p, (const double *)nullptr,
                 (const double *)nullptr, (const double *)nullptr, X, (double *)nullptr);
        launch_k(k_b_half_done, gs, 256, 0, q, (int)k, st);
        SAIT_TRY(apply(q, Bf.sv.p, Bf.sh.p));
        SAIT_CK(launch_spmm(A, SAIT_F64, (int)k, k, k, Bf.sh.p, false, Bf.t.p, false, q, nullptr));
        dots(q, act, 2, Bf.t.p, Bf.t.p, Bf.t.p, Bf.sv.p);
        launch_k(k_b_omega, gs, 256, 0, q, (int)k, st);
        launch_k(k_mc_update<2>, ge, 256, 0, q, n, (int)k, st, (const double *)Bf.ph.p, (const double *)Bf.sh.p,
                 (const double *)Bf.sv.p, (const double *)Bf.t.p, X, Bf.r.p);
        dots(q, act, 1, Bf.r.p, Bf.r.p, nullptr, nullptr);
        launch_k(k_b_check_r, gs, 256, 0, q, (int)k, st, (int)maxit);
        SAIT_CK(cudaGetLastError());
        return SAIT_OK;
    };
    int64_t graph_kernels = 0;
    // kPollB iterations and the count of active systems, captured as one graph
    auto poll_block = [&](cudaStream_t q) -> sait_status {
        for (int k2 = 0; k2 < kPollB; k2++) SAIT_TRY(iteration(q));
        SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), q));
        launch_k(k_b_count, gs, 256, 0, q, (int)k, (const int *)st.active, ctx->d_word);
        SAIT_CK(cudaGetLastError());
        return SAIT_OK;
    };
    DTemp<int> bodies;
    SAIT_CK(bodies.alloc(1, s0));
    int64_t loop_kernels = 0;
    if (ctx->device_loop)
        SAIT_TRY(capture_loop(ctx, cs, poll_block, ctx->d_word, bodies.p, (int)cdiv(maxit, kPollB), &cleanup.loop,
                              &loop_kernels));
    if (!cleanup.loop) SAIT_TRY(capture(ctx, cs, poll_block, &cleanup.g, &graph_kernels));
    SAIT_TRY(sync_streams(ctx, s0, cs, ev));
    int total_iters = 0, graph_launches = 0;
    for (int round = 0;; round++) {
        SAIT_TRY(run_iterations(ctx, cs, cleanup.loop, cleanup.g, loop_kernels, graph_kernels, maxit, ctx->d_word,
                                bodies.p, h, &total_iters, &graph_launches));
        launch_k(k_mc_residual, ge, 256, 0, cs, n, (int)k, (const int32_t *)A->rp, (const int32_t *)A->ci,
                 (const double *)A->va, (const double *)X, B, Bf.r.p);
        dots(cs, nullptr, 1, Bf.r.p, Bf.r.p, nullptr, nullptr);
        launch_k(k_b_relres, gs, 256, 0, cs, (int)k, (const double *)Bf.red.p, (const double *)st.bnorm, Bf.relres.p);
        launch_k(k_b_restart, gs, 256, 0, cs, (int)k, st, (const double *)Bf.relres.p, tol, (int)maxit);
        SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), cs));
        launch_k(k_b_count, gs, 256, 0, cs, (int)k, (const int *)st.active, ctx->d_word);
        SAIT_CK(cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, cs));
        SAIT_CK(cudaStreamSynchronize(cs));
        if (h[0] == 0 || round >= 64) break;
        launch_k(k_mc_update<4>, ge, 256, 0, cs, n, (int)k, st, (const double *)Bf.r.p, (const double *)nullptr,
                 (const double *)Bf.v.p, (const double *)nullptr, Bf.rh.p, Bf.p.p);
    }
    std::vector<double> rr(k);
    std::vector<int32_t> its(k), sts(k);
    SAIT_CK(cudaMemcpyAsync(rr.data(), Bf.relres.p, k * sizeof(double), cudaMemcpyDeviceToHost, cs));
    SAIT_CK(cudaMemcpyAsync(its.data(), st.iters, k * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    SAIT_CK(cudaMemcpyAsync(sts.data(), st.state, k * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    if (rel_resid) SAIT_CK(cudaMemcpyAsync(rel_resid, Bf.relres.p, k * sizeof(double), cudaMemcpyDeviceToDevice, cs));
    if (iters) SAIT_CK(cudaMemcpyAsync(iters, st.iters, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, cs));
    SAIT_CK(cudaStreamSynchronize(cs));
    sait_batch_info bi{};
    bi.nsys = k;
    sait_status result = SAIT_OK;
    for (int q = 0; q < k; q++) {
        bi.max_rel_resid = std::max(bi.max_rel_resid, rr[q]);
        bi.max_iters = std::max(bi.max_iters, its[q]);
        bi.converged += rr[q] <= tol ? 1 : 0;
        if (sts[q] == 3) result = SAIT_ERR_NONFINITE;
        else if (sts[q] == 2 && result == SAIT_OK && rr[q] > tol) result = SAIT_ERR_BREAKDOWN;
    }
    bi.graph_replays = total_iters;
    bi.device_loop = cleanup.loop ? 1 : 0;
    bi.graph_launches = graph_launches;
    if (info) *info = bi;
    if (result == SAIT_OK && bi.converged < k) result = SAIT_ERR_NOT_CONVERGED;
    SAIT_TRY(sync_streams(ctx, cs, s0, ev));
    if (result != SAIT_OK) {
        char buf[160];
        snprintf(buf, sizeof(buf), "sait_bicgstab_multi: %s, %d of %d columns converged, max relres %.3e",
                 sait_status_string(result), bi.converged, (int)k, bi.max_rel_resid);
        return ctx_fail(ctx, result, buf);
    }
    return SAIT_OK;
}

// ---- tile-size autotuning ---------------------------------------------------------
// Times the schedule-dependent part of one batched iteration (the per-tile dot
// kernel and the per-system reduction, the reductions that every BiCGSTAB
// step runs four to five times) for each candidate tile size on the caller's
// batch, and keeps the fastest in the context for later batched solves.
extern "C" sait_status sait_batch_autotune(sait_ctx ctx, int64_t n, int32_t nsys, const int64_t *sys_ptr,
                                           sait_batch_tune_report *report) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (n < 0 || nsys < 1 || !sys_ptr || !report)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_batch_autotune: bad argument");
    cudaStream_t s = ctx->stream;
    const int64_t cand[] = {512, 1024, 2048, 4096, 8192};
    const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
    *report = sait_batch_tune_report{};
    report->ncand = nc;
    int *h = (int *)ctx->h_pinned;
    int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
    DTemp<double> x, red;
    SAIT_CK(x.alloc(std::max<int64_t>(n, 1), s));
    SAIT_CK(red.alloc((size_t)nsys * 3, s));
    SAIT_CK(cudaMemsetAsync(x.p, 0, std::max<int64_t>(n, 1) * sizeof(double), s));
    cudaEvent_t e0, e1;
    SAIT_CK(cudaEventCreate(&e0));
    SAIT_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    sait_status st = SAIT_OK;
    for (int c = 0; c < nc && st == SAIT_OK; c++) {
        const int64_t tile = cand[c];
        DTemp<int32_t> tcnt, tsys;
        DTemp<int64_t> tptr, tbeg, tend;
        DTemp<double> partial;
        cudaError_t e = tcnt.alloc(nsys, s);
        if (e == cudaSuccess) e = tptr.alloc(nsys + 1, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_word, 0, sizeof(int), s);
        if (e != cudaSuccess) { st = ctx_cuda(ctx, e, "sait_batch_autotune", __FILE__, __LINE__); break; }
        launch_k(k_tile_count, (unsigned)cdiv(nsys, 256), 256, 0, s, (int)nsys, sys_ptr, tile, tcnt.p, ctx->d_word);
        e = scan_i32(tcnt.p, tptr.p, nsys, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64, tptr.p + nsys, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64 + 1, sys_ptr + nsys, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = ctx_cuda(ctx, e, "sait_batch_autotune", __FILE__, __LINE__); break; }
        if (h[0] != 0 || h64[1] != n) {
            st = ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_batch_autotune: sys_ptr must be non-decreasing to n");
            break;
        }
        const int64_t ntiles = h64[0];
        e = tsys.alloc(std::max<int64_t>(ntiles, 1), s);
        if (e == cudaSuccess) e = tbeg.alloc(std::max<int64_t>(ntiles, 1), s);
        if (e == cudaSuccess) e = tend.alloc(std::max<int64_t>(ntiles, 1), s);
        if (e == cudaSuccess) e = partial.alloc((size_t)std::max<int64_t>(ntiles, 1) * 3, s);
        if (e != cudaSuccess) { st = ctx_cuda(ctx, e, "sait_batch_autotune", __FILE__, __LINE__); break; }
        launch_k(k_tile_fill, (unsigned)cdiv(nsys, 256), 256, 0, s, (int)nsys, sys_ptr, tile, (const int64_t *)tptr.p,
                 tsys.p, tbeg.p, tend.p);
        const unsigned gt = (unsigned)ntiles, gs = (unsigned)cdiv(nsys, 256);
        auto one = [&]() {
            launch_k(k_bt_dots, gt, kT, 0, s, (const int32_t *)tsys.p, (const int64_t *)tbeg.p, (const int64_t *)tend.p,
                     (const int *)nullptr, 2, (const double *)x.p, (const double *)x.p, (const double *)x.p,
                     (const double *)x.p, (const double *)nullptr, (const double *)nullptr, partial.p);
            launch_k(k_bt_reduce, gs, 256, 0, s, (int)nsys, (const int64_t *)tptr.p, (const int *)nullptr, 2,
                     (const double *)partial.p, red.p);
        };
        for (int w = 0; w < 3; w++) one();
        constexpr int reps = 10;
        e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps; r++) one();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { st = ctx_cuda(ctx, e, "sait_batch_autotune", __FILE__, __LINE__); break; }
        report->tile_rows[c] = (int32_t)tile;
        report->us[c] = ms * 1e3f / reps;
        if (report->us[c] < best) {
            best = report->us[c];
            report->chosen = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == SAIT_OK) ctx->batch_tile = cand[report->chosen];
    return st;
}

extern "C" sait_status sait_ctx_set_batch_tile(sait_ctx ctx, int64_t rows) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (rows < 32 || rows > (1 << 20)) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_ctx_set_batch_tile: rows out of range");
    ctx->batch_tile = rows;
    return SAIT_OK;
}
