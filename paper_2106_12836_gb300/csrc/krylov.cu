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
    int ticket;      // GMRES: blocks of the dot sweep that finished (last-block pattern)
    int sweep;       // GMRES: 1 when the update sweep of this step runs
    int stop_after;  // GMRES: stop the cycle once column j-1 is rotated
    double gamma_last;
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
    pdl_wait();
    pdl_trigger();
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

// Precision on GB300: its FP64 pipe (1.2 TFLOP/s measured, against 63.5
// TFLOP/s FP32) would bound FP64 Gram-Schmidt passes far below HBM speed, so
// the final basis vectors are kept as (hi, m16) pairs: hi = the vector's top
// 24 bits in FP32 and m16 = its next 16 bits (split_hi16), ~2^-39 relative in
// six bytes; FP64 columns hold only the tentative vectors the products read.
// The dots run in FP32 on hi, the updates in double-float on (hi, m16) with
// error-free two-sums, and a few FP64 operations per entry and step remain.
//
// Layout: the kernels below work on n rounded up to a multiple of 4 rows with
// zero padding, so they move 16-byte vectors (four rows per thread) and never
// need a ragged tail; the basis columns' leading dimension ldv adds kColPad
// more entries, so that the columns do not all start at the same offset
// modulo a large power of two.
__device__ __forceinline__ float4 load_w4(const double2 *w, int64_t i4) {
    const double2 a = w[2 * i4], b = w[2 * i4 + 1];
    return make_float4(hi_part(a.x), hi_part(a.y), hi_part(b.x), hi_part(b.y));
}

// ---- GMRES with delayed reorthogonalization (DCGS2) --------------------------
// Classical Gram-Schmidt twice, with the second pass of each Arnoldi vector
// delayed to the next step (Bielich, Langou, Thomas, Swirydowicz, Yamazaki and
// Boman, "Low-synch Gram-Schmidt with delayed reorthogonalization for Krylov
// solvers", Parallel Computing 2022), written here for right-preconditioned
// GMRES.  Step j holds the final orthonormal v_0 .. v_{j-1} and a tentative
// u_j = w1 / eta (w1 stored unnormalized in column j, eta = ||w1||):
//   w = A M w1                                (the SAIT apply and A product)
//   one sweep:  c = V^T w1 / eta,  d = V^T w / eta,  delta = w1^T w / eta^2
//   gamma = sqrt(1 - c.c);  v_j = (u_j - V c) / gamma     (u_j reorthogonalized)
//   column j-1 becomes final: H(0:j-1, j-1) += eta c, H(j, j-1) = eta gamma
//   A M v_j = (w/eta - V_{j+1} H c) / gamma, so its first-pass coefficients
//   follow from d, delta and t = H c without another sweep, and
//   one sweep:  v_j and the next tentative w1' = A M v_j - V_{j+1} h_j.
// Two sweeps over the basis per step instead of four; the Givens rotation of a
// column is applied once it is final, so convergence is seen one step later.
// Precision as above: dots in FP32 on the hi parts, updates in double-float on
// the (hi, m16) pairs.
constexpr int kDCH = 8;          // basis vectors per chunk of the dual dot sweep
constexpr int kDotThreads = 1024; // dual dot sweep: one block of 1024 threads per SM
constexpr int kUpdPre = 16;      // basis vectors an update thread prefetches before its wait
constexpr int kColPad = 32;      // extra entries per basis column (see the layout in sait_gmres)

// Everything the last block of the dot sweep and the Givens step touch.
struct DcgsState {
    float *part;           // dot partials, column-major: part[slot * ldp + block]
    int ldp;               // leading dimension (>= blocks, multiple of 4, padding zero)
    const float *upart;    // ||w1||^2 of the update sweep's blocks (j >= 1), nbu of them
    int nbu;
    double *Hr, *R, *cs, *sn, *g;  // raw Hessenberg, rotated copy, rotations, rhs (ld m + 1)
    double *coef, *kk;             // update weights: coef = [p (j), r (j)], kk = [k1, k2, k3]
    Scal *sc;
    int *calls;            // timer-group counter (or null)
    int m;
};

// One unit of the dual sweep: batch q0 .. q0 + 7 of the basis over one tile
// (32 float4 rows) with that tile's u and w in registers.  The batch's 16 dot
// products over the tile are summed across the warp and added to the warp's
// shared slots wacc[q] (V_q . U) and wacc[j + q] (V_q . W).
__device__ __forceinline__ void dual_unit(int64_t i, bool ok, int q0, int j, const float4 *__restrict__ V,
                                          int64_t ldv4, const float4 &u, const float4 &w, float *wacc, int lane) {
    float4 vv[kDCH];
#pragma unroll
    for (int t = 0; t < kDCH; t++)
        vv[t] = ok && q0 + t < j ? __ldg(V + (int64_t)(q0 + t) * ldv4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    float v[2 * kDCH];  // v[t] = V_{q0+t} . U, v[kDCH + t] = V_{q0+t} . W over this lane's 4 rows
#pragma unroll
    for (int t = 0; t < kDCH; t++) {
        float a = vv[t].x * u.x;
        a = fmaf(vv[t].y, u.y, a);
        a = fmaf(vv[t].z, u.z, a);
        v[t] = fmaf(vv[t].w, u.w, a);
        float b = vv[t].x * w.x;
        b = fmaf(vv[t].y, w.y, b);
        b = fmaf(vv[t].z, w.z, b);
        v[kDCH + t] = fmaf(vv[t].w, w.w, b);
    }
    // warp sum of the 16 values by recursive halving: at offset o a lane keeps
    // the half of its values picked by its lane bit o and adds the partner's
    // copy of that half (16 shuffles for 16 sums instead of 80); afterwards
    // lanes 2i and 2i + 1 hold the sum of value i
#pragma unroll
    for (int h = kDCH, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int e = 0; e < h; e++) {
            const float send = up ? v[e] : v[e + h];
            const float keep = up ? v[e + h] : v[e];
            v[e] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    const int vi = lane >> 1, tt = vi & (kDCH - 1);
    if (!(lane & 1) && q0 + tt < j) wacc[(vi < kDCH ? 0 : j) + q0 + tt] += v[0];
}

// The dual sweep of one warp over tiles of 32 float4 rows (128 rows).  Warps
// take whole tiles round robin for as many full rounds as there are, so the
// GPU's warps read one contiguous front of rows of every vector at a time
// (DRAM streams that far better than one run per warp scattered over the
// columns) and load each tile's u and w once; the tiles left over are cut
// into units (tile, batch of 8 vectors), also taken round robin, so no warp
// holds more than one unit beyond another.  wacc[2j] gets U . W.
__device__ __forceinline__ void dual_sweep_warp(int64_t n4, const float4 *__restrict__ V, int64_t ldv4, int j,
                                                const float4 *__restrict__ U, const double2 *__restrict__ W,
                                                float *wacc) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * kDotThreads + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kDotThreads) >> 5;
    const int nbat = j > 0 ? (j + kDCH - 1) / kDCH : 1;
    const int64_t ntiles = (n4 + 31) / 32, main_tiles = ntiles / nw * nw;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float ad = 0.0f;
    auto tile_uw = [&](int64_t tile, bool first, int64_t &i, bool &ok, float4 &u, float4 &w) {
        i = tile * 32 + lane;
        ok = i < n4;
        u = ok ? U[i] : z4;
        w = ok ? load_w4(W, i) : z4;
        if (first) {
            ad = fmaf(u.x, w.x, ad);
            ad = fmaf(u.y, w.y, ad);
            ad = fmaf(u.z, w.z, ad);
            ad = fmaf(u.w, w.w, ad);
        }
    };
    for (int64_t tile = gw; tile < main_tiles; tile += nw) {  // whole tiles
        int64_t i;
        bool ok;
        float4 u, w;
        tile_uw(tile, true, i, ok, u, w);
        for (int q0 = 0; q0 < j; q0 += kDCH) dual_unit(i, ok, q0, j, V, ldv4, u, w, wacc, lane);
    }
    const int64_t units = (ntiles - main_tiles) * nbat;  // the rest as (tile, batch) units
    for (int64_t un = gw; un < units; un += nw) {
        const int64_t tile = main_tiles + un / nbat;
        const int bat = (int)(un % nbat);
        int64_t i;
        bool ok;
        float4 u, w;
        tile_uw(tile, bat == 0, i, ok, u, w);
        if (bat * kDCH < j) dual_unit(i, ok, bat * kDCH, j, V, ldv4, u, w, wacc, lane);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ad += __shfl_xor_sync(0xffffffffu, ad, o);
    if (lane == 0) wacc[2 * j] += ad;
}

// Sum of the FP32 values x[0 .. cnt) (a 16-byte aligned run, cnt a multiple of 4)
// by a group of LPC lanes (LPC = 8, 16 or 32, aligned in the warp), returned to
// all of them; each lane issues its loads (up to KQ float4) together, so the
// sum costs one L2 round trip for up to 4 LPC KQ values.
template <int LPC, int KQ>
__device__ __forceinline__ float group_sum(const float *x, int cnt, int sub) {
    const float4 *x4 = (const float4 *)x;
    const int c4 = cnt / 4;
    float s = 0.0f;
    for (int i0 = 0; i0 < c4; i0 += LPC * KQ) {
        float4 a[KQ];
#pragma unroll
        for (int u = 0; u < KQ; u++) {
            const int i = i0 + sub + LPC * u;
            a[u] = i < c4 ? __ldcg(x4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < KQ; u++) s += (a[u].x + a[u].y) + (a[u].z + a[u].w);
    }
#pragma unroll
    for (int o = 1; o < LPC; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// colsum[q] = sum over the dot sweep's blocks of part[q * ldp + b], q < ncol:
// LPC lanes per column, so that ncol columns of cnt partials take one or two rounds.
template <int LPC, int KQ>
__device__ __forceinline__ void column_sums(const DcgsState &S, int ncol, int cnt, double *colsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kPerWarp = 32 / LPC;
    const int groups = (kDotThreads / 32) * kPerWarp;
    for (int q0 = 0; q0 < ncol; q0 += groups) {
        const int q = q0 + warp * kPerWarp + lane / LPC;
        const float v = group_sum<LPC, KQ>(S.part + (int64_t)(q < ncol ? q : 0) * S.ldp, cnt, lane % LPC);
        if (q < ncol && lane % LPC == 0) colsum[q] = widen_exact(v);
    }
}

// The scalar step of DCGS2 step j, run by the last block of the dot sweep once
// every block's partial sums are in.  dots (reduced here) = [c' (j), d' (j),
// delta']; eta^2 = ||w1||^2 from the update sweep's partials (j >= 1; eta = beta
// at j = 0).  Column j-1 of H becomes final (its rotation is applied later, by
// dcgs_givens); writes coef = [p (j), r (j)], kk = [k1, k2, k3] and the first-pass
// column j of H, or with `close` only finalizes column j-1.
//
// GB300's FP64 pipe issues about two thread operations per cycle per SM with
// a 64-cycle dependent latency (sqrt and division about 650), so this step
// keeps FP64 work short and off the wide paths: the partial sums are added in
// FP32 (they are FP32 dot products already), the scalar recurrences run on
// one thread and are broadcast through shared memory, reciprocal square roots
// replace square roots and divisions, and t = H c is split over eight
// threads per row.
__device__ void dcgs_scalar_step(const DcgsState &S, int j, int close, int nbd) {
    __shared__ double colsum[2 * kMaxRestart + 2];
    __shared__ double c2[kMaxRestart + 1], dh[kMaxRestart + 1], tv[kMaxRestart + 2];
    __shared__ float c2f[kMaxRestart + 1], dhf[kMaxRestart + 1];
    __shared__ double s_cc, s_cd, s_e2, s_eta, s_ie, s_ig, s_gamma, s_av;
    __shared__ int s_ok;
    __shared__ float e2w[kDotThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarp = kDotThreads / 32;
    Scal *sc = S.sc;
    const int ncol = 2 * j + 1;
    // the update sweep's ||w1||^2 partials, loaded now (summed after the column sums)
    constexpr int kE = 4;
    float ep[kE];
#pragma unroll
    for (int u = 0; u < kE; u++) {
        const int i = tid + u * kDotThreads;
        ep[u] = j >= 1 && i < S.nbu ? __ldcg(S.upart + i) : 0.0f;
    }
    // the H entries of t = H c (below), loaded now so that their latency overlaps
    // the partial sums: warps 1.. take row i = (tid - 32) / kTR, kTR threads per row
    constexpr int kTR = 16, kTH = 4;
    const int rid = (tid - 32) / kTR, sub = (tid - 32) % kTR;
    double hreg[kTH];
    const bool tpre = warp != 0 && !close && j <= kTH * kTR && rid <= j;
    if (tpre) {
#pragma unroll
        for (int u = 0; u < kTH; u++) {
            const int k = (rid > 0 ? rid - 1 : 0) + sub + kTR * u;
            hreg[u] = k < j ? S.Hr[(int64_t)k * (S.m + 1) + rid] : 0.0;
        }
    }
    // (1) column sums of the partials: a warp, half warp or quarter warp per column
    const int cnt = (nbd + 3) / 4 * 4;
    if (ncol <= nwarp) column_sums<32, 5>(S, ncol, cnt, colsum);
    else if (ncol <= 2 * nwarp) column_sums<16, 10>(S, ncol, cnt, colsum);
    else column_sums<8, 10>(S, ncol, cnt, colsum);
    if (j >= 1) {  // ||w1||^2: every thread adds a few partials, then the block
        float s0 = 0.0f;
        for (int i = tid + kE * kDotThreads; i < S.nbu; i += kDotThreads) s0 += __ldcg(S.upart + i);
#pragma unroll
        for (int u = 0; u < kE; u++) s0 += ep[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        if (lane == 0) e2w[warp] = s0;
    }
    __syncthreads();
    if (tid == 0 && j >= 1) {
        float e = 0.0f;
        for (int w2 = 0; w2 < nwarp; w2++) e += e2w[w2];
        s_e2 = (double)e;
    }
    // (2) eta = ||w1|| (one thread)
    double *Hc = S.Hr + (int64_t)(j - 1) * (S.m + 1);  // column j-1 (j >= 1)
    if (tid == 0) {
        double eta, ie;
        if (j >= 1) {
            ie = rsqrt(s_e2);
            eta = s_e2 * ie;
        } else {
            eta = sc->beta;
            ie = 1.0 / eta;
        }
        const int ok = eta > 0.0 && isfinite(eta) && isfinite(ie);
        if (!ok) {  // invariant subspace (or a non-finite vector)
            if (S.calls) atomicAdd(S.calls, 1);
            if (!isfinite(eta)) sc->state = 3;
            sc->sweep = 0;
            if (j >= 1) {
                Hc[j] = 0.0;
                sc->stop_after = 1;   // rotate column j-1, then stop
            } else {
                sc->jdone = 0;
                sc->active = 0;
            }
        }
        s_ok = ok;
        s_eta = eta;
        s_ie = ie;
    }
    __syncthreads();
    if (!s_ok) return;
    const double eta = s_eta, ie = s_ie;
    for (int q = tid; q < j; q += kDotThreads) {
        c2[q] = colsum[q] * ie;
        dh[q] = colsum[j + q] * ie;
        c2f[q] = narrow_rn(c2[q]);
        dhf[q] = narrow_rn(dh[q]);
    }
    __syncthreads();
    // (3) warp 0: cc = c.c and cd = c.d; the other warps: t = H c.  In FP32:
    // c and d come from FP32 dot products and carry absolute errors of order
    // 2^-24 already, which FP32 sums of their products do not raise, while one
    // SM's FP64 pipe would spend microseconds on these few hundred terms.
    if (warp == 0) {
        float a = 0.0f, b = 0.0f;
        for (int q = lane; q < j; q += 32) {
            a = fmaf(c2f[q], c2f[q], a);
            b = fmaf(c2f[q], dhf[q], b);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            s_cc = widen_exact(a);
            s_cd = widen_exact(b);
        }
    } else if (!close) {
        const float etaf = narrow_rn(eta);
        // t_i = sum_{k = max(i-1,0)}^{j-1} H(i,k) c_k over the final columns, with
        // column j-1 taken as H(i,j-1) + eta c_i; H(j,j-1) = eta gamma is added below
        const int rows_per_round = (kDotThreads - 32) / kTR;
        for (int i0 = 0; i0 <= j; i0 += rows_per_round) {
            const int i = i0 + rid;
            float a = 0.0f;
            if (i <= j) {
                const int kb = (i > 0 ? i - 1 : 0) + sub;
                if (i0 == 0 && tpre) {
#pragma unroll
                    for (int u = 0; u < kTH; u++) {
                        const int k = kb + kTR * u;
                        if (k < j) {
                            const float hf = narrow_rn(hreg[u]);
                            const float h = k == j - 1 ? (i < j ? fmaf(etaf, c2f[i], hf) : 0.0f) : hf;
                            a = fmaf(h, c2f[k], a);
                        }
                    }
                } else {
                    for (int k = kb; k < j; k += kTR) {
                        float h = narrow_rn(S.Hr[(int64_t)k * (S.m + 1) + i]);
                        if (k == j - 1) h = i < j ? fmaf(etaf, c2f[i], h) : 0.0f;
                        a = fmaf(h, c2f[k], a);
                    }
                }
            }
#pragma unroll
            for (int o = 1; o < kTR; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (i <= j && sub == 0) tv[i] = widen_exact(a);
        }
    }
    __syncthreads();
    if (j >= 1)  // column j-1 final: H(0:j-1, j-1) += eta c (t above read the old column)
        for (int q = tid; q < j; q += kDotThreads) Hc[q] = fma(eta, c2[q], Hc[q]);
    // (4) gamma = sqrt(1 - c.c) and the scalars of column j (one thread)
    if (tid == 0) {
        const double om = 1.0 - s_cc;
        const double ig = om > 0.0 ? rsqrt(om) : 0.0;
        const double gamma = om > 0.0 ? om * ig : 0.0;
        if (S.calls) atomicAdd(S.calls, 1);
        if (j >= 1) Hc[j] = eta * gamma;
        sc->gamma_last = gamma;
        sc->sweep = (!close && gamma > 0.0) ? 1 : 0;
        sc->stop_after = (close || !(gamma > 0.0)) ? 1 : 0;
        if (!close && gamma > 0.0) {
            // first-pass coefficients of A M v_j (tentative column j): a_j and the
            // weights k1, k2, k3 of the update
            const double dl = colsum[2 * j] * ie * ie;
            const double tj = j >= 1 ? fma(eta * gamma, c2[j - 1], tv[j]) : 0.0;
            const double cj = ((dl - s_cd) * ig - tj) * ig;
            const double av = fma(gamma, cj, tj);
            S.Hr[(int64_t)j * (S.m + 1) + j] = cj;
            S.kk[0] = ie * ig;            // v_j   = k1 w1 - V p
            S.kk[1] = ie * ig;            // w1'   = k2 w - k3 w1 - V r
            S.kk[2] = av * ie * ig * ig;
            s_av = av;
        }
        s_ig = ig;
        s_gamma = gamma;
    }
    __syncthreads();
    const double gamma = s_gamma, ig = s_ig;
    if (close || !(gamma > 0.0)) return;
    const double av = s_av;
    double *Hj = S.Hr + (int64_t)j * (S.m + 1);
    for (int q = tid; q < j; q += kDotThreads) {
        const double c1 = (dh[q] - tv[q]) * ig;
        Hj[q] = c1;
        const double aV = fma(gamma, c1, tv[q]);
        S.coef[q] = c2[q] * ig;                          // p
        S.coef[j + q] = (aV - av * ig * c2[q]) * ig;     // r
    }
}

// Dual dot sweep of DCGS2 step j over the blocks' rows; the last block to finish
// then runs the scalar step.  remaining/close: see dcgs_givens.
__global__ void __launch_bounds__(kDotThreads, 1)
k_dcgs_dot(int64_t n4, const float4 *__restrict__ V, int64_t ldv4, int j, const float4 *__restrict__ U,
           const double2 *__restrict__ W, DcgsState S, int close) {
    pdl_wait();
    pdl_trigger();
    if (S.sc->active == 0) return;
    extern __shared__ float wacc_all[];  // per warp: the 2j + 1 sums of its tiles
    __shared__ int s_last;
    const int nslot = 2 * j + 1, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < (kDotThreads / 32) * nslot; t += kDotThreads) wacc_all[t] = 0.0f;
    __syncthreads();
    dual_sweep_warp(n4, V, ldv4, j, U, W, wacc_all + warp * nslot);
    __syncthreads();
    for (int t = threadIdx.x; t < nslot; t += kDotThreads) {  // the block's partials, warps in order
        float sum = 0.0f;
        for (int w2 = 0; w2 < kDotThreads / 32; w2++) sum += wacc_all[w2 * nslot + t];
        S.part[(int64_t)t * S.ldp + blockIdx.x] = sum;
    }
    __syncthreads();
    // the last block to finish sums the partials (threadfence-reduction pattern)
    if (threadIdx.x == 0) {
        __threadfence();
        const int ticket = atomicAdd(&S.sc->ticket, 1);
        s_last = ticket == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) S.sc->ticket = 0;
    dcgs_scalar_step(S, j, close, gridDim.x);
}

// Column c = j-1 of H is final: copy it into R, apply the previous rotations,
// form rotation c and update g; then jdone = j, and the cycle stops when
// |g_{c+1}| <= tol ||b||, when j reaches `remaining` steps, at the end of the
// cycle, or when the scalar step asked for it (invariant subspace, gamma = 0).
// One warp; the rotations are a serial chain (thread 0).
__device__ void dcgs_givens(const DcgsState &S, int j, int remaining) {
    Scal *sc = S.sc;
    const int c = j - 1, m = S.m;
    const double *Hc = S.Hr + (int64_t)c * (m + 1);
    double *Rc = S.R + (int64_t)c * (m + 1);
    __shared__ double hc[kMaxRestart + 2];
    for (int i = threadIdx.x; i <= c + 1; i += 32) hc[i] = Hc[i];
    __syncwarp();
    if (threadIdx.x == 0) {
        double carry = hc[0];
        for (int i = 0; i < c; i++) {
            const double ci = S.cs[i], si = S.sn[i], b = hc[i + 1];
            hc[i] = fma(ci, carry, si * b);
            carry = fma(ci, b, -si * carry);
        }
        const double a = carry, b = hc[c + 1];
        double cc = 1.0, ss = 0.0;
        if (b != 0.0) {
            const double t = hypot(a, b);
            cc = a / t;
            ss = b / t;
        }
        S.cs[c] = cc;
        S.sn[c] = ss;
        hc[c] = fma(cc, a, ss * b);
        hc[c + 1] = 0.0;
        const double gc = S.g[c];
        S.g[c + 1] = -ss * gc;
        S.g[c] = cc * gc;
        const double est = fabs(ss * gc);
        sc->jdone = j;
        if (!isfinite(est)) {
            sc->state = 3;
            sc->active = 0;
        } else if (est <= sc->tolb || j >= remaining || sc->stop_after) {
            sc->active = 0;
        }
    }
    __syncwarp();
    for (int i = threadIdx.x; i <= c + 1; i += 32) Rc[i] = hc[i];
}

// The rotation of the last column at the end of a cycle (no update sweep follows).
__global__ void k_dcgs_givens(DcgsState S, int j, int remaining) {
    pdl_wait();
    if (S.sc->active == 0 || j < 1) return;
    dcgs_givens(S, j, remaining);
}

// The basis is kept as (hi, m16): hi = v truncated to 24 significant bits (as
// hi_part) and m16 = the next 16 bits of v's mantissa, rounded, an unsigned
// magnitude with hi's sign, so v = hi + sign(hi) m16 2^(E-39) (E = hi's
// unbiased exponent) to within 2^(E-40), ~2^-39 relative.  Six bytes per entry
// instead of eight for an FP32 (hi, lo) pair; the Arnoldi relation holds to
// ~1e-12, far below the 1e-8 the solver targets.  Values outside the normal
// FP32 range of hi keep hi = fl32(v) and m16 = 0.
__device__ __forceinline__ void split_hi16(double v, float &hi, unsigned short &m16) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ef = (int)((b >> 52) & 0x7ff) - 896;
    if (ef <= 0 || ef >= 255) {
        hi = hi_part_slow(v);
        m16 = 0;
        return;
    }
    const unsigned long long frac = b & ((1ULL << 52) - 1);
    hi = __uint_as_float(((unsigned)(b >> 63) << 31) | ((unsigned)ef << 23) | (unsigned)(frac >> 29));
    const unsigned r = (unsigned)(frac & ((1ULL << 29) - 1));  // the 29 bits below hi
    const unsigned m = (r + (1u << 12)) >> 13;
    m16 = (unsigned short)(m > 0xffffu ? 0xffffu : m);
}

// The low part without its constant factor: sign(hi) m16 2^E, exact in FP32
// (m16 < 2^16; 2^E is hi with its mantissa bits cleared).  The low part itself
// is this times 2^-39, a factor the callers fold into their coefficients, so a
// basis entry costs four operations to widen instead of a dozen.
constexpr float kTail = 0x1p-39f;
__device__ __forceinline__ float lo16_unscaled(float hi, unsigned short m16) {
    const float mf = __uint_as_float(0x4B000000u | (unsigned)m16) - 8388608.0f;
    return mf * __uint_as_float(__float_as_uint(hi) & 0xff800000u);
}

// df_term with the low part of the basis entry given unscaled (lu, from
// lo16_unscaled) and the coefficient's hi part premultiplied by kTail (as):
// lu * as equals lo * a exactly, so the sum matches df_term's.
__device__ __forceinline__ void df_term_t(float &S, float &E, float vh, float lu, float a, float al, float as) {
    const float p = __fmul_rn(vh, a);
    float e = __fmaf_rn(vh, a, -p);
    e = __fmaf_rn(vh, al, e);
    e = __fmaf_rn(lu, as, e);
    df_add(S, E, p, e);
}

// Block 0 applies the Givens rotation of column j-1 (dcgs_givens), concurrently
// with the sweep of the other blocks:
// v_j = k1 w1 - V p (stored as its (hi, m16) pair in column j of the basis) and
// w1' = k2 w - k3 w1 - V r (written over w in column j + 1, with its FP32
// copy for the next dual sweep); upart[b] = ||w1'||^2 (FP32) of sweep block b's
// rows.  Two rows per thread (8-byte hi and 4-byte m16 pair loads), so many
// resident warps hide the load latency.
__global__ void __launch_bounds__(kThreads, 4)
k_dcgs_update(int64_t n2, const float2 *__restrict__ Vh, const ushort2 *__restrict__ Vm, int64_t ldv2, int j,
              const double2 *wcol1, double2 *wcol, float2 *vh_out, ushort2 *vm_out, float2 *w32, float *upart,
              DcgsState S, int remaining) {
    // Everything this sweep reads but the coefficients is final before the dot
    // sweep starts, so the blocks that become resident while its last block
    // runs the scalar step pull their first rows into L2 before waiting.
    if (blockIdx.x > 0) {
        const int64_t i = (int64_t)(blockIdx.x - 1) * kThreads + threadIdx.x;
        if (i < n2) {
            prefetch_l2(wcol1 + i);
            prefetch_l2(wcol + i);
            for (int q = 0; q < min(j, kUpdPre); q++) {
                prefetch_l2(Vh + (int64_t)q * ldv2 + i);
                prefetch_l2(Vm + (int64_t)q * ldv2 + i);
            }
        }
    }
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x == 0) {
        if (threadIdx.x < 32 && S.sc->active != 0 && j >= 1) dcgs_givens(S, j, remaining);
        return;
    }
    // a stop decided by block 0 in this launch leaves the sweep's columns unused
    if (S.sc->active == 0 || S.sc->sweep == 0) return;
    const int bid = blockIdx.x - 1, nbs = gridDim.x - 1;
    __shared__ float ph[kMaxRestart + 1], rh[kMaxRestart + 1], rl[kMaxRestart + 1], rs[kMaxRestart + 1];
    __shared__ float red[kThreads / 32];
    const double *coef = S.coef;
    for (int q = threadIdx.x; q < j; q += kThreads) {
        ph[q] = (float)coef[q];
        split_pair(coef[j + q], rh[q], rl[q]);
        rs[q] = rh[q] * kTail;
    }
    __syncthreads();
    const double k1 = S.kk[0], k2 = S.kk[1], k3 = S.kk[2];
    float nrm = 0.0f;
    for (int64_t i = (int64_t)bid * kThreads + threadIdx.x; i < n2; i += (int64_t)nbs * kThreads) {
        // V p is the reorthogonalization correction: p = c / gamma holds the
        // residual projections (FP32-dot error level, |p| << 1), so V_hi p in FP32
        // is accurate to |p| 2^-24 -- far below the FP64 rounding of v_j.  V r
        // carries the O(1) projections and cancels: double-float.
        float S1[2] = {0.f, 0.f}, S2[2] = {0.f, 0.f}, E2[2] = {0.f, 0.f};
        auto term = [&](const float2 &h, const ushort2 &m, int q) {
            const float a = ph[q], b = rh[q], bl = rl[q], bs = rs[q];
            S1[0] = fmaf(h.x, a, S1[0]);
            S1[1] = fmaf(h.y, a, S1[1]);
            df_term_t(S2[0], E2[0], h.x, lo16_unscaled(h.x, m.x), b, bl, bs);
            df_term_t(S2[1], E2[1], h.y, lo16_unscaled(h.y, m.y), b, bl, bs);
        };
        int q = 0;
        for (; q + 8 <= j; q += 8) {  // eight basis vectors' loads in flight (96 B per thread)
            float2 h[8];
            ushort2 l[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                h[t] = __ldg(Vh + (int64_t)(q + t) * ldv2 + i);
                l[t] = __ldg(Vm + (int64_t)(q + t) * ldv2 + i);
            }
#pragma unroll
            for (int t = 0; t < 8; t++) term(h[t], l[t], q + t);
        }
        for (; q + 4 <= j; q += 4) {
            float2 h[4];
            ushort2 l[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                h[t] = __ldg(Vh + (int64_t)(q + t) * ldv2 + i);
                l[t] = __ldg(Vm + (int64_t)(q + t) * ldv2 + i);
            }
#pragma unroll
            for (int t = 0; t < 4; t++) term(h[t], l[t], q + t);
        }
        for (; q < j; q++) term(__ldg(Vh + (int64_t)q * ldv2 + i), __ldg(Vm + (int64_t)q * ldv2 + i), q);
        const double2 u = wcol1[i], w = wcol[i];
        const double v0 = fma(k1, u.x, -widen_exact(S1[0]));
        const double v1 = fma(k1, u.y, -widen_exact(S1[1]));
        const double x0 = fma(k2, w.x, fma(-k3, u.x, -(widen_exact(S2[0]) + widen_exact(E2[0]))));
        const double x1 = fma(k2, w.y, fma(-k3, u.y, -(widen_exact(S2[1]) + widen_exact(E2[1]))));
        float vh0, vh1;
        unsigned short vm0, vm1;
        split_hi16(v0, vh0, vm0);
        split_hi16(v1, vh1, vm1);
        wcol[i] = make_double2(x0, x1);
        vh_out[i] = make_float2(vh0, vh1);
        vm_out[i] = make_ushort2(vm0, vm1);
        const float xh0 = hi_part(x0), xh1 = hi_part(x1);
        w32[i] = make_float2(xh0, xh1);
        nrm = fmaf(xh0, xh0, nrm);
        nrm = fmaf(xh1, xh1, nrm);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w2 = 0; w2 < kThreads / 32; w2++) s += red[w2];
        upart[bid] = s;
    }
}

// FP32 copy (hi part) of an FP64 vector, four rows per thread
__global__ void k_hi4(int64_t n4, const double2 *__restrict__ x, float4 *y) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += (int64_t)gridDim.x * kThreads) {
        const double2 a = x[2 * i], b = x[2 * i + 1];
        float h[4], l;
        split_pair(a.x, h[0], l);
        split_pair(a.y, h[1], l);
        split_pair(b.x, h[2], l);
        split_pair(b.y, h[3], l);
        y[i] = make_float4(h[0], h[1], h[2], h[3]);
    }
}

// start of a cycle: eta = beta = ||r||, g = beta e_1
__global__ void k_dcgs_start(Scal *sc, double *g, int m) {
    const double beta = sqrt(sc->r0);
    sc->beta = beta;
    sc->active = 1;
    sc->jdone = 0;
    sc->state = 0;
    g[0] = beta;
    for (int i = 1; i <= m; i++) g[i] = 0.0;
}

// u = V y over the first *nvec basis vectors, V kept as (hi, m16) pairs: the
// sums in double-float on the FP32 pipe (y split once per block), u in FP64.
__global__ void __launch_bounds__(kThreads)
k_gemv_basis(int64_t n, const float *__restrict__ Vh, const unsigned short *__restrict__ Vm, int64_t ldv,
             const int *nvec_dev, const double *__restrict__ y, double *u) {
    __shared__ float yh[kMaxRestart + 1], yl[kMaxRestart + 1], ys[kMaxRestart + 1];
    const int nv = *nvec_dev;
    for (int q = threadIdx.x; q < nv; q += kThreads) {
        split_pair(y[q], yh[q], yl[q]);
        ys[q] = yh[q] * kTail;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        float S = 0.0f, E = 0.0f;
        int q = 0;
        for (; q + 8 <= nv; q += 8) {  // eight vectors' loads in flight together, summed in order
            float h[8];
            unsigned short l[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                h[t] = __ldg(Vh + (int64_t)(q + t) * ldv + i);
                l[t] = __ldg(Vm + (int64_t)(q + t) * ldv + i);
            }
#pragma unroll
            for (int t = 0; t < 8; t++) df_term_t(S, E, h[t], lo16_unscaled(h[t], l[t]), yh[q + t], yl[q + t], ys[q + t]);
        }
        for (; q < nv; q++) {
            const float h = __ldg(Vh + (int64_t)q * ldv + i);
            df_term_t(S, E, h, lo16_unscaled(h, __ldg(Vm + (int64_t)q * ldv + i)), yh[q], yl[q], ys[q]);
        }
        u[i] = widen_exact(S) + widen_exact(E);
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

// The same back substitution for restart lengths up to kHsolveSmem, by one
// warp: the triangle of R and g staged in shared memory with one parallel
// load, the reciprocals of the diagonal formed in parallel, then a chain of
// one multiply and one FMA per row with no block barrier (the kernel above
// waits on a global load and a division at every row)
constexpr int kHsolveSmem = 64;
__global__ void __launch_bounds__(32) k_hsolve_warp(const double *H, const double *g, double *y, int m, Scal *sc) {
    __shared__ double rs[kHsolveSmem * kHsolveSmem], rinv[kHsolveSmem], sv[kHsolveSmem];
    const int jd = sc->jdone, lane = threadIdx.x;
    for (int idx = lane; idx < jd * jd; idx += 32) {
        const int c = idx / jd, r = idx - c * jd;
        rs[idx] = r <= c ? H[(int64_t)c * (m + 1) + r] : 0.0;
    }
    bool zero = false;
    for (int k = lane; k < jd; k += 32) {
        sv[k] = g[k];
        const double d = H[(int64_t)k * (m + 1) + k];
        zero |= d == 0.0;
        rinv[k] = d == 0.0 ? 0.0 : 1.0 / d;
    }
    if (__any_sync(0xffffffffu, zero) && lane == 0) sc->state = 2;
    __syncwarp();
    for (int i = jd - 1; i >= 0; i--) {
        const double yi = sv[i] * rinv[i];
        const double *ri = rs + i * jd;
        for (int k = lane; k < i; k += 32) sv[k] = fma(-ri[k], yi, sv[k]);
        if (lane == 0) y[i] = yi;
        __syncwarp();
    }
}

// ---- BiCGSTAB kernels ---------------------------------------------------------
__global__ void k_bicg_init(Scal *sc) {  // r0 holds ||r||^2 of the (re)start residual
    sc->rho_old = sc->alpha = sc->omega = 1.0;
    sc->active = 1;
    sc->state = 0;
    sc->r2 = sc->r0;        // rho = (rh, r) with rh = r
    sc->r3 = sqrt(sc->r0);  // smallest residual norm of this recurrence
}


__global__ void k_bicg_p(int64_t n, const double *__restrict__ r, const double *__restrict__ v, double *p,
                         const Scal *sc) {
    if (sc->active == 0) return;
    const double beta = sc->beta_b, omega = sc->omega;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        p[i] = r[i] + beta * (p[i] - omega * v[i]);
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





// ---- fused BiCGSTAB steps ---------------------------------------------------
// The residual-side dot products are formed inside the vector updates that
// produce their operands, and each scalar step runs in the block that sums
// the per-block partials (fixed order), so an iteration reads s and r once
// and launches two reductions fewer.

// s = r - alpha v;  partial[b*3] = sum (s, s)
__global__ void __launch_bounds__(kThreads)
k_bicg_s_dot(int64_t n, const double *__restrict__ r, const double *__restrict__ v, double *s, const Scal *sc,
             double *partial) {
    if (sc->active == 0) return;
    const double alpha = sc->alpha;
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const double si = r[i] - alpha * v[i];
        s[i] = si;
        a = fma(si, si, a);
    }
    a = block_sum(a);
    if (threadIdx.x == 0) partial[blockIdx.x * 3] = a;
}

// x += alpha ph + omega sh;  r = s - omega t;  partial[b*3] = (r, r), [b*3+1] = (rh, r)
__global__ void __launch_bounds__(kThreads)
k_bicg_xr_dot(int64_t n, double *x, double *r, const double *__restrict__ ph, const double *__restrict__ sh,
              const double *__restrict__ s, const double *__restrict__ t, const double *__restrict__ rh,
              const Scal *sc, double *partial) {
    if (sc->active == 0) return;
    const double alpha = sc->alpha, omega = sc->omega;
    double a = 0.0, c = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        x[i] += alpha * ph[i] + omega * sh[i];
        const double ri = s[i] - omega * t[i];
        r[i] = ri;
        a = fma(ri, ri, a);
        c = fma(rh[i], ri, c);
    }
    a = block_sum(a);
    c = block_sum(c);
    if (threadIdx.x == 0) {
        partial[blockIdx.x * 3] = a;
        partial[blockIdx.x * 3 + 1] = c;
    }
}

// one block: sums nd columns of the partials into sc->r0, r1, then one scalar step
enum { kStepAlpha = 0, kStepCheckS = 1, kStepOmega = 2, kStepCheckR = 3 };
__global__ void __launch_bounds__(kThreads)
k_bicg_step(int step, int nd, const double *__restrict__ partial, int nb, Scal *sc, int remaining) {
    if (sc->active == 0) return;
    double q0 = 0.0, q1 = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) {
        q0 += partial[(int64_t)b * 3];
        if (nd > 1) q1 += partial[(int64_t)b * 3 + 1];
    }
    q0 = block_sum(q0);
    if (nd > 1) q1 = block_sum(q1);
    if (threadIdx.x != 0) return;
    sc->r0 = q0;
    sc->r1 = q1;
    if (step == kStepAlpha) {
        if (q0 == 0.0 || !isfinite(q0)) {
            sc->state = !isfinite(q0) ? 3 : 2;
            sc->active = 0;
            return;
        }
        sc->alpha = sc->rho / q0;
    } else if (step == kStepCheckS) {
        sc->jdone += 1;
        const double sn = sqrt(q0);
        if (!isfinite(sn)) { sc->state = 3; sc->active = 0; return; }
        if (sn <= sc->tolb) { sc->state = 4; sc->active = 0; }
    } else if (step == kStepOmega) {
        sc->omega = q0 == 0.0 ? 0.0 : q1 / q0;
    } else {  // check r; q1 = (rh, r) is the next rho
        sc->rho_old = sc->rho;
        sc->r2 = q1;
        const double rn = sqrt(q0);
        if (!isfinite(rn)) { sc->state = 3; sc->active = 0; return; }
        if (rn <= sc->tolb) { sc->state = 1; sc->active = 0; return; }
        if (sc->jdone >= remaining) { sc->active = 0; return; }
        // divergence guard: restart the recurrence from the current iterate once
        // the residual has grown four orders of magnitude above its minimum
        if (rn > 1e4 * sc->r3) { sc->state = 5; sc->active = 0; return; }
        sc->r3 = fmin(sc->r3, rn);
    }
}

// beta from rho = (rh, r) (sc->r2: the previous check step, or ||r||^2 at a restart)
__global__ void k_bicg_beta2(Scal *sc) {
    if (sc->active == 0) return;
    const double rho = sc->r2;
    sc->rho = rho;
    if (rho == 0.0 || sc->omega == 0.0 || !isfinite(rho)) {
        sc->state = !isfinite(rho) ? 3 : 2;
        sc->active = 0;
        return;
    }
    sc->beta_b = (rho / sc->rho_old) * (sc->alpha / sc->omega);
}

// ---- PCG kernels (Saad, Algorithm 9.1) ----------------------------------------------
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

// one block: the sum of the per-block partials (fixed order), then one scalar
// step of the iteration: alpha = rho / (p, q), the convergence test on
// ||r||^2, or beta = (r, z) / rho
enum { kPcgAlpha = 0, kPcgCheck = 1, kPcgBeta = 2 };
__global__ void __launch_bounds__(kThreads)
k_pcg_step(int step, const double *__restrict__ partial, int nb, Scal *sc, int remaining) {
    if (sc->active == 0) return;
    double q = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) q += partial[(int64_t)b * 3];
    q = block_sum(q);
    if (threadIdx.x != 0) return;
    sc->r0 = q;
    if (step == kPcgAlpha) {
        if (q == 0.0 || !isfinite(q)) {
            sc->state = isfinite(q) ? 2 : 3;
            sc->active = 0;
            return;
        }
        sc->alpha = sc->rho / q;
    } else if (step == kPcgCheck) {
        sc->jdone += 1;
        const double rn = sqrt(q);
        if (!isfinite(rn)) { sc->state = 3; sc->active = 0; return; }
        if (rn <= sc->tolb) { sc->state = 1; sc->active = 0; return; }
        if (sc->jdone >= remaining) sc->active = 0;
    } else {
        sc->beta_b = q / sc->rho;
        sc->rho = q;
    }
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

__global__ void k_bsub(int64_t n, const double *__restrict__ b, double *r) {
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        r[i] = b[i] - r[i];
}

cudaError_t residual(sait_ctx ctx, sait_mat A, const double *x, const double *b, double *r) {
    if (A->n > 0 && !A->force_csr && sell_ready(A, SAIT_F64)) {  // the SELL product, then r = b - A x
        cudaError_t e = launch_spmv(A, SAIT_F64, x, false, r, false, nullptr, ctx->stream);
        if (e != cudaSuccess) return e;
        launch_k(k_bsub, (unsigned)std::min<int64_t>(cdiv(A->n, kThreads), 8LL * ctx->num_sms), kThreads, 0,
                 ctx->stream, A->n, b, r);
        return cudaGetLastError();
    }
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
    DTemp<double> V, H, cs, sn, g, y, z, u, part;
    DTemp<float> V32, w32;      // the basis's hi parts; fl32(w) after pass 1
    DTemp<unsigned short> VM;  // the basis's m16 parts (see split_hi16)
    DTemp<Scal> scd;
    // rows padded to 16-byte vectors (n4 of them), and the columns' leading
    // dimension kColPad entries longer still: at power-of-two n the columns would
    // otherwise start at the same offset modulo every power of two up to n
    const int64_t n4 = (n + 3) / 4, ldv = 4 * n4 + kColPad;
    SAIT_CK(V.alloc((size_t)(m + 1) * ldv, s));
    SAIT_CK(V32.alloc((size_t)(m + 1) * ldv, s));
    SAIT_CK(VM.alloc((size_t)(m + 1) * ldv, s));
    SAIT_CK(w32.alloc((size_t)ldv, s));
    if (ldv > n) {  // the padding rows stay zero for the whole solve
        SAIT_CK(cudaMemset2DAsync(V.p + n, ldv * sizeof(double), 0, (ldv - n) * sizeof(double), m + 1, s));
        SAIT_CK(cudaMemset2DAsync(V32.p + n, ldv * sizeof(float), 0, (ldv - n) * sizeof(float), m + 1, s));
        SAIT_CK(cudaMemset2DAsync(VM.p + n, ldv * sizeof(unsigned short), 0, (ldv - n) * sizeof(unsigned short), m + 1, s));
        SAIT_CK(cudaMemsetAsync(w32.p + n, 0, (ldv - n) * sizeof(float), s));
    }
    SAIT_CK(H.alloc((size_t)(m + 1) * m, s));
    DTemp<double> R, coef, kk;
    SAIT_CK(R.alloc((size_t)(m + 1) * m, s));
    SAIT_CK(coef.alloc((size_t)2 * m + 2, s));
    SAIT_CK(kk.alloc(4, s));
    SAIT_CK(cs.alloc(m, s));
    SAIT_CK(sn.alloc(m, s));
    SAIT_CK(g.alloc(m + 1, s));
    SAIT_CK(y.alloc(m + 2, s));
    SAIT_CK(z.alloc(n, s));
    SAIT_CK(u.alloc(n, s));
    SAIT_CK(part.alloc((size_t)W.nb * 3, s));
    // DCGS2: dual dot sweep on one 1024-thread block per SM, partials column-major
    // (2m + 1 slots, leading dimension a multiple of 4, padding zero); update
    // sweep on up to 16 blocks of 256 per SM plus the Givens block
    const int nb_dot = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n4, kDotThreads), (int64_t)ctx->num_sms));
    const int ldp = (nb_dot + 3) / 4 * 4;
    const int nb_upd = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(2 * n4, kThreads), 16LL * ctx->num_sms));
    // per-warp sums of the dual sweep in dynamic shared memory (2j + 1 per warp)
    auto dot_smem = [](int j) { return (size_t)(kDotThreads / 32) * (2 * j + 1) * sizeof(float); };
    if (dot_smem(m) > 48 * 1024)
        SAIT_CK(cudaFuncSetAttribute(k_dcgs_dot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dot_smem(m)));
    DTemp<float> dpart, upart;
    SAIT_CK(dpart.alloc((size_t)(2 * m + 2) * ldp, s));
    SAIT_CK(cudaMemsetAsync(dpart.p, 0, (size_t)(2 * m + 2) * ldp * sizeof(float), s));
    SAIT_CK(upart.alloc((size_t)nb_upd, s));
    SAIT_CK(scd.alloc(1, s));
    SAIT_CK(cudaMemsetAsync(scd.p, 0, sizeof(Scal), s));
    W.partial = part.p;
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
        // r = b - A x -> column 0 (the first tentative vector, eta = beta = ||r||)
        SAIT_CK(residual(ctx, A, x, b, V.p));
        SAIT_CK(dots(ctx, W, n, 1, V.p, V.p, nullptr, nullptr, nullptr, nullptr, r0, nullptr));
        launch_k(k_dcgs_start, 1, 1, 0, s, sc, g.p, m);
        SAIT_CK(cudaGetLastError());
        SAIT_TRY(read_scal(ctx, sc, &hs));
        inf.rel_resid = hs.beta / bnorm;
        if (!std::isfinite(hs.beta)) { result = SAIT_ERR_NONFINITE; break; }
        if (inf.rel_resid <= tol) { result = SAIT_OK; break; }
        if (iters >= maxit) break;
        launch_k(k_hi4, egrid, kThreads, 0, s, n4, (const double2 *)V.p, (float4 *)w32.p);
        const int remaining = maxit - iters;
        const float4 *Vh4 = (const float4 *)V32.p;
        DcgsState S{dpart.p, ldp, upart.p, nb_upd, H.p, R.p, cs.p, sn.p, g.p, coef.p, kk.p, sc,
                    group_counter(ctx, SAIT_TIMER_ORTHO), m};
        auto ortho = [&](int j, int close) {
            double *wj = V.p + (size_t)j * ldv;
            const double2 *wn = (const double2 *)(close ? wj : V.p + (size_t)(j + 1) * ldv);
            ScopedTimer tm(ctx, SAIT_TIMER_ORTHO);
            S.calls = group_counter(ctx, SAIT_TIMER_ORTHO);  // counted only while this call is timed
            // each kernel may be scheduled while its predecessor drains
            (void)launch_pdl(k_dcgs_dot, nb_dot, kDotThreads, dot_smem(j), s, n4, Vh4, ldv / 4, j,
                             (const float4 *)w32.p, wn, S, close);
            if (!close)
                (void)launch_pdl(k_dcgs_update, 1 + nb_upd, kThreads, 0, s, 2 * n4, (const float2 *)V32.p,
                                 (const ushort2 *)VM.p, ldv / 2, j, (const double2 *)wj,
                                 (double2 *)(V.p + (size_t)(j + 1) * ldv), (float2 *)(V32.p + (size_t)j * ldv),
                                 (ushort2 *)(VM.p + (size_t)j * ldv), (float2 *)w32.p, upart.p, S, remaining);
            else
                (void)launch_pdl(k_dcgs_givens, 1, 32, 0, s, S, j, remaining);
        };
        for (int j = 0; j < m; j++) {
            double *wj = V.p + (size_t)j * ldv, *w = V.p + (size_t)(j + 1) * ldv;
            SAIT_TRY(precondition(ctx, P, wj, z.p, n, act));
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, z.p, false, w, false, act, s,
                                    group_counter(ctx, SAIT_TIMER_SPMV), true));
            }
            ortho(j, 0);
            SAIT_CK(cudaGetLastError());
            if ((j + 1) % poll == 0 || j + 1 == m) {
                SAIT_TRY(read_scal(ctx, sc, &hs));
                if (!hs.active) break;
            }
        }
        ortho(m, 1);  // the last column becomes final (no-op after an earlier stop)
        SAIT_CK(cudaGetLastError());
        SAIT_TRY(read_scal(ctx, sc, &hs));
        iters += hs.jdone;
        cycles++;
        if (hs.state == 3) { result = SAIT_ERR_NONFINITE; break; }
        if (m <= kHsolveSmem)
            launch_k(k_hsolve_warp, 1, 32, 0, s, (const double *)R.p, (const double *)g.p, y.p, m, sc);
        else
            launch_k(k_hsolve, 1, kThreads, 0, s, (const double *)R.p, (const double *)g.p, y.p, m, sc);
        launch_k(k_gemv_basis, egrid, kThreads, 0, s, n, (const float *)V32.p, (const unsigned short *)VM.p, ldv,
                 (const int *)&sc->jdone, (const double *)y.p, u.p);
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
        const unsigned vgrid = (unsigned)W.nb;  // the fused kernels write one partial per block
        for (int it = 0; it < remaining; it++) {
            launch_k(k_bicg_beta2, 1, 1, 0, s, sc);
            launch_k(k_bicg_p, egrid, kThreads, 0, s, n, r.p, v.p, p.p, sc);
            SAIT_TRY(precondition(ctx, P, p.p, ph.p, n, act));
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, ph.p, false, v.p, false, act, s,
                                    group_counter(ctx, SAIT_TIMER_SPMV)));
            }
            launch_k(k_dots, W.nb, kThreads, 0, s, n, 1, (const double *)rh.p, (const double *)v.p,
                     (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                     (const double *)nullptr, W.partial, act);
            launch_k(k_bicg_step, 1, kThreads, 0, s, (int)kStepAlpha, 1, (const double *)W.partial, W.nb, sc,
                     remaining);
            launch_k(k_bicg_s_dot, vgrid, kThreads, 0, s, n, (const double *)r.p, (const double *)v.p, sv.p,
                     (const Scal *)sc, W.partial);
            launch_k(k_bicg_step, 1, kThreads, 0, s, (int)kStepCheckS, 1, (const double *)W.partial, W.nb, sc,
                     remaining);
            launch_k(k_bicg_xhalf, egrid, kThreads, 0, s, n, x, ph.p, sc);
            launch_k(k_bicg_xhalf_done, 1, 1, 0, s, sc);
            SAIT_TRY(precondition(ctx, P, sv.p, sh.p, n, act));
            {
                ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
                SAIT_CK(launch_spmv(A, SAIT_F64, sh.p, false, t.p, false, act, s,
                                    group_counter(ctx, SAIT_TIMER_SPMV)));
            }
            launch_k(k_dots, W.nb, kThreads, 0, s, n, 2, (const double *)t.p, (const double *)t.p,
                     (const double *)t.p, (const double *)sv.p, (const double *)nullptr, (const double *)nullptr,
                     W.partial, act);
            launch_k(k_bicg_step, 1, kThreads, 0, s, (int)kStepOmega, 2, (const double *)W.partial, W.nb, sc,
                     remaining);
            launch_k(k_bicg_xr_dot, vgrid, kThreads, 0, s, n, x, r.p, (const double *)ph.p, (const double *)sh.p,
                     (const double *)sv.p, (const double *)t.p, (const double *)rh.p, (const Scal *)sc, W.partial);
            launch_k(k_bicg_step, 1, kThreads, 0, s, (int)kStepCheckR, 2, (const double *)W.partial, W.nb, sc,
                     remaining);
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
            launch_k(k_dots, W.nb, kThreads, 0, s, n, 1, (const double *)p.p, (const double *)q.p,
                     (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                     (const double *)nullptr, W.partial, act);
            launch_k(k_pcg_step, 1, kThreads, 0, s, (int)kPcgAlpha, (const double *)W.partial, W.nb, sc, (int)maxit);
            launch_k(k_pcg_xr, (unsigned)W.nb, kThreads, 0, s, n, x, r.p, (const double *)p.p, (const double *)q.p,
                     (const Scal *)sc, W.partial);
            launch_k(k_pcg_step, 1, kThreads, 0, s, (int)kPcgCheck, (const double *)W.partial, W.nb, sc, (int)maxit);
            SAIT_TRY(precondition(ctx, P, r.p, z.p, n, act));
            launch_k(k_dots, W.nb, kThreads, 0, s, n, 1, (const double *)r.p, (const double *)z.p,
                     (const double *)nullptr, (const double *)nullptr, (const double *)nullptr,
                     (const double *)nullptr, W.partial, act);
            launch_k(k_pcg_step, 1, kThreads, 0, s, (int)kPcgBeta, (const double *)W.partial, W.nb, sc, (int)maxit);
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
