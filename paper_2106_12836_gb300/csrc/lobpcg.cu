// LOBPCG with a SAIT preconditioner (Knyazev 2001; the block eigensolver of
// the paper's eigenvalue experiments, Section 4.4, where SAIT is applied to a
// block of vectors as two sparse matrix-matrix products).
//
// Blocks are row-major n x p FP64 arrays.  Per iteration:
//   R = A X - X diag(lambda); column residuals; soft locking of converged columns
//   W = T R(:, active)                    (sait_apply_multi: one pass over M_L, M_U)
//   W = W - X (X^T W); W = W L^{-T} with W^T W = L L^T      (Cholesky QR)
//   P(:, active), A P(:, active) orthonormalised the same way (dropped if singular)
//   Rayleigh-Ritz on S = [X W P]: G_A = S^T A S, G_B = S^T S (FP64), one-block
//   dense solve: Cholesky of G_B, C = L^{-1} G_A L^{-T}, parallel cyclic
//   Jacobi, coefficients L^{-T} Y(:, 0:k)
//   X = S c, A X = (A S) c, P = [W P] c(k:, :), A P likewise.
// The Gram matrices and block products keep ~48-bit accuracy in double-float
// arithmetic on the FP32 pipe (GB300's FP64 rate would bound them otherwise);
// the Rayleigh-Ritz solve itself runs in FP64 on the device.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int kT = 256;
constexpr int kMaxK = 20;           // block size limit (the Gram kernel holds <= 16 x 256 outputs)
constexpr int kMaxM = 3 * kMaxK;    // Rayleigh-Ritz size limit
constexpr int kRows = 32;           // rows per shared-memory tile of the Gram kernel

// partial[b][a*q + c] = sum over block b's rows of Y[i, a] Z[i, c], in
// double-float: the rows are staged in shared memory as (hi, lo) FP32 pairs
// and every product is accumulated with error-free two-sums, so the Gram
// entries keep ~48-bit accuracy while running on the FP32 pipe (FP64 FMAs
// would bound this kernel on GB300).  Each thread owns a 4 x 4 tile of
// outputs (16-byte shared loads, four products per loaded value) for one
// residue class of the staged rows; SYM forms only the tiles on or above the
// diagonal (the reduction mirrors them).  Phases are summed in a fixed order.
constexpr int kGramSmem = 32 * 1024;  // bytes of dynamic shared memory of k_gram

__device__ __forceinline__ float comp(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

template <bool SYM>
__global__ void __launch_bounds__(kT)
k_gram(int64_t n, int p, const double *__restrict__ Y, int64_t ldy, int q, const double *__restrict__ Z,
       int64_t ldz, double *partial) {
    extern __shared__ float4 smf4[];
    const int p4 = (p + 3) / 4, q4 = (q + 3) / 4;
    float4 *yh = smf4, *yl = yh + kRows * p4, *zh = yl + kRows * p4, *zl = zh + kRows * q4;
    const int nmt = SYM ? p4 * (p4 + 1) / 2 : p4 * q4;
    const int nph = kT / nmt;
    const int mt = threadIdx.x % nmt, ph = threadIdx.x / nmt;
    const bool active = ph < nph;
    int ta = 0, tc = 0;
    if (SYM) {
        int rem = mt;
        while (rem >= p4 - ta) {
            rem -= p4 - ta;
            ta++;
        }
        tc = ta + rem;
    } else {
        ta = mt / q4;
        tc = mt % q4;
    }
    float S[16], E[16];
#pragma unroll
    for (int t = 0; t < 16; t++) S[t] = E[t] = 0.0f;
    float *yhf = (float *)yh, *ylf = (float *)yl, *zhf = (float *)zh, *zlf = (float *)zl;
    for (int64_t r0 = (int64_t)blockIdx.x * kRows; r0 < n; r0 += (int64_t)gridDim.x * kRows) {
        const int rows = (int)min((int64_t)kRows, n - r0);
        for (int e = threadIdx.x; e < kRows * p4 * 4; e += kT) {
            const int r = e / (p4 * 4), a = e % (p4 * 4);
            split_pair(r < rows && a < p ? Y[(r0 + r) * ldy + a] : 0.0, yhf[e], ylf[e]);
        }
        for (int e = threadIdx.x; e < kRows * q4 * 4; e += kT) {
            const int r = e / (q4 * 4), c = e % (q4 * 4);
            split_pair(r < rows && c < q ? Z[(r0 + r) * ldz + c] : 0.0, zhf[e], zlf[e]);
        }
        __syncthreads();
        if (active) {
            for (int r = ph; r < kRows; r += nph) {
                const float4 ah = yh[r * p4 + ta], al = yl[r * p4 + ta];
                const float4 bh = zh[r * q4 + tc], bl = zl[r * q4 + tc];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        df_term(S[i * 4 + j], E[i * 4 + j], comp(ah, i), comp(al, i), comp(bh, j), comp(bl, j));
            }
        }
        __syncthreads();
    }
    double *red = (double *)smf4;  // nph x nmt x 16
    if (active)
#pragma unroll
        for (int t = 0; t < 16; t++) red[((int64_t)ph * nmt + mt) * 16 + t] = df_value(S[t], E[t]);
    __syncthreads();
    const int pq = p * q;
    for (int o = threadIdx.x; o < pq; o += kT) {
        const int a = o / q, c = o % q;
        double v = 0.0;
        if (!SYM || a <= c) {
            const int xa = a / 4, xc = c / 4;
            const int m2 = SYM ? xa * p4 - xa * (xa - 1) / 2 + (xc - xa) : xa * q4 + xc;
            const int t = (a % 4) * 4 + (c % 4);
            for (int f = 0; f < nph; f++) v += red[((int64_t)f * nmt + m2) * 16 + t];
        }
        partial[(int64_t)blockIdx.x * pq + o] = v;
    }
}

// G[o] = sum_b partial[b][o] (FP64, fixed order); sym: G[a][c] = G[c][a] for a > c
__global__ void k_gram_reduce(int nb, int p, int q, int sym, const double *__restrict__ partial, double *G) {
    const int pq = p * q;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= pq) return;
    const int a = o / q, c = o % q;
    const int src = (sym && a > c) ? c * q + a : o;
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += partial[(int64_t)b * pq + src];
    G[o] = s;
}

// Y (n x p, ldy) = (accumulate ? Y : 0) + sign * Z (n x q, ldz) C (q x p, row-major, ldc),
// each output accumulated in double-float on the FP32 pipe (C staged as
// (hi, lo) pairs, Z split on load) and rounded to FP64 once
__global__ void __launch_bounds__(kT)
k_block_mul(int64_t n, int q, const double *__restrict__ Z, int64_t ldz, int p, const double *__restrict__ C,
            int ldc, double *Y, int64_t ldy, int accumulate, double sign) {
    __shared__ float ch[kMaxM * 16], cl[kMaxM * 16];
    const int c0 = blockIdx.y * 16;  // output columns c0 .. c0+15
    const int pc = min(16, p - c0);
    for (int e = threadIdx.x; e < q * 16; e += kT) {
        const int a = e / 16, b = e % 16;
        split_pair(b < pc ? C[a * ldc + c0 + b] : 0.0, ch[e], cl[e]);
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
        float S[16], E[16];
#pragma unroll
        for (int b = 0; b < 16; b++) S[b] = E[b] = 0.0f;
        const double *zr = Z + i * ldz;
        for (int a = 0; a < q; a++) {
            float zh, zl;
            split_pair(zr[a], zh, zl);
#pragma unroll
            for (int b = 0; b < 16; b++) df_term(S[b], E[b], zh, zl, ch[a * 16 + b], cl[a * 16 + b]);
        }
        double *yr = Y + i * ldy + c0;
#pragma unroll
        for (int b = 0; b < 16; b++) {
            if (b < pc) {
                const double v = df_value(S[b], E[b]);
                yr[b] = accumulate ? yr[b] + sign * v : sign * v;
            }
        }
    }
}

// Y[:, dst_off + t] = Z[:, idx[t]] for t < cnt (column gather between blocks)
__global__ void k_gather_cols(int64_t n, int cnt, const int *__restrict__ idx, const double *__restrict__ Z,
                              int64_t ldz, double *Y, int64_t ldy, int dst_off) {
    const int64_t tot = n * cnt;
    for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < tot; e += (int64_t)gridDim.x * kT) {
        const int64_t i = e / cnt;
        const int t = (int)(e % cnt);
        Y[i * ldy + dst_off + t] = Z[i * ldz + idx[t]];
    }
}

// S = [X W P], AS = [AX AW AP] (row-major n x m, m = k + na + np) in one pass:
// strided 2D copies of 16-column blocks run row by row on the copy engines
// and cost milliseconds at this shape
__global__ void k_assemble(int64_t n, int k, int na, int np, const double *__restrict__ X,
                           const double *__restrict__ W, const double *__restrict__ P, const double *__restrict__ AX,
                           const double *__restrict__ AW, const double *__restrict__ AP, double *S, double *AS) {
    const int m = k + na + np;
    const int64_t tot = n * m;
    for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < tot; e += (int64_t)gridDim.x * kT) {
        const int64_t i = e / m;
        const int t = (int)(e - i * m);
        double a, b;
        if (t < k) {
            a = X[i * k + t];
            b = AX[i * k + t];
        } else if (t < k + na) {
            a = W[i * na + t - k];
            b = AW[i * na + t - k];
        } else {
            a = P[i * np + t - k - na];
            b = AP[i * np + t - k - na];
        }
        S[e] = a;
        AS[e] = b;
    }
}

// R = AX - X diag(lambda); partial sums of ||R_j||^2 and ||X_j||^2
__global__ void __launch_bounds__(kT)
k_residual_block(int64_t n, int k, const double *__restrict__ AX, const double *__restrict__ X,
                 const double *__restrict__ lam, double *R, double *partial) {
    __shared__ double red[2][kT];
    const int c = threadIdx.x % k;
    const int rpp = kT / k, r0 = threadIdx.x / k;
    double sr = 0.0, sx = 0.0;
    if ((int)threadIdx.x < rpp * k) {
        const double l = lam[c];
        for (int64_t i = (int64_t)blockIdx.x * rpp + r0; i < n; i += (int64_t)gridDim.x * rpp) {
            const int64_t e = i * k + c;
            const double x = X[e], r = AX[e] - l * x;
            R[e] = r;
            sr = fma(r, r, sr);
            sx = fma(x, x, sx);
        }
    }
    red[0][threadIdx.x] = sr;
    red[1][threadIdx.x] = sx;
    __syncthreads();
    if ((int)threadIdx.x < k) {
        double a = 0.0, b = 0.0;
        for (int rr = 0; rr < rpp; rr++) {
            a += red[0][rr * k + threadIdx.x];
            b += red[1][rr * k + threadIdx.x];
        }
        partial[(int64_t)blockIdx.x * 2 * k + threadIdx.x] = a;
        partial[(int64_t)blockIdx.x * 2 * k + k + threadIdx.x] = b;
    }
}

// residual norms, soft-locking list of active columns (ascending), count
__global__ void k_res_finish(int k, int nb, const double *__restrict__ partial, const double *__restrict__ lam,
                             double tol, double *res, int *active, int *nact) {
    __shared__ int flag[kMaxK];
    const int c = threadIdx.x;
    if (c < k) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nb; q++) {
            a += partial[(int64_t)q * 2 * k + c];
            b += partial[(int64_t)q * 2 * k + k + c];
        }
        const double rr = sqrt(a) / (fabs(lam[c]) * sqrt(b));
        res[c] = rr;
        flag[c] = (rr > tol || !isfinite(rr)) ? 1 : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int na = 0;
        for (int j = 0; j < k; j++)
            if (flag[j]) active[na++] = j;
        *nact = na;
    }
}

// ---- small dense kernels (one block) ---------------------------------------------
// In-place lower Cholesky of G (m x m, leading dimension ld) in shared memory,
// right-looking: per column one reciprocal square root on one thread, then the
// column scaled and the trailing block updated in parallel (a left-looking
// form ran length-j FP64 dot chains on one thread, 64 cycles per operation).
// Returns 1 when a pivot is not above 1e-14 of the largest diagonal entry.
__device__ int dev_chol(int m, double *G, int ld) {
    __shared__ int fail;
    __shared__ double mx, s_ir;
    if (threadIdx.x == 0) {
        fail = 0;
        mx = 0.0;
        for (int i = 0; i < m; i++) mx = fmax(mx, G[i * ld + i]);
    }
    __syncthreads();
    for (int j = 0; j < m; j++) {
        if (threadIdx.x == 0) {
            const double d = G[j * ld + j];
            if (!(d > 1e-14 * mx)) fail = 1;
            const double ir = d > 0.0 ? rsqrt(d) : 1.0;
            G[j * ld + j] = d > 0.0 ? d * ir : 1.0;
            s_ir = ir;
        }
        __syncthreads();
        const double ir = s_ir;
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) G[i * ld + j] *= ir;
        __syncthreads();
        const int r = m - j - 1;
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
            const int i = j + 1 + e / r, l = j + 1 + e % r;
            if (l <= i) G[i * ld + l] = fma(-G[i * ld + j], G[l * ld + j], G[i * ld + l]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x)
        if (e % m > e / m) G[(e / m) * ld + e % m] = 0.0;
    __syncthreads();
    return fail;
}

// R = L^{-1} (lower triangular; leading dimensions ldl, ldr), one column per
// thread, with the reciprocals of the diagonal formed once and each row's sum
// split in two chains
__device__ void dev_tri_inv(int m, const double *L, int ldl, double *R, int ldr) {
    __shared__ double dinv[kMaxM];
    for (int i = threadIdx.x; i < m; i += blockDim.x) dinv[i] = 1.0 / L[i * ldl + i];
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        for (int i = 0; i < m; i++) {
            if (i < j) {
                R[i * ldr + j] = 0.0;
                continue;
            }
            double s0 = (i == j) ? 1.0 : 0.0, s1 = 0.0;
            int q = j;
            for (; q + 1 < i; q += 2) {
                s0 = fma(-L[i * ldl + q], R[q * ldr + j], s0);
                s1 = fma(-L[i * ldl + q + 1], R[(q + 1) * ldr + j], s1);
            }
            if (q < i) s0 = fma(-L[i * ldl + q], R[q * ldr + j], s0);
            R[i * ldr + j] = (s0 + s1) * dinv[i];
        }
    __syncthreads();
}

// Cholesky-QR factor for a block, with the Gram matrix equilibrated first
// (columns of very different norms, e.g. residuals of nearly converged
// columns, would otherwise fail the relative pivot test):
// D = diag(G)^{-1/2}, D G D = L L^T, out (m x m) = D L^{-T}; flag on failure.
__global__ void k_cholqr_factor(int m, const double *__restrict__ G, double *out, int *flag) {
    extern __shared__ double sm[];
    double *Gs = sm, *Ri = sm + m * m;
    __shared__ double dsc[kMaxM];
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
        const double g = G[a * m + a];
        dsc[a] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Gs[e] = G[e] * dsc[e / m] * dsc[e % m];
    __syncthreads();
    int f = dev_chol(m, Gs, m);
    if (threadIdx.x == 0)
        for (int a = 0; a < m; a++) f |= dsc[a] == 0.0;
    dev_tri_inv(m, Gs, m, Ri, m);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int a = e / m, b = e % m;
        out[e] = dsc[a] * Ri[b * m + a];  // D L^{-T}
    }
    if (threadIdx.x == 0) *flag = f;
}

// Cyclic Jacobi on the symmetric me x me matrix C (me even; shared memory,
// leading dimension ld), with the rotations accumulated into V: in round-robin
// order, so every step rotates me/2 disjoint pairs at once.  A pair whose
// off-diagonal entry is at most thr is not rotated.  Stops once the
// off-diagonal norm is at most stop, or after max_sweeps sweeps.  rot holds me
// values of type F, pr me ints.  ld = me + 1 keeps the column updates (lanes
// on consecutive rows) on distinct shared-memory banks; with ld = 48 every
// lane of a warp hit the same bank.
template <typename F>
__device__ void jacobi_sweeps(int me, int ld, F *C, F *V, F *rot, int *pr, F stop, F thr, int max_sweeps) {
    __shared__ F offn;
    __shared__ F opart[kT / 32];
    const int np = me / 2;
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        F o = F(0);
        for (int e = threadIdx.x; e < me * me; e += kT) {
            const int a = e / me, b = e % me;
            if (a != b) o += C[a * ld + b] * C[a * ld + b];
        }
        for (int d = 16; d > 0; d >>= 1) o += __shfl_xor_sync(0xffffffffu, o, d);
        if ((threadIdx.x & 31) == 0) opart[threadIdx.x >> 5] = o;
        __syncthreads();
        if (threadIdx.x == 0) {
            F t = F(0);
            for (int w = 0; w < kT / 32; w++) t += opart[w];
            offn = sqrt(t);
        }
        __syncthreads();
        if (offn <= stop) break;  // uniform: every thread reads the same shared value
        for (int step = 0; step < me - 1; step++) {
            // round-robin pairs: position 0 fixed, the others rotate
            for (int t = threadIdx.x; t < np; t += kT) {
                const int pa = t, pb = me - 1 - t;
                const int p = pa == 0 ? 0 : ((pa - 1 + step) % (me - 1)) + 1;
                const int q = ((pb - 1 + step) % (me - 1)) + 1;
                const int lo = min(p, q), hi = max(p, q);
                pr[2 * t] = lo;
                pr[2 * t + 1] = hi;
                const F apq = C[lo * ld + hi];
                F c = F(1), sn = F(0);
                if (fabs(apq) > thr) {
                    // symmetric 2x2 Schur decomposition: t = tan of the angle,
                    // sign(d) 2 a / (|d| + sqrt(d^2 + 4 a^2)) with d = a_hh - a_ll
                    const F d = C[hi * ld + hi] - C[lo * ld + lo];
                    const F tt = (d >= F(0) ? F(2) : F(-2)) * apq / (fabs(d) + sqrt(d * d + F(4) * apq * apq));
                    c = rsqrt(F(1) + tt * tt);
                    sn = tt * c;
                }
                rot[2 * t] = c;
                rot[2 * t + 1] = sn;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < np * me; e += kT) {  // C <- C J, V <- V J (columns)
                const int t = e / me, r = e % me;
                const int p = pr[2 * t], q = pr[2 * t + 1];
                const F c = rot[2 * t], sn = rot[2 * t + 1];
                if (sn == F(0)) continue;
                F a = C[r * ld + p], b = C[r * ld + q];
                C[r * ld + p] = c * a - sn * b;
                C[r * ld + q] = sn * a + c * b;
                a = V[r * ld + p];
                b = V[r * ld + q];
                V[r * ld + p] = c * a - sn * b;
                V[r * ld + q] = sn * a + c * b;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < np * me; e += kT) {  // C <- J^T C (rows)
                const int t = e / me, r = e % me;
                const int p = pr[2 * t], q = pr[2 * t + 1];
                const F c = rot[2 * t], sn = rot[2 * t + 1];
                if (sn == F(0)) continue;
                const F a = C[p * ld + r], b = C[q * ld + r];
                C[p * ld + r] = c * a - sn * b;
                C[q * ld + r] = sn * a + c * b;
            }
            __syncthreads();
        }
    }
}

// Y = op(A) B for me x me matrices in shared memory (leading dimension ld;
// op(A) = A^T when ta), one output entry per thread and pass, each sum split
// in four chains (one FP64 operation every 64 cycles per chain otherwise)
__device__ void smem_gemm(int me, int ld, const double *A, bool ta, const double *B, double *Y) {
    for (int e = threadIdx.x; e < me * me; e += kT) {
        const int a = e / me, b = e % me;
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        int q = 0;
        if (ta) {
            for (; q + 3 < me; q += 4)
#pragma unroll
                for (int u = 0; u < 4; u++) s[u] = fma(A[(q + u) * ld + a], B[(q + u) * ld + b], s[u]);
            for (; q < me; q++) s[0] = fma(A[q * ld + a], B[q * ld + b], s[0]);
        } else {
            for (; q + 3 < me; q += 4)
#pragma unroll
                for (int u = 0; u < 4; u++) s[u] = fma(A[a * ld + q + u], B[(q + u) * ld + b], s[u]);
            for (; q < me; q++) s[0] = fma(A[a * ld + q], B[q * ld + b], s[0]);
        }
        Y[a * ld + b] = (s[0] + s[1]) + (s[2] + s[3]);
    }
    __syncthreads();
}

// Rayleigh-Ritz: generalized symmetric eigenproblem GA c = theta GB c (m x m);
// theta[0:k] ascending and coefficients c (m x k) = L^{-T} Y(:, 0:k); flag = 1
// if GB is not numerically positive definite.
//
// The reduced matrix C = L^{-1} GA L^{-T} is diagonalised by Jacobi rotations
// in two phases.  One block runs this kernel, and one SM issues about two FP64
// operations per clock on GB300, so FP64 sweeps from the start (each rotating
// every entry of C and V me - 1 times) took about 3 ms at m = 48.  The first
// sweeps therefore run in FP32 on a rounded copy, down to an off-diagonal norm
// of 1e-6 ||C||_F; their rotations Q are made orthonormal in FP64 by two
// Newton-Schulz steps Q <- Q (3 I - Q^T Q) / 2 (orthogonality error 1e-7, then
// ~1e-14, then rounding level), C becomes Q^T C Q in FP64, and FP64 sweeps
// finish the diagonalisation from there (two, by quadratic convergence), so
// the result has the accuracy of an all-FP64 Jacobi run.  Every shared matrix
// has a leading dimension one above its order (no bank conflicts in the
// column-wise passes).
__global__ void __launch_bounds__(kT) k_rayleigh_ritz(int m, int k, const double *__restrict__ GA,
                                                      const double *__restrict__ GB, double *theta, double *coef,
                                                      int *flag) {
    extern __shared__ double sm[];
    const int me = m + (m & 1);  // even size for the round-robin ordering
    const int lm = m + 1, ld = me + 1;
    double *L = sm;              // m x m (ld lm)
    double *Li = L + m * lm;     // m x m (ld lm)
    double *T = Li + m * lm;     // m x m (ld lm)
    double *C = T + m * lm;      // me x me (ld ld)
    double *V = C + me * ld;     // me x me
    double *W = V + me * ld;     // me x me scratch
    double *X = W + me * ld;     // me x me scratch (the FP32 copies of C and V during the FP32 sweeps)
    double *rot = X + me * ld;   // me/2 x 2 (c, s)
    int *pr = (int *)(rot + me); // me/2 x 2 pair indices
    float *C32 = (float *)X, *V32 = C32 + me * ld;
    __shared__ double fro;
    for (int e = threadIdx.x; e < m * m; e += kT) {
        const int a = e / m, b = e % m;
        L[a * lm + b] = 0.5 * (GB[a * m + b] + GB[b * m + a]);
        T[a * lm + b] = 0.5 * (GA[a * m + b] + GA[b * m + a]);
    }
    __syncthreads();
    const int f = dev_chol(m, L, lm);
    if (threadIdx.x == 0) *flag = f;
    if (f) return;  // uniform: f is read from shared memory by every thread
    dev_tri_inv(m, L, lm, Li, lm);
    // C = Li T Li^T (padded to me with a decoupled large diagonal entry)
    for (int e = threadIdx.x; e < m * m; e += kT) {
        const int a = e / m, b = e % m;
        double s0 = 0.0, s1 = 0.0;
        int q = 0;
        for (; q + 1 <= a; q += 2) {
            s0 = fma(Li[a * lm + q], T[q * lm + b], s0);
            s1 = fma(Li[a * lm + q + 1], T[(q + 1) * lm + b], s1);
        }
        if (q <= a) s0 = fma(Li[a * lm + q], T[q * lm + b], s0);
        V[a * ld + b] = s0 + s1;  // temporary: Li T
    }
    __syncthreads();
    for (int e = threadIdx.x; e < me * me; e += kT) {
        const int a = e / me, b = e % me;
        double s0 = 0.0, s1 = 0.0;
        if (a < m && b < m) {
            int q = 0;
            for (; q + 1 <= b; q += 2) {
                s0 = fma(V[a * ld + q], Li[b * lm + q], s0);
                s1 = fma(V[a * ld + q + 1], Li[b * lm + q + 1], s1);
            }
            if (q <= b) s0 = fma(V[a * ld + q], Li[b * lm + q], s0);
        }
        C[a * ld + b] = s0 + s1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < me * me; e += kT) {
        const int a = e / me, b = e % me;
        if (a < b) {
            const double sv = 0.5 * (C[a * ld + b] + C[b * ld + a]);
            C[a * ld + b] = sv;
            C[b * ld + a] = sv;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0, f2 = 0.0;
        for (int i = 0; i < m; i++) mx = fmax(mx, fabs(C[i * ld + i]));
        if (me > m) C[m * ld + m] = 10.0 * mx + 1.0;  // sorted last
        for (int i = 0; i < me; i++)
            for (int j = 0; j < me; j++) f2 += C[i * ld + j] * C[i * ld + j];
        fro = sqrt(f2);
    }
    __syncthreads();
    // FP32 sweeps on a rounded copy
    for (int e = threadIdx.x; e < me * me; e += kT) {
        const int a = e / me, b = e % me;
        C32[a * ld + b] = (float)C[a * ld + b];
        V32[a * ld + b] = a == b ? 1.0f : 0.0f;
    }
    __syncthreads();
    const float fro32 = (float)fro;
    jacobi_sweeps<float>(me, ld, C32, V32, (float *)rot, pr, 1e-6f * fro32, 1e-9f * fro32 / (float)me, 20);
    // Q = their rotations, orthonormalised in FP64 (two Newton-Schulz steps)
    for (int e = threadIdx.x; e < me * me; e += kT) {
        const int a = e / me, b = e % me;
        V[a * ld + b] = (double)V32[a * ld + b];
    }
    __syncthreads();
    for (int it = 0; it < 2; it++) {
        smem_gemm(me, ld, V, true, V, W);  // Q^T Q
        for (int e = threadIdx.x; e < me * me; e += kT) {
            const int a = e / me, b = e % me;
            W[a * ld + b] = (a == b ? 1.5 : 0.0) - 0.5 * W[a * ld + b];
        }
        __syncthreads();
        smem_gemm(me, ld, V, false, W, X);  // Q (3 I - Q^T Q) / 2
        for (int e = threadIdx.x; e < me * me; e += kT) {
            const int a = e / me, b = e % me;
            V[a * ld + b] = X[a * ld + b];
        }
        __syncthreads();
    }
    // C <- Q^T C Q, symmetrised
    smem_gemm(me, ld, C, false, V, W);
    smem_gemm(me, ld, V, true, W, X);
    for (int e = threadIdx.x; e < me * me; e += kT) {
        const int a = e / me, b = e % me;
        C[a * ld + b] = 0.5 * (X[a * ld + b] + X[b * ld + a]);
    }
    __syncthreads();
    // FP64 sweeps to the stopping level: a pair whose off-diagonal entry is
    // already below thr cannot matter at that level and is not rotated
    jacobi_sweeps<double>(me, ld, C, V, rot, pr, 1e-15 * fro, 1e-17 * fro / me, 40);
    // sort: rank of each eigenvalue (ties by index), then pick the k smallest
    __shared__ int order[kMaxM + 2];
    for (int i = threadIdx.x; i < me; i += kT) {
        const double wi = C[i * ld + i];
        int rank = 0;
        for (int j = 0; j < me; j++) {
            const double wj = C[j * ld + j];
            rank += (wj < wi) || (wj == wi && j < i);
        }
        order[rank] = i;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += kT) theta[j] = C[order[j] * ld + order[j]];
    // coef = Li^T V(:, order[0:k])  (rows 0..m-1)
    for (int e = threadIdx.x; e < m * k; e += kT) {
        const int a = e / k, j = e % k;
        const int col = order[j];
        double s = 0.0;
        for (int q = a; q < m; q++) s += Li[q * lm + a] * V[q * ld + col];
        coef[a * k + j] = s;
    }
}

struct LWork {
    int nb = 1;
    DTemp<double> partial, G, G2, F, coef, theta, res, rpart;
    DTemp<int> flag, active, nact;
};

// G = Y^T Z (p x q); sym when the result is known to be symmetric (Y^T Y, S^T A S)
sait_status gram(sait_ctx ctx, LWork &w, int64_t n, const double *Y, int p, int64_t ldy, const double *Z, int q,
                 int64_t ldz, double *G, bool sym = false) {
    if (sym && p == q)
        launch_k(k_gram<true>, (unsigned)w.nb, kT, (size_t)kGramSmem, ctx->stream, n, p, Y, ldy, q, Z, ldz,
                 w.partial.p);
    else
        launch_k(k_gram<false>, (unsigned)w.nb, kT, (size_t)kGramSmem, ctx->stream, n, p, Y, ldy, q, Z, ldz,
                 w.partial.p);
    launch_k(k_gram_reduce, (unsigned)cdiv(p * q, 256), 256, 0, ctx->stream, w.nb, p, q, (int)(sym && p == q),
             (const double *)w.partial.p, G);
    SAIT_CK(cudaGetLastError());
    return SAIT_OK;
}

sait_status bmul(sait_ctx ctx, int64_t n, const double *Z, int q, int64_t ldz, const double *C, int p, int ldc,
                 double *Y, int64_t ldy, bool accumulate, double sign) {
    if (p <= 0 || q <= 0 || n == 0) return SAIT_OK;
    dim3 grid((unsigned)std::min<int64_t>(cdiv(n, kT), (int64_t)ctx->num_sms * 8), (unsigned)cdiv(p, 16));
    launch_k(k_block_mul, grid, kT, 0, ctx->stream, n, q, Z, ldz, p, C, ldc, Y, ldy, (int)accumulate, sign);
    SAIT_CK(cudaGetLastError());
    return SAIT_OK;
}

// Y (n x p) <- Y L^{-T}, AY likewise when given; returns 1 in *failed if singular
sait_status cholqr(sait_ctx ctx, LWork &w, int64_t n, double *Y, double *AY, int p, double *tmp, int *failed) {
    SAIT_TRY(gram(ctx, w, n, Y, p, p, Y, p, p, w.G.p, true));
    launch_k(k_cholqr_factor, 1, kT, (size_t)2 * p * p * sizeof(double), ctx->stream, p, (const double *)w.G.p,
             w.F.p, w.flag.p);
    SAIT_CK(cudaGetLastError());
    int *h = (int *)ctx->h_pinned;
    SAIT_CK(cudaMemcpyAsync(h, w.flag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SAIT_CK(cudaStreamSynchronize(ctx->stream));
    *failed = h[0];
    if (h[0]) return SAIT_OK;
    SAIT_TRY(bmul(ctx, n, Y, p, p, w.F.p, p, p, tmp, p, false, 1.0));
    SAIT_CK(cudaMemcpyAsync(Y, tmp, (size_t)n * p * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    if (AY) {
        SAIT_TRY(bmul(ctx, n, AY, p, p, w.F.p, p, p, tmp, p, false, 1.0));
        SAIT_CK(cudaMemcpyAsync(AY, tmp, (size_t)n * p * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return SAIT_OK;
}

}  // namespace

extern "C" sait_status sait_lobpcg(sait_ctx ctx, sait_mat A, sait_prec P, int32_t k, double *X, double *lambda,
                                   double tol, int32_t maxit, sait_info *info) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || k < 1 || k > kMaxK || 3 * (int64_t)k > A->n || !X || !lambda || !(tol > 0.0) || maxit < 0 ||
        (P && P->kind != 1) || (P && P->n != A->n))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG,
                        "sait_lobpcg: bad argument (1 <= k <= 20, 3k <= n, P a SAIT pair or NULL)");
    const int64_t n = A->n;
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    const size_t nk = (size_t)n * k;
    LWork w;
    w.nb = (int)std::min<int64_t>(cdiv(n, kRows), 2LL * ctx->num_sms);
    const int mmax = 3 * k;
    DTemp<double> AX, R, W, AW, Pb, AP, S, AS, tmp, Wt;
    for (DTemp<double> *d : {&AX, &R, &W, &AW, &Pb, &AP, &tmp, &Wt}) SAIT_CK(d->alloc(nk, s));
    SAIT_CK(S.alloc(nk * 3, s));
    SAIT_CK(AS.alloc(nk * 3, s));
    SAIT_CK(w.partial.alloc((size_t)w.nb * mmax * mmax, s));
    SAIT_CK(w.G.alloc((size_t)mmax * mmax, s));
    SAIT_CK(w.G2.alloc((size_t)mmax * mmax, s));
    SAIT_CK(w.F.alloc((size_t)mmax * mmax, s));
    SAIT_CK(w.coef.alloc((size_t)mmax * k, s));
    SAIT_CK(w.theta.alloc(k, s));
    SAIT_CK(w.res.alloc(k, s));
    const int rnb = (int)std::min<int64_t>(cdiv(n, kT / k), 2LL * ctx->num_sms);
    SAIT_CK(w.rpart.alloc((size_t)rnb * 2 * k, s));
    SAIT_CK(w.flag.alloc(1, s));
    SAIT_CK(w.active.alloc(kMaxK, s));
    SAIT_CK(w.nact.alloc(1, s));
    const size_t rr_smem = (size_t)(3 * mmax * (mmax + 1) + 4 * (mmax + 1) * (mmax + 2)) * sizeof(double) +
                           (size_t)(mmax + 2) * sizeof(double) + (size_t)(mmax + 2) * sizeof(int) + 64;
    SAIT_CK(cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_smem));
    SAIT_CK(cudaFuncSetAttribute(k_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramSmem));
    SAIT_CK(cudaFuncSetAttribute(k_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGramSmem));
    auto spmm_a = [&](const double *Z, int p, double *Y) -> sait_status {
        ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
        SAIT_CK(launch_spmm(A, SAIT_F64, p, p, p, Z, false, Y, false, s, group_counter(ctx, SAIT_TIMER_SPMV)));
        return SAIT_OK;
    };
    auto rayleigh_ritz = [&](int m, const double *Sp, const double *ASp, int *failed) -> sait_status {
        SAIT_TRY(gram(ctx, w, n, Sp, m, m, ASp, m, m, w.G.p, true));   // A symmetric
        SAIT_TRY(gram(ctx, w, n, Sp, m, m, Sp, m, m, w.G2.p, true));
        launch_k(k_rayleigh_ritz, 1, kT, rr_smem, s, m, (int)k, (const double *)w.G.p, (const double *)w.G2.p,
                 w.theta.p, w.coef.p, w.flag.p);
        SAIT_CK(cudaGetLastError());
        SAIT_CK(cudaMemcpyAsync(h, w.flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaStreamSynchronize(s));
        *failed = h[0];
        return SAIT_OK;
    };
    sait_info inf{0, 0, 0, 0, 0.0};
    // initial Rayleigh-Ritz on span(X)
    int failed = 0;
    SAIT_TRY(cholqr(ctx, w, n, X, nullptr, k, tmp.p, &failed));
    if (failed) return ctx_fail(ctx, SAIT_ERR_BREAKDOWN, "sait_lobpcg: initial block is rank deficient");
    SAIT_TRY(spmm_a(X, k, AX.p));
    SAIT_TRY(rayleigh_ritz(k, X, AX.p, &failed));
    if (failed) return ctx_fail(ctx, SAIT_ERR_BREAKDOWN, "sait_lobpcg: initial Gram matrix singular");
    SAIT_TRY(bmul(ctx, n, X, k, k, w.coef.p, k, k, tmp.p, k, false, 1.0));
    SAIT_CK(cudaMemcpyAsync(X, tmp.p, nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SAIT_TRY(bmul(ctx, n, AX.p, k, k, w.coef.p, k, k, tmp.p, k, false, 1.0));
    SAIT_CK(cudaMemcpyAsync(AX.p, tmp.p, nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SAIT_CK(cudaMemcpyAsync(lambda, w.theta.p, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
    bool havep = false;
    sait_status result = SAIT_ERR_NOT_CONVERGED;
    std::vector<double> hres(k);
    for (int it = 0; it <= maxit; it++) {
        launch_k(k_residual_block, (unsigned)rnb, kT, 0, s, n, (int)k, (const double *)AX.p, (const double *)X,
                 (const double *)lambda, R.p, w.rpart.p);
        launch_k(k_res_finish, 1, 32 * (int)cdiv(k, 32), 0, s, (int)k, rnb, (const double *)w.rpart.p,
                 (const double *)lambda, tol, w.res.p, w.active.p, w.nact.p);
        SAIT_CK(cudaGetLastError());
        SAIT_CK(cudaMemcpyAsync(h, w.nact.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaMemcpyAsync(hres.data(), w.res.p, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaStreamSynchronize(s));
        const int na = h[0];
        inf.rel_resid = *std::max_element(hres.begin(), hres.end());
        if (!std::isfinite(inf.rel_resid)) { result = SAIT_ERR_NONFINITE; break; }
        if (na == 0) { result = SAIT_OK; break; }
        if (it == maxit) break;
        inf.iters = it + 1;
        // W = T R(:, active), orthogonalised against X, orthonormal
        const unsigned gg = (unsigned)std::min<int64_t>(cdiv(n * na, kT), (int64_t)ctx->num_sms * 16);
        launch_k(k_gather_cols, gg, kT, 0, s, n, na, (const int *)w.active.p, (const double *)R.p, (int64_t)k, Wt.p,
                 (int64_t)na, 0);
        if (P) SAIT_TRY(apply_multi_impl(ctx, P->lo, P->up, na, Wt.p, na, W.p, na, tmp.p));
        else SAIT_CK(cudaMemcpyAsync(W.p, Wt.p, (size_t)n * na * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SAIT_TRY(gram(ctx, w, n, X, k, k, W.p, na, na, w.G.p));                 // X^T W (k x na)
        SAIT_TRY(bmul(ctx, n, X, k, k, w.G.p, na, na, W.p, na, true, -1.0));    // W -= X (X^T W)
        SAIT_TRY(cholqr(ctx, w, n, W.p, nullptr, na, tmp.p, &failed));
        if (failed) { result = SAIT_ERR_BREAKDOWN; break; }
        SAIT_TRY(spmm_a(W.p, na, AW.p));
        int np = 0;
        if (havep) {  // P(:, active), A P(:, active)
            launch_k(k_gather_cols, gg, kT, 0, s, n, na, (const int *)w.active.p, (const double *)Pb.p, (int64_t)k,
                     Wt.p, (int64_t)na, 0);
            launch_k(k_gather_cols, gg, kT, 0, s, n, na, (const int *)w.active.p, (const double *)AP.p, (int64_t)k,
                     tmp.p, (int64_t)na, 0);
            SAIT_CK(cudaMemcpyAsync(Pb.p, Wt.p, (size_t)n * na * sizeof(double), cudaMemcpyDeviceToDevice, s));
            SAIT_CK(cudaMemcpyAsync(AP.p, tmp.p, (size_t)n * na * sizeof(double), cudaMemcpyDeviceToDevice, s));
            SAIT_TRY(cholqr(ctx, w, n, Pb.p, AP.p, na, tmp.p, &failed));
            np = failed ? 0 : na;
        }
        bool done = false;
        for (int attempt = 0; attempt < 2 && !done; attempt++) {
            const int m = k + na + np;
            // S = [X W P], AS = [AX AW AP] (row-major n x m)
            launch_k(k_assemble, (unsigned)std::min<int64_t>(cdiv(n * m, kT), (int64_t)ctx->num_sms * 16), kT, 0, s,
                     n, (int)k, na, np, (const double *)X, (const double *)W.p, (const double *)Pb.p,
                     (const double *)AX.p, (const double *)AW.p, (const double *)AP.p, S.p, AS.p);
            SAIT_CK(cudaGetLastError());
            SAIT_TRY(rayleigh_ritz(m, S.p, AS.p, &failed));
            if (failed) {
                if (np) { np = 0; continue; }  // drop P and retry
                result = SAIT_ERR_BREAKDOWN;
                break;
            }
            // X = S c, P = [W P] c(k:, :); A X and A P are formed by products with A
            // rather than as AS c: that is as cheap and keeps them from drifting away
            // from A X over the iterations (the residuals need them to ~1e-14 ||A||)
            SAIT_TRY(bmul(ctx, n, S.p, m, m, w.coef.p, k, k, X, k, false, 1.0));
            SAIT_TRY(bmul(ctx, n, S.p + k, na + np, m, w.coef.p + (size_t)k * k, k, k, Pb.p, k, false, 1.0));
            SAIT_TRY(spmm_a(X, k, AX.p));
            SAIT_TRY(spmm_a(Pb.p, k, AP.p));
            SAIT_CK(cudaMemcpyAsync(lambda, w.theta.p, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
            havep = true;
            done = true;
        }
        if (!done) break;
    }
    if (info) *info = inf;
    SAIT_CK(cudaStreamSynchronize(s));
    if (result != SAIT_OK) {
        char buf[160];
        snprintf(buf, sizeof(buf), "sait_lobpcg: %s after %d iterations, max residual %.3e", sait_status_string(result),
                 inf.iters, inf.rel_resid);
        return ctx_fail(ctx, result, buf);
    }
    return SAIT_OK;
}
