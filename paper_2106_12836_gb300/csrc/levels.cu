// Level scheduling for the exact triangular solves and for ILU(0).
//
// The level of row i is 0 if it depends on no other row, else 1 + the largest
// level among the rows it depends on (columns j < i for a lower factor,
// j > i for an upper one).  Rows of one level are independent, so each level
// is one parallel launch.  Levels are found on the GPU by repeated in-place
// relaxation sweeps (monotone, so a sweep that changes nothing proves the
// fixed point), then rows are bucketed by level with a counting sort.
//
// These are the "exact triangular solvers" that SAIT replaces (Section 3.1)
// and the level-0 ILU factorisation that supplies SAIT's input (Section 4).
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace {

__global__ void k_level_sweep(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              int lower, int32_t *lev, int *changed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = 0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        if (lower ? j < i : j > i) {
            const int lj = *((volatile int32_t *)lev + j);
            l = max(l, lj + 1);
        }
    }
    if (l != lev[i]) {
        lev[i] = l;
        *changed = 1;
    }
}

__global__ void k_level_hist(int64_t n, const int32_t *__restrict__ lev, int32_t *hist, int *maxlev) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(&hist[lev[i]], 1);
    atomicMax(maxlev, lev[i]);
}

__global__ void k_level_scatter(int64_t n, const int32_t *__restrict__ lev, const int64_t *__restrict__ ptr,
                                int32_t *cursor, int32_t *rows) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = lev[i];
    rows[ptr[l] + atomicAdd(&cursor[l], 1)] = (int32_t)i;
}

// x_i = (b_i - sum_{j on the strict side} T_ij x_j) / T_ii, G lanes per row.
template <int G>
__global__ void __launch_bounds__(256)
k_trisolve_level(const int32_t *__restrict__ rows, int cnt, const int32_t *__restrict__ rp,
                 const int32_t *__restrict__ ci, const double *__restrict__ va, int lower,
                 const double *__restrict__ b, double *__restrict__ x) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = gid / G;
    const int lane = threadIdx.x & (G - 1);
    double s = 0.0, d = 0.0;
    int i = -1;
    if (r < cnt) {
        i = rows[r];
        for (int k = rp[i] + lane; k < rp[i + 1]; k += G) {
            const int j = ci[k];
            if (j == i) d = va[k];
            else s = fma(va[k], x[j], s);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if (r < cnt && lane == 0) x[i] = (b[i] - s) / d;
}

// ILU(0), IKJ order (Saad, Algorithm 10.4), one warp per row of a level.
// For each k < i in row i (ascending): a_ik /= a_kk, then a_ij -= a_ik a_kj for
// every j > k of row k that is also in row i's pattern.
__global__ void __launch_bounds__(256)
k_ilu0_level(const int32_t *__restrict__ rows, int cnt, const int32_t *__restrict__ rp,
             const int32_t *__restrict__ ci, const int32_t *__restrict__ dpos, double *a, int *err) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= cnt) return;  // uniform per warp
    const int i = rows[w];
    const int b = rp[i], e = rp[i + 1];
    for (int q = b; q < e; q++) {
        const int k = ci[q];
        if (k >= i) break;
        const double ukk = a[dpos[k]];
        if (ukk == 0.0 || !isfinite(ukk)) {
            if (lane == 0) atomicOr(err, 1);
            return;
        }
        const double aik = a[q] / ukk;
        __syncwarp();
        if (lane == 0) a[q] = aik;
        for (int f = dpos[k] + 1 + lane; f < rp[k + 1]; f += 32) {
            const int j = ci[f];
            int lo = b, hi = e - 1;  // binary search for j in row i
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int c = ci[mid];
                if (c == j) { a[mid] = fma(-aik, a[f], a[mid]); break; }
                if (c < j) lo = mid + 1; else hi = mid - 1;
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        const double d = a[dpos[i]];
        if (d == 0.0 || !isfinite(d)) atomicOr(err, 1);
    }
}

__global__ void k_diag_pos(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           int32_t *dpos, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = -1;
    for (int k = rp[i]; k < rp[i + 1]; k++)
        if (ci[k] == i) p = k;
    dpos[i] = p;
    if (p < 0) atomicOr(err, 2);
}

__global__ void k_lu_counts(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            int32_t *lc, int32_t *uc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = 1, u = 0;  // L stores its unit diagonal explicitly
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        if (ci[k] < i) l++;
        else u++;
    }
    lc[i] = l;
    uc[i] = u;
}

__global__ void k_lu_fill(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ a, const int64_t *__restrict__ lrp64,
                          const int64_t *__restrict__ urp64, int32_t *lrp, int32_t *lci, double *lva,
                          int32_t *urp, int32_t *uci, double *uva) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        lrp[n] = (int32_t)lrp64[n];
        urp[n] = (int32_t)urp64[n];
        return;
    }
    int64_t lo = lrp64[i], uo = urp64[i];
    lrp[i] = (int32_t)lo;
    urp[i] = (int32_t)uo;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        if (j < i) { lci[lo] = j; lva[lo] = a[k]; lo++; }
        else { uci[uo] = j; uva[uo] = a[k]; uo++; }
    }
    lci[lo] = (int32_t)i;
    lva[lo] = 1.0;
}

}  // namespace

void free_levels(LevelSchedule *L) {
    if (L->rows) cudaFree(L->rows);
    L->rows = nullptr;
    L->ptr.clear();
    L->nlev = 0;
}

sait_status build_levels(sait_ctx ctx, const int32_t *rp, const int32_t *ci, int64_t n, bool lower,
                         LevelSchedule *out) {
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    out->nlev = 0;
    out->ptr.assign(1, 0);
    if (n == 0) return SAIT_OK;
    DTemp<int32_t> lev;
    SAIT_CK(lev.alloc(n, s));
    SAIT_CK(cudaMemsetAsync(lev.p, 0, n * sizeof(int32_t), s));
    const unsigned grid = (unsigned)cdiv(n, 256);
    // Relaxation: in batches of 8 sweeps; the flag is reset before the last
    // sweep of a batch, so it reports whether that sweep changed anything.
    for (int64_t sweeps = 0;; sweeps += 8) {
        if (sweeps > n + 16) return ctx_fail(ctx, SAIT_ERR_CUDA, "level sweeps did not converge");
        for (int t = 0; t < 7; t++)
            launch_k(k_level_sweep, grid, 256, 0, s, n, rp, ci, lower, lev.p, ctx->d_word + 8);
        SAIT_CK(cudaMemsetAsync(ctx->d_word + 8, 0, sizeof(int), s));
        launch_k(k_level_sweep, grid, 256, 0, s, n, rp, ci, lower, lev.p, ctx->d_word + 8);
        SAIT_CK(cudaGetLastError());
        SAIT_CK(cudaMemcpyAsync(h, ctx->d_word + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaStreamSynchronize(s));
        if (h[0] == 0) break;
    }
    DTemp<int32_t> hist, cursor;
    SAIT_CK(hist.alloc(n, s));
    SAIT_CK(cursor.alloc(n, s));
    SAIT_CK(cudaMemsetAsync(hist.p, 0, n * sizeof(int32_t), s));
    SAIT_CK(cudaMemsetAsync(cursor.p, 0, n * sizeof(int32_t), s));
    SAIT_CK(cudaMemsetAsync(ctx->d_word + 9, 0, sizeof(int), s));
    launch_k(k_level_hist, grid, 256, 0, s, n, lev.p, hist.p, ctx->d_word + 9);
    SAIT_CK(cudaGetLastError());
    SAIT_CK(cudaMemcpyAsync(h + 1, ctx->d_word + 9, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    const int nlev = h[1] + 1;
    DTemp<int64_t> ptr;
    SAIT_CK(ptr.alloc(nlev + 1, s));
    SAIT_CK(scan_i32(hist.p, ptr.p, nlev, s));
    SAIT_CK(cudaMalloc((void **)&out->rows, n * sizeof(int32_t)));
    launch_k(k_level_scatter, grid, 256, 0, s, n, lev.p, ptr.p, cursor.p, out->rows);
    SAIT_CK(cudaGetLastError());
    std::vector<int64_t> hp(nlev + 1);
    SAIT_CK(cudaMemcpyAsync(hp.data(), ptr.p, (nlev + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    out->nlev = nlev;
    out->ptr.resize(nlev + 1);
    out->max_width = 0;
    for (int l = 0; l <= nlev; l++) out->ptr[l] = (int32_t)hp[l];
    for (int l = 0; l < nlev; l++) out->max_width = std::max(out->max_width, out->ptr[l + 1] - out->ptr[l]);
    return SAIT_OK;
}

cudaError_t launch_trisolve(const sait_mat_s *T, const LevelSchedule &lev, bool lower, const double *b,
                            double *x, cudaStream_t s) {
    const int G = std::min(T->lanes, 8);
    for (int l = 0; l < lev.nlev; l++) {
        const int cnt = lev.ptr[l + 1] - lev.ptr[l];
        const int32_t *rows = lev.rows + lev.ptr[l];
        const unsigned grid = (unsigned)cdiv((int64_t)cnt * G, 256);
        switch (G) {
            case 2: launch_k(k_trisolve_level<2>, grid, 256, 0, s, rows, cnt, T->rp, T->ci, T->va, lower, b, x); break;
            case 4: launch_k(k_trisolve_level<4>, grid, 256, 0, s, rows, cnt, T->rp, T->ci, T->va, lower, b, x); break;
            default: launch_k(k_trisolve_level<8>, grid, 256, 0, s, rows, cnt, T->rp, T->ci, T->va, lower, b, x); break;
        }
    }
    return cudaGetLastError();
}

extern "C" sait_status sait_ilu0(sait_ctx ctx, const sait_csr *A, sait_mat *L, sait_mat *U) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || !L || !U) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_ilu0: null argument");
    *L = *U = nullptr;
    ScopedTimer tm(ctx, SAIT_TIMER_ILU);
    sait_mat W = nullptr;  // validated working copy of A, overwritten with L\U
    SAIT_TRY(sait_mat_create_csr(ctx, A, &W));
    const int64_t n = W->n;
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    sait_status st = SAIT_OK;
    LevelSchedule lev;
    DTemp<int32_t> dpos, lc, uc;
    DTemp<int64_t> lrp, urp;
    sait_mat Lm = nullptr, Um = nullptr;
    const unsigned grid = (unsigned)cdiv(std::max<int64_t>(n, 1), 256);
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        st = ctx_cuda(ctx, e, what, __FILE__, __LINE__);
    };
    cudaError_t e = dpos.alloc(n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_word, 0, sizeof(int), s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 setup"); goto done; }
    if (n > 0) launch_k(k_diag_pos, grid, 256, 0, s, n, W->rp, W->ci, dpos.p, ctx->d_word);
    e = cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 diagonal"); goto done; }
    if (h[0]) { st = ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_ilu0: missing diagonal entry"); goto done; }
    st = build_levels(ctx, W->rp, W->ci, n, true, &lev);
    if (st != SAIT_OK) goto done;
    for (int l = 0; l < lev.nlev; l++) {
        const int cnt = lev.ptr[l + 1] - lev.ptr[l];
        launch_k(k_ilu0_level, (unsigned)cdiv((int64_t)cnt * 32, 256), 256, 0, s, 
            lev.rows + lev.ptr[l], cnt, W->rp, W->ci, dpos.p, W->va, ctx->d_word);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 factorisation"); goto done; }
    if (h[0]) { st = ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_ilu0: zero or non-finite pivot"); goto done; }
    // split into L (unit diagonal stored) and U
    e = lc.alloc(n, s);
    if (e == cudaSuccess) e = uc.alloc(n, s);
    if (e == cudaSuccess) e = lrp.alloc(n + 1, s);
    if (e == cudaSuccess) e = urp.alloc(n + 1, s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 split"); goto done; }
    if (n > 0) launch_k(k_lu_counts, grid, 256, 0, s, n, W->rp, W->ci, lc.p, uc.p);
    e = scan_i32(lc.p, lrp.p, n, s);
    if (e == cudaSuccess) e = scan_i32(uc.p, urp.p, n, s);
    {
        int64_t *h64 = (int64_t *)ctx->h_pinned;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64, lrp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64 + 1, urp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 split"); goto done; }
        st = mat_alloc(ctx, n, h64[0], &Lm);
        if (st == SAIT_OK) st = mat_alloc(ctx, n, h64[1], &Um);
        if (st != SAIT_OK) goto done;
    }
    launch_k(k_lu_fill, (unsigned)cdiv(n + 1, 256), 256, 0, s, n, W->rp, W->ci, W->va, lrp.p, urp.p, Lm->rp,
                                                         Lm->ci, Lm->va, Um->rp, Um->ci, Um->va);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 split"); goto done; }
    Lm->lanes = choose_lanes(n, Lm->nnz);
    Um->lanes = choose_lanes(n, Um->nnz);
    *L = Lm;
    *U = Um;
    Lm = Um = nullptr;
done:
    if (Lm) sait_mat_destroy(Lm);
    if (Um) sait_mat_destroy(Um);
    free_levels(&lev);
    cudaStreamSynchronize(s);
    sait_mat_destroy(W);
    return st;
}
