// Level scheduling for the exact triangular solves and for ILU(0).
//
// Row i depends on the rows j on the strict side of row i (j < i for a lower
// factor, j > i for an upper one).  Rows whose dependencies are all finished
// form the next level set and are independent of one another.  The level sets
// are found by a frontier sweep over the transposed dependency graph (Kahn's
// topological order): one launch per level processes the current frontier and
// releases its dependents, whose in-degree drops to zero, into the next one.
// ILU(0) is fused into that sweep (a row is factored in the launch of its
// level), so the factorisation costs one launch per level and O(nnz) work.
//
// These are the "exact triangular solvers" that SAIT replaces (Section 3.1)
// and the level-0 ILU factorisation that supplies SAIT's input (Section 4).
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace {

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

// ---- dependency graph and frontier sweep ----------------------------------------
__global__ void k_dep_count(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            int lower, int32_t *indeg, int32_t *tcnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        if (lower ? j < i : j > i) {
            c++;
            atomicAdd(tcnt + j, 1);
        }
    }
    indeg[i] = c;
}

__global__ void k_dep_fill(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           int lower, const int64_t *__restrict__ trp, int32_t *tfill, int32_t *tcol) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        if (lower ? j < i : j > i) tcol[trp[j] + atomicAdd(tfill + j, 1)] = (int32_t)i;
    }
}

// q[0] begin and q[1] end of the current level in `order`, q[2] append tail,
// q[3] number of levels found; lptr[l] = start of level l in `order`.
__global__ void k_front0(int64_t n, const int32_t *__restrict__ indeg, int32_t *order, int *q) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || indeg[i] != 0) return;
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(q + 2, __popc(act));
    base = __shfl_sync(act, base, leader);
    order[base + __popc(act & ((1u << lane) - 1u))] = (int32_t)i;
}

__global__ void k_front_init(int *q, int32_t *lptr) {
    q[0] = 0;
    q[1] = q[2];
    q[3] = q[2] > 0 ? 1 : 0;
    lptr[0] = 0;
    lptr[1] = q[2];
}


// ILU(0), IKJ order (Saad, Algorithm 10.4), for row i whose dependencies are
// final, from precomputed update triples (q, f, p): for each L entry q of row
// i (column k, ascending) a_iq /= a_kk, then a_p -= a_iq a_f for the entries
// f of U row k (past its diagonal) that match position p of row i.  The
// triples replace the pattern searches, so the chain of dependent loads per
// row is short; the fma chain per entry is the IKJ one.
__device__ __forceinline__ void ilu0_row_triples(int i, const int32_t *__restrict__ rp,
                                                 const int32_t *__restrict__ dpos, const int32_t *__restrict__ ldiag,
                                                 const int64_t *__restrict__ tp, const int3 *__restrict__ tr,
                                                 double *a, int *err) {
    const int b = rp[i], dq = dpos[i];
    int64_t t = tp[i];
    const int64_t te = tp[i + 1];
    for (int q = b; q < dq; q++) {
        const double ukk = a[ldiag[q]];
        if (ukk == 0.0 || !isfinite(ukk)) {
            atomicOr(err, 1);
            return;
        }
        const double aik = a[q] / ukk;
        a[q] = aik;
        for (; t < te; t++) {
            const int3 x = tr[t];
            if (x.x != q) break;
            a[x.z] = fma(-aik, a[x.y], a[x.z]);
        }
    }
    const double d = a[dq];
    if (d == 0.0 || !isfinite(d)) atomicOr(err, 1);
}

// Symbolic ILU(0) step, a thread per row: ldiag[q] = position of a_kk for the
// L entries q of row i (column k), and the triples (q, f, p) with ci[f] ==
// ci[p], f in U row k past its diagonal, p in row i past q.  Counts only
// (into cnt) when tr is null.
__global__ void k_ilu_triples(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const int32_t *__restrict__ dpos, int32_t *ldiag, const int64_t *__restrict__ tp,
                              int32_t *cnt, int3 *tr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = rp[i], e = rp[i + 1], dq = dpos[i];
    int64_t out = tr ? tp[i] : 0;
    int c = 0;
    for (int q = b; q < dq; q++) {
        const int k = ci[q];
        const int dk = dpos[k];
        if (!tr) ldiag[q] = dk;
        int p = q + 1;
        for (int f = dk + 1; f < rp[k + 1]; f++) {
            const int j = ci[f];
            while (p < e && ci[p] < j) p++;
            if (p < e && ci[p] == j) {
                if (tr) tr[out++] = make_int3(q, f, p);
                else c++;
            }
        }
    }
    if (!tr) cnt[i] = c;
}

// One level, a thread per frontier row: factor it (ILU) from its triples,
// then release its dependents; a dependent whose in-degree reaches zero joins
// the next level (one queue atomic per warp).  The last block to finish
// publishes the next level, so a level costs one launch.
template <bool ILU>
__global__ void __launch_bounds__(256)
k_front_step(int32_t *order, int *q, int32_t *lptr, unsigned *done_blocks, const int64_t *__restrict__ trp,
             const int32_t *__restrict__ tcol, int32_t *indeg, const int32_t *__restrict__ rp,
             const int32_t *__restrict__ dpos, const int32_t *__restrict__ ldiag, const int64_t *__restrict__ tp,
             const int3 *__restrict__ tr, double *a, int *err) {
    const int begin = q[0], end = q[1];
    const int lane = threadIdx.x & 31;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = begin + gt; r - lane < end; r += nt) {  // warp-uniform trip count
        const bool valid = r < end;
        const int i = valid ? order[r] : 0;
        if (ILU && valid) ilu0_row_triples(i, rp, dpos, ldiag, tp, tr, a, err);
        int64_t t = valid ? trp[i] : 0;
        const int64_t te = valid ? trp[i + 1] : 0;
        while (__any_sync(0xffffffffu, t < te)) {
            bool rel = false;
            int d = 0;
            if (t < te) {
                d = tcol[t];
                rel = atomicSub(indeg + d, 1) == 1;
                t++;
            }
            const unsigned m = __ballot_sync(0xffffffffu, rel);
            if (m) {
                const int leader = __ffs(m) - 1;
                int pos = 0;
                if (lane == leader) pos = atomicAdd(q + 2, __popc(m));
                pos = __shfl_sync(0xffffffffu, pos, leader);
                if (rel) order[pos + __popc(m & ((1u << lane) - 1u))] = d;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done_blocks, 1u) == gridDim.x - 1) {  // every block of this level is done
            __threadfence();
            const int tail = atomicAdd(q + 2, 0);
            q[0] = end;
            q[1] = tail;
            if (tail > end) {
                const int l = q[3] + 1;
                q[3] = l;
                lptr[l] = tail;
            }
            *done_blocks = 0;
            __threadfence();
        }
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

// Frontier sweep over the dependency graph of (rp, ci); fills `out` (level
// sets on the device, level pointers on the host) when given, and factors
// ILU(0) in place in `a` when `a` is given (err_word collects pivot errors).
sait_status frontier_schedule(sait_ctx ctx, const int32_t *rp, const int32_t *ci, int64_t n, bool lower,
                              const int32_t *dpos, double *a, int *err_word, LevelSchedule *out) {
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    if (out) {
        out->nlev = 0;
        out->ptr.assign(1, 0);
    }
    if (n == 0) return SAIT_OK;
    const unsigned grid = (unsigned)cdiv(n, 256);
    DTemp<int32_t> indeg, tcnt, order, lptr;
    DTemp<int64_t> trp;
    DTemp<int32_t> tcol;
    DTemp<int> q;
    SAIT_CK(indeg.alloc(n, s));
    SAIT_CK(tcnt.alloc(n, s));
    SAIT_CK(order.alloc(n, s));
    SAIT_CK(lptr.alloc(n + 2, s));
    SAIT_CK(trp.alloc(n + 1, s));
    SAIT_CK(q.alloc(4, s));
    SAIT_CK(cudaMemsetAsync(tcnt.p, 0, n * sizeof(int32_t), s));
    SAIT_CK(cudaMemsetAsync(q.p, 0, 4 * sizeof(int), s));
    launch_k(k_dep_count, grid, 256, 0, s, n, rp, ci, (int)lower, indeg.p, tcnt.p);
    SAIT_CK(scan_i32(tcnt.p, trp.p, n, s));
    int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
    SAIT_CK(cudaMemcpyAsync(h64, trp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    SAIT_CK(tcol.alloc(h64[0], s));
    SAIT_CK(cudaMemsetAsync(tcnt.p, 0, n * sizeof(int32_t), s));  // reused as fill cursors
    launch_k(k_dep_fill, grid, 256, 0, s, n, rp, ci, (int)lower, (const int64_t *)trp.p, tcnt.p, tcol.p);
    launch_k(k_front0, grid, 256, 0, s, n, (const int32_t *)indeg.p, order.p, q.p);
    launch_k(k_front_init, 1, 1, 0, s, q.p, lptr.p);
    SAIT_CK(cudaGetLastError());
    const bool ilu = a != nullptr;
    // ILU: the update triples of every row (symbolic, all rows in parallel)
    DTemp<int32_t> ldiag, tcnt2;
    DTemp<int64_t> tp;
    DTemp<int3> tr;
    if (ilu) {
        SAIT_CK(cudaMemcpyAsync(h, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaStreamSynchronize(s));
        SAIT_CK(ldiag.alloc(std::max<int64_t>(h[0], 1), s));
        SAIT_CK(tcnt2.alloc(n, s));
        SAIT_CK(tp.alloc(n + 1, s));
        launch_k(k_ilu_triples, grid, 256, 0, s, n, rp, ci, dpos, ldiag.p, (const int64_t *)nullptr, tcnt2.p,
                 (int3 *)nullptr);
        SAIT_CK(scan_i32(tcnt2.p, tp.p, n, s));
        SAIT_CK(cudaMemcpyAsync(h64 + 1, tp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaStreamSynchronize(s));
        SAIT_CK(tr.alloc(std::max<int64_t>(h64[1], 1), s));
        launch_k(k_ilu_triples, grid, 256, 0, s, n, rp, ci, dpos, ldiag.p, (const int64_t *)tp.p, tcnt2.p, tr.p);
        SAIT_CK(cudaGetLastError());
    }
    // few blocks: the level work is short and every block of a level meets at one counter
    const unsigned sgrid = (unsigned)std::min<int64_t>(cdiv(n, 256), (int64_t)ctx->num_sms * 2);
    DTemp<unsigned> done_blocks;
    SAIT_CK(done_blocks.alloc(1, s));
    SAIT_CK(cudaMemsetAsync(done_blocks.p, 0, sizeof(unsigned), s));
    // kBatch levels (one launch each) are captured once in a CUDA graph and
    // replayed until the frontier is empty; a level past the last one is a
    // no-op (empty frontier), so replaying whole batches is safe
    constexpr int kBatch = 32;
    cudaGraphExec_t gexec = nullptr;
    {
        cudaStream_t cs;
        SAIT_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        const int64_t launches0 = g_sait_launches;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int t = 0; t < kBatch; t++) {
                if (ilu)
                    launch_k(k_front_step<true>, sgrid, 256, 0, cs, order.p, q.p, lptr.p, done_blocks.p,
                             (const int64_t *)trp.p, (const int32_t *)tcol.p, indeg.p, rp, dpos,
                             (const int32_t *)ldiag.p, (const int64_t *)tp.p, (const int3 *)tr.p, a, err_word);
                else
                    launch_k(k_front_step<false>, sgrid, 256, 0, cs, order.p, q.p, lptr.p, done_blocks.p,
                             (const int64_t *)trp.p, (const int32_t *)tcol.p, indeg.p, rp, dpos,
                             (const int32_t *)nullptr, (const int64_t *)nullptr, (const int3 *)nullptr, a, err_word);
            }
            cudaError_t e1 = cudaGetLastError();
            e = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
        }
        g_sait_launches = launches0;  // captured, not executed
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            if (gexec) cudaGraphExecDestroy(gexec);
            return ctx_cuda(ctx, e, "frontier graph", __FILE__, __LINE__);
        }
    }
    sait_status st = SAIT_OK;
    for (int64_t batch = 0;; batch++) {
        if (batch * kBatch > n + 64) {
            st = ctx_fail(ctx, SAIT_ERR_CUDA, "level schedule did not terminate");
            break;
        }
        cudaError_t e = cudaGraphLaunch(gexec, s);
        g_sait_launches += kBatch;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, q.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = ctx_cuda(ctx, e, "frontier sweep", __FILE__, __LINE__);
            break;
        }
        if (h[0] == h[1]) break;  // empty frontier: every row is scheduled
    }
    cudaGraphExecDestroy(gexec);
    if (st != SAIT_OK) return st;
    if (h[1] != n) return ctx_fail(ctx, SAIT_ERR_CUDA, "level schedule lost rows");
    if (out) {
        const int nlev = h[3];
        out->nlev = nlev;
        out->ptr.resize(nlev + 1);
        SAIT_CK(cudaMemcpyAsync(out->ptr.data(), lptr.p, (nlev + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaMalloc((void **)&out->rows, n * sizeof(int32_t)));
        SAIT_CK(cudaMemcpyAsync(out->rows, order.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        SAIT_CK(cudaStreamSynchronize(s));
        out->max_width = 0;
        for (int l = 0; l < nlev; l++) out->max_width = std::max(out->max_width, out->ptr[l + 1] - out->ptr[l]);
    }
    return SAIT_OK;
}

sait_status build_levels(sait_ctx ctx, const int32_t *rp, const int32_t *ci, int64_t n, bool lower,
                         LevelSchedule *out) {
    return frontier_schedule(ctx, rp, ci, n, lower, nullptr, nullptr, nullptr, out);
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
    SAIT_TRY(mat_copy_csr(ctx, A, &W));
    const int64_t n = W->n;
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    sait_status st = SAIT_OK;
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
    e = cudaMemsetAsync(ctx->d_word, 0, sizeof(int), s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_ilu0 setup"); goto done; }
    st = frontier_schedule(ctx, W->rp, W->ci, n, true, dpos.p, W->va, ctx->d_word, nullptr);
    if (st != SAIT_OK) goto done;
    e = cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s);
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
        int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
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
    cudaStreamSynchronize(s);
    sait_mat_destroy(W);
    return st;
}
