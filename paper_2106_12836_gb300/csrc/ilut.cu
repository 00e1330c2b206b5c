// ILUT(tau, lfil) on the GPU (Saad, Iterative Methods for Sparse Linear
// Systems, Algorithm 10.6): threshold ILU factors for SAIT (Section 4 feeds
// SAIT with level-0, level-1 and threshold ILU factors).
//
// Row i needs the finished U rows of every k it eliminates, and which k those
// are is only known while the row is being eliminated (fill creates new
// ones), so no level schedule can be computed in advance.  The kernel is
// therefore sync-free: persistent warps take rows in increasing order from an
// atomic ticket, and a warp that reaches column k of its row waits for the flag
// of row k.  Every row k < i was taken earlier by a running warp that itself
// waits only on smaller rows, so the waits always end; each is still bounded
// (kSpinLimit polls, or the context's wait limit), after which the kernel records a timeout and all warps
// leave.
//
// One warp holds its working row w in a shared-memory hash table (column ->
// value).  The elimination visits columns k < i in increasing order, found by
// a warp-wide minimum over the table, so fill-in created on the way is seen.
// For each k: w_k /= u_kk, the first dropping rule, then w_j = fma(-w_k, u_kj,
// w_j) with one lane per entry of U row k.  The same fma chain in the same
// order as the plain row-by-row algorithm gives bit-identical factors.  Then
// the second rule: entries below tau_i are dropped and the lfil largest of
// the L part and of the U part are kept (ties keep the smaller column).  Rows
// are written into fixed slots of lfil entries and compacted to CSR at the end.
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace {

constexpr int kWarps = 4;                 // warps per block
constexpr int kHash = 512;                // working-row slots per warp (power of two)
constexpr int kMaxFill = kHash / 2;       // entries of w beyond which the row is rejected
constexpr int kMaxLfil = 32;
constexpr long long kSpinLimit = 1LL << 22;  // polls of one dependency flag

enum : int { kErrPivot = 1, kErrFill = 2, kErrTimeout = 4 };

struct Slots {
    int32_t *lcol, *lcnt;
    double *lval;
    int32_t *ucol, *ucnt;
    double *uval, *udiag;
    int *done;
};

struct WarpSmem {
    int keys[kHash];
    double vals[kHash];
    int ckey[kHash / 2];
    double cval[kHash / 2];
    int kkey[kMaxLfil];
    double kval[kMaxLfil];
    int nfill;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ unsigned hash_of(int c) { return ((unsigned)c * 2654435761u) & (kHash - 1); }

// Slot of column c, claimed if absent (value 0).  -1 when the row is full.
__device__ int hash_insert(WarpSmem &S, int c) {
    unsigned h = hash_of(c);
    for (int probe = 0; probe < kHash; probe++) {
        const int old = atomicCAS(&S.keys[h], -1, c);
        if (old == c) return (int)h;
        if (old == -1) {
            if (atomicAdd(&S.nfill, 1) >= kMaxFill) return -1;
            return (int)h;
        }
        h = (h + 1) & (kHash - 1);
    }
    return -1;
}

__device__ int hash_find(const WarpSmem &S, int c) {
    unsigned h = hash_of(c);
    for (int probe = 0; probe < kHash; probe++) {
        const int k = S.keys[h];
        if (k == c) return (int)h;
        if (k == -1) return -1;
        h = (h + 1) & (kHash - 1);
    }
    return -1;
}

// Second dropping rule on one part: candidates are the slots whose column
// satisfies `part` (-1 lower, +1 upper relative to row i) with |w| >= tau_i
// and w != 0; the lfil largest are written, ascending by column, to
// col/val[0..cnt).  Returns cnt.
__device__ int keep_part(WarpSmem &S, int lane, int64_t i, int part, double tau_i, int lfil, int32_t *col,
                         double *val) {
    // compact the candidates
    int nc = 0;
    for (int base = 0; base < kHash; base += 32) {
        const int s = base + lane;
        const int c = S.keys[s];
        const double v = S.vals[s];
        const bool side = c >= 0 && (part < 0 ? c < i : c > i);
        const bool pred = side && v != 0.0 && fabs(v) >= tau_i;
        const unsigned m = __ballot_sync(0xffffffffu, pred);
        if (pred) {
            const int pos = nc + __popc(m & ((1u << lane) - 1u));
            S.ckey[pos] = c;
            S.cval[pos] = v;
        }
        nc += __popc(m);
    }
    __syncwarp();
    // rank by magnitude (ties: smaller column first); keep rank < lfil
    int nk = 0;
    for (int base = 0; base < nc; base += 32) {
        const int a = base + lane;
        bool keep = false;
        int ka = 0;
        double va = 0.0;
        if (a < nc) {
            ka = S.ckey[a];
            va = S.cval[a];
            const double ma = fabs(va);
            int rank = 0;
            for (int b = 0; b < nc && rank < lfil; b++) {
                const double mb = fabs(S.cval[b]);
                if (mb > ma || (mb == ma && S.ckey[b] < ka)) rank++;
            }
            keep = rank < lfil;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int pos = nk + __popc(m & ((1u << lane) - 1u));
            S.kkey[pos] = ka;
            S.kval[pos] = va;
        }
        nk += __popc(m);
    }
    __syncwarp();
    // write ascending by column
    if (lane < nk) {
        const int c = S.kkey[lane];
        int pos = 0;
        for (int b = 0; b < nk; b++) pos += S.kkey[b] < c;
        col[pos] = c;
        val[pos] = S.kval[lane];
    }
    __syncwarp();
    return nk;
}

// Waits (lane 0 polls, bounded) until row k is published.  Returns false on a
// timeout or when another warp reported an error.
__device__ bool wait_row(const int *done, int64_t k, int *err, int lane, long long limit) {
    int ok = 1;
    if (lane == 0) {
        long long polls = 0;
        unsigned ns = 32;
        while (ld_acquire(done + k) == 0) {
            if (ld_volatile(err) != 0) { ok = 0; break; }
            if (++polls > limit) {
                atomicOr(err, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(ns);
            if (ns < 256) ns <<= 1;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) (void)ld_acquire(done + k);  // every lane orders its reads of row k after the flag
    return ok != 0;
}

__global__ void __launch_bounds__(kWarps * 32)
k_ilut(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ va,
       double tau, int lfil, Slots out, unsigned long long *ticket, int *err, long long limit) {
    __shared__ WarpSmem smem[kWarps];
    const int lane = threadIdx.x & 31;
    WarpSmem &S = smem[threadIdx.x >> 5];
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = ld_volatile(err) ? (unsigned long long)n : atomicAdd(ticket, 1ULL);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)n) return;
        const int64_t i = (int64_t)t;
        // clear the working row
        for (int s = lane; s < kHash; s += 32) {
            S.keys[s] = -1;
            S.vals[s] = 0.0;
        }
        if (lane == 0) S.nfill = 0;
        __syncwarp();
        // w = a_i*, tau_i = tau ||a_i*||_2 (sum of squares in column order, no contraction)
        const int e0 = rp[i], e1 = rp[i + 1];
        bool full = false;
        for (int e = e0 + lane; e < e1; e += 32) {
            const int s = hash_insert(S, ci[e]);
            if (s < 0) full = true;
            else S.vals[s] = va[e];
        }
        __syncwarp();
        double tau_i = 0.0;
        if (lane == 0) {
            double ss = 0.0;
            for (int e = e0; e < e1; e++) ss = __dadd_rn(ss, __dmul_rn(va[e], va[e]));
            tau_i = __dmul_rn(tau, sqrt(ss));
            if (hash_insert(S, (int)i) < 0) full = true;  // the diagonal always has a slot
        }
        tau_i = __shfl_sync(0xffffffffu, tau_i, 0);
        __syncwarp();
        // elimination over k < i in increasing order
        int k = -1;
        for (;;) {
            if (__any_sync(0xffffffffu, full)) {
                if (lane == 0) atomicOr(err, kErrFill);
                return;
            }
            int best = INT_MAX, bslot = -1;
            for (int s = lane; s < kHash; s += 32) {
                const int c = S.keys[s];
                if (c > k && c < i && c < best) { best = c; bslot = s; }
            }
            const int m = __reduce_min_sync(0xffffffffu, best);
            if (m == INT_MAX) break;
            k = m;
            const unsigned who = __ballot_sync(0xffffffffu, best == m);
            const int slot = __shfl_sync(0xffffffffu, bslot, __ffs(who) - 1);
            double wk = S.vals[slot];
            if (wk == 0.0) continue;
            if (!wait_row(out.done, k, err, lane, limit)) return;
            wk = wk / __ldcg(out.udiag + k);
            __syncwarp();
            if (fabs(wk) < tau_i) {  // first dropping rule
                if (lane == 0) S.vals[slot] = 0.0;
                __syncwarp();
                continue;
            }
            if (lane == 0) S.vals[slot] = wk;
            const int cnt = __ldcg(out.ucnt + k);
            if (lane < cnt) {
                const int64_t f = k * (int64_t)lfil + lane;
                const int j = __ldcg(out.ucol + f);
                const double u = __ldcg(out.uval + f);
                const int s = hash_insert(S, j);
                if (s < 0) full = true;
                else S.vals[s] = fma(-wk, u, S.vals[s]);
            }
            __syncwarp();
        }
        // pivot
        const int ds = hash_find(S, (int)i);
        const double piv = ds >= 0 ? S.vals[ds] : 0.0;
        if (piv == 0.0 || !isfinite(piv)) {
            if (lane == 0) atomicOr(err, kErrPivot);
            return;
        }
        const int64_t off = i * (int64_t)lfil;
        const int nl = keep_part(S, lane, i, -1, tau_i, lfil, out.lcol + off, out.lval + off);
        const int nu = keep_part(S, lane, i, +1, tau_i, lfil, out.ucol + off, out.uval + off);
        if (lane == 0) {
            out.lcnt[i] = nl;
            out.ucnt[i] = nu;
            out.udiag[i] = piv;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(out.done + i, 1);
    }
}

__global__ void k_ilut_counts(int64_t n, const int32_t *__restrict__ lcnt, const int32_t *__restrict__ ucnt,
                              int32_t *lc, int32_t *uc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    lc[i] = lcnt[i] + 1;  // L stores its unit diagonal
    uc[i] = ucnt[i] + 1;  // U stores its pivot
}

__global__ void k_ilut_fill(int64_t n, int lfil, Slots in, const int64_t *__restrict__ lrp64,
                            const int64_t *__restrict__ urp64, int32_t *lrp, int32_t *lci, double *lva,
                            int32_t *urp, int32_t *uci, double *uva) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        lrp[n] = (int32_t)lrp64[n];
        urp[n] = (int32_t)urp64[n];
        return;
    }
    int64_t lo = lrp64[i], uo = urp64[i];
    lrp[i] = (int32_t)lo;
    urp[i] = (int32_t)uo;
    const int64_t off = i * (int64_t)lfil;
    for (int t = 0; t < in.lcnt[i]; t++, lo++) {
        lci[lo] = in.lcol[off + t];
        lva[lo] = in.lval[off + t];
    }
    lci[lo] = (int32_t)i;
    lva[lo] = 1.0;
    uci[uo] = (int32_t)i;
    uva[uo] = in.udiag[i];
    uo++;
    for (int t = 0; t < in.ucnt[i]; t++, uo++) {
        uci[uo] = in.ucol[off + t];
        uva[uo] = in.uval[off + t];
    }
}

}  // namespace

extern "C" sait_status sait_ilut(sait_ctx ctx, const sait_csr *A, double tau, int32_t lfil, sait_mat *L,
                                 sait_mat *U) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || !L || !U || !(tau >= 0.0) || lfil < 0) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_ilut: bad argument");
    if (lfil > kMaxLfil) return ctx_fail(ctx, SAIT_ERR_UNSUPPORTED, "sait_ilut: lfil above 32");
    *L = *U = nullptr;
    ScopedTimer tm(ctx, SAIT_TIMER_ILU);
    sait_mat W = nullptr;  // validated copy of A
    SAIT_TRY(mat_copy_csr(ctx, A, &W));
    const int64_t n = W->n;
    cudaStream_t s = ctx->stream;
    sait_status st = SAIT_OK;
    const int64_t n1 = std::max<int64_t>(n, 1), ns = std::max<int64_t>(n * (int64_t)lfil, 1);
    DTemp<int32_t> lcol, ucol, lcnt, ucnt, lc, uc;
    DTemp<double> lval, uval, udiag;
    DTemp<int> done, err;
    DTemp<unsigned long long> ticket;
    DTemp<int64_t> lrp, urp;
    sait_mat Lm = nullptr, Um = nullptr;
    int *h = (int *)ctx->h_pinned;
    Slots sl{};
    cudaError_t e = lcol.alloc(ns, s);
    if (e == cudaSuccess) e = ucol.alloc(ns, s);
    if (e == cudaSuccess) e = lval.alloc(ns, s);
    if (e == cudaSuccess) e = uval.alloc(ns, s);
    if (e == cudaSuccess) e = lcnt.alloc(n1, s);
    if (e == cudaSuccess) e = ucnt.alloc(n1, s);
    if (e == cudaSuccess) e = udiag.alloc(n1, s);
    if (e == cudaSuccess) e = done.alloc(n1, s);
    if (e == cudaSuccess) e = err.alloc(1, s);
    if (e == cudaSuccess) e = ticket.alloc(1, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(done.p, 0, n1 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket.p, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        st = ctx_cuda(ctx, e, "sait_ilut setup", __FILE__, __LINE__);
        goto done_;
    }
    sl = Slots{lcol.p, lcnt.p, lval.p, ucol.p, ucnt.p, uval.p, udiag.p, done.p};
    if (n > 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ilut, kWarps * 32, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        const int64_t blocks = std::min<int64_t>((int64_t)per_sm * ctx->num_sms, cdiv(n, kWarps));
        launch_k(k_ilut, (unsigned)blocks, kWarps * 32, 0, s, n, (const int32_t *)W->rp, (const int32_t *)W->ci,
                 (const double *)W->va, tau, (int)lfil, sl, ticket.p, err.p,
                 (long long)(ctx->wait_limit > 0 ? ctx->wait_limit : kSpinLimit));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = ctx_cuda(ctx, e, "sait_ilut factorisation", __FILE__, __LINE__);
            goto done_;
        }
        if (h[0] & kErrTimeout) {
            st = ctx_fail(ctx, SAIT_ERR_TIMEOUT, "sait_ilut: a row dependency wait ran out");
            goto done_;
        }
        if (h[0] & kErrFill) {
            st = ctx_fail(ctx, SAIT_ERR_UNSUPPORTED, "sait_ilut: a working row exceeded 256 entries");
            goto done_;
        }
        if (h[0] & kErrPivot) {
            st = ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_ilut: zero or non-finite pivot");
            goto done_;
        }
    }
    e = lc.alloc(n1, s);
    if (e == cudaSuccess) e = uc.alloc(n1, s);
    if (e == cudaSuccess) e = lrp.alloc(n + 1, s);
    if (e == cudaSuccess) e = urp.alloc(n + 1, s);
    if (e == cudaSuccess && n > 0)
        launch_k(k_ilut_counts, (unsigned)cdiv(n, 256), 256, 0, s, n, (const int32_t *)lcnt.p,
                 (const int32_t *)ucnt.p, lc.p, uc.p);
    if (e == cudaSuccess) e = scan_i32(lc.p, lrp.p, n, s);
    if (e == cudaSuccess) e = scan_i32(uc.p, urp.p, n, s);
    {
        int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64, lrp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64 + 1, urp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = ctx_cuda(ctx, e, "sait_ilut compaction", __FILE__, __LINE__);
            goto done_;
        }
        st = mat_alloc(ctx, n, h64[0], &Lm);
        if (st == SAIT_OK) st = mat_alloc(ctx, n, h64[1], &Um);
        if (st != SAIT_OK) goto done_;
    }
    launch_k(k_ilut_fill, (unsigned)cdiv(n + 1, 256), 256, 0, s, n, (int)lfil, sl, (const int64_t *)lrp.p,
             (const int64_t *)urp.p, Lm->rp, Lm->ci, Lm->va, Um->rp, Um->ci, Um->va);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        st = ctx_cuda(ctx, e, "sait_ilut compaction", __FILE__, __LINE__);
        goto done_;
    }
    *L = Lm;
    *U = Um;
    Lm = Um = nullptr;
done_:
    if (Lm) sait_mat_destroy(Lm);
    if (Um) sait_mat_destroy(Um);
    cudaStreamSynchronize(s);
    sait_mat_destroy(W);
    return st;
}
