// Level scheduling for the exact triangular solves and for ILU(0).
//
// Row i depends on the rows j on the strict side of row i (j < i for a lower
// factor, j > i for an upper one).  Rows whose dependencies are all finished
// form the next level set and are independent of one another.  The level sets
// are found by a frontier sweep over the transposed dependency graph (Kahn's
// topological order): one launch per level processes the current frontier and
// releases its dependents, whose in-degree drops to zero, into the next one.
//
// These are the "exact triangular solvers" that SAIT replaces (Section 3.1),
// and the same sweep factors ILU(0) and ILU(1), SAIT's input (Section 4): a
// row is factored in the launch of its level, so the factorisation costs one
// launch per level and O(nnz) work.
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

// Level 0: the rows without dependencies, appended to order[0 ..) with lcnt[0]
// as the tail (one atomic per warp).
__global__ void k_front0(int64_t n, const int32_t *__restrict__ indeg, int32_t *order, int32_t *lcnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || indeg[i] != 0) return;
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(lcnt, __popc(act));
    base = __shfl_sync(act, base, leader);
    order[base + __popc(act & ((1u << lane) - 1u))] = (int32_t)i;
}

// Symbolic ILU step on a fixed pattern, a thread per row: ldiag[q] = position
// of u_kk for the L entries q of row i (column k), and the update triples
// (q, f, p) with ci[f] == ci[p], f in U row k past its diagonal, p in row i
// past q, ordered by q then f (the IKJ order).  Counts only (into cnt) when tr
// is null.
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

// kLuG lanes per row: each lane takes one entry per round, its position in L or
// U is the count of the group's earlier L or U entries (a ballot), so the row's
// order is kept and its loads are in flight together
constexpr int kLuG = 8;
__global__ void k_lu_fill(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ a, const int64_t *__restrict__ lrp64,
                          const int64_t *__restrict__ urp64, int32_t *lrp, int32_t *lci, double *lva,
                          int32_t *urp, int32_t *uci, double *uva) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kLuG;
    const int sub = threadIdx.x & (kLuG - 1);
    const unsigned gmask = ((1u << kLuG) - 1u) << ((threadIdx.x & 31) & ~(kLuG - 1));
    if (i > n) return;  // whole groups leave together
    if (i == n) {
        if (sub == 0) {
            lrp[n] = (int32_t)lrp64[n];
            urp[n] = (int32_t)urp64[n];
        }
        return;
    }
    const int64_t lo = lrp64[i], uo = urp64[i];
    if (sub == 0) {
        lrp[i] = (int32_t)lo;
        urp[i] = (int32_t)uo;
    }
    const unsigned below = (1u << sub) - 1u;
    const int shift = (threadIdx.x & 31) & ~(kLuG - 1);
    int lc = 0, uc = 0;
    for (int base = rp[i]; base < rp[i + 1]; base += kLuG) {
        const int k = base + sub;
        const bool valid = k < rp[i + 1];
        const int j = valid ? ci[k] : 0;
        const double v = valid ? a[k] : 0.0;
        const bool isl = valid && j < i, isu = valid && j >= i;
        const unsigned bl = (__ballot_sync(gmask, isl) >> shift) & ((1u << kLuG) - 1u);
        const unsigned bu = (__ballot_sync(gmask, isu) >> shift) & ((1u << kLuG) - 1u);
        if (isl) {
            const int64_t d = lo + lc + __popc(bl & below);
            lci[d] = j;
            lva[d] = v;
        }
        if (isu) {
            const int64_t d = uo + uc + __popc(bu & below);
            uci[d] = j;
            uva[d] = v;
        }
        lc += __popc(bl);
        uc += __popc(bu);
    }
    if (sub == 0) {
        lci[lo + lc] = (int32_t)i;
        lva[lo + lc] = 1.0;
    }
}

// ---- ILU(p), p = 0 or 1 -------------------------------------------------------------
// The factorisation (Saad, Algorithm 10.4 on a fixed pattern; Algorithm 10.5
// chooses the pattern) runs on the pattern S = A's pattern for ILU(0) and
// S = A's pattern plus the level-1 fill for ILU(1).  Level-1 fill of row i is
// {j : (i,k) and (k,j) in A's pattern, k < i, j > k}: the level of an entry
// depends only on levels already fixed, and for p = 1 only on A's pattern,
// so the rows of S are built independently.  Entries outside S are never
// pivots and never feed an entry of S, so eliminating on S gives the
// level-of-fill factors with the same fma chains.
constexpr int kIluThreads = 256;
constexpr int kIluCap = 512;               // candidate columns per row for the ILU(1) pattern
enum : int { kIluErrPivot = 1, kIluErrRow = 8 };

// ILU(1) pattern of row i, one warp: the columns of A's row i, then the strict U
// part of A's row k for every L column k, deduplicated and ranked.  Count pass
// (ci_s null): cnt[i] = |S_i|.  Fill pass: sorted columns, A's values (0 for
// fill) and the diagonal position.
__global__ void __launch_bounds__(kIluThreads)
k_ilu1_pattern(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
               const double *__restrict__ va, const int32_t *__restrict__ dpos, int32_t *cnt,
               const int64_t *__restrict__ rp_s, int32_t *ci_s, double *va_s, int32_t *dpos_s, int *err) {
    __shared__ int cand[kIluThreads / 32][kIluCap];
    __shared__ unsigned char first[kIluThreads / 32][kIluCap];
    const int lane = threadIdx.x & 31;
    int *C = cand[threadIdx.x >> 5];
    unsigned char *F = first[threadIdx.x >> 5];
    const int64_t i = ((int64_t)blockIdx.x * kIluThreads + threadIdx.x) >> 5;
    if (i >= n) return;
    const int b = rp[i], e = rp[i + 1], dq = dpos[i];
    int nc = e - b;
    bool over = nc > kIluCap;
    if (!over)
        for (int q = b + lane; q < e; q += 32) C[q - b] = ci[q];  // A's row first (unique, sorted)
    for (int q = b; q < dq && !over; q++) {  // then the strict U part of A's row k = ci[q]
        const int k = ci[q];
        const int fb = dpos[k] + 1, fe = rp[k + 1];
        if (nc + (fe - fb) > kIluCap) { over = true; break; }
        for (int f = fb + lane; f < fe; f += 32) C[nc + f - fb] = ci[f];
        nc += fe - fb;
    }
    __syncwarp();
    if (over) {
        if (lane == 0) atomicOr(err, kIluErrRow);
        return;
    }
    for (int x = lane; x < nc; x += 32) {  // first occurrence of its column?
        const int c = C[x];
        bool f = true;
        for (int y = 0; y < x && f; y++) f = C[y] != c;
        F[x] = f;
    }
    __syncwarp();
    int uniq = 0;
    for (int x = lane; x < nc; x += 32) {
        if (!F[x]) continue;
        uniq++;
        if (ci_s) {
            const int c = C[x];
            int rank = 0;  // distinct columns below c
            for (int y = 0; y < nc; y++) rank += F[y] && C[y] < c;
            const int64_t o = rp_s[i] + rank;
            ci_s[o] = c;
            va_s[o] = x < e - b ? va[b + x] : 0.0;
            if (c == (int)i) dpos_s[i] = (int32_t)o;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) uniq += __shfl_xor_sync(0xffffffffu, uniq, o);
    if (!ci_s && lane == 0) cnt[i] = uniq;
}

__global__ void k_i64_to_i32(int64_t n, const int64_t *__restrict__ in, int32_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = (int32_t)in[i];
}

struct IluNum {                // the numeric ILU of a level sweep (null a: no factorisation)
    const int32_t *dpos, *ldiag;  // diagonal position per row; position of u_kk per L entry
    const int64_t *tp;            // update triples of row i: tr[tp[i] .. tp[i+1])
    const int3 *tr;
    double *a;                    // values on the pattern, overwritten with L\U
    int *err;
};

// Row i of the factorisation, one thread, once the rows it depends on are
// final (earlier levels).  Every load of the row is issued before the
// arithmetic: the L entries, their pivots u_kk and the update triples with
// their u_kj.  When no update lands on an L position (the 5- and 7-point
// stencils with ILU(0)) the divisions a_ik / u_kk are independent and run
// together; then a_ij -= l_ik u_kj in (k, j) order, the IKJ fma chain of each
// entry.  Longer rows, and rows whose updates reach their own L part, run the
// IKJ loop entry by entry.  One thread per row keeps the FP64 work of a level
// off GB300's narrow FP64 pipe, which a warp per row (one lane busy in each
// FP64 instruction) had kept half occupied.
constexpr int kRowL = 4, kRowT = 4;

__device__ __forceinline__ void ilu_row_thread(int i, const int32_t *__restrict__ rp, const IluNum &F) {
    const int b = rp[i], dq = F.dpos[i];
    const int nl = dq - b;
    const int64_t t0 = F.tp[i];
    const int nt = (int)(F.tp[i + 1] - t0);
    double *a = F.a;
    bool fast = nl <= kRowL && nt <= kRowT;
    int3 tr[kRowT];
    double uf[kRowT], lv[kRowL], ukk[kRowL];
    if (fast) {
#pragma unroll
        for (int t = 0; t < kRowT; t++)
            if (t < nt) {
                tr[t] = F.tr[t0 + t];
                fast = fast && tr[t].z >= dq;
            }
    }
    if (fast) {
#pragma unroll
        for (int q = 0; q < kRowL; q++)
            if (q < nl) {
                lv[q] = a[b + q];
                ukk[q] = a[F.ldiag[b + q]];
            }
#pragma unroll
        for (int t = 0; t < kRowT; t++)
            if (t < nt) uf[t] = a[tr[t].y];
#pragma unroll
        for (int q = 0; q < kRowL; q++)
            if (q < nl) {
                lv[q] = lv[q] / ukk[q];  // l_ik = a_ik / u_kk
                a[b + q] = lv[q];
            }
#pragma unroll
        for (int t = 0; t < kRowT; t++)
            if (t < nt) {
                const int qq = tr[t].x - b;
                double l = lv[0];
#pragma unroll
                for (int q = 1; q < kRowL; q++) l = q == qq ? lv[q] : l;
                a[tr[t].z] = fma(-l, uf[t], a[tr[t].z]);  // a_ij -= l_ik u_kj
            }
    } else {
        int64_t t = t0;
        const int64_t te = t0 + nt;
        for (int q = b; q < dq; q++) {
            const double aik = a[q] / a[F.ldiag[q]];
            a[q] = aik;
            for (; t < te; t++) {
                const int3 y = F.tr[t];
                if (y.x != q) break;
                a[y.z] = fma(-aik, a[y.y], a[y.z]);
            }
        }
    }
    const double piv = a[dq];
    if (!(piv != 0.0) || !isfinite(piv)) atomicOr(F.err, kIluErrPivot);
}

// Level l of the sweep, a thread per row and role: level l is order[lptr[l] ..)
// with lcnt[l] rows (final when this launch starts).  Each row releases its
// dependents (kDep at a time, their atomics in flight together) and is
// factored (with F.a); a dependent whose in-degree reaches zero joins level
// l + 1 at a position from one atomic on lcnt[l + 1] per warp and round.  The
// row's factorisation and the releases are independent (the dependents run in
// a later launch), so they run in different warps at the same time.  Block 0
// publishes lptr[l + 1] for the next launch, so a level costs one launch and
// no hand-off between blocks.
constexpr int kDep = 8;

template <bool ILU>
__global__ void __launch_bounds__(kIluThreads, 4)
k_level(int l, int32_t *order, int32_t *lptr, int32_t *lcnt, const int64_t *__restrict__ trp,
        const int32_t *__restrict__ tcol, int32_t *indeg, const int32_t *__restrict__ rp, IluNum F) {
    pdl_wait();
    pdl_trigger();
    const int begin = lptr[l], cnt = lcnt[l];
    if (cnt == 0) return;
    const int next = begin + cnt;
    if (blockIdx.x == 0 && threadIdx.x == 0) lptr[l + 1] = next;
    const int lane = threadIdx.x & 31;
    // With ILU the warps come in pairs over the same 32 rows: the even warp
    // factors them, the odd one releases their dependents.  A thread's loads
    // wait behind its own atomics, so one thread doing both would serialise
    // the two round-trip chains; two warps run them side by side.
    const int64_t gw = ((int64_t)blockIdx.x * kIluThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kIluThreads) >> 5;
    const int64_t unit = ILU ? gw >> 1 : gw, nunits = ILU ? nwarps >> 1 : nwarps;
    const bool factor = ILU && !(gw & 1);
    for (int64_t r = unit * 32 + lane; r - lane < cnt; r += nunits * 32) {  // warp-uniform
        const bool valid = r < cnt;
        const int i = valid ? order[begin + r] : 0;
        if (factor) {
            if (valid) ilu_row_thread(i, rp, F);
            continue;
        }
        int64_t t = valid ? trp[i] : 0;
        const int64_t te = valid ? trp[i + 1] : 0;
        int dd[kDep];
        unsigned relm = 0;
        auto release = [&]() {
            relm = 0;
#pragma unroll
            for (int u = 0; u < kDep; u++) dd[u] = t + u < te ? tcol[t + u] : -1;
#pragma unroll
            for (int u = 0; u < kDep; u++)
                if (dd[u] >= 0 && atomicSub(indeg + dd[u], 1) == 1) relm |= 1u << u;
            t += kDep;
        };
        release();
        for (;;) {  // warp-uniform: append this round's released rows, then the next round
            const int c = __popc(relm);
            int incl = c;  // inclusive prefix of the released counts over the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total) {
                int base = 0;
                if (lane == 31) base = atomicAdd(lcnt + l + 1, total);
                base = __shfl_sync(0xffffffffu, base, 31) + incl - c;
#pragma unroll
                for (int u = 0; u < kDep; u++)
                    if (relm >> u & 1u) {
                        const int d = dd[u];
                        order[next + base++] = d;
                        // the next launch reads these first: have them in L2 by then
                        prefetch_l2(rp + d);
                        prefetch_l2(trp + d);
                        if (ILU) {
                            prefetch_l2(F.dpos + d);
                            prefetch_l2(F.tp + d);
                        }
                    }
            }
            if (!__any_sync(0xffffffffu, t < te)) break;
            release();
        }
    }
}

}  // namespace

void free_levels(LevelSchedule *L) {
    if (L->rows) cudaFree(L->rows);
    L->rows = nullptr;
    L->ptr.clear();
    L->nlev = 0;
}

// Level sweep over the dependency graph of (rp, ci): one launch of k_level per
// level (programmatic dependent launches, 32 per host check of the frontier).
// Fills `out` (level sets on the device, level pointers on the host) when
// given, and factors on the pattern when F.a is given.
sait_status level_sweep(sait_ctx ctx, const int32_t *rp, const int32_t *ci, int64_t n, bool lower,
                        const IluNum &F, LevelSchedule *out) {
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    if (out) {
        out->nlev = 0;
        out->ptr.assign(1, 0);
    }
    if (n == 0) return SAIT_OK;
    constexpr int kBatch = 32;
    const unsigned grid = (unsigned)cdiv(n, 256);
    const int64_t nl_cap = n + 2 * kBatch + 2;  // levels never exceed n
    DTemp<int32_t> indeg, tcnt, order, lptr, lcnt, tcol;
    DTemp<int64_t> trp;
    SAIT_CK(indeg.alloc(n, s));
    SAIT_CK(tcnt.alloc(n, s));
    SAIT_CK(order.alloc(n, s));
    SAIT_CK(lptr.alloc(nl_cap, s));
    SAIT_CK(lcnt.alloc(nl_cap, s));
    SAIT_CK(trp.alloc(n + 1, s));
    SAIT_CK(cudaMemsetAsync(tcnt.p, 0, n * sizeof(int32_t), s));
    SAIT_CK(cudaMemsetAsync(lcnt.p, 0, nl_cap * sizeof(int32_t), s));
    SAIT_CK(cudaMemsetAsync(lptr.p, 0, sizeof(int32_t), s));
    launch_k(k_dep_count, grid, 256, 0, s, n, rp, ci, (int)lower, indeg.p, tcnt.p);
    SAIT_CK(scan_i32(tcnt.p, trp.p, n, s));
    int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
    SAIT_CK(cudaMemcpyAsync(h64, trp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    SAIT_CK(tcol.alloc(std::max<int64_t>(h64[0], 1), s));
    SAIT_CK(cudaMemsetAsync(tcnt.p, 0, n * sizeof(int32_t), s));  // reused as fill cursors
    launch_k(k_dep_fill, grid, 256, 0, s, n, rp, ci, (int)lower, (const int64_t *)trp.p, tcnt.p, tcol.p);
    launch_k(k_front0, grid, 256, 0, s, n, (const int32_t *)indeg.p, order.p, lcnt.p);
    SAIT_CK(cudaGetLastError());
    const bool ilu = F.a != nullptr;
    int per_sm = 0;
    cudaError_t oe = ilu ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<true>, kIluThreads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_level<false>, kIluThreads, 0);
    if (oe != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const unsigned lgrid = (unsigned)std::min<int64_t>((int64_t)per_sm * ctx->num_sms, cdiv(n, kIluThreads));
    // kBatch levels per batch; the frontier check of batch b is read while batch
    // b + 1 runs (a batch past the last level is 32 no-op launches)
    auto launch_batch = [&](int l0) -> cudaError_t {
        for (int t = 0; t < kBatch; t++) {
            cudaError_t e = ilu ? launch_pdl(k_level<true>, lgrid, kIluThreads, 0, s, l0 + t, order.p, lptr.p,
                                             lcnt.p, (const int64_t *)trp.p, (const int32_t *)tcol.p, indeg.p, rp, F)
                                : launch_pdl(k_level<false>, lgrid, kIluThreads, 0, s, l0 + t, order.p, lptr.p,
                                             lcnt.p, (const int64_t *)trp.p, (const int32_t *)tcol.p, indeg.p, rp, F);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    int l0 = 0;
    cudaError_t le = launch_batch(0);
    for (;; l0 += kBatch) {
        if (le != cudaSuccess) return ctx_cuda(ctx, le, "level sweep", __FILE__, __LINE__);
        if (l0 > n) return ctx_fail(ctx, SAIT_ERR_CUDA, "level schedule did not terminate");
        SAIT_CK(cudaMemcpyAsync(h, lcnt.p + l0 + kBatch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        le = launch_batch(l0 + kBatch);  // runs while the host waits for the check
        SAIT_CK(cudaStreamSynchronize(s));
        if (h[0] == 0) break;  // empty frontier: every row is scheduled
    }
    l0 += kBatch;  // the batch launched last
    // level sizes: levels past the last one are empty
    std::vector<int32_t> cnts((size_t)l0 + kBatch + 1);
    SAIT_CK(cudaMemcpyAsync(cnts.data(), lcnt.p, cnts.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    int nlev = 0;
    int64_t rows = 0;
    while (nlev < (int)cnts.size() && cnts[nlev] > 0) rows += cnts[nlev++];
    if (rows != n) return ctx_fail(ctx, SAIT_ERR_CUDA, "level schedule lost rows");
    if (out) {
        out->nlev = nlev;
        out->ptr.resize(nlev + 1);
        out->ptr[0] = 0;
        out->max_width = 0;
        for (int l = 0; l < nlev; l++) {
            out->ptr[l + 1] = out->ptr[l] + cnts[l];
            out->max_width = std::max(out->max_width, cnts[l]);
        }
        SAIT_CK(cudaMalloc((void **)&out->rows, n * sizeof(int32_t)));
        SAIT_CK(cudaMemcpyAsync(out->rows, order.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        SAIT_CK(cudaStreamSynchronize(s));
    }
    return SAIT_OK;
}

sait_status build_levels(sait_ctx ctx, const int32_t *rp, const int32_t *ci, int64_t n, bool lower,
                         LevelSchedule *out) {
    return level_sweep(ctx, rp, ci, n, lower, IluNum{}, out);
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

extern "C" sait_status sait_iluk(sait_ctx ctx, const sait_csr *A, int32_t level, sait_mat *L, sait_mat *U) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || !L || !U || level < 0) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_iluk: bad argument");
    if (level > 1) return ctx_fail(ctx, SAIT_ERR_UNSUPPORTED, "sait_iluk: level of fill above 1");
    *L = *U = nullptr;
    ScopedTimer tm(ctx, SAIT_TIMER_ILU);
    sait_mat W = nullptr;  // validated working copy of A (ILU(0): overwritten with L\U)
    SAIT_TRY(mat_copy_csr(ctx, A, &W));
    const int64_t n = W->n, n1 = std::max<int64_t>(n, 1);
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);
    sait_status st = SAIT_OK;
    DTemp<int32_t> dpos, lc, uc, cnt, ldiag, rp_s, ci_s, dpos_s;
    DTemp<int64_t> lrp, urp, rp64, tp;
    DTemp<double> va_s;
    DTemp<int3> tr;
    DTemp<int> err;
    sait_mat Lm = nullptr, Um = nullptr;
    const int32_t *prp = W->rp, *pci = W->ci, *pdpos = nullptr;
    double *pva = W->va;
    int64_t nnz_s = W->nnz;
    const unsigned grid = (unsigned)cdiv(n1, 256);
    const unsigned wgrid = (unsigned)cdiv(n1 * 32, kIluThreads);  // a warp per row (ILU(1) pattern)
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        st = ctx_cuda(ctx, e, what, __FILE__, __LINE__);
    };
    cudaError_t e = dpos.alloc(n1, s);
    if (e == cudaSuccess) e = err.alloc(1, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, sizeof(int), s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_iluk setup"); goto done_; }
    if (n > 0) launch_k(k_diag_pos, grid, 256, 0, s, n, W->rp, W->ci, dpos.p, err.p);
    e = cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_iluk diagonal"); goto done_; }
    if (h[0]) { st = ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_iluk: missing diagonal entry"); goto done_; }
    pdpos = dpos.p;
    if (level == 1 && n > 0) {  // the ILU(1) pattern S, built row by row
        e = cnt.alloc(n1, s);
        if (e == cudaSuccess) e = rp64.alloc(n + 1, s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_iluk pattern"); goto done_; }
        launch_k(k_ilu1_pattern, wgrid, kIluThreads, 0, s, n, (const int32_t *)W->rp, (const int32_t *)W->ci,
                 (const double *)W->va, (const int32_t *)dpos.p, cnt.p, (const int64_t *)nullptr, (int32_t *)nullptr,
                 (double *)nullptr, (int32_t *)nullptr, err.p);
        e = scan_i32(cnt.p, rp64.p, n, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64, rp64.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_iluk pattern"); goto done_; }
        if (h[0]) { st = ctx_fail(ctx, SAIT_ERR_UNSUPPORTED, "sait_iluk: a row's level-1 candidates exceed 512"); goto done_; }
        nnz_s = h64[0];
        if (nnz_s > INT_MAX) { st = ctx_fail(ctx, SAIT_ERR_UNSUPPORTED, "sait_iluk: more than 2^31 entries"); goto done_; }
        e = rp_s.alloc(n + 1, s);
        if (e == cudaSuccess) e = ci_s.alloc(std::max<int64_t>(nnz_s, 1), s);
        if (e == cudaSuccess) e = va_s.alloc(std::max<int64_t>(nnz_s, 1), s);
        if (e == cudaSuccess) e = dpos_s.alloc(n1, s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_iluk pattern"); goto done_; }
        launch_k(k_i64_to_i32, (unsigned)cdiv(n + 1, 256), 256, 0, s, n, (const int64_t *)rp64.p, rp_s.p);
        launch_k(k_ilu1_pattern, wgrid, kIluThreads, 0, s, n, (const int32_t *)W->rp, (const int32_t *)W->ci,
                 (const double *)W->va, (const int32_t *)dpos.p, cnt.p, (const int64_t *)rp64.p, ci_s.p, va_s.p,
                 dpos_s.p, err.p);
        prp = rp_s.p;
        pci = ci_s.p;
        pva = va_s.p;
        pdpos = dpos_s.p;
    }
    if (n > 0) {  // update triples, then the level sweep with the numeric rows
        e = ldiag.alloc(std::max<int64_t>(nnz_s, 1), s);
        if (e == cudaSuccess) e = cnt.alloc(n1, s);
        if (e == cudaSuccess) e = tp.alloc(n + 1, s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_iluk triples"); goto done_; }
        launch_k(k_ilu_triples, grid, 256, 0, s, n, prp, pci, pdpos, ldiag.p, (const int64_t *)nullptr, cnt.p,
                 (int3 *)nullptr);
        e = scan_i32(cnt.p, tp.p, n, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h64 + 1, tp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = tr.alloc(std::max<int64_t>(h64[1], 1), s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_iluk triples"); goto done_; }
        launch_k(k_ilu_triples, grid, 256, 0, s, n, prp, pci, pdpos, ldiag.p, (const int64_t *)tp.p, cnt.p, tr.p);
        st = level_sweep(ctx, prp, pci, n, true, IluNum{pdpos, ldiag.p, tp.p, tr.p, pva, err.p}, nullptr);
        if (st != SAIT_OK) goto done_;
        e = cudaMemcpyAsync(h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { cuda_fail(e, "sait_iluk factorisation"); goto done_; }
        if (h[0] & kIluErrPivot) { st = ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_iluk: zero or non-finite pivot"); goto done_; }
        if (h[0]) { st = ctx_fail(ctx, SAIT_ERR_CUDA, "sait_iluk: factorisation failed"); goto done_; }
    }
    // split into L (unit diagonal stored) and U
    e = lc.alloc(n1, s);
    if (e == cudaSuccess) e = uc.alloc(n1, s);
    if (e == cudaSuccess) e = lrp.alloc(n + 1, s);
    if (e == cudaSuccess) e = urp.alloc(n + 1, s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_iluk split"); goto done_; }
    if (n > 0) launch_k(k_lu_counts, grid, 256, 0, s, n, prp, pci, lc.p, uc.p);
    e = scan_i32(lc.p, lrp.p, n, s);
    if (e == cudaSuccess) e = scan_i32(uc.p, urp.p, n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h64, lrp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h64 + 1, urp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_iluk split"); goto done_; }
    st = mat_alloc(ctx, n, h64[0], &Lm);
    if (st == SAIT_OK) st = mat_alloc(ctx, n, h64[1], &Um);
    if (st != SAIT_OK) goto done_;
    launch_k(k_lu_fill, (unsigned)cdiv((n + 1) * kLuG, 256), 256, 0, s, n, prp, pci, (const double *)pva, lrp.p, urp.p,
             Lm->rp, Lm->ci, Lm->va, Um->rp, Um->ci, Um->va);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cuda_fail(e, "sait_iluk split"); goto done_; }
    Lm->lanes = choose_lanes(n, Lm->nnz);
    Um->lanes = choose_lanes(n, Um->nnz);
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

extern "C" sait_status sait_ilu0(sait_ctx ctx, const sait_csr *A, sait_mat *L, sait_mat *U) {
    return sait_iluk(ctx, A, 0, L, U);
}
