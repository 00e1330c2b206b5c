// SAIT build (Algorithms 1-3): M = sum_{i < m_terms} T~^i D^-1 by the Horner
// recursion M_k D = T~ (M_{k-1} D) + I (equation Recursive), one sparse
// product per term with the dropping rule fused into the product kernel.
//
// Per product:
//   1. k_rowub      upper bound of each output row: 1 + sum_k nnz((M D)_k) over
//                   the columns k of T~'s row (or |S_i| when masked by a pattern);
//                   rows above kWarpMaxUb go to an overflow list;
//   2. scan         row slots of the output (int64 offsets, gaps allowed);
//   3. k_spgemm_warp one warp per row: shared-memory hash accumulator, products
//                   taken in ascending k with FP64 fma, +1 on the diagonal, drop
//                   rule, in-place compaction and a bitonic sort by column;
//      k_spgemm_dense one block per overflow row with a dense global accumulator
//                   and an ordered block compaction.
// The iterate keeps its gapped layout (offset + count per row) between
// products; the last product also applies the column scaling by D^-1, and a
// final pass compacts the rows into CSR.
//
// Every output value is the same chain of fma's as the oracle's dense
// accumulator (ascending k, starting from 0), so the FP64 values are
// reproduced bit for bit.
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace {

constexpr int kWarps = 8;                  // warps per block in k_spgemm_warp
constexpr int kHashCap = 512;              // hash slots per warp
constexpr int kWarpMaxUb = kHashCap / 2;   // rows whose bound exceeds this go to the dense kernel
constexpr int kDenseThreads = 256;

enum { kDropNone = 0, kDropAbs = 1, kDropRowRel = 2, kDropPattern = 3 };
enum { E_UNSORTED = 1, E_SIDE = 2, E_PIVOT = 4, E_HASH = 8 };

struct WarpSmem {
    int32_t keys[kHashCap];
    double vals[kHashCap];
    uint8_t touched[kHashCap];
};

// ---- step 1 of Algorithm 1: D^-1 and T~ = I - D^-1 T -----------------------
__global__ void k_split_check(int64_t n, const int32_t *__restrict__ rp,
                              const int32_t *__restrict__ ci, const double *__restrict__ va,
                              int lower, double *__restrict__ dinv, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = rp[i], e = rp[i + 1];
    int nd = 0, bits = 0;
    double d = 0.0;
    for (int k = b; k < e; k++) {
        const int c = ci[k];
        if (k > b && c <= ci[k - 1]) bits |= E_UNSORTED;
        if (c == i) { nd++; d = va[k]; }
        else if (lower ? c > i : c < i) bits |= E_SIDE;
    }
    if (nd != 1 || d == 0.0 || !isfinite(d)) bits |= E_PIVOT;
    else dinv[i] = 1.0 / d;
    if (bits) atomicOr(err, bits);
}

// Rows of T~ = rows of T without the diagonal; entry -(d_i^-1 T_ij).
__global__ void k_split_fill(int64_t n, const int32_t *__restrict__ rp,
                             const int32_t *__restrict__ ci, const double *__restrict__ va,
                             const double *__restrict__ dinv, int32_t *__restrict__ tt_rp,
                             int32_t *__restrict__ tt_ci, double *__restrict__ tt_va) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) { tt_rp[n] = rp[n] - (int32_t)n; return; }
    int o = rp[i] - (int)i;
    tt_rp[i] = o;
    const double di = dinv[i];
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        if (ci[k] == i) continue;
        tt_ci[o] = ci[k];
        tt_va[o] = -(di * va[k]);
        o++;
    }
}

// M D = I in the gapped layout.
__global__ void k_identity(int64_t n, int64_t *off, int32_t *cnt, int32_t *ci, double *va) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    off[i] = i;
    cnt[i] = 1;
    ci[i] = (int32_t)i;
    va[i] = 1.0;
}

// Row bins by the symbolic bound u (products + 1): 0: u <= 8, 1: u <= 16,
// 2: u <= 32 (register kernels, lanes hold one product each), 3: u <= kWarpMaxUb
// (shared-memory hash), 4: longer rows (dense accumulator).  Masked iterations
// of the pattern rule use the hash and dense kernels only.
constexpr int kBins = 5;

__global__ void k_rowub(int64_t n, const int32_t *__restrict__ tt_rp,
                        const int32_t *__restrict__ tt_ci, const int32_t *__restrict__ m_cnt,
                        int masked, const int32_t *__restrict__ s_cnt, int64_t *__restrict__ ub,
                        int *bin_count, int32_t *__restrict__ bin_rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ int s_n[kBins], s_base[kBins];
    if (threadIdx.x < kBins) s_n[threadIdx.x] = 0;
    __syncthreads();
    int bin = -1, rank = 0;
    if (i < n) {
        int64_t u;
        if (masked) {
            u = s_cnt ? s_cnt[i] : 1;
            bin = u <= kWarpMaxUb ? 3 : 4;
        } else {
            u = 1;
            for (int e = tt_rp[i]; e < tt_rp[i + 1]; e++) u += m_cnt[tt_ci[e]];
            bin = u <= 8 ? 0 : u <= 16 ? 1 : u <= 32 ? 2 : u <= kWarpMaxUb ? 3 : 4;
        }
        ub[i] = u;
        rank = atomicAdd(&s_n[bin], 1);  // position within the block's share of the bin
    }
    __syncthreads();
    // block-aggregated append: one global atomic per (block, bin); the counters
    // are few, so per-warp atomics on them serialised
    if (threadIdx.x < kBins) s_base[threadIdx.x] = s_n[threadIdx.x] ? atomicAdd(bin_count + threadIdx.x, s_n[threadIdx.x]) : 0;
    __syncthreads();
    if (bin >= 0) bin_rows[(int64_t)bin * n + s_base[bin] + rank] = (int32_t)i;
}

__device__ __forceinline__ int hslot(int32_t j, int logcap) {
    return (int)(((uint32_t)j * 0x9E3779B1u) >> (32 - logcap));
}

// Insert key j (or find it if present); -1 if the table is full.
__device__ __forceinline__ int hinsert(int32_t *keys, int32_t j, int logcap) {
    const int mask = (1 << logcap) - 1;
    int s = hslot(j, logcap);
    for (int probe = 0; probe <= mask; probe++) {
        int32_t old = atomicCAS(&keys[s], -1, j);
        if (old == -1 || old == j) return s;
        s = (s + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ int hfind(const int32_t *keys, int32_t j, int logcap) {
    const int mask = (1 << logcap) - 1;
    int s = hslot(j, logcap);
    for (int probe = 0; probe <= mask; probe++) {
        int32_t k = keys[s];
        if (k == j) return s;
        if (k == -1) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per output row (rows with bound <= kWarpMaxUb).
template <bool MASKED>
__global__ void __launch_bounds__(kWarps * 32)
k_spgemm_warp(int nrows, const int32_t *__restrict__ rows, const int32_t *__restrict__ tt_rp, const int32_t *__restrict__ tt_ci,
              const double *__restrict__ tt_va, const int64_t *__restrict__ m_off,
              const int32_t *__restrict__ m_cnt, const int32_t *__restrict__ m_ci,
              const double *__restrict__ m_va, const int64_t *__restrict__ s_off,
              const int32_t *__restrict__ s_cnt, const int32_t *__restrict__ s_ci,
              const int64_t *__restrict__ ub, const int64_t *__restrict__ o_off,
              int32_t *__restrict__ o_cnt, int32_t *__restrict__ o_ci, double *__restrict__ o_va,
              int kind, double tau, const double *__restrict__ dinv_scale, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem *W = reinterpret_cast<WarpSmem *>(smem_raw) + warp;
    int32_t *keys = W->keys;
    double *vals = W->vals;
    uint8_t *touched = W->touched;
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool thresholded = (kind == kDropAbs || kind == kDropRowRel);

    for (int r = blockIdx.x * kWarps + warp; r < nrows; r += gridDim.x * kWarps) {
        const int32_t i = rows[r];
        const int64_t u = ub[i];
        int logcap = 5;
        while ((1 << logcap) < 2 * u) logcap++;
        const int cap = 1 << logcap;
        for (int s = lane; s < cap; s += 32) { keys[s] = -1; vals[s] = 0.0; touched[s] = 0; }
        __syncwarp();
        bool bad = false;
        if (MASKED) {  // the pattern S_i, entries start at 0 and untouched
            if (s_off) {
                const int64_t sb = s_off[i];
                const int sc = s_cnt[i];
                for (int t = lane; t < sc; t += 32) bad |= hinsert(keys, s_ci[sb + t], logcap) < 0;
            } else if (lane == 0) {
                bad |= hinsert(keys, (int32_t)i, logcap) < 0;
            }
            __syncwarp();
        }
        // T~ (M D): ascending k, one fma per (k, j); the j of one row k are distinct
        const int tb = tt_rp[i], te = tt_rp[i + 1];
        for (int e = tb; e < te; e++) {
            const int32_t k = tt_ci[e];
            const double t = tt_va[e];
            const int64_t mb = m_off[k];
            const int mc = m_cnt[k];
            for (int f = lane; f < mc; f += 32) {
                const int32_t j = m_ci[mb + f];
                const double v = m_va[mb + f];
                int s = MASKED ? hfind(keys, j, logcap) : hinsert(keys, j, logcap);
                if (s >= 0) {
                    vals[s] = fma(t, v, vals[s]);
                    touched[s] = 1;
                } else if (!MASKED) {
                    bad = true;
                }
            }
            __syncwarp();
        }
        // + I
        if (lane == 0) {
            int s = MASKED ? hfind(keys, (int32_t)i, logcap) : hinsert(keys, (int32_t)i, logcap);
            if (s >= 0) { vals[s] = vals[s] + 1.0; touched[s] = 1; }
            else bad = true;
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, E_HASH);
        // dropping rule on the whole row
        double thr = tau;
        if (kind == kDropRowRel) {
            double mx = 0.0;
            for (int s = lane; s < cap; s += 32)
                if (keys[s] >= 0 && touched[s]) mx = fmax(mx, fabs(vals[s]));
            thr = tau * warp_max(mx);
        }
        int cnt = 0;
        for (int c = 0; c < cap; c += 32) {
            const int s = c + lane;
            const int32_t key = keys[s];
            const double v = vals[s];
            bool keep = key >= 0 && touched[s];
            if (keep && thresholded && key != i) keep = !(fabs(v) < thr);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int pos = cnt + __popc(m & lt_mask);
            __syncwarp();
            if (keep) { keys[pos] = key; vals[pos] = v; }
            cnt += __popc(m);
            __syncwarp();
        }
        // bitonic sort of keys[0..P) by column, P = next power of two >= cnt
        int P = 1;
        while (P < cnt) P <<= 1;
        for (int s = cnt + lane; s < P; s += 32) keys[s] = INT_MAX;
        __syncwarp();
        for (int k2 = 2; k2 <= P; k2 <<= 1) {
            for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                for (int t = lane; t < P; t += 32) {
                    const int o = t ^ j2;
                    if (o > t) {
                        const int32_t a = keys[t], b = keys[o];
                        const bool up = (t & k2) == 0;
                        if ((a > b) == up) {
                            keys[t] = b; keys[o] = a;
                            const double va_ = vals[t];
                            vals[t] = vals[o]; vals[o] = va_;
                        }
                    }
                }
                __syncwarp();
            }
        }
        const int64_t ob = o_off[i];
        for (int t = lane; t < cnt; t += 32) {
            const int32_t j = keys[t];
            const double v = vals[t];
            o_ci[ob + t] = j;
            o_va[ob + t] = dinv_scale ? v * dinv_scale[j] : v;
        }
        if (lane == 0) o_cnt[i] = cnt;
        __syncwarp();
    }
}

// Register-resident product for short rows: a group of W lanes owns one
// row, lane p holds the p-th product T~_ik (M D)_kj in the order (k ascending,
// then j ascending), the lane after the last product holds the diagonal.  A
// stable sort by column (ranks from shuffles) puts the products of one column
// next to each other in ascending k; a segmented chain then forms
// acc_j = fma(T~_ik, (MD)_kj, acc_j) in that order -- the oracle's chain.
template <int W>
__global__ void __launch_bounds__(256)
k_spgemm_reg(int nrows, const int32_t *__restrict__ rows, const int32_t *__restrict__ tt_rp,
             const int32_t *__restrict__ tt_ci, const double *__restrict__ tt_va,
             const int64_t *__restrict__ m_off, const int32_t *__restrict__ m_cnt,
             const int32_t *__restrict__ m_ci, const double *__restrict__ m_va,
             const int64_t *__restrict__ o_off, int32_t *__restrict__ o_cnt, int32_t *__restrict__ o_ci,
             double *__restrict__ o_va, int kind, double tau, const double *__restrict__ dinv_scale) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t g = gt / W;
    if (g >= nrows) return;  // whole groups leave together
    const int gl = threadIdx.x & (W - 1);
    const int gbase = (threadIdx.x & 31) & ~(W - 1);
    const unsigned gmask = W == 32 ? 0xffffffffu : (((1u << W) - 1u) << gbase);
    const unsigned lt = (1u << gl) - 1u;
    const int i = rows[g];
    const int tb = tt_rp[i], nt = tt_rp[i + 1] - tb;
    int kk = 0, cnt = 0;
    int64_t off = 0;
    double t = 0.0;
    if (gl < nt) {
        kk = tt_ci[tb + gl];
        t = tt_va[tb + gl];
        off = m_off[kk];
        cnt = m_cnt[kk];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        const int v = __shfl_up_sync(gmask, incl, o, W);
        if (gl >= o) incl += v;
    }
    const int start = incl - cnt;
    const int pc = __shfl_sync(gmask, incl, W - 1, W);  // number of products (< W)
    int my_e = 0;
    for (int e2 = 0; e2 < nt; e2++) {
        const int st = __shfl_sync(gmask, start, e2, W);
        if (st <= gl) my_e = e2;
    }
    const double t_my = __shfl_sync(gmask, t, my_e, W);
    const int64_t off_my = __shfl_sync(gmask, off, my_e, W);
    const int start_my = __shfl_sync(gmask, start, my_e, W);
    int key = INT_MAX;
    double mv = 0.0;
    if (gl < pc) {
        key = m_ci[off_my + gl - start_my];
        mv = m_va[off_my + gl - start_my];
    } else if (gl == pc) {
        key = i;  // + I
    }
    // stable ranks by column
    int rank = 0;
#pragma unroll
    for (int q = 0; q < W; q++) {
        const int kq = __shfl_sync(gmask, key, q, W);
        rank += (kq < key) || (kq == key && q < gl);
    }
    int src = 0;
#pragma unroll
    for (int q = 0; q < W; q++) {
        const int rq = __shfl_sync(gmask, rank, q, W);
        if (rq == gl) src = q;
    }
    const int skey = __shfl_sync(gmask, key, src, W);
    const double st_ = __shfl_sync(gmask, t_my, src, W);
    const double sm = __shfl_sync(gmask, mv, src, W);
    const bool sdiag = __shfl_sync(gmask, (int)(gl == pc), src, W) != 0;
    const int prev_key = __shfl_up_sync(gmask, skey, 1, W);
    const bool head = gl == 0 || prev_key != skey;
    const unsigned heads = (__ballot_sync(gmask, head) >> gbase) & (W == 32 ? 0xffffffffu : ((1u << W) - 1u));
    const int hpos = 31 - __clz(heads & (lt | (1u << gl)));
    const int pos = gl - hpos;
    double acc = 0.0;
    if (sdiag) acc = 0.0 + 1.0;
    else if (pos == 0 && skey != INT_MAX) acc = fma(st_, sm, 0.0);
    for (int step = 1; step < nt; step++) {
        const double prev = __shfl_up_sync(gmask, acc, 1, W);
        if (pos == step && !sdiag) acc = fma(st_, sm, prev);
    }
    const int next_key = __shfl_down_sync(gmask, skey, 1, W);
    const bool tail = skey != INT_MAX && (gl == W - 1 || next_key != skey);
    // The magnitude tests run on the IEEE bit patterns (non-negative doubles
    // order like their encodings), which keeps them off GB300's narrow FP64
    // pipe: |acc| < thr  <=>  absbits(acc) < bits(thr) for thr >= 0, and a
    // NaN (encoding above infinity) is kept, as !(NaN < thr) keeps it.
    constexpr unsigned long long kAbs = 0x7fffffffffffffffULL, kInf = 0x7ff0000000000000ULL;
    const unsigned long long ab = (unsigned long long)__double_as_longlong(acc) & kAbs;
    double thr = tau;
    if (kind == kDropRowRel) {
        unsigned long long mb = tail && ab <= kInf ? ab : 0ULL;  // the row maximum ignores NaN
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(gmask, mb, o, W);
            mb = ob > mb ? ob : mb;
        }
        thr = tau * __longlong_as_double((long long)mb);
    }
    bool keep = tail;
    if (keep && (kind == kDropAbs || kind == kDropRowRel) && skey != i)
        keep = !(ab < (unsigned long long)__double_as_longlong(thr));
    const unsigned km = (__ballot_sync(gmask, keep) >> gbase) & (W == 32 ? 0xffffffffu : ((1u << W) - 1u));
    if (keep) {
        const int64_t dst = o_off[i] + __popc(km & lt);
        o_ci[dst] = skey;
        o_va[dst] = dinv_scale ? acc * dinv_scale[skey] : acc;
    }
    if (gl == 0) o_cnt[i] = __popc(km);
}

// Exclusive scan of a 0/1 flag over a block of kDenseThreads threads.
__device__ __forceinline__ int block_flag_scan(bool f, int *total) {
    __shared__ int wt[kDenseThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wt[warp] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kDenseThreads / 32; w++) {
        if (w < warp) before += wt[w];
        tot += wt[w];
    }
    __syncthreads();
    *total = tot;
    return before + __popc(m & ((1u << lane) - 1u));
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double wm[kDenseThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max(v);
    if (lane == 0) wm[warp] = v;
    __syncthreads();
    double r = 0.0;
#pragma unroll
    for (int w = 0; w < kDenseThreads / 32; w++) r = fmax(r, wm[w]);
    __syncthreads();
    return r;
}

// One block per overflow row; dense accumulator acc/st of n entries per block.
// st[j] == 2i+1: touched in row i; st[j] == 2i: in S_i but not yet touched.
template <bool MASKED>
__global__ void __launch_bounds__(kDenseThreads)
k_spgemm_dense(int nrows, const int32_t *__restrict__ rows, int64_t n,
               const int32_t *__restrict__ tt_rp, const int32_t *__restrict__ tt_ci,
               const double *__restrict__ tt_va, const int64_t *__restrict__ m_off,
               const int32_t *__restrict__ m_cnt, const int32_t *__restrict__ m_ci,
               const double *__restrict__ m_va, const int64_t *__restrict__ s_off,
               const int32_t *__restrict__ s_cnt, const int32_t *__restrict__ s_ci,
               const int64_t *__restrict__ o_off, int32_t *__restrict__ o_cnt,
               int32_t *__restrict__ o_ci, double *__restrict__ o_va, int kind, double tau,
               const double *__restrict__ dinv_scale, double *acc_all, uint32_t *st_all) {
    __shared__ int lo_s, hi_s;
    double *acc = acc_all + (int64_t)blockIdx.x * n;
    uint32_t *st = st_all + (int64_t)blockIdx.x * n;
    const bool thresholded = (kind == kDropAbs || kind == kDropRowRel);
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int32_t i = rows[r];
        const uint32_t TT = 2u * (uint32_t)i + 1u, PP = 2u * (uint32_t)i;
        if (threadIdx.x == 0) { lo_s = INT_MAX; hi_s = -1; }
        __syncthreads();
        if (MASKED) {
            if (s_off) {
                const int64_t sb = s_off[i];
                for (int t = threadIdx.x; t < s_cnt[i]; t += kDenseThreads) {
                    const int32_t j = s_ci[sb + t];
                    st[j] = PP;
                    acc[j] = 0.0;
                    atomicMin(&lo_s, j);
                    atomicMax(&hi_s, j);
                }
            } else if (threadIdx.x == 0) {
                st[i] = PP;
                acc[i] = 0.0;
                atomicMin(&lo_s, i);
                atomicMax(&hi_s, i);
            }
            __syncthreads();
        }
        for (int e = tt_rp[i]; e < tt_rp[i + 1]; e++) {
            const int32_t k = tt_ci[e];
            const double t = tt_va[e];
            const int64_t mb = m_off[k];
            const int mc = m_cnt[k];
            for (int f = threadIdx.x; f < mc; f += kDenseThreads) {
                const int32_t j = m_ci[mb + f];
                const double v = m_va[mb + f];
                const uint32_t sj = st[j];
                if (MASKED) {
                    if (sj == PP || sj == TT) { acc[j] = fma(t, v, acc[j]); st[j] = TT; }
                } else if (sj != TT) {
                    st[j] = TT;
                    acc[j] = fma(t, v, 0.0);
                    atomicMin(&lo_s, j);
                    atomicMax(&hi_s, j);
                } else {
                    acc[j] = fma(t, v, acc[j]);
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (st[i] == TT) acc[i] = acc[i] + 1.0;
            else { acc[i] = 0.0 + 1.0; st[i] = TT; }
            atomicMin(&lo_s, i);
            atomicMax(&hi_s, i);
        }
        __syncthreads();
        const int lo = lo_s, hi = hi_s;
        double thr = tau;
        if (kind == kDropRowRel) {
            double mx = 0.0;
            for (int j = lo + threadIdx.x; j <= hi; j += kDenseThreads)
                if (st[j] == TT) mx = fmax(mx, fabs(acc[j]));
            thr = tau * block_max(mx);
        }
        const int64_t ob = o_off[i];
        int base = 0;
        for (int c = lo; c <= hi; c += kDenseThreads) {
            const int j = c + threadIdx.x;
            bool keep = j <= hi && st[j] == TT;
            double v = keep ? acc[j] : 0.0;
            if (keep && thresholded && j != i) keep = !(fabs(v) < thr);
            int tot;
            const int pos = block_flag_scan(keep, &tot);
            if (keep) {
                o_ci[ob + base + pos] = j;
                o_va[ob + base + pos] = dinv_scale ? v * dinv_scale[j] : v;
            }
            base += tot;
        }
        if (threadIdx.x == 0) o_cnt[i] = base;
        __syncthreads();
    }
}

// Gapped rows -> CSR.  kCompactG lanes per row (a SAIT row holds a few tens of
// entries at most, so a warp per row left most lanes idle), each lane moving
// two entries per round with both loads in flight.
constexpr int kCompactG = 8;
__global__ void k_compact(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ cnt,
                          const int32_t *__restrict__ ci, const double *__restrict__ va,
                          const int64_t *__restrict__ rp64, int32_t *__restrict__ rp,
                          int32_t *__restrict__ oci, double *__restrict__ ova) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kCompactG;
    const int sub = threadIdx.x & (kCompactG - 1);
    if (w > n) return;
    if (w == n) {
        if (sub == 0) rp[n] = (int32_t)rp64[n];
        return;
    }
    const int64_t src = off[w], dst = rp64[w];
    const int c = cnt[w];
    if (sub == 0) rp[w] = (int32_t)dst;
    for (int t = sub; t < c; t += 2 * kCompactG) {
        const bool two = t + kCompactG < c;
        const int32_t c0 = ci[src + t];
        const double v0 = va[src + t];
        const int32_t c1 = two ? ci[src + t + kCompactG] : 0;
        const double v1 = two ? va[src + t + kCompactG] : 0.0;
        oci[dst + t] = c0;
        ova[dst + t] = v0;
        if (two) {
            oci[dst + t + kCompactG] = c1;
            ova[dst + t + kCompactG] = v1;
        }
    }
}

// M = D^-1 (a single series term).
__global__ void k_diag_inverse(int64_t n, const double *dinv, int32_t *rp, int32_t *ci, double *va) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    rp[i] = (int32_t)i;
    if (i < n) { ci[i] = (int32_t)i; va[i] = 1.0 * dinv[i]; }
}

struct Iterate {
    DTemp<int64_t> off;
    DTemp<int32_t> cnt, ci;
    DTemp<double> va;
};

struct View {
    const int64_t *off;
    const int32_t *cnt;
    const int32_t *ci;
    const double *va;
};

View view_of(const Iterate &it) { return View{it.off.p, it.cnt.p, it.ci.p, it.va.p}; }

void move_iterate(Iterate &dst, Iterate &src) {
    dst.off.release(); dst.cnt.release(); dst.ci.release(); dst.va.release();
    dst.off.s = src.off.s; dst.off.p = src.off.take();
    dst.cnt.s = src.cnt.s; dst.cnt.p = src.cnt.take();
    dst.ci.s = src.ci.s; dst.ci.p = src.ci.take();
    dst.va.s = src.va.s; dst.va.p = src.va.take();
}

}  // namespace

extern "C" sait_status sait_build(sait_ctx ctx, sait_mat T, sait_uplo uplo, int32_t m_terms,
                                  sait_drop drop, sait_dtype store, sait_mat *out) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!T || !out) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: null matrix or output");
    *out = nullptr;
    if (m_terms < 1) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: m_terms < 1");
    if (uplo != SAIT_LOWER && uplo != SAIT_UPPER)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: bad uplo");
    if (drop.kind < SAIT_DROP_NONE || drop.kind > SAIT_DROP_HYBRID)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: bad drop kind");
    if ((drop.kind == SAIT_DROP_ABS || drop.kind == SAIT_DROP_ROWREL || drop.kind == SAIT_DROP_HYBRID) &&
        !(drop.tau >= 0.0 && drop.tau < 1.0))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: tau must lie in [0, 1)");
    if ((drop.kind == SAIT_DROP_PATTERN || drop.kind == SAIT_DROP_HYBRID) && drop.p < 0)
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: p < 0");
    if (!store_valid(store))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: bad storage type");
    const int64_t n = T->n, nnzT = T->nnz;
    cudaStream_t s = ctx->stream;
    ScopedTimer tm(ctx, SAIT_TIMER_BUILD);
    int *h = (int *)ctx->h_pinned;
    int64_t *h64 = (int64_t *)((char *)ctx->h_pinned + 256);  // apart from the int words

    // ---- split and validate
    DTemp<double> dinv;
    SAIT_CK(dinv.alloc(n, s));
    SAIT_CK(cudaMemsetAsync(ctx->d_word, 0, sizeof(int), s));
    if (n > 0)
        launch_k(k_split_check, (unsigned)cdiv(n, 256), 256, 0, s, n, T->rp, T->ci, T->va,
                                                             uplo == SAIT_LOWER, dinv.p, ctx->d_word);
    SAIT_CK(cudaGetLastError());
    SAIT_CK(cudaMemcpyAsync(h, ctx->d_word, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAIT_CK(cudaStreamSynchronize(s));
    if (h[0] & E_UNSORTED) return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_build: unsorted columns");
    if (h[0] & E_SIDE)
        return ctx_fail(ctx, SAIT_ERR_NOT_TRIANGULAR, "sait_build: entry on the wrong side of the diagonal");
    if (h[0] & E_PIVOT)
        return ctx_fail(ctx, SAIT_ERR_ZERO_PIVOT, "sait_build: missing, zero or non-finite diagonal");

    sait_mat M = nullptr;
    if (m_terms == 1) {
        SAIT_TRY(mat_alloc(ctx, n, n, &M));
        launch_k(k_diag_inverse, (unsigned)cdiv(n + 1, 256), 256, 0, s, n, dinv.p, M->rp, M->ci, M->va);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { sait_mat_destroy(M); return ctx_cuda(ctx, e, "k_diag_inverse", __FILE__, __LINE__); }
    } else {
        const int64_t ntt = nnzT - n;
        DTemp<int32_t> tt_rp, tt_ci;
        DTemp<double> tt_va;
        SAIT_CK(tt_rp.alloc(n + 1, s));
        SAIT_CK(tt_ci.alloc(ntt, s));
        SAIT_CK(tt_va.alloc(ntt, s));
        launch_k(k_split_fill, (unsigned)cdiv(n + 1, 256), 256, 0, s, n, T->rp, T->ci, T->va, dinv.p,
                                                                 tt_rp.p, tt_ci.p, tt_va.p);
        SAIT_CK(cudaGetLastError());

        const int smem = kWarps * (int)sizeof(WarpSmem);
        SAIT_CK(cudaFuncSetAttribute(k_spgemm_warp<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        SAIT_CK(cudaFuncSetAttribute(k_spgemm_warp<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem));

        // owned: the current iterate when it is not the pattern S; cur: a view
        Iterate owned, S;
        bool have_S = false;
        SAIT_CK(owned.off.alloc(n, s));
        SAIT_CK(owned.cnt.alloc(n, s));
        SAIT_CK(owned.ci.alloc(n, s));
        SAIT_CK(owned.va.alloc(n, s));
        if (n > 0)
            launch_k(k_identity, (unsigned)cdiv(n, 256), 256, 0, s, n, owned.off.p, owned.cnt.p, owned.ci.p,
                                                             owned.va.p);
        SAIT_CK(cudaGetLastError());
        View cur = view_of(owned);
        const bool pattern = drop.kind == SAIT_DROP_PATTERN;

        DTemp<int64_t> ub;
        DTemp<int32_t> bins;  // kBins row lists of up to n rows each
        SAIT_CK(ub.alloc(n, s));
        SAIT_CK(bins.alloc((size_t)kBins * n, s));
        int *bin_count = ctx->d_word + kWordBins;
        int *hash_err = ctx->d_word + kWordBuildErr;
        SAIT_CK(cudaMemsetAsync(hash_err, 0, sizeof(int), s));
        for (int it = 1; it < m_terms; it++) {
            const bool masked = pattern && it > drop.p;
            const int kind = pattern ? kDropNone
                             : drop.kind == SAIT_DROP_HYBRID ? (it <= drop.p ? kDropNone : kDropAbs)
                                                             : (int)drop.kind;
            const bool last = it == m_terms - 1;
            const int32_t *s_cnt = masked && have_S ? S.cnt.p : nullptr;
            const int64_t *s_off = masked && have_S ? S.off.p : nullptr;
            const int32_t *s_ci = masked && have_S ? S.ci.p : nullptr;
            SAIT_CK(cudaMemsetAsync(bin_count, 0, kBins * sizeof(int), s));
            if (n > 0)
                launch_k(k_rowub, (unsigned)cdiv(n, 256), 256, 0, s, n, (const int32_t *)tt_rp.p,
                         (const int32_t *)tt_ci.p, cur.cnt, (int)masked, s_cnt, ub.p, bin_count, bins.p);
            SAIT_CK(cudaGetLastError());
            Iterate nx;
            SAIT_CK(nx.off.alloc(n + 1, s));
            SAIT_CK(scan_i64(ub.p, nx.off.p, n, s));
            SAIT_CK(cudaMemcpyAsync(h64, nx.off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            SAIT_CK(cudaMemcpyAsync(h + 4, bin_count, kBins * sizeof(int), cudaMemcpyDeviceToHost, s));
            SAIT_CK(cudaStreamSynchronize(s));
            const int64_t total = h64[0];
            int nbin[kBins];
            for (int q = 0; q < kBins; q++) nbin[q] = h[4 + q];
            SAIT_CK(nx.cnt.alloc(n, s));
            SAIT_CK(nx.ci.alloc(total, s));
            SAIT_CK(nx.va.alloc(total, s));
            const double *scale = last ? dinv.p : nullptr;
            const double tau = drop.tau;
            const int32_t *rows0 = bins.p, *rows1 = bins.p + n, *rows2 = bins.p + 2 * n;
            const int32_t *rows3 = bins.p + 3 * n, *rows4 = bins.p + 4 * n;
            // short rows: register kernels (never masked)
            launch_k(k_spgemm_reg<8>, (unsigned)cdiv((int64_t)nbin[0] * 8, 256), 256, 0, s, nbin[0], rows0,
                     (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                     cur.cnt, cur.ci, cur.va, (const int64_t *)nx.off.p, nx.cnt.p, nx.ci.p, nx.va.p, kind, tau,
                     scale);
            launch_k(k_spgemm_reg<16>, (unsigned)cdiv((int64_t)nbin[1] * 16, 256), 256, 0, s, nbin[1], rows1,
                     (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                     cur.cnt, cur.ci, cur.va, (const int64_t *)nx.off.p, nx.cnt.p, nx.ci.p, nx.va.p, kind, tau,
                     scale);
            launch_k(k_spgemm_reg<32>, (unsigned)cdiv((int64_t)nbin[2] * 32, 256), 256, 0, s, nbin[2], rows2,
                     (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                     cur.cnt, cur.ci, cur.va, (const int64_t *)nx.off.p, nx.cnt.p, nx.ci.p, nx.va.p, kind, tau,
                     scale);
            SAIT_CK(cudaGetLastError());
            if (nbin[3] > 0) {
                const unsigned grid = (unsigned)std::min<int64_t>(cdiv(nbin[3], kWarps), (int64_t)ctx->num_sms * 4);
                if (masked)
                    launch_k(k_spgemm_warp<true>, grid, kWarps * 32, smem, s, nbin[3], rows3,
                             (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                             cur.cnt, cur.ci, cur.va, s_off, s_cnt, s_ci, (const int64_t *)ub.p,
                             (const int64_t *)nx.off.p, nx.cnt.p, nx.ci.p, nx.va.p, kind, tau, scale, hash_err);
                else
                    launch_k(k_spgemm_warp<false>, grid, kWarps * 32, smem, s, nbin[3], rows3,
                             (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                             cur.cnt, cur.ci, cur.va, s_off, s_cnt, s_ci, (const int64_t *)ub.p,
                             (const int64_t *)nx.off.p, nx.cnt.p, nx.ci.p, nx.va.p, kind, tau, scale, hash_err);
                SAIT_CK(cudaGetLastError());
            }
            const int novf = nbin[4];
            if (novf > 0) {
                // dense accumulators, bounded to about 2 GB of scratch
                const int64_t per = n * (int64_t)(sizeof(double) + sizeof(uint32_t));
                const int64_t nb = std::max<int64_t>(
                    1, std::min<int64_t>({(int64_t)novf, (int64_t)128, (int64_t)(2LL << 30) / per}));
                DTemp<double> acc;
                DTemp<uint32_t> stp;
                SAIT_CK(acc.alloc(nb * n, s));
                SAIT_CK(stp.alloc(nb * n, s));
                SAIT_CK(cudaMemsetAsync(stp.p, 0xff, nb * n * sizeof(uint32_t), s));
                if (masked)
                    launch_k(k_spgemm_dense<true>, (unsigned)nb, kDenseThreads, 0, s, novf, rows4, n,
                             (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                             cur.cnt, cur.ci, cur.va, s_off, s_cnt, s_ci, (const int64_t *)nx.off.p, nx.cnt.p,
                             nx.ci.p, nx.va.p, kind, tau, scale, acc.p, stp.p);
                else
                    launch_k(k_spgemm_dense<false>, (unsigned)nb, kDenseThreads, 0, s, novf, rows4, n,
                             (const int32_t *)tt_rp.p, (const int32_t *)tt_ci.p, (const double *)tt_va.p, cur.off,
                             cur.cnt, cur.ci, cur.va, s_off, s_cnt, s_ci, (const int64_t *)nx.off.p, nx.cnt.p,
                             nx.ci.p, nx.va.p, kind, tau, scale, acc.p, stp.p);
                SAIT_CK(cudaGetLastError());
            }
            move_iterate(owned, nx);   // frees the previous owned iterate (stream-ordered)
            cur = view_of(owned);
            if (pattern && it == drop.p) {  // keep the sparsity pattern S of M
                move_iterate(S, owned);
                cur = view_of(S);
                have_S = true;
            }
        }
        const View fin = cur;
        // compaction into CSR
        SAIT_CK(cudaMemcpyAsync(h + 3, ctx->d_word + kWordBuildErr, sizeof(int), cudaMemcpyDeviceToHost, s));
        DTemp<int64_t> rp64;
        SAIT_CK(rp64.alloc(n + 1, s));
        SAIT_CK(scan_i32(fin.cnt, rp64.p, n, s));
        SAIT_CK(cudaMemcpyAsync(h64 + 1, rp64.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SAIT_CK(cudaStreamSynchronize(s));
        if (h[3] & E_HASH) return ctx_fail(ctx, SAIT_ERR_CUDA, "sait_build: hash table overflow");
        const int64_t nnzM = h64[1];
        if (nnzM >= (int64_t)INT_MAX)
            return ctx_fail(ctx, SAIT_ERR_UNSUPPORTED, "sait_build: nnz(M) >= 2^31");
        SAIT_TRY(mat_alloc(ctx, n, nnzM, &M));
        launch_k(k_compact, (unsigned)cdiv((n + 1) * kCompactG, 256), 256, 0, s, n, fin.off, fin.cnt, fin.ci, fin.va,
                                                                   rp64.p, M->rp, M->ci, M->va);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { sait_mat_destroy(M); return ctx_cuda(ctx, e, "k_compact", __FILE__, __LINE__); }
    }
    M->lanes = choose_lanes(M->n, M->nnz);
    sait_status st = mat_prepare_store(ctx, M, store);
    if (st != SAIT_OK) { sait_mat_destroy(M); return st; }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { sait_mat_destroy(M); return ctx_cuda(ctx, e, "sait_build", __FILE__, __LINE__); }
    *out = M;
    return SAIT_OK;
}
