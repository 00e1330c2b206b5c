// Sliced ELLPACK (SELL-32) copies of CSR matrices and their products.
//
// Rows are cut into slices of 32 consecutive rows; slice s stores its entries
// column-major, padded to the longest row of the slice: entry k of the row in
// slot position p = 32 s + l sits at soff[s] + 32 k + l.  Padding has column -1
// and value 0 and is skipped.  Slot positions are the rows themselves unless
// natural order would pad more than 20%: then rows are sorted by length,
// longest first (stable), inside windows of kSigma rows (SELL-C-sigma with
// C = 32, sigma = kSigma), sperm[p] names the row at position p, and a
// product writes y[sperm[p]].  A warp owns one slice and lane l one row, so
// every load of columns and values is a full 128-byte (int32 / FP32) or
// 256-byte (FP64) coalesced line, and four column slots are loaded before
// they are used to keep enough bytes in flight per warp.  For the PDE factors
// of the SAIT path, whose rows of a slice have almost the same length, the
// padding costs 0.2-1% of the entries.
#include <algorithm>

#include "internal.cuh"

namespace {

// column slots loaded ahead per lane: enough bytes in flight per warp for
// 8-byte values with 4, for 4- and 2-byte values with 8
template <typename TV> struct Ahead { static constexpr int value = 8; };
template <> struct Ahead<double> { static constexpr int value = 4; };



// streaming loads: columns and values are read once per product
__device__ __forceinline__ int32_t lds(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ double lds(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float lds(const float *p) { return __ldcs(p); }
__device__ __forceinline__ __nv_bfloat16 lds(const __nv_bfloat16 *p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_bfloat16(u);
}

template <typename TV, typename A, typename TX, typename TY>
__global__ void __launch_bounds__(256)
k_spmv_sell(int64_t n, int64_t nslices, const int64_t *__restrict__ soff, const int32_t *__restrict__ ci,
            const TV *__restrict__ va, const TX *__restrict__ x, TY *__restrict__ y,
            const int *__restrict__ active, int *calls, const int32_t *__restrict__ perm) {
    constexpr int kU = Ahead<TV>::value;
    pdl_wait();
    pdl_trigger();
    if (active && *active == 0) return;
    if (calls && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(calls, 1);
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int64_t b = soff[s];
    const int len = (int)((soff[s + 1] - b) >> 5);
    const int32_t *c = ci + b + lane;
    const TV *v = va + b + lane;
    using VT = decltype(Load<A, TV>::get(TV{}));
    using XT = decltype(XCast<A, TX>::get(TX{}));
    A acc{};
    int k = 0;
    // kU column slots per round, the last round predicated: every load of a
    // round is issued before the first use, also for short rows
    for (; k < len; k += kU) {
        const int m = min(kU, len - k);
        int32_t cc[kU];
        VT vv[kU];
        XT xx[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            cc[u] = u < m ? lds(c + 32 * u) : -1;
            vv[u] = u < m ? Load<A, TV>::get(lds(v + 32 * u)) : (VT)0;
        }
#pragma unroll
        for (int u = 0; u < kU; u++) xx[u] = cc[u] >= 0 ? XCast<A, TX>::get(__ldg(x + cc[u])) : (XT)0;
#pragma unroll
        for (int u = 0; u < kU; u++)
            if (cc[u] >= 0) mac(acc, vv[u], xx[u]);
        c += 32 * kU;
        v += 32 * kU;
    }
    const int64_t p = s * 32 + lane;
    if (p < n) put_out(y + (perm ? (int64_t)perm[p] : p), acc);
}

// SELL-C-sigma order: inside each window of kSigma rows (one block), the rank
// of a row is the number of rows in the window that are longer, or as long
// and earlier; perm[window start + rank] = row
constexpr int kSigma = 256;
__global__ void __launch_bounds__(kSigma) k_sigma_perm(int64_t n, const int32_t *__restrict__ rp, int32_t *perm) {
    __shared__ int len[kSigma];
    const int t = threadIdx.x;
    const int64_t w0 = (int64_t)blockIdx.x * kSigma, row = w0 + t;
    const int l = row < n ? rp[row + 1] - rp[row] : -1;
    len[t] = l;
    __syncthreads();
    if (row >= n) return;
    int rank = 0;
    for (int q = 0; q < kSigma; q++) {
        const int lq = len[q];
        rank += lq > l || (lq == l && q < t);
    }
    perm[w0 + rank] = (int32_t)row;
}

// slice lengths (in column slots) and the padded-entry count per slice
__global__ void k_sell_len(int64_t n, int64_t nslices, const int32_t *__restrict__ rp,
                           const int32_t *__restrict__ perm, int64_t *slots) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int64_t p = s * 32 + lane;
    const int64_t row = p < n ? (perm ? (int64_t)perm[p] : p) : -1;
    int len = row >= 0 ? rp[row + 1] - rp[row] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) slots[s] = 32LL * len;
}

__device__ __forceinline__ void put(double *p, double v) { *p = v; }
__device__ __forceinline__ void put(float *p, double v) { *p = (float)v; }
__device__ __forceinline__ void put(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }

template <typename TV>
__global__ void k_sell_fill(int64_t n, int64_t nslices, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ va,
                            const int64_t *__restrict__ soff, const int32_t *__restrict__ perm, int32_t *sci,
                            TV *sva, bool fill_cols) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;
    const int64_t p = s * 32 + lane;
    const int64_t row = p < n ? (perm ? (int64_t)perm[p] : p) : -1;
    const int64_t b = soff[s];
    const int len = (int)((soff[s + 1] - b) >> 5);
    const int rb = row >= 0 ? rp[row] : 0, re = row >= 0 ? rp[row + 1] : 0;
    for (int k = 0; k < len; k++) {
        const int64_t dst = b + 32LL * k + lane;
        const bool in = rb + k < re;
        if (fill_cols) sci[dst] = in ? ci[rb + k] : -1;
        put(sva + dst, in ? va[rb + k] : 0.0);
    }
}

template <typename TV, typename TA, typename TX, typename TY>
cudaError_t sell_launch(const sait_mat_s *A, const TV *va, const TX *x, TY *y, const int *active,
                        cudaStream_t s, int *calls, bool pdl) {
    const unsigned grid = (unsigned)cdiv(A->nslices * 32, 256);
    if (pdl)
        return launch_pdl(k_spmv_sell<TV, TA, TX, TY>, grid, 256, 0, s, A->n, A->nslices, (const int64_t *)A->soff,
                          (const int32_t *)A->sci, va, x, y, active, calls,
                          (const int32_t *)A->sperm);
    launch_k(k_spmv_sell<TV, TA, TX, TY>, grid, 256, 0, s, A->n, A->nslices, (const int64_t *)A->soff,
             (const int32_t *)A->sci, va, x, y, active, calls,
                          (const int32_t *)A->sperm);
    return cudaGetLastError();
}

template <typename TV, typename TA>
cudaError_t sell_xy(const sait_mat_s *A, const TV *va, const void *x, bool x_f32, void *y, bool y_f32,
                    const int *active, cudaStream_t s, int *calls, bool pdl) {
    if (x_f32) {
        if (y_f32) return sell_launch<TV, TA>(A, va, (const float *)x, (float *)y, active, s, calls, pdl);
        return sell_launch<TV, TA>(A, va, (const float *)x, (double *)y, active, s, calls, pdl);
    }
    if (y_f32) return sell_launch<TV, TA>(A, va, (const double *)x, (float *)y, active, s, calls, pdl);
    return sell_launch<TV, TA>(A, va, (const double *)x, (double *)y, active, s, calls, pdl);
}

}  // namespace

// Build the SELL-32 structure of M (natural order, or sorted in windows of kSigma
// rows, when its padding stays below 20%) and the value array of the requested
// storage precision.
sait_status mat_prepare_sell(sait_ctx ctx, sait_mat M, sait_dtype store) {
    cudaStream_t s = ctx->stream;
    const int64_t n = M->n;
    if (n == 0 || M->sell_rejected) return SAIT_OK;
    const int64_t nslices = cdiv(n, 32);
    const unsigned grid = (unsigned)cdiv(nslices * 32, 256);
    if (!M->soff) {
        DTemp<int64_t> slots;
        SAIT_CK(slots.alloc(nslices, s));
        int64_t *soff = nullptr;
        int32_t *perm = nullptr;
        SAIT_CK(mat_array(ctx, M, (void **)&soff, (nslices + 1) * sizeof(int64_t)));
        // padded entries in natural order, and sorted in windows if that pads more than 20%
        auto count = [&](const int32_t *pm, int64_t *total) -> cudaError_t {
            launch_k(k_sell_len, grid, 256, 0, s, n, nslices, (const int32_t *)M->rp, pm, slots.p);
            cudaError_t e = scan_i64(slots.p, soff, nslices, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(total, soff + nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            return e;
        };
        const double cap = 1.2 * (double)std::max<int64_t>(M->nnz, 1);
        int64_t total = 0;
        cudaError_t e = count(nullptr, &total);
        if (e == cudaSuccess && (double)total > cap) {
            e = mat_array(ctx, M, (void **)&perm, (size_t)n * sizeof(int32_t));
            if (e == cudaSuccess) {
                launch_k(k_sigma_perm, (unsigned)cdiv(n, kSigma), kSigma, 0, s, n, (const int32_t *)M->rp, perm);
                e = count(perm, &total);
            }
        }
        if (e != cudaSuccess || (double)total > cap) {
            cudaFreeAsync(soff, s);
            if (perm) cudaFreeAsync(perm, s);
            if (e != cudaSuccess) return ctx_cuda(ctx, e, "mat_prepare_sell", __FILE__, __LINE__);
            M->sell_rejected = true;  // too ragged even sorted: products stay on CSR
            return SAIT_OK;
        }
        M->soff = soff;
        M->sperm = perm;
        M->nslices = nslices;
        M->sell_nnz = total;
        SAIT_CK(mat_array(ctx, M, (void **)&M->sci, std::max<int64_t>(total, 1) * sizeof(int32_t)));
        SAIT_CK(mat_array(ctx, M, (void **)&M->sva64, std::max<int64_t>(total, 1) * sizeof(double)));
        launch_k(k_sell_fill<double>, grid, 256, 0, s, n, nslices, (const int32_t *)M->rp,
                 (const int32_t *)M->ci, (const double *)M->va, (const int64_t *)M->soff,
                 (const int32_t *)M->sperm, M->sci, M->sva64, true);
        SAIT_CK(cudaGetLastError());
    }
    const int64_t total = M->sell_nnz;
    store = store_base(store);
    if (store == SAIT_F32 && !M->sva32) {
        SAIT_CK(mat_array(ctx, M, (void **)&M->sva32, std::max<int64_t>(total, 1) * sizeof(float)));
        launch_k(k_sell_fill<float>, grid, 256, 0, s, n, nslices, (const int32_t *)M->rp,
                 (const int32_t *)M->ci, (const double *)M->va, (const int64_t *)M->soff,
                 (const int32_t *)M->sperm, M->sci, M->sva32, false);
        SAIT_CK(cudaGetLastError());
    } else if (store == SAIT_BF16 && !M->sva16) {
        SAIT_CK(mat_array(ctx, M, (void **)&M->sva16, std::max<int64_t>(total, 1) * sizeof(__nv_bfloat16)));
        launch_k(k_sell_fill<__nv_bfloat16>, grid, 256, 0, s, n, nslices, (const int32_t *)M->rp,
                 (const int32_t *)M->ci, (const double *)M->va, (const int64_t *)M->soff,
                 (const int32_t *)M->sperm, M->sci, M->sva16, false);
        SAIT_CK(cudaGetLastError());
    }
    return SAIT_OK;
}

bool sell_ready(const sait_mat_s *A, sait_dtype store) {
    if (!A->soff) return false;
    store = store_base(store);
    return store == SAIT_F64 ? A->sva64 != nullptr : store == SAIT_F32 ? A->sva32 != nullptr
                                                                          : A->sva16 != nullptr;
}

cudaError_t launch_spmv_sell(const sait_mat_s *A, sait_dtype store, const void *x, bool x_f32, void *y,
                             bool y_f32, const int *active, cudaStream_t s, int *calls, bool pdl) {
    switch (store) {
        case SAIT_F32: return sell_xy<float, float>(A, A->sva32, x, x_f32, y, y_f32, active, s, calls, pdl);
        case SAIT_BF16: return sell_xy<__nv_bfloat16, float>(A, A->sva16, x, x_f32, y, y_f32, active, s, calls, pdl);
        case SAIT_F32_X64: return sell_xy<float, DF>(A, A->sva32, x, x_f32, y, y_f32, active, s, calls, pdl);
        case SAIT_BF16_X64:
            return sell_xy<__nv_bfloat16, DF>(A, A->sva16, x, x_f32, y, y_f32, active, s, calls, pdl);
        default: return sell_xy<double, double>(A, A->sva64, x, x_f32, y, y_f32, active, s, calls, pdl);
    }
}
