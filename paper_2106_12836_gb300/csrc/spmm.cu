// Multi-right-hand-side products Y = A X (X, Y row-major n x k with leading
// dimension ld) and the SAIT block apply Z = M_U (M_L R).
//
// A group of G lanes owns one row; lane l handles columns l, l + G, ... of
// the block.  The group loads G entries of the row at a time (one per lane)
// and broadcasts each (column, value) pair with shuffles, so every entry of A
// is read once per product whatever k is, and for each entry the group reads
// the G consecutive values X[c, :] -- one coalesced line.  With the block of
// k columns, the matrix traffic of one apply is shared by k vectors (the
// block eigensolver and many-right-hand-side cases).
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.cuh"

namespace {


template <int G, int CPL, typename TV, typename A, typename TX, typename TY>
__global__ void __launch_bounds__(256)
k_spmm_csr(int64_t n, int k, int64_t ldx, int64_t ldy, const int32_t *__restrict__ rp,
           const int32_t *__restrict__ ci, const TV *__restrict__ va, const TX *__restrict__ X,
           TY *__restrict__ Y, int *calls) {
    if (calls && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(calls, 1);
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int gl = threadIdx.x & (G - 1);
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    if (row >= n) return;  // whole groups leave together
    using VT = decltype(Load<A, TV>::get(TV{}));
    A acc[CPL];
#pragma unroll
    for (int t = 0; t < CPL; t++) acc[t] = A{};
    const int b = rp[row], e = rp[row + 1];
    for (int base = b; base < e; base += G) {
        const int idx = base + gl;
        const int c_l = idx < e ? __ldg(ci + idx) : 0;
        const VT v_l = idx < e ? Load<A, TV>::get(va[idx]) : (VT)0;
        const int cnt = min(G, e - base);
        for (int u = 0; u < cnt; u++) {
            const int c = __shfl_sync(gmask, c_l, u, G);
            const VT v = __shfl_sync(gmask, v_l, u, G);
            const TX *xr = X + (int64_t)c * ldx;
#pragma unroll
            for (int t = 0; t < CPL; t++) {
                const int col = gl + t * G;
                if (col < k) mac(acc[t], v, XCast<A, TX>::get(__ldg(xr + col)));
            }
        }
    }
    TY *yr = Y + row * ldy;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
        const int col = gl + t * G;
        if (col < k) put_out(yr + col, acc[t]);
    }
}

__device__ __forceinline__ void put4(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void put4(double *p, float a, float b, float c, float d) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(widen_exact(a), widen_exact(b));
    reinterpret_cast<double2 *>(p)[1] = make_double2(widen_exact(c), widen_exact(d));
}

// entries of a row gathered per trip in k_spmm_f32x4, and the resident blocks
// per SM asked of the compiler (at most 40 registers): 128^3 x 64 FP32 apply
// 1.52 ms with 2 entries, 1.44 ms with 4, 1.39 ms with 4 and 6 blocks per SM
constexpr int kX4Entries = 4;
constexpr int kX4MinBlocks = 6;

// FP32 arithmetic on an FP32 block X with k = 4 G columns: a group of G lanes
// owns a row and each lane gathers four consecutive columns of X[c, :] with
// one 16-byte load, so one warp serves 32 / G rows and each entry costs a
// fraction of the instructions of k_spmm_csr's one-column-per-lane form
// (which issued about 26 warp instructions per entry for k = 64 and was
// issue- and latency-bound).  kX4Entries entries per trip, all gathers
// issued first.  Every column sums the row's entries in entry order with fmaf, as
// k_spmm_csr does, so the two kernels give the same bits.  Needs X, Y
// 16-byte aligned and ldx, ldy multiples of 4.
template <int G, int U, typename TV, typename TY>
__global__ void __launch_bounds__(256, kX4MinBlocks)
k_spmm_f32x4(int64_t n, int64_t ldx, int64_t ldy, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
             const TV *__restrict__ va, const float *__restrict__ X, TY *__restrict__ Y, int *calls) {
    if (calls && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(calls, 1);
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int gl = threadIdx.x & (G - 1);
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    if (row >= n) return;  // whole groups leave together
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    const float4 *X4 = reinterpret_cast<const float4 *>(X) + gl;
    const int64_t ld4 = ldx / 4;
    const int b = rp[row], e = rp[row + 1];
    auto add = [&](float v, const float4 &x) {
        a0 = fmaf(v, x.x, a0);
        a1 = fmaf(v, x.y, a1);
        a2 = fmaf(v, x.z, a2);
        a3 = fmaf(v, x.w, a3);
    };
    for (int base = b; base < e; base += G) {
        const int idx = base + gl;
        const int c_l = idx < e ? __ldg(ci + idx) : 0;
        const float v_l = idx < e ? Load<float, TV>::get(va[idx]) : 0.0f;
        const int cnt = min(G, e - base);
        int u = 0;
        for (; u + U <= cnt; u += U) {  // U entries per trip, all gathers issued first
            float4 xv[U];
            float vv[U];
#pragma unroll
            for (int t = 0; t < U; t++) {
                const int c = __shfl_sync(gmask, c_l, u + t, G);
                vv[t] = __shfl_sync(gmask, v_l, u + t, G);
                xv[t] = __ldg(X4 + c * ld4);
            }
#pragma unroll
            for (int t = 0; t < U; t++) add(vv[t], xv[t]);
        }
        for (; u < cnt; u++) {
            const int c = __shfl_sync(gmask, c_l, u, G);
            const float v = __shfl_sync(gmask, v_l, u, G);
            add(v, __ldg(X4 + c * ld4));
        }
    }
    put4(Y + row * ldy + 4 * gl, a0, a1, a2, a3);
}

template <int G, typename TV, typename TY>
void launch_x4(const sait_mat_s *A, const TV *va, int64_t ldx, int64_t ldy, const float *X, TY *Y, cudaStream_t s,
               int *calls) {
    constexpr int U = G < kX4Entries ? G : kX4Entries;
    launch_k(k_spmm_f32x4<G, U, TV, TY>, (unsigned)cdiv(A->n * G, 256), 256, 0, s, A->n, ldx, ldy,
             (const int32_t *)A->rp, (const int32_t *)A->ci, va, X, Y, calls);
}

// the four-column form for k in {8, 16, 32, 64, 128} with aligned blocks; false: not applicable
template <typename TV, typename TY>
bool launch_f32x4(const sait_mat_s *A, const TV *va, int k, int64_t ldx, int64_t ldy, const float *X, TY *Y,
                  cudaStream_t s, int *calls) {
    if (ldx % 4 || ldy % 4 || ((uintptr_t)X & 15) || ((uintptr_t)Y & 15)) return false;
    switch (k) {
        case 8: launch_x4<2>(A, va, ldx, ldy, X, Y, s, calls); return true;
        case 16: launch_x4<4>(A, va, ldx, ldy, X, Y, s, calls); return true;
        case 32: launch_x4<8>(A, va, ldx, ldy, X, Y, s, calls); return true;
        case 64: launch_x4<16>(A, va, ldx, ldy, X, Y, s, calls); return true;
        case 128: launch_x4<32>(A, va, ldx, ldy, X, Y, s, calls); return true;
        default: return false;
    }
}

template <int G, int CPL, typename TV, typename TA, typename TX, typename TY>
void launch_gc(const sait_mat_s *A, const TV *va, int k, int64_t ldx, int64_t ldy, const TX *X, TY *Y,
               cudaStream_t s, int *calls) {
    launch_k(k_spmm_csr<G, CPL, TV, TA, TX, TY>, (unsigned)cdiv(A->n * G, 256), 256, 0, s, A->n, k, ldx, ldy,
             (const int32_t *)A->rp, (const int32_t *)A->ci, va, X, Y, calls);
}

template <typename TV, typename TA, typename TX, typename TY>
void launch_shape(const sait_mat_s *A, const TV *va, int k, int64_t ldx, int64_t ldy, const TX *X, TY *Y,
                  cudaStream_t s, int *calls) {
    if (k <= 1) launch_gc<2, 1, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else if (k <= 2) launch_gc<2, 1, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else if (k <= 4) launch_gc<4, 1, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else if (k <= 8) launch_gc<8, 1, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else if (k <= 16) launch_gc<16, 1, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else if (k <= 32) launch_gc<32, 1, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else if (k <= 64) launch_gc<32, 2, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
    else launch_gc<32, 4, TV, TA>(A, va, k, ldx, ldy, X, Y, s, calls);
}

template <typename TV, typename TA>
cudaError_t spmm_xy(const sait_mat_s *A, const TV *va, int k, int64_t ldx, int64_t ldy, const void *X,
                    bool x_f32, void *Y, bool y_f32, cudaStream_t s, int *calls) {
    if constexpr (std::is_same<TA, float>::value) {
        if (x_f32) {
            const bool done = y_f32 ? launch_f32x4(A, va, k, ldx, ldy, (const float *)X, (float *)Y, s, calls)
                                    : launch_f32x4(A, va, k, ldx, ldy, (const float *)X, (double *)Y, s, calls);
            if (done) return cudaGetLastError();
        }
    }
    if (x_f32) {
        if (y_f32) launch_shape<TV, TA>(A, va, k, ldx, ldy, (const float *)X, (float *)Y, s, calls);
        else launch_shape<TV, TA>(A, va, k, ldx, ldy, (const float *)X, (double *)Y, s, calls);
    } else {
        if (y_f32) launch_shape<TV, TA>(A, va, k, ldx, ldy, (const double *)X, (float *)Y, s, calls);
        else launch_shape<TV, TA>(A, va, k, ldx, ldy, (const double *)X, (double *)Y, s, calls);
    }
    return cudaGetLastError();
}

// Y = fl32(X), n x k row-major with leading dimensions ldx and k, rounded to
// nearest (narrow_rn): the rounding the FP32 products otherwise apply to every
// gathered entry of X
__global__ void k_narrow_block(int64_t n, int k, int64_t ldx, const double *__restrict__ X, float *__restrict__ Y) {
    const int64_t total = n * k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / k;
        Y[i] = narrow_rn(X[r * ldx + (i - r * k)]);
    }
}

}  // namespace

cudaError_t launch_spmm(const sait_mat_s *A, sait_dtype store, int k, int64_t ldx, int64_t ldy, const void *X,
                        bool x_f32, void *Y, bool y_f32, cudaStream_t s, int *calls) {
    if (A->n == 0 || k <= 0) return cudaSuccess;
    switch (store) {
        case SAIT_F32:
            return spmm_xy<float, float>(A, (const float *)A->va32, k, ldx, ldy, X, x_f32, Y, y_f32, s, calls);
        case SAIT_BF16:
            return spmm_xy<__nv_bfloat16, float>(A, (const __nv_bfloat16 *)A->va16, k, ldx, ldy, X, x_f32, Y, y_f32,
                                                 s, calls);
        // The block products of the X64 modes keep FP64 arithmetic: with many
        // columns the double-float split of every gathered X entry costs more
        // than the FP64 FMA it replaces (measured 11.0 vs 4.5 ms, 128^3 x 64).
        case SAIT_F32_X64:
            return spmm_xy<float, double>(A, (const float *)A->va32, k, ldx, ldy, X, x_f32, Y, y_f32, s, calls);
        case SAIT_BF16_X64:
            return spmm_xy<__nv_bfloat16, double>(A, (const __nv_bfloat16 *)A->va16, k, ldx, ldy, X, x_f32, Y,
                                                  y_f32, s, calls);
        default:
            return spmm_xy<double, double>(A, (const double *)A->va, k, ldx, ldy, X, x_f32, Y, y_f32, s, calls);
    }
}

extern "C" sait_status sait_spmm(sait_ctx ctx, sait_mat A, int32_t k, const double *X, int64_t ldx, double *Y,
                                 int64_t ldy) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!A || k < 0 || ldx < k || ldy < k || (A->n > 0 && k > 0 && (!X || !Y)))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_spmm: bad argument");
    ScopedTimer tm(ctx, SAIT_TIMER_SPMV);
    SAIT_CK(launch_spmm(A, A->store, k, ldx, ldy, X, false, Y, false, ctx->stream,
                        group_counter(ctx, SAIT_TIMER_SPMV)));
    return SAIT_OK;
}

sait_status apply_multi_impl(sait_ctx ctx, sait_mat ML, sait_mat MU, int k, const double *R, int64_t ldr,
                             double *Z, int64_t ldz, void *W) {
    const bool f64 = store_x64(ML->store) && store_x64(MU->store);
    ScopedTimer tm(ctx, SAIT_TIMER_APPLY);
    if (!f64 && !store_x64(ML->store)) {
        // FP32 products round every gathered entry of R: round R once into the
        // second half of the n x k-double scratch and gather 4-byte values
        float *R32 = (float *)W + (size_t)ML->n * k;
        if (ldr == k) {
            SAIT_CK(launch_narrow((int64_t)ML->n * k, R, R32, nullptr, ctx->stream, ctx->num_sms));
        } else {
            const unsigned blocks = (unsigned)std::min<int64_t>(cdiv((int64_t)ML->n * k, 256), 8LL * ctx->num_sms);
            launch_k(k_narrow_block, blocks, 256, 0, ctx->stream, ML->n, k, ldr, R, R32);
        }
        SAIT_CK(launch_spmm(ML, ML->store, k, k, k, R32, true, W, true, ctx->stream,
                            group_counter(ctx, SAIT_TIMER_APPLY)));
    } else {
        SAIT_CK(launch_spmm(ML, ML->store, k, ldr, k, R, false, W, !f64, ctx->stream,
                            group_counter(ctx, SAIT_TIMER_APPLY)));
    }
    SAIT_CK(launch_spmm(MU, MU->store, k, k, ldz, W, !f64, Z, false, ctx->stream, nullptr));
    return SAIT_OK;
}

extern "C" sait_status sait_apply_multi(sait_ctx ctx, sait_mat ML, sait_mat MU, int32_t k, const double *R,
                                        int64_t ldr, double *Z, int64_t ldz) {
    if (!ctx) return SAIT_ERR_INVALID_ARG;
    if (!ML || !MU || ML->n != MU->n || k < 0 || ldr < k || ldz < k || (ML->n > 0 && k > 0 && (!R || !Z)))
        return ctx_fail(ctx, SAIT_ERR_INVALID_ARG, "sait_apply_multi: bad argument");
    if (ML->n == 0 || k == 0) return SAIT_OK;
    DTemp<double> W;  // n x k intermediate (FP64, or FP32 in its first half)
    SAIT_CK(W.alloc((size_t)ML->n * k, ctx->stream));
    return apply_multi_impl(ctx, ML, MU, k, R, ldr, Z, ldz, W.p);
}
