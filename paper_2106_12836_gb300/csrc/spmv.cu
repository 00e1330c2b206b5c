// CSR sparse matrix-vector products y = A x.
//
// G consecutive lanes of a warp own one row and stride over its entries, so a
// warp reads 32 consecutive (column, value) pairs per step when rows are at
// least G long; partial sums are combined with warp shuffles.  The value type
// is the matrix's storage precision: FP64 values accumulate in FP64, FP32 and
// BF16 values in FP32 (the SAIT matrices approximate T^-1 anyway, so their
// product precision can be reduced; Section 3.1).
#include <type_traits>

#include "internal.cuh"

namespace {



template <int G, typename TV, typename A, typename TX, typename TY>
__global__ void __launch_bounds__(256)
k_spmv_csr(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
           const TV *__restrict__ va, const TX *__restrict__ x, TY *__restrict__ y,
           const int *__restrict__ active, int *calls) {
    if (active && *active == 0) return;  // uniform over the grid
    if (calls && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(calls, 1);
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gid / G;
    const int lane = threadIdx.x & (G - 1);
    A s{};
    if (row < n) {
        const int b = rp[row], e = rp[row + 1];
        for (int k = b + lane; k < e; k += G) mac(s, Load<A, TV>::get(va[k]), XCast<A, TX>::get(__ldg(x + ci[k])));
    }
    if constexpr (std::is_same<A, DF>::value) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            DF t;
            t.S = __shfl_xor_sync(0xffffffffu, s.S, o);
            t.E = __shfl_xor_sync(0xffffffffu, s.E, o);
            df_merge(s, t);
        }
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (row < n && lane == 0) put_out(y + row, s);
}

template <typename TV, typename TA, typename TX, typename TY>
cudaError_t launch_g(int G, int64_t n, const int32_t *rp, const int32_t *ci, const TV *va,
                     const TX *x, TY *y, const int *active, cudaStream_t s, int *calls) {
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (unsigned)cdiv(n * G, threads);
    switch (G) {
        case 2: launch_k(k_spmv_csr<2, TV, TA, TX, TY>, blocks, threads, 0, s, n, rp, ci, va, x, y, active, calls); break;
        case 4: launch_k(k_spmv_csr<4, TV, TA, TX, TY>, blocks, threads, 0, s, n, rp, ci, va, x, y, active, calls); break;
        case 8: launch_k(k_spmv_csr<8, TV, TA, TX, TY>, blocks, threads, 0, s, n, rp, ci, va, x, y, active, calls); break;
        case 16: launch_k(k_spmv_csr<16, TV, TA, TX, TY>, blocks, threads, 0, s, n, rp, ci, va, x, y, active, calls); break;
        default: launch_k(k_spmv_csr<32, TV, TA, TX, TY>, blocks, threads, 0, s, n, rp, ci, va, x, y, active, calls); break;
    }
    return cudaGetLastError();
}

template <typename TV, typename TA>
cudaError_t launch_xy(const sait_mat_s *A, const TV *va, const void *x, bool x_f32, void *y,
                      bool y_f32, const int *active, cudaStream_t s, int *calls) {
    const int G = A->lanes;
    if (x_f32) {
        if (y_f32)
            return launch_g<TV, TA>(G, A->n, A->rp, A->ci, va, (const float *)x, (float *)y, active, s, calls);
        return launch_g<TV, TA>(G, A->n, A->rp, A->ci, va, (const float *)x, (double *)y, active, s, calls);
    }
    if (y_f32)
        return launch_g<TV, TA>(G, A->n, A->rp, A->ci, va, (const double *)x, (float *)y, active, s, calls);
    return launch_g<TV, TA>(G, A->n, A->rp, A->ci, va, (const double *)x, (double *)y, active, s, calls);
}

__global__ void k_cast(const double *__restrict__ src, float *d32, __nv_bfloat16 *d16, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = src[i];
        if (d32) d32[i] = (float)v;
        if (d16) d16[i] = __double2bfloat16(v);
    }
}

// y = fl32(x) with round to nearest even (narrow_rn, integer operations), the
// rounding the FP32 products otherwise apply to every gathered entry of x
__global__ void k_narrow(int64_t n, const double *__restrict__ x, float *__restrict__ y,
                         const int *__restrict__ active) {
    pdl_wait();
    pdl_trigger();
    if (active && *active == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = narrow_rn(x[i]);
}

}  // namespace

cudaError_t launch_narrow(int64_t n, const double *x, float *y, const int *active, cudaStream_t s, int num_sms) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(cdiv(n, 256), (int64_t)num_sms * 8);
    return launch_pdl(k_narrow, blocks, 256, 0, s, n, x, y, active);
}

int choose_lanes(int64_t n, int64_t nnz) {
    double avg = n > 0 ? (double)nnz / (double)n : 1.0;
    int G = 2;
    while (G < 32 && G * 2 <= avg) G *= 2;
    return G;
}

cudaError_t launch_spmv(const sait_mat_s *A, sait_dtype store, const void *x, bool x_f32, void *y,
                        bool y_f32, const int *active, cudaStream_t s, int *calls, bool pdl) {
    if (!A->force_csr && sell_ready(A, store))
        return launch_spmv_sell(A, store, x, x_f32, y, y_f32, active, s, calls, pdl);
    switch (store) {
        case SAIT_F32: return launch_xy<float, float>(A, A->va32, x, x_f32, y, y_f32, active, s, calls);
        case SAIT_BF16: return launch_xy<__nv_bfloat16, float>(A, A->va16, x, x_f32, y, y_f32, active, s, calls);
        case SAIT_F32_X64: return launch_xy<float, DF>(A, A->va32, x, x_f32, y, y_f32, active, s, calls);
        case SAIT_BF16_X64:
            return launch_xy<__nv_bfloat16, DF>(A, A->va16, x, x_f32, y, y_f32, active, s, calls);
        default: return launch_xy<double, double>(A, A->va, x, x_f32, y, y_f32, active, s, calls);
    }
}

cudaError_t cast_values(const double *src, float *d32, __nv_bfloat16 *d16, int64_t nnz,
                        cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    unsigned blocks = (unsigned)std::min<int64_t>(cdiv(nnz, 256), 152 * 16);
    launch_k(k_cast, blocks, 256, 0, s, src, d32, d16, nnz);
    return cudaGetLastError();
}
