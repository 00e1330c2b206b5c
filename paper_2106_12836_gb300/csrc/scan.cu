// Exclusive prefix sums (int32 or int64 input, int64 output) in three passes:
// per-tile scan, scan of the tile totals, and a tile offset add.
#include "internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kThreads / 32 ? warp_tot[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < kThreads / 32) warp_tot[lane] = wi - w;
        if (lane == kThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = incl - v + warp_tot[warp];
    __syncthreads();
    return r;
}

template <typename Tin>
__global__ void __launch_bounds__(kThreads) k_scan_tiles(const Tin *__restrict__ in, int64_t n,
                                                         int64_t *__restrict__ out,
                                                         int64_t *__restrict__ tile_sums) {
    __shared__ int64_t tot;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < kItems; q++) {
        int64_t idx = base + q;
        v[q] = idx < n ? (int64_t)in[idx] : 0;
        s += v[q];
    }
    int64_t run = block_excl_scan(s, &tot);
#pragma unroll
    for (int q = 0; q < kItems; q++) {
        int64_t idx = base + q;
        if (idx < n) out[idx] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile totals in place; total -> *total_out.
__global__ void __launch_bounds__(kThreads) k_scan_sums(int64_t *sums, int64_t ntiles,
                                                        int64_t *total_out) {
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kThreads) {
        int64_t idx = b + threadIdx.x;
        int64_t v = idx < ntiles ? sums[idx] : 0;
        int64_t e = block_excl_scan(v, &tot);
        if (idx < ntiles) sums[idx] = e + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_off) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += tile_off[idx / kTile];
}

template <typename Tin>
cudaError_t scan_impl(const Tin *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    int64_t ntiles = cdiv(n, kTile);
    int64_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sums, ntiles * sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
    launch_k(k_scan_tiles<Tin>, (unsigned)ntiles, kThreads, 0, s, in, n, out, sums);
    launch_k(k_scan_sums, 1, kThreads, 0, s, sums, ntiles, out + n);
    launch_k(k_scan_add, (unsigned)cdiv(n, 256), 256, 0, s, out, n, sums);
    e = cudaGetLastError();
    cudaFreeAsync(sums, s);
    return e;
}

}  // namespace

cudaError_t scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}
cudaError_t scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}
