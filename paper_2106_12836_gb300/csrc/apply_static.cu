// SAIT apply that allocates nothing.
//
// sait_apply obtains its intermediate vector w = M_L r from the stream-ordered
// pool.  Some callers cannot let a library allocate device memory when they
// apply the preconditioner: loops with hard latency budgets that forbid
// allocator calls, and frameworks or embedded runtimes that hand out all device
// memory from their own pools, sized once at start-up.  sait_apply_static
// keeps w in a fixed array compiled into the library instead.  The array exists
// once per device that loads the library and stays allocated until the
// process exits.
#include <mutex>

#include "internal.cuh"

namespace {

// 2^21 entries of 8 bytes: 16 MiB per device.  Holds w in FP64, or in FP32
// when either SAIT matrix is stored in reduced precision.
__device__ __align__(256) double g_apply_scratch[SAIT_APPLY_STATIC_MAX_N];

constexpr int kMaxDevices = 128;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_apply_scratch on the current device.  In host code the
// symbol itself is only a host-side stand-in, so its address is looked up once
// per device and cached.  A device reset frees the array with everything else
// on the device; sait_ctx_create (which every caller needs again after a reset,
// to rebuild its matrices) drops the cached address through
// static_apply_forget, so the next call looks it up again.
cudaError_t scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

void static_apply_forget(int dev) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (dev >= 0 && dev < kMaxDevices) g_scratch_addr[dev] = nullptr;
}

extern "C" sait_status sait_apply_static(sait_mat ML, sait_mat MU, const double *r, double *z, void *stream) {
    if (!ML || !MU || ML->n != MU->n || (ML->n > 0 && (!r || !z))) return SAIT_ERR_INVALID_ARG;
    if (ML->n > (int64_t)SAIT_APPLY_STATIC_MAX_N) return SAIT_ERR_UNSUPPORTED;
    if (ML->n == 0) return SAIT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices || dev != ML->device ||
        dev != MU->device) {
        cudaGetLastError();
        return SAIT_ERR_INVALID_ARG;
    }
    void *w = nullptr;
    if (scratch_address(dev, &w) != cudaSuccess) {
        cudaGetLastError();
        return SAIT_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool f64 = store_x64(ML->store) && store_x64(MU->store);
    cudaError_t e = launch_spmv(ML, ML->store, r, false, w, !f64, nullptr, s);
    if (e == cudaSuccess) e = launch_spmv(MU, MU->store, w, !f64, z, false, nullptr, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SAIT_ERR_CUDA;
    }
    return SAIT_OK;
}
