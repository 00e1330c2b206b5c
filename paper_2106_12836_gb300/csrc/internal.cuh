// Internal declarations shared by the translation units of libsait.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sait.h"

// d_word layout: [0] per-call error flags, [2..6] SpGEMM
// row-bin counters, [8..9] level analysis, [10] SpGEMM error flags, [16 + g]
// device-side call counters of timer group g (incremented by kernels that did
// real work).
constexpr int kWordBins = 2;
constexpr int kWordBuildErr = 10;
constexpr int kCounterBase = 16;

struct TimerRec {
    int group;
    cudaEvent_t a, b;
};

struct sait_ctx_s {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 1;
    std::string last_error;
    int *d_word = nullptr;     // device scratch words (error flags, counters)
    void *h_pinned = nullptr;  // pinned host staging (4 KB)
    bool timing = false;
    unsigned timing_groups = ~0u;  // groups timed while timing is on (bit per sait_timer)
    int timing_every = 1;          // a timed group records one call in timing_every
    int64_t group_seen[SAIT_TIMER_COUNT] = {};  // calls of each group since timing was set
    bool group_live[SAIT_TIMER_COUNT] = {};     // the group's current call records events
    std::vector<TimerRec> pending;
    std::vector<cudaEvent_t> spare;
    double ms[SAIT_TIMER_COUNT] = {};
    int64_t host_calls[SAIT_TIMER_COUNT] = {};
    int64_t launch_base = 0;
    int64_t batch_tile = 2048;  // rows per tile of the batched solver's schedule (sait_batch_autotune)
    int64_t wait_limit = 0;     // polls of a device-side dependency wait (0: the kernel's default)
    int device_loop = 1;        // batched solvers: iterate inside a WHILE graph node (0: host replays)
};

// Kernel launches made by this host thread (graph kernel nodes included).
extern thread_local int64_t g_sait_launches;

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
    kernel<<<grid, block, smem, s>>>(args...);
    ++g_sait_launches;
}

// Programmatic dependent launch: the kernel may be scheduled while its
// predecessor in the stream drains; it must call pdl_wait() before touching
// any memory the predecessor writes.  A dependent grid starts only after every
// block of the predecessor has called pdl_trigger() or exited, so waiting
// blocks never hold back the predecessor.  Both calls are no-ops in a kernel
// launched without the attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++g_sait_launches;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// A hint that pulls the line holding p into L2 (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Event pair around a group of launches on the context stream (timing on only).
struct ScopedTimer {
    sait_ctx ctx;
    int group;
    cudaEvent_t a = nullptr;
    ScopedTimer(sait_ctx c, int g);
    ~ScopedTimer();
};
// device counter of a timer group while its current call is timed, else null
int *group_counter(sait_ctx ctx, int group);

struct sait_mat_s {
    int64_t n = 0, nnz = 0;
    int32_t *rp = nullptr;
    int32_t *ci = nullptr;
    double *va = nullptr;           // FP64 values (always present)
    float *va32 = nullptr;          // FP32 copy (on demand)
    __nv_bfloat16 *va16 = nullptr;  // BF16 copy (on demand)
    sait_dtype store = SAIT_F64;
    int device = 0;
    int lanes = 8;                  // lanes per row for CSR products
    bool pooled = false;            // arrays from the stream-ordered pool (see mat_array)
    // SELL-32 copy for products (built on demand; see sell.cu)
    bool sell_rejected = false;     // padding above 20% even sorted: products stay on CSR
    bool force_csr = false;         // set by sait_mat_autotune when CSR products won
    int64_t nslices = 0, sell_nnz = 0;
    int64_t *soff = nullptr;
    int32_t *sperm = nullptr;       // SELL-C-sigma: row held by slot position p (null: natural order)
    int32_t *sci = nullptr;
    double *sva64 = nullptr;
    float *sva32 = nullptr;
    __nv_bfloat16 *sva16 = nullptr;
};

// A device array of M from the context's stream-ordered pool: a large
// cudaMalloc maps fresh memory and its cudaFree synchronises the device, both
// per matrix, while the pool hands back memory freed earlier (the ILU factors,
// SAIT factors and their SELL copies are rebuilt for every system).
// sait_mat_destroy synchronises the device before returning pooled arrays,
// since cudaFree does not wait for work still using them.
cudaError_t mat_array(sait_ctx ctx, sait_mat M, void **p, size_t bytes);

struct LevelSchedule {
    int32_t nlev = 0;
    int32_t *rows = nullptr;            // device: rows ordered by level
    std::vector<int32_t> ptr;           // host: level l is rows[ptr[l] .. ptr[l+1])
    int32_t max_width = 0;
};

struct sait_prec_s {
    int kind = 0;  // 1 SAIT pair, 2 exact ILU, 3 Jacobi sweeps
    bool pooled = false;        // tmp from the stream-ordered pool (kind 1, see mat_array)
    int sweeps = 0;             // kind 3: sweeps per triangle
    double *dinv = nullptr;     // kind 3: 1 / diag(L) then 1 / diag(U), 2n
    sait_mat lo = nullptr, up = nullptr;
    LevelSchedule lev_lo, lev_up;
    double *tmp = nullptr;      // n-vector scratch
    int64_t n = 0;
    int device = 0;
    // CUDA graph of the level-scheduled substitution (input/output buffers fixed)
    cudaGraphExec_t graph = nullptr;
    int64_t graph_kernels = 0;  // kernel nodes in the graph
    double *gin = nullptr, *gout = nullptr;
};

// ---- error helpers ---------------------------------------------------------
sait_status ctx_fail(sait_ctx ctx, sait_status st, const std::string &msg);
sait_status jacobi_apply(sait_ctx ctx, sait_prec P, const double *r, double *z, const int *active);
sait_status ctx_cuda(sait_ctx ctx, cudaError_t e, const char *what, const char *file, int line);

#define SAIT_CK(call)                                                         \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ctx_cuda(ctx, e_, #call, __FILE__, __LINE__); \
    } while (0)

#define SAIT_TRY(expr)                          \
    do {                                        \
        sait_status s_ = (expr);                \
        if (s_ != SAIT_OK) return s_;           \
    } while (0)

// Stream-ordered device temporary, freed on scope exit (on the same stream).
template <class T>
struct DTemp {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    DTemp() = default;
    DTemp(const DTemp &) = delete;
    DTemp &operator=(const DTemp &) = delete;
    ~DTemp() { release(); }
    cudaError_t alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        return cudaMallocAsync((void **)&p, (count ? count : 1) * sizeof(T), st);
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
    T *take() {
        T *q = p;
        p = nullptr;
        return q;
    }
};

__host__ __device__ static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Double-float arithmetic on the FP32 pipe.  GB300 runs FP64 at 1/53 of its
// FP32 rate, so long FP64 reductions and block products carry ~48-bit values
// as (hi, lo) FP32 pairs instead, with error-free transformations.
//
// Knuth's two-sum of (S, p) into S plus the rounding error added to E; the
// _rn intrinsics keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void df_add(float &S, float &E, float p, float e) {
    const float sn = __fadd_rn(S, p);
    const float bb = __fsub_rn(sn, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(sn, bb)), __fsub_rn(p, bb));
    S = sn;
    E = __fadd_rn(E, __fadd_rn(err, e));
}

// one double-float product term (vh + vl)(a + al), without the lo*lo part
__device__ __forceinline__ void df_term(float &S, float &E, float vh, float vl, float a, float al) {
    const float p = __fmul_rn(vh, a);
    float e = __fmaf_rn(vh, a, -p);
    e = __fmaf_rn(vh, al, e);
    e = __fmaf_rn(vl, a, e);
    df_add(S, E, p, e);
}

// Out-of-line conversions for the rare values outside the integer paths
// below.  Kept out of line so that the compiler cannot evaluate them
// speculatively for every value: on GB300 a float <-> double conversion takes
// the narrow FP64 pipe, and a speculated one per vector entry made the
// Gram-Schmidt sweeps FP64-pipe bound.
static __device__ __noinline__ void split_pair_slow(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}
static __device__ __noinline__ float hi_part_slow(double v) { return (float)v; }

// (hi, lo) with hi = v truncated to 24 significant bits and lo the next 23
// bits of v, both taken from the IEEE-754 fields with integer operations and
// one exact FP32 subtraction, so no FP64 or conversion instruction is spent
// (conversions from FP64 share GB300's narrow FP64 pipe).  |lo| < 2^-23 |hi|
// and |v - hi - lo| < 2^-46 |v|.  Values outside 2^-75 <= |v| < 2^128 take
// the conversion path.
__device__ __forceinline__ void split_pair(double v, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const int ef = e - 896;  // FP32 biased exponent of hi (1023 - 127 = 896)
    const int el = e - 919;  // FP32 biased exponent whose mantissa ulp weighs the fraction bits 6..28
    if (e <= 948 || ef >= 255) {
        split_pair_slow(v, hi, lo);
        return;
    }
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned long long frac = b & ((1ULL << 52) - 1);
    hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(frac >> 29));
    const unsigned base = (unsigned)el << 23;
    const unsigned mid = (unsigned)(frac >> 6) & ((1u << 23) - 1);  // fraction bits 6..28
    lo = __fsub_rn(__uint_as_float(sign | base | mid), __uint_as_float(sign | base));
}

// v truncated to FP32 (the hi part of split_pair) with integer operations
__device__ __forceinline__ float hi_part(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const int ef = e - 896;
    if (ef <= 0 || ef >= 255) return hi_part_slow(v);
    return __uint_as_float(((unsigned)(b >> 63) << 31) | ((unsigned)ef << 23) |
                           (unsigned)((b & ((1ULL << 52) - 1)) >> 29));
}

// Exact FP32 -> FP64 widening from the IEEE-754 fields with integer
// operations only (zero, subnormal, infinite and NaN inputs included, no
// branch).  On GB300 a hardware float-to-double conversion occupies the narrow
// FP64 pipe longer than a DFMA, and the sweeps and products widen one value
// per row.
__device__ __forceinline__ double widen_exact(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    unsigned m = b & 0x7fffffu;
    unsigned ed = e + 896u;                                   // normal
    const int sh = __clz(m | 1u) - 8;                         // subnormal: bring the leading 1 to bit 23
    const unsigned ms = (m << sh) & 0x7fffffu;
    ed = e == 0xffu ? 0x7ffu : ed;                            // infinity / NaN
    ed = e == 0u ? (m ? 897u - (unsigned)sh : 0u) : ed;       // subnormal / zero
    m = (e == 0u && m) ? ms : m;
    const unsigned hi = (b & 0x80000000u) | (ed << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)((m & 7u) << 29));
}

static __device__ __noinline__ float narrow_slow(double v) { return (float)v; }

// FP64 -> FP32 rounded to nearest (ties to even) with integer operations:
// the 23 leading fraction bits, rounded up when the 29 dropped bits exceed
// half an FP32 ulp or equal it with an odd last bit (a carry moves into the
// exponent, and past the largest finite value gives infinity, as IEEE
// rounding does).  |v| < 2^-126 gives a signed zero (no FP32 subnormals);
// |v| >= 2^128, infinities and NaNs take the conversion instruction.  The
// products of FP32- and BF16-stored matrices narrow one FP64 vector entry per
// matrix entry, which as conversions would keep GB300's FP64 pipe busy.
__device__ __forceinline__ float narrow_rn(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ef = (int)((b >> 52) & 0x7ff) - 896;
    const unsigned sign = (unsigned)(b >> 63) << 31;
    if (ef >= 255) return narrow_slow(v);
    if (ef <= 0) return __uint_as_float(sign);
    const unsigned long long frac = b & ((1ULL << 52) - 1);
    const unsigned m = (unsigned)(frac >> 29);
    const unsigned rest = (unsigned)frac & ((1u << 29) - 1);
    const unsigned up = (rest > (1u << 28)) | ((rest == (1u << 28)) & (m & 1u));
    return __uint_as_float(sign | ((((unsigned)ef << 23) | m) + up));
}

// S + E as an FP64 value
__device__ __forceinline__ double df_value(float S, float E) { return (double)S + (double)E; }

// Double-float accumulator of the *_X64 storage modes: products of the rounded
// (exact FP32) matrix values with FP64 or FP32 vector entries, summed with
// error-free transformations, ~48 significant bits without FP64 instructions.
struct DF {
    float S = 0.0f, E = 0.0f;
};
__device__ __forceinline__ void mac(DF &acc, float v, double x) {
    float xh, xl;
    split_pair(x, xh, xl);
    const float p = __fmul_rn(xh, v);
    float e = __fmaf_rn(xh, v, -p);
    e = __fmaf_rn(xl, v, e);
    df_add(acc.S, acc.E, p, e);
}
__device__ __forceinline__ void mac(DF &acc, float v, float x) {
    const float p = __fmul_rn(x, v);
    df_add(acc.S, acc.E, p, __fmaf_rn(x, v, -p));
}
__device__ __forceinline__ void mac(double &acc, double v, double x) { acc = fma(v, x, acc); }
__device__ __forceinline__ void mac(float &acc, float v, float x) { acc = fmaf(v, x, acc); }
// b into a (both double-float partial sums)
__device__ __forceinline__ void df_merge(DF &a, const DF &b) { df_add(a.S, a.E, b.S, b.E); }
__device__ __forceinline__ double acc_value(const DF &a) { return df_value(a.S, a.E); }
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ float acc_value(float a) { return a; }
// vector entry as the multiplier type of accumulator A
template <typename A, typename TX> struct XCast {
    __device__ __forceinline__ static A get(TX x) { return (A)x; }
};
template <> struct XCast<float, double> {
    __device__ __forceinline__ static float get(double x) { return narrow_rn(x); }
};
template <typename TX> struct XCast<DF, TX> {
    __device__ __forceinline__ static TX get(TX x) { return x; }
};

// accumulator A stored as output element type TY (FP32 sums widen exactly and
// FP64 sums narrow with integer operations, see widen_exact and narrow_rn)
__device__ __forceinline__ void put_out(double *p, double a) { *p = a; }
__device__ __forceinline__ void put_out(double *p, float a) { *p = widen_exact(a); }
__device__ __forceinline__ void put_out(double *p, const DF &a) { *p = widen_exact(a.S) + widen_exact(a.E); }
__device__ __forceinline__ void put_out(float *p, float a) { *p = a; }
__device__ __forceinline__ void put_out(float *p, double a) { *p = narrow_rn(a); }
__device__ __forceinline__ void put_out(float *p, const DF &a) { *p = narrow_rn(widen_exact(a.S) + widen_exact(a.E)); }

// Exact widening of stored FP32 / BF16 values to FP64 (a hardware
// conversion; integer bit assembly measured slower on GB300).
__device__ __forceinline__ double widen(float f) { return (double)f; }
__device__ __forceinline__ double widen(__nv_bfloat16 b) {
    return widen(__uint_as_float((uint32_t)__bfloat16_as_ushort(b) << 16));
}
__device__ __forceinline__ double widen(double v) { return v; }

// value of storage type TV in accumulator type A
template <typename A, typename TV> struct Load;
template <typename TV> struct Load<double, TV> {
    __device__ __forceinline__ static double get(TV v) { return widen(v); }
};
template <> struct Load<float, float> {
    __device__ __forceinline__ static float get(float v) { return v; }
};
template <> struct Load<float, __nv_bfloat16> {
    __device__ __forceinline__ static float get(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct Load<DF, float> {
    __device__ __forceinline__ static float get(float v) { return v; }
};
template <> struct Load<DF, __nv_bfloat16> {
    __device__ __forceinline__ static float get(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// FP64 arithmetic in products with this storage (values converted exactly)
static inline bool store_x64(sait_dtype s) { return s == SAIT_F64 || s == SAIT_F32_X64 || s == SAIT_BF16_X64; }
// which value array a storage mode reads
static inline sait_dtype store_base(sait_dtype s) {
    return s == SAIT_F32_X64 ? SAIT_F32 : s == SAIT_BF16_X64 ? SAIT_BF16 : s;
}
static inline bool store_valid(int s) { return s >= SAIT_F64 && s <= SAIT_BF16_X64; }

// ---- internal launchers (one translation unit each) -------------------------
// scan.cu: out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
cudaError_t scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
cudaError_t scan_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);

// spmv.cu
int choose_lanes(int64_t n, int64_t nnz);
// y = A x for the value storage of A; x/y element types given by flags.
cudaError_t launch_spmv(const sait_mat_s *A, sait_dtype store, const void *x, bool x_f32, void *y,
                        bool y_f32, const int *active, cudaStream_t s, int *calls = nullptr, bool pdl = false);
// y = fl32(x), rounded to nearest (the narrowing of the FP32 products' inputs)
cudaError_t launch_narrow(int64_t n, const double *x, float *y, const int *active, cudaStream_t s, int num_sms);
cudaError_t cast_values(const double *src, float *d32, __nv_bfloat16 *d16, int64_t nnz,
                        cudaStream_t s);

// spmm.cu
cudaError_t launch_spmm(const sait_mat_s *A, sait_dtype store, int k, int64_t ldx, int64_t ldy, const void *X,
                        bool x_f32, void *Y, bool y_f32, cudaStream_t s, int *calls);
sait_status apply_multi_impl(sait_ctx ctx, sait_mat ML, sait_mat MU, int k, const double *R, int64_t ldr,
                             double *Z, int64_t ldz, void *W);

// sell.cu
sait_status mat_prepare_sell(sait_ctx ctx, sait_mat M, sait_dtype store);
bool sell_ready(const sait_mat_s *A, sait_dtype store);
cudaError_t launch_spmv_sell(const sait_mat_s *A, sait_dtype store, const void *x, bool x_f32, void *y,
                             bool y_f32, const int *active, cudaStream_t s, int *calls, bool pdl = false);

// levels.cu
sait_status build_levels(sait_ctx ctx, const int32_t *rp, const int32_t *ci, int64_t n, bool lower,
                         LevelSchedule *out);
void free_levels(LevelSchedule *L);
cudaError_t launch_trisolve(const sait_mat_s *T, const LevelSchedule &lev, bool lower,
                            const double *b, double *x, cudaStream_t s);

// apply_static.cu: drop the cached device address of the static apply's array
void static_apply_forget(int dev);

// mat helpers (api.cu)
sait_status mat_copy_csr(sait_ctx ctx, const sait_csr *A, sait_mat *out);  // validated copy, CSR only
sait_status mat_alloc(sait_ctx ctx, int64_t n, int64_t nnz, sait_mat *out);
sait_status mat_prepare_store(sait_ctx ctx, sait_mat M, sait_dtype store);
sait_status prec_apply_impl(sait_ctx ctx, sait_prec P, const double *r, double *z,
                            const int *active);
