// Shared device/host helpers of the OT IPM library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "ot_ipm.h"

namespace ot {

// ---------------------------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};

extern std::atomic<int64_t> g_launches;
void set_thread_error(const char *msg);

#define OT_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            return ::ot::Error{e_ == cudaErrorMemoryAllocation ? OT_ERR_OOM : OT_ERR_CUDA,  \
                               std::string(#call) + ": " + cudaGetErrorString(e_)};        \
        }                                                                                  \
    } while (0)

#define OT_TRY(expr)                                                                       \
    do {                                                                                   \
        ::ot::Error e2_ = (expr);                                                          \
        if (e2_.code != OT_OK) return e2_;                                                 \
    } while (0)

#define OT_LAUNCHED()                                                                      \
    do {                                                                                   \
        ::ot::g_launches.fetch_add(1, std::memory_order_relaxed);                          \
        cudaError_t e3_ = cudaGetLastError();                                              \
        if (e3_ != cudaSuccess)                                                            \
            return ::ot::Error{OT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e3_)}; \
    } while (0)

inline Error ok() { return Error{OT_OK, std::string()}; }

// ------------------------------------------------------------------------ kernel timing
// Opt-in CUDA-event timing of the main kernels, recorded on the stream each kernel is
// launched on (ot_kernel_timing_enable / ot_kernel_timing_read in the C ABI).
enum KernelId : int {
    KT_SCAN_HIST = 0, KT_SCAN_GATHER, KT_RECHECK, KT_PCG64, KT_PCG32, KT_LDL_NUMERIC, KT_LDL_SOLVE,
    KT_D32_FACTOR, KT_D32_APPLY, KT_DCG, KT_COUNT
};
void ktimer_begin(int id, cudaStream_t st);
void ktimer_end(int id, cudaStream_t st);
// algorithmic work (bytes or flops, per kernel id) accumulated while timing is on
void ktimer_add_work(int id, double work);
inline Error fail(int code, const std::string &m) { return Error{code, m}; }

// ------------------------------------------------------------------------ small utilities
constexpr int kWarp = 32;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Monotone maps to unsigned keys: a < b (as reals) <=> key(a) < key(b).  -0.0 and +0.0 map
// to different keys but are never compared as distinct values by the callers (they filter
// d < 0 first).
__host__ __device__ inline uint64_t f64_key(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double f64_from_key(uint64_t k) {
    uint64_t b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// ------------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_min(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_down_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    return x;
}

// Deterministic block sum (fixed order); result valid in thread 0.  `sh` needs
// blockDim.x/32 doubles.  Ends with a __syncthreads so `sh` can be reused.
template <typename T>
__device__ __forceinline__ T block_sum(T x, T *sh) {
    x = warp_sum(x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_min(double x, double *sh) {
    x = warp_min(x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    double r = INFINITY;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmin(r, sh[w]);
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------ grid barrier
// Sense-free generation barrier for kernels launched cooperatively (co-residency is then
// guaranteed).  bar[0] = arrival count (bar[1] unused).  Every wait is bounded: after
// ~kSpinLimit polls the barrier records OT_ERR_TIMEOUT in *err and returns false; callers
// leave the kernel as soon as a barrier returns false.
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, int *err) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int okv = 1;
        if (nblocks > 1) {
            // bar[0] counts arrivals over the whole launch (zeroed before it): the barrier this
            // arrival belongs to opens when the count reaches the next multiple of nblocks, so
            // the last arrival releases it by itself (no reset, no second word on the path)
            __threadfence();
            const unsigned arrived = atomicAdd(bar, 1u);
            const unsigned target = (arrived / nblocks + 1u) * nblocks;
            unsigned spins = 0;
            while ((int)(ld_acquire_gpu(bar) - target) < 0) {
                if (++spins > kSpinLimit || *(volatile int *)err) {
                    atomicCAS(err, 0, (int)OT_ERR_TIMEOUT);
                    okv = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        s_ok = okv;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace ot
