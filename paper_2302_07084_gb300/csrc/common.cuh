// Shared device helpers of the LightNE 2.0 GB300 path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lne.h"

namespace lne {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies
// with Weyl-sequence key bumps. Counter-based, so every (sample, block) pair
// has its own independent 128-bit output.
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ u32x4 philox10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        uint32_t lo1 = 0xCD9E8D57u * c.z;
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        u32x4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Error state shared by host code of the library.
struct Status {
    int code = 0;
    std::string msg;
};

#define LNE_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            return ::lne::cuda_fail(#expr, _e, __FILE__, __LINE__);                 \
        }                                                                           \
    } while (0)

#define LNE_LAUNCH_CHECK()                                                          \
    do {                                                                            \
        ::lne::count_launch();                                                      \
        cudaError_t _e = cudaGetLastError();                                        \
        if (_e != cudaSuccess) return ::lne::cuda_fail("kernel launch", _e, __FILE__, __LINE__); \
    } while (0)

#define LNE_TRY(expr)                                                               \
    do {                                                                            \
        int _r = (expr);                                                            \
        if (_r != 0) return _r;                                                     \
    } while (0)

// Records the failure in the thread's last-error slot and returns LNE_ERR_CUDA
// (or LNE_ERR_OOM for allocation failures).
int cuda_fail(const char *what, cudaError_t e, const char *file, int line);
// Process-wide count of kernel launches made by this library.
void count_launch();
// The calling thread's tracer (set by every context entry point; NULL = none).
struct Tracer;
void set_tracer(Tracer *t);
Tracer *get_tracer();
// Kernels counted so far (count_launch); add_launches counts n kernels that a
// CUDA graph replay runs.
int64_t launches_now();
void add_launches(int64_t n);
// Named timing regions: when the calling context has tracing on, a region
// records a CUDA event pair on the launching stream around its kernels.
void trace_begin(const char *name, cudaStream_t st);
void trace_end(cudaStream_t st);
struct TraceScope {
    cudaStream_t st;
    TraceScope(const char *name, cudaStream_t s) : st(s) { trace_begin(name, s); }
    ~TraceScope() { trace_end(st); }
};
#define LNE_CAT2(a, b) a##b
#define LNE_CAT(a, b) LNE_CAT2(a, b)
#define LNE_TRACE(name, st) ::lne::TraceScope LNE_CAT(_lne_trace_, __LINE__)(name, st)
int fail(int code, const std::string &msg);
const std::string &last_message();
void clear_message();

// Whether (kernel, device) has had its dynamic shared-memory limit raised,
// and the mark set once it has (thread-safe).
bool smem_limit_raised(const void *kernel, int dev);
void mark_smem_limit_raised(const void *kernel, int dev);

// Let `kernel` use as much dynamic shared memory as the device allows beside
// its static shared memory. The value is the same on every call, so host
// threads that launch the kernel concurrently cannot lower the limit under one
// another's launch; it is set once per kernel and device (the attribute
// calls take microseconds of host time, which would stall a stream of short
// kernels).
template <typename Kernel>
inline int allow_dynamic_smem(Kernel kernel) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e, __FILE__, __LINE__);
    if (smem_limit_raised(reinterpret_cast<const void *>(kernel), dev)) return 0;
    cudaFuncAttributes fa;
    int optin = 0;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return cuda_fail("cudaFuncSetAttribute", e, __FILE__, __LINE__);
    mark_smem_limit_raised(reinterpret_cast<const void *>(kernel), dev);
    return 0;
}

// Streaming multiprocessors of the current device (queried once per device
// and cached): grids are sized in multiples of it.
int num_sms();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

}  // namespace lne
