// Exclusive prefix sums used to turn per-tile / per-bucket / per-row counts
// into offsets. One CTA walks the array in chunks (the arrays scanned here are
// at most a few million entries: tiles, buckets or rows), so the result is
// deterministic and needs no inter-CTA protocol.
#include "runtime.h"

namespace lne {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;

// One CTA per row: row b scans in[b * stride .. + n) into out[b * stride ..],
// out[b * stride + n] = the row total (in and out may be the same array).
template <typename In>
__global__ void __launch_bounds__(kScanThreads) scan_exclusive_kernel(const In *in, int64_t *out,
                                                                      int64_t n, int64_t stride = 0) {
    in += (int64_t)blockIdx.x * stride;
    out += (int64_t)blockIdx.x * stride;
    __shared__ int64_t warp_sums[kScanThreads / 32];
    __shared__ int64_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    const int64_t chunk = (int64_t)kScanThreads * kScanItems;
    for (int64_t base = 0; base < n; base += chunk) {
        int64_t v[kScanItems];
        int64_t local = 0;
        const int64_t i0 = base + (int64_t)tid * kScanItems;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            int64_t idx = i0 + j;
            v[j] = idx < n ? (int64_t)in[idx] : 0;
            local += v[j];
        }
        // inclusive warp scan of the per-thread totals
        int64_t x = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            if (lane < kScanThreads / 32) warp_sums[lane] = w;   // inclusive
        }
        __syncthreads();
        const int64_t carry = carry_s;
        int64_t run = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + x - local;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            int64_t idx = i0 + j;
            if (idx < n) out[idx] = run;
            run += v[j];
        }
        __syncthreads();
        if (tid == kScanThreads - 1) carry_s = run;
        __syncthreads();
    }
    if (tid == 0) out[n] = carry_s;
}

}  // namespace

int scan_exclusive_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    {
        LNE_TRACE("scan_exclusive", st);
        scan_exclusive_kernel<uint32_t><<<1, kScanThreads, 0, st>>>(in, out, n);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int scan_exclusive_rows_i64(int64_t *data, int64_t rows, int64_t n, cudaStream_t st) {
    if (rows <= 0) return 0;
    LNE_TRACE("scan_rows", st);
    scan_exclusive_kernel<int64_t><<<(unsigned)rows, kScanThreads, 0, st>>>(data, data, n, n + 1);
    LNE_LAUNCH_CHECK();
    return 0;
}

int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    {
        LNE_TRACE("scan_exclusive", st);
        scan_exclusive_kernel<int64_t><<<1, kScanThreads, 0, st>>>(in, out, n);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

}  // namespace lne
