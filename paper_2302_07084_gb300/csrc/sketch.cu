// Sparse sign test matrix for the randomized SVD (Algorithm 4; Sec. 4.2
// names very sparse and sparse sign projections as cheaper alternatives to
// the Gaussian Omega; the construction follows Tropp et al., SISC 2019).
//
// Omega (n x c) has exactly zeta nonzeros +-1 per row, at distinct columns
// chosen by Floyd's subset sampling from Philox4x32-10 words: row i reads the
// words of counters (i, b, 0, 0x53505253), b = 0, 1, ..., with the Gaussian
// sketch's key; words 0..zeta-1 drive Floyd's steps, word zeta holds the signs
// (bit k set: the k-th chosen column is -1). A row is packed into 16 bytes:
// the column bytes in .x/.y/.z (zeta <= 12, c <= 255) and the sign bits in .w.
//
// Y = M Omega then costs zeta terms per nonzero of M instead of c: a warp
// takes a row of M, each lane one nonzero m_ik at a time, and adds +-m_ik into
// the zeta columns of Omega row k. The sums are kept in 64-bit fixed point
// (2^-32 units) in shared memory, so they are exact and independent of the
// order; each entry of Y is the sum rounded once to FP32.
#include <cmath>

#include "common.cuh"
#include "runtime.h"

namespace lne {
namespace {

constexpr uint32_t kSparseSignTag = 0x53505253u;
constexpr uint32_t kVerySparseTag = 0x56535250u;
constexpr int kSsWarps = 2;
constexpr int kSsUnroll = 4;

__device__ __forceinline__ uint32_t word_of(const u32x4 (&b)[4], int k) {
    const u32x4 &v = b[k >> 2];
    const int t = k & 3;
    return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
}

__global__ void sparse_sign_kernel(int64_t n, int c, int zeta, uint32_t k0, uint32_t k1,
                                   uint4 *__restrict__ packed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        u32x4 b[4];
        const int nblk = (zeta + 1 + 3) / 4;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < nblk) b[q] = philox10(u32x4{(uint32_t)i, (uint32_t)q, 0u, kSparseSignTag}, k0, k1);
        uint32_t col[kMaxSketchZeta];
#pragma unroll
        for (int k = 0; k < kMaxSketchZeta; ++k) {
            if (k >= zeta) break;
            // Floyd: j = c - zeta + k; t = word mod (j + 1); t unless taken, else j
            const uint32_t j = (uint32_t)(c - zeta + k);
            const uint32_t t = word_of(b, k) % (j + 1u);
            bool taken = false;
#pragma unroll
            for (int e = 0; e < kMaxSketchZeta; ++e)
                if (e < k) taken |= col[e] == t;
            col[k] = taken ? j : t;
        }
        uint4 pk = make_uint4(0u, 0u, 0u, word_of(b, zeta) & ((1u << zeta) - 1u));
#pragma unroll
        for (int k = 0; k < kMaxSketchZeta; ++k) {
            if (k >= zeta) break;
            const uint32_t v = col[k] << (8 * (k & 3));
            if (k < 4) pk.x |= v; else if (k < 8) pk.y |= v; else pk.z |= v;
        }
        packed[i] = pk;
    }
}

// Very sparse projection (Li, Hastie and Church, KDD 2006; Sec. 4.2 names it
// beside the sparse sign matrix): entry (i, j) is +1 if word j mod 4 of counter
// (i, j / 4, 0, 0x56535250) is below thr = floor(2^32 / (2 s)), -1 if it is in
// [thr, 2 thr), else 0. Row i is packed like a sparse sign row, with its
// nonzero count in bits 16..19 of .w; a row with more than kMaxSketchZeta
// nonzeros sets status[2] (its extra entries are dropped).
__global__ void very_sparse_kernel(int64_t n, int c, uint32_t thr, uint32_t k0, uint32_t k1,
                                   uint4 *__restrict__ packed, int *__restrict__ status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint4 pk = make_uint4(0u, 0u, 0u, 0u);
        int cnt = 0;
        for (int b = 0; b < (c + 3) / 4; ++b) {
            const u32x4 blk = philox10(u32x4{(uint32_t)i, (uint32_t)b, 0u, kVerySparseTag}, k0, k1);
            const uint32_t ws[4] = {blk.x, blk.y, blk.z, blk.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = 4 * b + t;
                const uint32_t w = ws[t];
                const bool pos = w < thr, neg = !pos && (w - thr) < thr;
                if (j >= c || !(pos || neg)) continue;
                if (cnt == kMaxSketchZeta) {
                    atomicExch(status + 2, 1);
                    continue;
                }
                const uint32_t v = (uint32_t)j << (8 * (cnt & 3));
                if (cnt < 4) pk.x |= v; else if (cnt < 8) pk.y |= v; else pk.z |= v;
                if (neg) pk.w |= 1u << cnt;
                ++cnt;
            }
        }
        pk.w |= (uint32_t)cnt << 16;
        packed[i] = pk;
    }
}

__device__ __forceinline__ int packed_col(const uint4 &pk, int k) {
    const uint32_t w = k < 4 ? pk.x : k < 8 ? pk.y : pk.z;
    return (int)((w >> (8 * (k & 3))) & 255u);
}

__global__ void sparse_sign_dense_kernel(int64_t n, int c, int zeta, const uint4 *__restrict__ packed,
                                         float *__restrict__ out, int64_t ld) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float *row = out + i * ld;
        for (int j = 0; j < c; ++j) row[j] = 0.f;
        const uint4 pk = packed[i];
        const int z = zeta > 0 ? zeta : (int)((pk.w >> 16) & 15u);
        for (int k = 0; k < z; ++k) row[packed_col(pk, k)] = (pk.w >> k) & 1u ? -1.f : 1.f;
    }
}

// A warp per row of M. Lane l adds the terms of nonzeros l, l + 32, ... of
// the row into its own fixed-point row, stored interleaved (entry (l, col) at
// col * 32 + l) so that the 32 lanes always hit 32 different banks; plain
// shared loads and stores, no atomics. At the end of the row lane j sums
// column j over the 32 lane rows, starting at lane row j so that the lanes
// again read different banks (integers: any order gives the same sum), and
// clears them.
__global__ void __launch_bounds__(kSsWarps * 32) sparse_sign_product_kernel(
    int64_t n, const int64_t *__restrict__ indptr, const int32_t *__restrict__ indices,
    const float *__restrict__ data, const uint4 *__restrict__ packed, int zeta, int c, float *__restrict__ Y,
    int64_t ldy) {
    extern __shared__ long long s_acc[];   // kSsWarps x c x 32
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long *wacc = s_acc + (size_t)warp * 32 * c;
    for (int j = 0; j < c; ++j) wacc[j * 32 + lane] = 0;
    __syncwarp();
    const int64_t nw = (int64_t)gridDim.x * kSsWarps;
    for (int64_t i = (int64_t)blockIdx.x * kSsWarps + warp; i < n; i += nw) {
        const int64_t a0 = __ldg(indptr + i), a1 = __ldg(indptr + i + 1);
        // Software pipeline over chunks of kSsUnroll nonzeros per lane: while
        // chunk t is added up, the Omega rows of chunk t + 1 and the indices
        // and values of chunk t + 2 are on their way.
        int32_t kn[kSsUnroll], kf[kSsUnroll];
        float mn[kSsUnroll], mf[kSsUnroll];
        uint4 pc[kSsUnroll], pn[kSsUnroll];
        float mc[kSsUnroll];
        auto load_idx = [&](int64_t ab, int32_t (&k)[kSsUnroll], float (&m)[kSsUnroll]) {
#pragma unroll
            for (int u = 0; u < kSsUnroll; ++u) {
                const int64_t a = ab + 32 * u;
                k[u] = a < a1 ? __ldg(indices + a) : -1;
                m[u] = a < a1 ? __ldg(data + a) : 0.f;
            }
        };
        auto load_rows = [&](const int32_t (&k)[kSsUnroll], uint4 (&pk)[kSsUnroll]) {
#pragma unroll
            for (int u = 0; u < kSsUnroll; ++u)
                pk[u] = k[u] >= 0 ? __ldg(packed + k[u]) : make_uint4(0u, 0u, 0u, 0u);
        };
        const int64_t step = 32 * kSsUnroll;
        load_idx(a0 + lane, kn, mc);
        load_rows(kn, pc);
        load_idx(a0 + lane + step, kn, mn);
        for (int64_t ab = a0 + lane; ab < a1; ab += step) {
            load_idx(ab + 2 * step, kf, mf);
            load_rows(kn, pn);
#pragma unroll
            for (int u = 0; u < kSsUnroll; ++u) {
                // m 2^32 is exact in FP32; rounding it to an integer moves it by at most 2^-33
                const long long q = __float2ll_rn(mc[u] * 4294967296.0f);
                // the zeta columns of one Omega row are distinct: their loads,
                // adds and stores are independent of one another (only the
                // next nonzero's may touch the same entries)
                const int z = zeta > 0 ? zeta : (int)((pc[u].w >> 16) & 15u);   // 0: per-row count
                long long v[kMaxSketchZeta];
#pragma unroll
                for (int k = 0; k < kMaxSketchZeta; ++k)
                    if (k < z) v[k] = wacc[packed_col(pc[u], k) * 32 + lane];
#pragma unroll
                for (int k = 0; k < kMaxSketchZeta; ++k)
                    if (k < z) wacc[packed_col(pc[u], k) * 32 + lane] = v[k] + ((pc[u].w >> k) & 1u ? -q : q);
            }
#pragma unroll
            for (int u = 0; u < kSsUnroll; ++u) {
                pc[u] = pn[u];
                mc[u] = mn[u];
                kn[u] = kf[u];
                mn[u] = mf[u];
            }
        }
        __syncwarp();
        float *yr = Y + i * ldy;
        for (int j = lane; j < c; j += 32) {
            long long sum = 0;
            long long *col = wacc + j * 32;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const int r = (l + j) & 31;
                sum += col[r];
                col[r] = 0;
            }
            yr[j] = __ll2float_rn(sum) * 2.3283064365386963e-10f;   // * 2^-32, exact
        }
        __syncwarp();
    }
}

int check_sparse_sign(int64_t n, int c, int zeta) {
    if (n < 0 || c < 1 || c > 255) return fail(LNE_ERR_INVALID, "sparse sign sketch needs 1 <= c <= 255");
    if (zeta < 1 || zeta > kMaxSketchZeta || zeta > c)
        return fail(LNE_ERR_INVALID, "sparse sign sketch needs 1 <= zeta <= min(12, c)");
    return 0;
}

unsigned rows_grid(int64_t n, int per_block) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, (int64_t)per_block), num_sms() * 16));
}

int check_very_sparse(int64_t n, int c, double s) {
    if (n < 0 || c < 1 || c > 255) return fail(LNE_ERR_INVALID, "very sparse projection needs 1 <= c <= 255");
    if (!(s >= 1.0) || !std::isfinite(s)) return fail(LNE_ERR_INVALID, "very sparse projection needs s >= 1");
    return 0;
}

}  // namespace

double very_sparse_s(int64_t n, double s) { return s > 0.0 ? s : std::sqrt((double)std::max<int64_t>(n, 1)); }

int very_sparse_sketch(Workspace &ws, int64_t n, int c, double s, uint64_t seed, const uint4 **packed,
                       cudaStream_t st) {
    s = very_sparse_s(n, s);
    LNE_TRY(check_very_sparse(n, c, s));
    uint4 *pk = nullptr;
    int *status = nullptr;
    LNE_TRY(ws.get("sketch.packed", (size_t)std::max<int64_t>(n, 1), &pk));
    LNE_TRY(device_status(ws, &status, st));
    const uint32_t thr = (uint32_t)std::floor(4294967296.0 / (2.0 * s));
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu) ^ 0x4f4d4547u;
    const uint32_t k1 = (uint32_t)(seed >> 32);
    if (n > 0) {
        LNE_TRACE("sketch", st);
        very_sparse_kernel<<<rows_grid(n, 256), 256, 0, st>>>(n, c, thr, k0, k1, pk, status);
        LNE_LAUNCH_CHECK();
    }
    *packed = pk;
    return 0;
}

int very_sparse_dense(Workspace &ws, int64_t n, int c, double s, uint64_t seed, float *out, int64_t ld,
                      cudaStream_t st) {
    if (ld < c) return fail(LNE_ERR_INVALID, "ld must be >= c");
    const uint4 *pk = nullptr;
    LNE_TRY(very_sparse_sketch(ws, n, c, s, seed, &pk, st));
    if (n > 0) {
        LNE_TRACE("sketch", st);
        sparse_sign_dense_kernel<<<rows_grid(n, 256), 256, 0, st>>>(n, c, 0, pk, out, ld);
        LNE_LAUNCH_CHECK();
    }
    return status_check(ws, st);
}

int very_sparse_spmm(Workspace &ws, const CsrView &M, int c, double s, uint64_t seed, float *Y, int64_t ldy,
                     cudaStream_t st) {
    if (ldy < c) return fail(LNE_ERR_INVALID, "ldy must be >= c");
    const uint4 *pk = nullptr;
    LNE_TRY(very_sparse_sketch(ws, M.n, c, s, seed, &pk, st));
    if (M.n > 0) {
        LNE_TRACE("sparse_sign_spmm", st);
        const int smem = kSsWarps * 32 * c * (int)sizeof(long long);
        LNE_TRY(allow_dynamic_smem(sparse_sign_product_kernel));
        sparse_sign_product_kernel<<<rows_grid(M.n, kSsWarps), kSsWarps * 32, smem, st>>>(
            M.n, M.indptr, M.indices, M.data, pk, 0, c, Y, ldy);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int sparse_sign_sketch(Workspace &ws, int64_t n, int c, int zeta, uint64_t seed, const uint4 **packed,
                       cudaStream_t st) {
    LNE_TRY(check_sparse_sign(n, c, zeta));
    uint4 *pk = nullptr;
    LNE_TRY(ws.get("sketch.packed", (size_t)std::max<int64_t>(n, 1), &pk));
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu) ^ 0x4f4d4547u;
    const uint32_t k1 = (uint32_t)(seed >> 32);
    if (n > 0) {
        LNE_TRACE("sketch", st);
        sparse_sign_kernel<<<rows_grid(n, 256), 256, 0, st>>>(n, c, zeta, k0, k1, pk);
        LNE_LAUNCH_CHECK();
    }
    *packed = pk;
    return 0;
}

int sparse_sign_dense(Workspace &ws, int64_t n, int c, int zeta, uint64_t seed, float *out, int64_t ld,
                      cudaStream_t st) {
    if (ld < c) return fail(LNE_ERR_INVALID, "ld must be >= c");
    const uint4 *pk = nullptr;
    LNE_TRY(sparse_sign_sketch(ws, n, c, zeta, seed, &pk, st));
    if (n > 0) {
        LNE_TRACE("sketch", st);
        sparse_sign_dense_kernel<<<rows_grid(n, 256), 256, 0, st>>>(n, c, zeta, pk, out, ld);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int sparse_sign_spmm(Workspace &ws, const CsrView &M, int c, int zeta, uint64_t seed, float *Y, int64_t ldy,
                     cudaStream_t st) {
    if (ldy < c) return fail(LNE_ERR_INVALID, "ldy must be >= c");
    const uint4 *pk = nullptr;
    LNE_TRY(sparse_sign_sketch(ws, M.n, c, zeta, seed, &pk, st));
    if (M.n > 0) {
        LNE_TRACE("sparse_sign_spmm", st);
        const int smem = kSsWarps * 32 * c * (int)sizeof(long long);
        LNE_TRY(allow_dynamic_smem(sparse_sign_product_kernel));
        sparse_sign_product_kernel<<<rows_grid(M.n, kSsWarps), kSsWarps * 32, smem, st>>>(
            M.n, M.indptr, M.indices, M.data, pk, zeta, c, Y, ldy);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

}  // namespace lne
