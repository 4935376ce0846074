// Sparse sign test matrix for the randomized SVD (Algorithm 4; Sec. 3.2
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
#include "common.cuh"
#include "runtime.h"

namespace lne {
namespace {

constexpr uint32_t kSparseSignTag = 0x53505253u;
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
        for (int k = 0; k < zeta; ++k) row[packed_col(pk, k)] = (pk.w >> k) & 1u ? -1.f : 1.f;
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
                long long v[kMaxSketchZeta];
#pragma unroll
                for (int k = 0; k < kMaxSketchZeta; ++k)
                    if (k < zeta) v[k] = wacc[packed_col(pc[u], k) * 32 + lane];
#pragma unroll
                for (int k = 0; k < kMaxSketchZeta; ++k)
                    if (k < zeta) wacc[packed_col(pc[u], k) * 32 + lane] = v[k] + ((pc[u].w >> k) & 1u ? -q : q);
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

}  // namespace

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
