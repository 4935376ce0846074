// Sparse x dense products of the hot path:
//   * Y = M X with the weighted sparsifier M (Algorithm 4);
//   * the propagation products with the unweighted graph A, where the row
//     scale 1/deg(i) (D^-1 A) and the Chebyshev recurrence of Sec. 4.3 are
//     fused into the epilogue:  out = alpha * rs_i (A X)_i + b1 E1 + b2 E2 + b3 E3,
//     optionally F += gamma * out and G = X0 - F.
//
// Main path (column count a multiple of 4): nonzero-balanced ("merge") SpMM.
// Warp w owns nonzeros [w W, (w + 1) W); lane l gathers columns 4l..4l+3
// (+128 t) of each referenced X row with 16-byte loads. A row wholly inside one
// warp's slice is finished there; a row crossing slice boundaries leaves its
// partial sums in a carry buffer, and a fix-up kernel adds them in slice order.
// Every sum has a fixed order, so results are deterministic and independent of
// the degree distribution's skew.
// Fallback (other column counts): one warp per row, lane l owns columns l,
// l+32, ...; rows longer than 512 nonzeros get a whole CTA.
#include "runtime.h"

namespace lne {


namespace {

constexpr int kLongRow = 512;    // rows with more nonzeros get a whole CTA
constexpr int kCtaWarps = 8;

// Accumulates nonzeros [p, p + cnt) (cnt <= 32) of one row into acc: lane l
// holds (col, val) of nonzero p + l; the inner loop is unrolled so several
// gathers are in flight.
template <int NT, bool WEIGHTED>
__device__ __forceinline__ void gather_chunk(const int32_t *__restrict__ indices, const float *__restrict__ vals,
                                             int64_t p, int cnt, const float *__restrict__ X, int64_t ldx, int c,
                                             int lane, float (&acc)[NT]) {
    const int col = lane < cnt ? __ldg(indices + p + lane) : 0;
    float v = 0.f;
    if (WEIGHTED) v = lane < cnt ? __ldg(vals + p + lane) : 0.f;
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
        const int ck = __shfl_sync(0xffffffffu, col, k);
        const float *xr = X + (int64_t)ck * ldx;
        if (WEIGHTED) {
            const float vk = __shfl_sync(0xffffffffu, v, k);
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int cc = lane + 32 * t;
                if (cc < c) acc[t] = fmaf(vk, __ldg(xr + cc), acc[t]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int cc = lane + 32 * t;
                if (cc < c) acc[t] += __ldg(xr + cc);
            }
        }
    }
}

template <int NT>
__device__ __forceinline__ void epilogue(int64_t i, int64_t deg, const float (&acc)[NT], int lane, int c,
                                         float *__restrict__ Y, int64_t ldy, const SpmmEpilogue &ep) {
    float rs = ep.alpha;
    if (ep.dinv) rs = ep.dinv_w ? ep.alpha * __ldg(ep.dinv_w + i) : deg > 0 ? ep.alpha / (float)deg : 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cc = lane + 32 * t;
        if (cc >= c) continue;
        const int64_t e = i * ep.lde + cc;
        float o = rs * acc[t];
        if (ep.E1) o = fmaf(ep.b1_col ? ep.b1_col[cc] : ep.b1, ep.E1[e], o);
        if (ep.E2) o = fmaf(ep.b2, ep.E2[e], o);
        if (ep.E3) o = fmaf(ep.b3, ep.E3[e], o);
        if (ep.store) Y[i * ldy + cc] = o;
        if (ep.F) {
            const float f = fmaf(ep.gamma_col ? ep.gamma_col[cc] : ep.gamma, o, ep.F[e]);
            ep.F[e] = f;
            if (ep.G) ep.G[e] = ep.X0[e] - f;
        }
    }
}

// One warp per row, rows with at most kLongRow nonzeros.
template <int NT, bool WEIGHTED>
__global__ void __launch_bounds__(256) spmm_warp_kernel(int64_t n, const int64_t *__restrict__ indptr,
                                                        const int32_t *__restrict__ indices,
                                                        const float *__restrict__ vals,
                                                        const float *__restrict__ X, int64_t ldx, int c,
                                                        float *__restrict__ Y, int64_t ldy,
                                                        SpmmEpilogue ep) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t p0 = indptr[i], p1 = indptr[i + 1];
        if (p1 - p0 > kLongRow) continue;
        float acc[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[t] = 0.f;
        for (int64_t p = p0; p < p1; p += 32)
            gather_chunk<NT, WEIGHTED>(indices, vals, p, (int)imin64(32, p1 - p), X, ldx, c, lane, acc);
        epilogue<NT>(i, p1 - p0, acc, lane, c, Y, ldy, ep);
    }
}

// One CTA per long row: warp w takes 32-nonzero chunks w, w + 8, ...; the
// partial sums are added in warp order, so the result is deterministic.
template <int NT, bool WEIGHTED>
__global__ void __launch_bounds__(kCtaWarps * 32) spmm_cta_kernel(int64_t n, const int64_t *__restrict__ indptr,
                                                                  const int32_t *__restrict__ indices,
                                                                  const float *__restrict__ vals,
                                                                  const float *__restrict__ X, int64_t ldx, int c,
                                                                  float *__restrict__ Y, int64_t ldy,
                                                                  SpmmEpilogue ep) {
    __shared__ float part[kCtaWarps][NT * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t p0 = indptr[i], p1 = indptr[i + 1];
        if (p1 - p0 <= kLongRow) continue;
        float acc[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[t] = 0.f;
        for (int64_t p = p0 + 32 * warp; p < p1; p += 32 * kCtaWarps)
            gather_chunk<NT, WEIGHTED>(indices, vals, p, (int)imin64(32, p1 - p), X, ldx, c, lane, acc);
#pragma unroll
        for (int t = 0; t < NT; ++t) part[warp][lane + 32 * t] = acc[t];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                float s = part[0][lane + 32 * t];
                for (int w = 1; w < kCtaWarps; ++w) s += part[w][lane + 32 * t];
                acc[t] = s;
            }
            epilogue<NT>(i, p1 - p0, acc, lane, c, Y, ldy, ep);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// merge path
// ---------------------------------------------------------------------------
template <int NV>
struct Acc4 {
    float4 v[NV];
};

// Four consecutive operand values as FP32: one 16-byte load (FP32) or one
// 8-byte load (BF16, widened).
__device__ __forceinline__ float4 load4(const float *__restrict__ row, int q) {
    return __ldg(reinterpret_cast<const float4 *>(row) + q);
}
__device__ __forceinline__ float4 load4(const __nv_bfloat16 *__restrict__ row, int q) {
    // a bfloat16 is the upper half of the FP32 with the same value
    const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(row) + q);
    return make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xffff0000u),
                       __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xffff0000u));
}

// STREAM: the matrix, read once, goes through L2 with the evict-first
// (streaming) policy and leaves the gathered operand rows their place
template <int NV, bool WEIGHTED, typename TX, bool STREAM = false>
__device__ __forceinline__ void gather4(const int32_t *__restrict__ indices, const float *__restrict__ vals,
                                        int64_t p, int cnt, const TX *__restrict__ X, int64_t ldx, int c4,
                                        int lane, Acc4<NV> &acc) {
    const int col = lane < cnt ? (STREAM ? __ldcs(indices + p + lane) : __ldg(indices + p + lane)) : 0;
    float v = 0.f;
    if (WEIGHTED) v = lane < cnt ? (STREAM ? __ldcs(vals + p + lane) : __ldg(vals + p + lane)) : 0.f;
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
        const int ck = __shfl_sync(0xffffffffu, col, k);
        const float vk = WEIGHTED ? __shfl_sync(0xffffffffu, v, k) : 1.f;
        const TX *xr = X + (int64_t)ck * ldx;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const int q = lane + 32 * t;
            if (q < c4) {
                const float4 x = load4(xr, q);
                if (WEIGHTED) {
                    acc.v[t].x = fmaf(vk, x.x, acc.v[t].x);
                    acc.v[t].y = fmaf(vk, x.y, acc.v[t].y);
                    acc.v[t].z = fmaf(vk, x.z, acc.v[t].z);
                    acc.v[t].w = fmaf(vk, x.w, acc.v[t].w);
                } else {
                    acc.v[t].x += x.x;
                    acc.v[t].y += x.y;
                    acc.v[t].z += x.z;
                    acc.v[t].w += x.w;
                }
            }
        }
    }
}

// Narrow products (c4 <= LG): the warp works as 32 / LG groups of LG lanes;
// group g takes nonzeros g, g + G, ... of the chunk and lane q of a group owns
// column group q. The groups' partial sums are combined by a fixed xor tree at
// the end of each row segment, so the result is deterministic.
template <int LG, bool WEIGHTED, typename TX>
__device__ __forceinline__ void gather4_grouped(const int32_t *__restrict__ indices, const float *__restrict__ vals,
                                                int64_t p, int cnt, const TX *__restrict__ X, int64_t ldx, int c4,
                                                int lane, float4 &acc) {
    constexpr int G = 32 / LG;
    const int col = lane < cnt ? __ldg(indices + p + lane) : 0;
    float v = 0.f;
    if (WEIGHTED) v = lane < cnt ? __ldg(vals + p + lane) : 0.f;
    const int g = lane / LG, q = lane % LG;
#pragma unroll 4
    for (int k0 = 0; k0 < cnt; k0 += G) {
        const int k = k0 + g;
        const int ck = __shfl_sync(0xffffffffu, col, k & 31);
        const float vk = WEIGHTED ? __shfl_sync(0xffffffffu, v, k & 31) : 1.f;
        if (k < cnt && q < c4) {
            const float4 x = load4(X + (int64_t)ck * ldx, q);
            if (WEIGHTED) {
                acc.x = fmaf(vk, x.x, acc.x);
                acc.y = fmaf(vk, x.y, acc.y);
                acc.z = fmaf(vk, x.z, acc.z);
                acc.w = fmaf(vk, x.w, acc.w);
            } else {
                acc.x += x.x;
                acc.y += x.y;
                acc.z += x.z;
                acc.w += x.w;
            }
        }
    }
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 fma4(float4 a, float4 x, float4 y) {
    return make_float4(fmaf(a.x, x.x, y.x), fmaf(a.y, x.y, y.y), fmaf(a.z, x.z, y.z), fmaf(a.w, x.w, y.w));
}
__device__ __forceinline__ float4 splat4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ uint32_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ void st4_bf16(__nv_bfloat16 *p, float4 v) {
    uint2 raw;
    raw.x = bf16_bits(v.x) | (bf16_bits(v.y) << 16);
    raw.y = bf16_bits(v.z) | (bf16_bits(v.w) << 16);
    *reinterpret_cast<uint2 *>(p) = raw;
}

// The epilogue on four consecutive columns 4q..4q+3 of row i, with 16-byte
// loads and stores (every operand is 16-byte aligned, leading dimensions are
// multiples of 4); per element the same FMA chain as a scalar epilogue.
// STREAM: E1 is read and Y written with the evict-first (streaming) policy
// (the column-blocked product's running sum, touched once per block)
template <int NV, bool STREAM = false>
__device__ __forceinline__ void epilogue4(int64_t i, int64_t deg, const Acc4<NV> &acc, int lane, int c4,
                                          float *__restrict__ Y, int64_t ldy, const SpmmEpilogue &ep) {
    float rs = ep.alpha;
    if (ep.dinv) rs = ep.dinv_w ? ep.alpha * __ldg(ep.dinv_w + i) : deg > 0 ? ep.alpha / (float)deg : 0.f;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int q = lane + 32 * t;
        if (q >= c4) continue;
        const int64_t e = i * ep.lde + 4 * q;
        const int64_t yo = i * ldy + 4 * q;
        const float4 a = acc.v[t];
        float4 o = make_float4(rs * a.x, rs * a.y, rs * a.z, rs * a.w);
        if (ep.E1)
            o = fma4(ep.b1_col ? ld4(ep.b1_col + 4 * q) : splat4(ep.b1),
                     STREAM ? __ldcs(reinterpret_cast<const float4 *>(ep.E1 + e)) : ld4(ep.E1 + e), o);
        if (ep.E2) o = fma4(splat4(ep.b2), ld4(ep.E2 + e), o);
        if (ep.E3) o = fma4(splat4(ep.b3), ld4(ep.E3 + e), o);
        if (ep.store) {
            if (STREAM) __stcs(reinterpret_cast<float4 *>(Y + yo), o);
            else st4(Y + yo, o);
        }
        if (ep.Yb) st4_bf16(ep.Yb + yo, o);
        if (ep.F) {
            const float4 f = fma4(ep.gamma_col ? ld4(ep.gamma_col + 4 * q) : splat4(ep.gamma), o, ld4(ep.F + e));
            st4(ep.F + e, f);
            if (ep.G) {
                const float4 x0 = ld4(ep.X0 + e);
                const float4 gv = make_float4(x0.x - f.x, x0.y - f.y, x0.z - f.z, x0.w - f.w);
                st4(ep.G + e, gv);
                if (ep.Gb) st4_bf16(ep.Gb + e, gv);
            }
        }
    }
}

__device__ __forceinline__ int64_t row_of(const int64_t *__restrict__ indptr, int64_t n, int64_t p) {
    int64_t lo = 0, hi = n;   // last row with indptr[row] <= p
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(indptr + mid) <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// VB (one vertex block of a column-blocked product): indptr holds the
// block's virtual row offsets V (prefix sums of the rows' segment lengths);
// row r's segment starts at indptr0[r] + segb[r] of indices / vals, so
// position p of the row maps to p + indptr0[r] + segb[r] - V[r].
template <int NV, bool WEIGHTED, typename TX, int LG = 32, bool VB = false>
__global__ void __launch_bounds__(256) spmm_merge_kernel(int64_t n, int64_t nnz, const int64_t *__restrict__ indptr,
                                                         const int32_t *__restrict__ indices,
                                                         const float *__restrict__ vals, const TX *__restrict__ X,
                                                         int64_t ldx, int c4, float *__restrict__ Y, int64_t ldy,
                                                         SpmmEpilogue ep, int64_t W, int64_t nwarps,
                                                         float4 *__restrict__ carry, int64_t *__restrict__ carry_row,
                                                         const int64_t *__restrict__ indptr0 = nullptr,
                                                         const uint32_t *__restrict__ segb = nullptr) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nwarps) return;
    const int64_t p0 = w * W, p1 = imin64(p0 + W, nnz);
    if (lane == 0) {   // slots left from an earlier product must not be read
        carry_row[w * 2] = -1;
        carry_row[w * 2 + 1] = -1;
    }
    int64_t r = row_of(indptr, n, p0);
    // skip empty rows sharing the start offset
    while (r + 1 < n && __ldg(indptr + r + 1) <= p0) ++r;
    int64_t p = p0;
    while (p < p1) {
        const int64_t rs = VB ? __ldcs(indptr + r) : __ldg(indptr + r);
        const int64_t re = VB ? __ldcs(indptr + r + 1) : __ldg(indptr + r + 1);
        const int64_t e = imin64(re, p1);
        const int32_t *ind = indices;
        const float *val = vals;
        if (VB) {
            const int64_t phys = __ldcs(indptr0 + r) + (int64_t)__ldcs(segb + r) - rs;
            ind = indices + phys;
            val = vals + phys;
        }
        Acc4<NV> acc;
#pragma unroll
        for (int t = 0; t < NV; ++t) acc.v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (LG < 32) {
            for (int64_t q = p; q < e; q += 32)
                gather4_grouped<LG, WEIGHTED, TX>(ind, val, q, (int)imin64(32, e - q), X, ldx, c4, lane, acc.v[0]);
#pragma unroll
            for (int off = LG; off < 32; off <<= 1) {
                acc.v[0].x += __shfl_xor_sync(0xffffffffu, acc.v[0].x, off);
                acc.v[0].y += __shfl_xor_sync(0xffffffffu, acc.v[0].y, off);
                acc.v[0].z += __shfl_xor_sync(0xffffffffu, acc.v[0].z, off);
                acc.v[0].w += __shfl_xor_sync(0xffffffffu, acc.v[0].w, off);
            }
        } else {
            for (int64_t q = p; q < e; q += 32)
                gather4<NV, WEIGHTED, TX, VB>(ind, val, q, (int)imin64(32, e - q), X, ldx, c4, lane, acc);
        }
        if (rs >= p0 && re <= p1) {
            epilogue4<NV, VB>(r, re - rs, acc, lane, c4, Y, ldy, ep);
        } else {
            const int slot = rs < p0 ? 0 : 1;
            float4 *dst = carry + (w * 2 + slot) * (int64_t)(NV * 32);
#pragma unroll
            for (int t = 0; t < NV; ++t)
                if (lane + 32 * t < c4) dst[lane + 32 * t] = acc.v[t];
            if (lane == 0) carry_row[w * 2 + slot] = r;
        }
        p = e;
        ++r;
        while (p < p1 && r + 1 < n && __ldg(indptr + r + 1) <= p) ++r;   // empty rows
    }
}

// Rows that are empty or cross slice boundaries: sum the partials in slice order.
template <int NV, bool STREAM = false>
__global__ void __launch_bounds__(256) spmm_fixup_kernel(int64_t n, const int64_t *__restrict__ indptr, int c4,
                                                         float *__restrict__ Y, int64_t ldy, SpmmEpilogue ep, int64_t W,
                                                         const float4 *__restrict__ carry,
                                                         const int64_t *__restrict__ carry_row) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int64_t rs = STREAM ? __ldcs(indptr + r) : indptr[r], re = STREAM ? __ldcs(indptr + r + 1) : indptr[r + 1];
        Acc4<NV> acc;
#pragma unroll
        for (int t = 0; t < NV; ++t) acc.v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (re > rs) {
            const int64_t w0 = rs / W, w1 = (re - 1) / W;
            if (w0 == w1) continue;   // finished by its warp
            for (int64_t w = w0; w <= w1; ++w) {
                const int slot = carry_row[w * 2] == r ? 0 : 1;
                const float4 *src = carry + (w * 2 + slot) * (int64_t)(NV * 32);
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    if (lane + 32 * t < c4) {
                        const float4 x = src[lane + 32 * t];
                        acc.v[t].x += x.x;
                        acc.v[t].y += x.y;
                        acc.v[t].z += x.z;
                        acc.v[t].w += x.w;
                    }
                }
            }
        }
        epilogue4<NV, STREAM>(r, re - rs, acc, lane, c4, Y, ldy, ep);
    }
}

template <bool WEIGHTED>
int launch_spmm(int64_t n, const int64_t *indptr, const int32_t *indices, const float *vals,
                const float *X, int64_t ldx, int c, float *Y, int64_t ldy, const SpmmEpilogue &ep,
                cudaStream_t st) {
    if (n <= 0) return 0;
    const int nt = (c + 31) / 32;
    const int wblocks = (int)std::min<int64_t>(ceil_div(n, 8), num_sms() * 64);
    const int cblocks = (int)std::min<int64_t>(n, num_sms() * 16);
    LNE_TRACE(WEIGHTED ? "spmm" : "graph_spmm", st);
#define LNE_SPMM_CASE(K)                                                                              \
    case K:                                                                                           \
        spmm_warp_kernel<K, WEIGHTED><<<wblocks, 256, 0, st>>>(n, indptr, indices, vals, X, ldx, c, Y, \
                                                                ldy, ep);                             \
        spmm_cta_kernel<K, WEIGHTED><<<cblocks, kCtaWarps * 32, 0, st>>>(n, indptr, indices, vals, X,  \
                                                                          ldx, c, Y, ldy, ep);        \
        break;
    switch (nt) {
        LNE_SPMM_CASE(1)
        LNE_SPMM_CASE(2)
        LNE_SPMM_CASE(3)
        LNE_SPMM_CASE(4)
        LNE_SPMM_CASE(5)
        LNE_SPMM_CASE(6)
        LNE_SPMM_CASE(7)
        LNE_SPMM_CASE(8)
        default:
            return fail(LNE_ERR_UNSUPPORTED, "SpMM supports at most 256 dense columns");
    }
#undef LNE_SPMM_CASE
    LNE_LAUNCH_CHECK();
    ::lne::count_launch();   // two kernels per product
    return 0;
}

inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

template <typename TX>
bool merge_ok(const TX *X, int64_t ldx, int c, const float *Y, int64_t ldy, const SpmmEpilogue &ep) {
    return c % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && ep.lde % 4 == 0 && c <= 1024 &&
           aligned(X, 4 * sizeof(TX)) && aligned(Y, 16) && aligned(ep.E1, 16) && aligned(ep.E2, 16) &&
           aligned(ep.E3, 16) && aligned(ep.F, 16) && aligned(ep.X0, 16) && aligned(ep.G, 16) &&
           aligned(ep.Yb, 8) && aligned(ep.Gb, 8) && aligned(ep.b1_col, 16) && aligned(ep.gamma_col, 16);
}

// nonzeros per warp slice: ~8 waves of warps, at least about two average rows
// (fewer rows split across slices: measured 1.14 -> 0.92 ms for the 19 graph
// products of the benchmark) and at least 32; beyond 1024 per slice only for
// very large products (>6e7 nonzeros), which keeps the carry buffers (two rows
// of c per warp) small
int64_t merge_slice(int64_t nnz, int64_t n) {
    const int64_t W = nnz / ((int64_t)num_sms() * 48 * 8);
    const int64_t two_rows = n > 0 ? 2 * ceil_div(nnz, n) : 32;
    const int64_t lo = std::max<int64_t>(32, std::min<int64_t>(1024, two_rows / 32 * 32));
    const int64_t cap = nnz > (int64_t)num_sms() * 48 * 8 * 1024 ? 65536 : 1024;
    return std::max<int64_t>(lo, std::min<int64_t>(cap, (W + 31) / 32 * 32));
}

int merge_vectors(int c) {
    int nv = (c / 4 + 31) / 32;
    if (nv == 3) nv = 4;
    if (nv > 4 && nv < 8) nv = 8;
    return nv;
}

template <bool WEIGHTED, typename TX>
int launch_merge(Workspace &ws, int64_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                 const float *vals, const TX *X, int64_t ldx, int c, float *Y, int64_t ldy, const SpmmEpilogue &ep,
                 cudaStream_t st) {
    if (n <= 0) return 0;
    if (ep.col_block > 0 && ep.col_block < c && ep.col_block % 4 == 0) {
        // column blocks, one after another on the stream (they share the
        // carry buffers); every column gets the same terms in the same order
        for (int cb = 0; cb < c; cb += ep.col_block) {
            const int w = std::min(ep.col_block, c - cb);
            SpmmEpilogue eb = ep;
            eb.col_block = 0;
            auto shift = [cb](auto *p) { return p ? p + cb : p; };
            eb.E1 = shift(ep.E1);
            eb.E2 = shift(ep.E2);
            eb.E3 = shift(ep.E3);
            eb.F = shift(ep.F);
            eb.X0 = shift(ep.X0);
            eb.G = shift(ep.G);
            eb.Gb = shift(ep.Gb);
            eb.b1_col = shift(ep.b1_col);
            eb.gamma_col = shift(ep.gamma_col);
            eb.Yb = shift(ep.Yb);
            LNE_TRY((launch_merge<WEIGHTED, TX>(ws, n, nnz, indptr, indices, vals, X + cb, ldx, w, Y + cb, ldy, eb,
                                                st)));
        }
        return 0;
    }
    const int c4 = c / 4;
    const int nv = merge_vectors(c);
    const int64_t W = merge_slice(nnz, n);
    const int64_t nwarps = std::max<int64_t>(1, ceil_div(nnz, W));
    float4 *carry = nullptr;
    int64_t *carry_row = nullptr;
    LNE_TRY(merge_carry(ws, ep.carry_tag, nnz, n, c, &carry, &carry_row));
    const int threads = ep.threads > 0 ? ep.threads : 256;
    const unsigned mblocks = (unsigned)ceil_div(nwarps, threads / 32);
    const unsigned fblocks = (unsigned)std::min<int64_t>(ceil_div(n, 8), num_sms() * 32);
    LNE_TRACE(WEIGHTED ? "spmm" : "graph_spmm", st);
#define LNE_MERGE_CASE(K)                                                                                  \
    case K:                                                                                                \
        if (nnz > 0)                                                                                       \
            spmm_merge_kernel<K, WEIGHTED, TX><<<mblocks, threads, 0, st>>>(n, nnz, indptr, indices, vals, X, ldx, \
                                                                     c4, Y, ldy, ep, W, nwarps, carry,     \
                                                                     carry_row);                           \
        spmm_fixup_kernel<K><<<fblocks, 256, 0, st>>>(n, indptr, c4, Y, ldy, ep, W, carry, carry_row);      \
        break;
#define LNE_MERGE_GROUPED(LGV)                                                                              \
    {                                                                                                       \
        if (nnz > 0)                                                                                        \
            spmm_merge_kernel<1, WEIGHTED, TX, LGV><<<mblocks, threads, 0, st>>>(                          \
                n, nnz, indptr, indices, vals, X, ldx, c4, Y, ldy, ep, W, nwarps, carry, carry_row);        \
        spmm_fixup_kernel<1><<<fblocks, 256, 0, st>>>(n, indptr, c4, Y, ldy, ep, W, carry, carry_row);      \
    }
    // weighted products with at most 16 float4 column groups: several nonzeros
    // per warp step (the graph products keep one, so batched propagation sums
    // in the same order as a single candidate's)
    if (WEIGHTED && c4 <= 8) LNE_MERGE_GROUPED(8)
    else if (WEIGHTED && c4 <= 16) LNE_MERGE_GROUPED(16)
    else switch (nv) {
        LNE_MERGE_CASE(1)
        LNE_MERGE_CASE(2)
        LNE_MERGE_CASE(4)
        LNE_MERGE_CASE(8)
        default:
            return fail(LNE_ERR_UNSUPPORTED, "SpMM supports at most 1024 dense columns");
    }
#undef LNE_MERGE_CASE
#undef LNE_MERGE_GROUPED
    LNE_LAUNCH_CHECK();
    ::lne::count_launch();
    return 0;
}

// Segments of the rows of a CSR matrix (columns sorted within rows) by
// vertex blocks [b << shift, (b + 1) << shift): seg[b n + i] = the number of
// row i's nonzeros with column < b << shift (b = 0..nb). A warp per row;
// unsorted rows set *unsorted.
__global__ void __launch_bounds__(256) vblock_seg_kernel(int64_t n, const int64_t *__restrict__ indptr,
                                                         const int32_t *__restrict__ indices, int shift, int nb,
                                                         uint32_t *__restrict__ seg, int *__restrict__ unsorted) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int64_t rs = __ldg(indptr + i), len = __ldg(indptr + i + 1) - rs;
        if (lane == 0) seg[i] = 0;   // block 0
        int prev = 0;                // block of the element before the chunk (0 before the first)
        for (int64_t k0 = 0; k0 < len; k0 += 32) {
            const int64_t k = k0 + lane;
            const bool valid = k < len;
            const int col = valid ? __ldg(indices + rs + k) : 0;
            if (valid && (col < 0 || (int64_t)col >= n)) *unsorted = 1;   // not a valid column: no blocking
            const int blk = valid ? min(max(col, 0) >> shift, nb - 1) : nb;
            int before = __shfl_up_sync(0xffffffffu, blk, 1);
            if (lane == 0) before = prev;
            if (valid) {
                if (blk < before) *unsorted = 1;
                for (int b = before + 1; b <= blk; ++b) seg[(int64_t)b * n + i] = (uint32_t)k;
            }
            prev = __shfl_sync(0xffffffffu, blk, 31);
        }
        const int last = len > 0 ? min(max(__ldg(indices + rs + len - 1), 0) >> shift, nb - 1) : 0;
        for (int b = last + 1 + lane; b <= nb; b += 32) seg[(int64_t)b * n + i] = (uint32_t)len;
    }
}

// V[b (n + 1) + i] = the length of row i's segment in block b (scanned in place afterwards)
__global__ void vblock_len_kernel(int64_t n, int nb, const uint32_t *__restrict__ seg, int64_t *__restrict__ V) {
    const int64_t total = (int64_t)nb * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / n, i = e - b * n;
        V[b * (n + 1) + i] = (int64_t)(seg[(b + 1) * n + i] - seg[b * n + i]);
    }
}

__global__ void vblock_totals_kernel(int64_t n, int nb, const int64_t *__restrict__ V, int64_t *__restrict__ out) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) out[b] = V[(int64_t)b * (n + 1) + n];
}

// The column-blocked product Y = alpha M X: vertex block b of the columns
// (a bounded region of operand rows) at a time, each block's partial product added
// to Y in block order by the epilogue (Y = partial + Y for b > 0); the last
// block also writes the BF16 copy. Deterministic: fixed block order, and
// within a block the merge kernel's fixed order.
template <typename TX>
int launch_merge_vb(Workspace &ws, const CsrView &M, const TX *X, int64_t ldx, int c, float *Y, int64_t ldy,
                    const SpmmEpilogue &ep, cudaStream_t st) {
    const VBlocks &vb = *M.vb;
    const int64_t n = M.n;
    const int c4 = c / 4;
    const int nv = merge_vectors(c);
    for (int b = 0; b < vb.nb; ++b) {
        const int64_t nnzb = vb.nnz[(size_t)b];
        const int64_t *V = vb.V + (int64_t)b * (n + 1);
        const uint32_t *segb = vb.seg + (int64_t)b * n;
        SpmmEpilogue eb;
        eb.lde = ldy;
        eb.alpha = ep.alpha;
        eb.threads = ep.threads;
        eb.carry_tag = ep.carry_tag;
        if (b > 0) {
            eb.E1 = Y;
            eb.b1 = 1.f;
        }
        if (b == vb.nb - 1) eb.Yb = ep.Yb;
        const int64_t W = merge_slice(nnzb, n);
        const int64_t nwarps = std::max<int64_t>(1, ceil_div(nnzb, W));
        float4 *carry = nullptr;
        int64_t *carry_row = nullptr;
        LNE_TRY(merge_carry(ws, eb.carry_tag, nnzb, n, c, &carry, &carry_row));
        const int threads = eb.threads > 0 ? eb.threads : 256;
        const unsigned mblocks = (unsigned)ceil_div(nwarps, threads / 32);
        const unsigned fblocks = (unsigned)std::min<int64_t>(ceil_div(n, 8), num_sms() * 32);
        LNE_TRACE("spmm", st);
#define LNE_VB_CASE(K)                                                                                           \
    case K:                                                                                                      \
        if (nnzb > 0)                                                                                            \
            spmm_merge_kernel<K, true, TX, 32, true><<<mblocks, threads, 0, st>>>(                               \
                n, nnzb, V, M.indices, M.data, X, ldx, c4, Y, ldy, eb, W, nwarps, carry, carry_row, M.indptr, segb); \
        spmm_fixup_kernel<K, true><<<fblocks, 256, 0, st>>>(n, V, c4, Y, ldy, eb, W, carry, carry_row);         \
        break;
        switch (nv) {
            LNE_VB_CASE(1)
            LNE_VB_CASE(2)
            LNE_VB_CASE(4)
            LNE_VB_CASE(8)
            default:
                return fail(LNE_ERR_UNSUPPORTED, "SpMM supports at most 1024 dense columns");
        }
#undef LNE_VB_CASE
        LNE_LAUNCH_CHECK();
        ::lne::count_launch();
    }
    return 0;
}


}  // namespace

int vblock_shift_for(int mode, int64_t n, int c, int elem_bytes) {
    if (mode < 0 || n <= 0) return 0;
    if (mode > 0) return (int64_t)1 << mode < n ? mode : 0;
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        return 0;
    const double row = (double)c * elem_bytes;
    if ((double)n * row <= (double)l2) return 0;   // the whole operand fits in L2
    // the largest blocks whose operand rows take at most 2.5 times L2:
    // measured on a 10M-vertex graph (c = 144, BF16 operand), blocks of
    // 0.6, 1.2, 2.4 and 4.8 times L2 took the products from 614 ms to 614,
    // 558, 550 and 574 ms; L2-sized blocks do not help, the random row
    // gathers are bound by the memory system's request throughput, not by
    // DRAM bytes, and more passes over Y cost more than the hits save
    int shift = 10;
    while (shift < 30 && (double)((int64_t)1 << (shift + 1)) * row <= 2.5 * (double)l2) ++shift;
    return (int64_t)1 << shift < n ? shift : 0;
}

int vblocks_build(Workspace &ws, const CsrView &M, int shift, VBlocks *vb, bool *ok, cudaStream_t st) {
    *ok = false;
    const int64_t n = M.n;
    if (shift <= 0 || n <= 0 || M.nnz <= 0) return 0;
    const int nb = (int)ceil_div(n, (int64_t)1 << shift);
    if (nb < 2) return 0;
    uint32_t *seg = nullptr;
    int64_t *V = nullptr, *tot = nullptr;
    int *flag = nullptr;
    LNE_TRY(ws.get("vb.seg", (size_t)(nb + 1) * (size_t)n, &seg));
    LNE_TRY(ws.get("vb.V", (size_t)nb * (size_t)(n + 1), &V));
    LNE_TRY(ws.get("vb.tot", (size_t)nb, &tot));
    LNE_TRY(ws.get("vb.flag", 1, &flag));
    LNE_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
    {
        LNE_TRACE("vblock_seg", st);
        const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n, 8), num_sms() * 32);
        vblock_seg_kernel<<<blocks, 256, 0, st>>>(n, M.indptr, M.indices, shift, nb, seg, flag);
        LNE_LAUNCH_CHECK();
        vblock_len_kernel<<<(unsigned)(num_sms() * 16), 256, 0, st>>>(n, nb, seg, V);
        LNE_LAUNCH_CHECK();
    }
    LNE_TRY(scan_exclusive_rows_i64(V, nb, n, st));
    vblock_totals_kernel<<<1, 256, 0, st>>>(n, nb, V, tot);
    LNE_LAUNCH_CHECK();
    std::vector<int64_t> h((size_t)nb);
    int unsorted = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(h.data(), tot, sizeof(int64_t) * (size_t)nb, cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(&unsorted, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (unsorted) return 0;
    vb->shift = shift;
    vb->nb = nb;
    vb->seg = seg;
    vb->V = V;
    vb->nnz = std::move(h);
    *ok = true;
    return 0;
}

// Partial products of k-slices (P[z] = the slice's n x c block, z = 0..ks-1)
// summed in slice order into Y: deterministic.
__global__ void slice_sum_kernel(const float *__restrict__ P, int ks, int64_t n, int c, float *__restrict__ Y,
                                 int64_t ldy) {
    const int64_t total = n * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        float v = P[e];
        for (int z = 1; z < ks; ++z) v += P[(int64_t)z * total + e];
        const int64_t r = e / c;
        Y[r * ldy + (e - r * c)] = v;
    }
}

int slice_sum(const float *P, int ks, int64_t n, int c, float *Y, int64_t ldy, cudaStream_t st) {
    LNE_TRACE("slice_sum", st);
    slice_sum_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n * c, 256), num_sms() * 16)), 256, 0,
                       st>>>(P, ks, n, c, Y, ldy);
    LNE_LAUNCH_CHECK();
    return 0;
}

int merge_carry(Workspace &ws, const char *tag, int64_t nnz, int64_t n, int c, float4 **carry,
                int64_t **carry_row) {
    const int64_t nwarps = std::max<int64_t>(1, ceil_div(nnz, merge_slice(nnz, n)));
    const std::string t = tag ? tag : "spmm.carry";
    LNE_TRY(ws.get(t + ".c", (size_t)nwarps * 2 * merge_vectors(c) * 32, carry));
    LNE_TRY(ws.get(t + ".r", (size_t)nwarps * 2, carry_row));
    return 0;
}


int spmm(Workspace &ws, const CsrView &M, const float *X, int64_t ldx, int c, float *Y, int64_t ldy,
         cudaStream_t st) {
    SpmmEpilogue ep;
    ep.lde = ldy;
    if (M.vb && merge_ok(X, ldx, c, Y, ldy, ep)) return launch_merge_vb<float>(ws, M, X, ldx, c, Y, ldy, ep, st);
    if (merge_ok(X, ldx, c, Y, ldy, ep))
        return launch_merge<true, float>(ws, M.n, M.nnz, M.indptr, M.indices, M.data, X, ldx, c, Y, ldy, ep, st);
    return launch_spmm<true>(M.n, M.indptr, M.indices, M.data, X, ldx, c, Y, ldy, ep, st);
}

int spmm_bf16(Workspace &ws, const CsrView &M, const __nv_bfloat16 *X, int64_t ldx, int c, float *Y, int64_t ldy,
              __nv_bfloat16 *Yb, cudaStream_t st) {
    SpmmEpilogue ep;
    ep.lde = ldy;
    ep.Yb = Yb;
    if (!merge_ok(X, ldx, c, Y, ldy, ep)) return fail(LNE_ERR_UNSUPPORTED, "BF16 operands need c and ld multiples of 4");
    if (M.vb) return launch_merge_vb<__nv_bfloat16>(ws, M, X, ldx, c, Y, ldy, ep, st);
    return launch_merge<true, __nv_bfloat16>(ws, M.n, M.nnz, M.indptr, M.indices, M.data, X, ldx, c, Y, ldy, ep, st);
}

int graph_spmm_bf16(Workspace &ws, const GraphView &g, const __nv_bfloat16 *X, int64_t ldx, int c, float *Y,
                    int64_t ldy, const SpmmEpilogue &ep, cudaStream_t st) {
    if (!merge_ok(X, ldx, c, Y, ldy, ep)) return fail(LNE_ERR_UNSUPPORTED, "BF16 operands need c and ld multiples of 4");
    if (g.w) {   // weighted: sum_y A_xy X_y, scaled by 1 / d_x
        SpmmEpilogue ew = ep;
        ew.dinv_w = ep.dinv ? g.dinv : nullptr;
        return launch_merge<true, __nv_bfloat16>(ws, g.n, g.nnz, g.indptr, g.indices, g.wf, X, ldx, c, Y, ldy, ew,
                                                 st);
    }
    return launch_merge<false, __nv_bfloat16>(ws, g.n, g.nnz, g.indptr, g.indices, nullptr, X, ldx, c, Y, ldy, ep, st);
}

namespace {
__global__ void to_bf16_kernel(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}
}  // namespace

int to_bf16(const float *in, __nv_bfloat16 *out, int64_t count, cudaStream_t st) {
    if (count <= 0) return 0;
    LNE_TRACE("to_bf16", st);
    to_bf16_kernel<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), num_sms() * 16), 256, 0, st>>>(in, out, count);
    LNE_LAUNCH_CHECK();
    return 0;
}

int graph_spmm(Workspace &ws, const GraphView &g, const float *X, int64_t ldx, int c, float *Y, int64_t ldy,
               const SpmmEpilogue &ep, cudaStream_t st) {
    if (g.w) {   // weighted: sum_y A_xy X_y, scaled by 1 / d_x
        SpmmEpilogue ew = ep;
        ew.dinv_w = ep.dinv ? g.dinv : nullptr;
        if (merge_ok(X, ldx, c, Y, ldy, ew))
            return launch_merge<true, float>(ws, g.n, g.nnz, g.indptr, g.indices, g.wf, X, ldx, c, Y, ldy, ew, st);
        return launch_spmm<true>(g.n, g.indptr, g.indices, g.wf, X, ldx, c, Y, ldy, ew, st);
    }
    if (merge_ok(X, ldx, c, Y, ldy, ep))
        return launch_merge<false, float>(ws, g.n, g.nnz, g.indptr, g.indices, nullptr, X, ldx, c, Y, ldy, ep, st);
    return launch_spmm<false>(g.n, g.indptr, g.indices, nullptr, X, ldx, c, Y, ldy, ep, st);
}

}  // namespace lne
