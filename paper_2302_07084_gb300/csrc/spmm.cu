// Sparse x dense products of the hot path:
//   * Y = M X with the weighted sparsifier M (Algorithm 4, lines 3 and 5);
//   * the propagation products with the unweighted graph A, where the row
//     scale 1/deg(i) (D^-1 A) and the Chebyshev recurrence of Sec. 3.3 are
//     fused into the epilogue:  out = alpha * rs_i (A X)_i + b1 E1 + b2 E2 + b3 E3,
//     optionally F += gamma * out and G = X0 - F.
//
// One warp per row; lane l owns columns l, l+32, ...; the row's column indices
// and values are read 32 at a time and broadcast by shuffles. Rows are
// summed in CSR order, so results are deterministic.
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
    if (ep.dinv) rs = deg > 0 ? ep.alpha / (float)deg : 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cc = lane + 32 * t;
        if (cc >= c) continue;
        const int64_t e = i * ep.lde + cc;
        float o = rs * acc[t];
        if (ep.E1) o = fmaf(ep.b1, ep.E1[e], o);
        if (ep.E2) o = fmaf(ep.b2, ep.E2[e], o);
        if (ep.E3) o = fmaf(ep.b3, ep.E3[e], o);
        if (ep.store) Y[i * ldy + cc] = o;
        if (ep.F) {
            const float f = fmaf(ep.gamma, o, ep.F[e]);
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

template <bool WEIGHTED>
int launch_spmm(int64_t n, const int64_t *indptr, const int32_t *indices, const float *vals,
                const float *X, int64_t ldx, int c, float *Y, int64_t ldy, const SpmmEpilogue &ep,
                cudaStream_t st) {
    if (n <= 0) return 0;
    const int nt = (c + 31) / 32;
    const int wblocks = (int)std::min<int64_t>(ceil_div(n, 8), 152 * 64);
    const int cblocks = (int)std::min<int64_t>(n, 152 * 16);
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

}  // namespace

int spmm(const CsrView &M, const float *X, int64_t ldx, int c, float *Y, int64_t ldy, cudaStream_t st) {
    SpmmEpilogue ep;
    ep.lde = ldy;
    return launch_spmm<true>(M.n, M.indptr, M.indices, M.data, X, ldx, c, Y, ldy, ep, st);
}

int graph_spmm(const GraphView &g, const float *X, int64_t ldx, int c, float *Y, int64_t ldy,
               const SpmmEpilogue &ep, cudaStream_t st) {
    return launch_spmm<false>(g.n, g.indptr, g.indices, nullptr, X, ldx, c, Y, ldy, ep, st);
}

}  // namespace lne
