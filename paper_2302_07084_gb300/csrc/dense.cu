// Dense stages of the randomized SVD (Algorithm 4) on the GPU:
//
//   sketch         Omega = randn(n, c) from Philox4x32-10 words (Box-Muller).
//   gram           G = Y^T Y to FP64 accuracy: per-CTA partial Grams over row
//                  blocks in error-free float-pair arithmetic, summed in FP64
//                  in a fixed order so the result is reproducible.
//   chol           G = R^T R (upper Cholesky) in FP64, one CTA.
//   trsm_rows      Q = Y R^-1 by forward substitution per row (FP32): each
//                  row's solve is backward stable, so Y = Q R holds to FP32
//                  rounding whatever the conditioning of R.
//   right_multiply out = Y W for a small FP64 W (rounded to FP32), FP32 FMA.
//   cholqr2        Q = Y R1^-1, then again: the orthonormalisation used in
//                  place of eigSVD inside the power iteration (same range).
//   small_svd      SVD of the c x c factor R: FP32 one-sided Jacobi, then
//                  Ogita-Aishima refinement in FP64, so Y = Q R gives left
//                  singular vectors Q U_R -- the final eigSVD of Algorithm 4.
//   sign_fix_embed largest-magnitude entry of each column made positive, and
//                  X = U Sigma^{1/2} (Sec. 4.2).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "jacobi_order.h"
#include "runtime.h"

namespace lne {
namespace {

// ---------------------------------------------------------------------------
// Gaussian sketch
// ---------------------------------------------------------------------------
__device__ __forceinline__ float log_unit(uint32_t w) {
    // ln((w + 0.5) / 2^32); near 1 use log1p of the exact integer distance.
    if (w >= 0x80000000u) {
        uint32_t m = 0u - w;   // 2^32 - w, in 1 .. 2^31
        return log1pf(-((float)m - 0.5f) * 2.3283064365386963e-10f);
    }
    return logf(((float)w + 0.5f) * 2.3283064365386963e-10f);
}

__global__ void sketch_kernel(int64_t n, int c, uint32_t k0, uint32_t k1, float *__restrict__ out,
                              int64_t ld) {
    const int nblk = (c + 3) / 4;
    const int64_t total = n * nblk;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / nblk;
        const int cb = (int)(idx - i * nblk);
        u32x4 w = philox10(u32x4{(uint32_t)i, (uint32_t)cb, 0u, 0u}, k0, k1);
        float r0 = sqrtf(-2.0f * log_unit(w.x));
        float r1 = sqrtf(-2.0f * log_unit(w.z));
        float s0, c0, s1, c1;
        sincospif(2.0f * (((float)w.y + 0.5f) * 2.3283064365386963e-10f), &s0, &c0);
        sincospif(2.0f * (((float)w.w + 0.5f) * 2.3283064365386963e-10f), &s1, &c1);
        float z[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
        float *row = out + i * ld + 4 * cb;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (4 * cb + t < c) row[t] = z[t];
    }
}

// ---------------------------------------------------------------------------
// Gram with FP64 accuracy from FP32 arithmetic: thread (ti, tj, half), ti <= tj,
// owns 4 rows of an 8x8 tile of the upper half. Every product a*b is split exactly into
// p + e (p = fl(a b), e = fma(a, b, -p)); p enters a float pair (hi, lo) by
// an error-free two-sum, e and the two-sum's error go to lo. The pair carries
// ~46 significant bits over a CTA's rows; CTAs are summed in FP64. FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU, so this
// is several times faster than FP64 FMAs. The _rn intrinsics keep the
// compiler from contracting the error-free transformations.
// ---------------------------------------------------------------------------
constexpr int kGramRows = 32;   // rows staged per step

constexpr int kGramThreads = 384;

__global__ void __launch_bounds__(kGramThreads) gram_partial_kernel(const float *__restrict__ Y, int64_t n, int c,
                                                                    int64_t ld, int64_t rows_per_cta,
                                                                    double *__restrict__ partial) {
    extern __shared__ float ys[];   // kGramRows x cp
    const int cp = (c + 7) & ~7;
    const int nt = cp / 8;
    const int nitems = nt * (nt + 1);   // (tile, half): rows 0-3 or 4-7 of an 8x8 tile
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = imin64(n, r0 + rows_per_cta);
    // items are processed in groups of kGramThreads (uniform trip count for the barriers)
    for (int g0 = 0; g0 < nitems; g0 += kGramThreads) {
        const int item = g0 + tid;
        const bool active = item < nitems;
        int ti = 0, tj = 0;
        const int half = item & 1;
        if (active) {
            int rem = item >> 1;
            while (rem >= nt - ti) {
                rem -= nt - ti;
                ++ti;
            }
            tj = ti + rem;
        }
        const int xa = ti * 8 + half * 4;
        float hi[4][8], lo[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) hi[a][b] = lo[a][b] = 0.f;
        for (int64_t base = r0; base < r1; base += kGramRows) {
            const int rows = (int)imin64(kGramRows, r1 - base);
#pragma unroll 4
            for (int e = tid; e < kGramRows * cp; e += kGramThreads) {
                int rr = e / cp, cc = e - rr * cp;
                ys[e] = (rr < rows && cc < c) ? Y[(base + rr) * ld + cc] : 0.f;
            }
            __syncthreads();
            if (active) {
                for (int rr = 0; rr < rows; ++rr) {
                    const float *yr = ys + rr * cp;
                    float av[4], bv[8];
#pragma unroll
                    for (int t = 0; t < 4; ++t) av[t] = yr[xa + t];
#pragma unroll
                    for (int t = 0; t < 8; ++t) bv[t] = yr[tj * 8 + t];
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 8; ++y) {
                            const float p = __fmul_rn(av[x], bv[y]);
                            const float e = fmaf(av[x], bv[y], -p);
                            const float h = hi[x][y];
                            const float s = __fadd_rn(h, p);
                            const float bb = __fsub_rn(s, h);
                            const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
                            hi[x][y] = s;
                            lo[x][y] = __fadd_rn(lo[x][y], __fadd_rn(err, e));
                        }
                }
            }
            __syncthreads();
        }
        if (active) {
            double *P = partial + (int64_t)blockIdx.x * cp * cp;
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y)
                    P[(xa + x) * cp + tj * 8 + y] = (double)hi[x][y] + (double)lo[x][y];
        }
    }
}

// G[a][b] = G[b][a] = sum over CTAs of the partials of the upper entry
// (a, b): 8 lanes per entry, lane q summing partials q, q + 8, ..., then a
// fixed shuffle tree, so the order is the same on every run. (The (a, b)
// entry lives in tile (a/8, b/8); tiles with a/8 == b/8 hold both orders,
// tiles above the diagonal only (a, b).)
constexpr int kGramRedLanes = 8;

__global__ void gram_reduce_kernel(const double *__restrict__ partial, int nblk, int c,
                                   double *__restrict__ G) {
    constexpr int kPerWarp = 32 / kGramRedLanes;   // entries per warp and step
    const int cp = (c + 7) & ~7;
    const int nup = c * (c + 1) / 2;
    const int lane = threadIdx.x & 31, q = lane % kGramRedLanes;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the warp's lanes take the same trip count (the shuffles need all of them)
    for (int64_t ub = warp * kPerWarp; ub < nup; ub += nwarps * kPerWarp) {
        const int64_t u = ub + lane / kGramRedLanes;
        const bool live = u < nup;
        int a = 0, b = 0;
        if (live) {   // u-th upper entry in row order: row a holds c - a entries
            int rem = (int)u;
            while (rem >= c - a) {
                rem -= c - a;
                ++a;
            }
            b = a + rem;
        }
        double s = 0.0;
        if (live)
            for (int k = q; k < nblk; k += kGramRedLanes) s += partial[(int64_t)k * cp * cp + a * cp + b];
#pragma unroll
        for (int off = kGramRedLanes / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (live && q == 0) {
            G[a * c + b] = s;
            G[b * c + a] = s;
        }
    }
}

// 1/sqrt(a) of a positive finite FP64 pivot by two Newton steps
// y <- y (3 - a y^2) / 2 from the FP32 estimate (which has 24 bits; two steps
// pass FP64's 53), so no FP64 square root or division runs on this GPU's
// narrow FP64 pipe; pivots outside FP32's range take the plain route.
__device__ __forceinline__ double pivot_rsqrt(double a) {
    double y = (double)rsqrtf((float)a);
    if (!(y > 0.0) || !isfinite(y)) return 1.0 / sqrt(a);
    y = y * fma(-0.5 * a, y * y, 1.5);
    return y * fma(-0.5 * a, y * y, 1.5);
}

// ---------------------------------------------------------------------------
// Cholesky (upper, G = R^T R), one CTA, FP64. Right-looking: for each k the
// pivot row is scaled by 1/sqrt(pivot) and the trailing upper triangle takes
// the rank-1 update.
// ---------------------------------------------------------------------------
constexpr int kCholThreads = 1024;
constexpr int kMaxSmemC = 160;

__global__ void __launch_bounds__(kCholThreads) chol_kernel(const double *__restrict__ G, int c,
                                                            double *__restrict__ R, int *__restrict__ status) {
    extern __shared__ double sm[];
    const bool in_smem = c <= kMaxSmemC;
    double *A = in_smem ? sm : R;
    __shared__ double s_inv;
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kCholThreads / 32;
    for (int e = tid; e < c * c; e += kCholThreads) A[e] = G[e];
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < c; ++k) {
        if (tid == 0) {
            const double akk = A[k * c + k];
            if (!(akk > 0.0) || !isfinite(akk)) {
                if (!bad) bad = k + 1;
                A[k * c + k] = 1.0;
                s_inv = 1.0;
            } else {
                const double y = pivot_rsqrt(akk);
                A[k * c + k] = akk * y;
                s_inv = y;
            }
        }
        __syncthreads();
        const double inv = s_inv;
        for (int j = k + 1 + tid; j < c; j += kCholThreads) A[k * c + j] *= inv;
        __syncthreads();
        for (int i = k + 1 + warp; i < c; i += nw) {
            const double aki = A[k * c + i];
            for (int j = i + lane; j < c; j += 32) A[i * c + j] = fma(-aki, A[k * c + j], A[i * c + j]);
        }
        __syncthreads();
    }
    for (int e = tid; e < c * c; e += kCholThreads) {
        const int i = e / c, j = e - i * c;
        if (in_smem) R[e] = j >= i ? A[e] : 0.0;
        else if (j < i) R[e] = 0.0;
    }
    if (tid == 0 && bad && *status == 0) *status = bad;   // sticky: only a breakdown writes
}

// Blocked Cholesky over many SMs (FP64), for the matrix sizes where the
// one-CTA kernel is bound by a single SM's FP64 rate. Panels of kCholB rows:
// the panel phase (chol_panel_body) factors the diagonal block,
// R11^T R11 = A11, and solves R11^T R12 = A12 for the panel's row block; the
// update phase (chol_update_body, one CTA per 16 x 16 upper tile) subtracts
// R12^T R12 from the trailing matrix. A is the working copy (row-major, upper
// triangle significant) and ends as R. Both phases of every panel run in one
// cooperative launch (chol_coop_kernel), separated by grid barriers.
//
// The panel's row block is spread over ceil((c - k1) / 16) CTAs, 16 columns
// each; every CTA factors the small diagonal block itself (identically), so
// no CTA waits for another. Since other CTAs may still be reading A11 while
// one has finished, R11 goes to a scratch block (written by CTA 0) and is
// copied into A in the update phase, or directly by a panel that runs as a
// single CTA.
constexpr int kCholB = 16;

// The panel of rows k0.. for the 16-column block bx of R12 (nb blocks).
__device__ __forceinline__ void chol_panel_body(double *__restrict__ A, int c, int k0, int *__restrict__ status,
                                                double *__restrict__ r11, int bx, int nb) {
    __shared__ double s11[kCholB][kCholB + 1];
    __shared__ double sinv[kCholB];
    const int tid = threadIdx.x;
    const int bs = min(kCholB, c - k0), k1 = k0 + bs;
    for (int e = tid; e < bs * bs; e += blockDim.x) {
        const int i = e / bs, j = e - i * bs;
        s11[i][j] = A[(size_t)(k0 + i) * c + k0 + j];
    }
    __syncthreads();
    // unblocked factorisation of the diagonal block, one entry (ti, tj) per thread
    const int ti = tid >> 4, tj = tid & 15;
    for (int t = 0; t < bs; ++t) {
        if (tid == 0) {
            const double att = s11[t][t];
            double d = 1.0, y = 1.0;
            if (!(att > 0.0) || !isfinite(att)) {
                if (bx == 0 && *status == 0) *status = k0 + t + 1;
            } else {
                y = pivot_rsqrt(att);
                d = att * y;
            }
            s11[t][t] = d;
            sinv[t] = y;
        }
        __syncthreads();
        if (ti == t && tj > t && tj < bs) s11[t][tj] *= sinv[t];
        __syncthreads();
        if (ti > t && tj >= ti && tj < bs) s11[ti][tj] = fma(-s11[t][ti], s11[t][tj], s11[ti][tj]);
        __syncthreads();
    }
    // R12: 16 lanes per column; lane i holds x_i and subtracts r_ti x_t as
    // soon as x_t is final (the same terms in the same order as a row-by-row
    // forward substitution)
    {
        const int li = tid & 15;
        const int j = k1 + bx * 16 + (tid >> 4);
        const bool live = j < c && li < bs;
        double x = live ? A[(size_t)(k0 + li) * c + j] : 0.0;
        for (int t = 0; t < bs; ++t) {
            if (li == t) x *= sinv[t];
            const double xt = __shfl_sync(0xffffffffu, x, t, 16);
            if (li > t && li < bs) x = fma(-s11[t][li], xt, x);
        }
        if (live) A[(size_t)(k0 + li) * c + j] = x;
    }
    // R11 (and zeros left of the diagonal in the panel's rows)
    if (bx == 0)
        for (int e = tid; e < bs * bs; e += blockDim.x) {
            const int i = e / bs, j = e - i * bs;
            r11[e] = j >= i ? s11[i][j] : 0.0;
        }
    if (nb == 1)
        for (int e = tid; e < bs * k1; e += blockDim.x) {
            const int i = e / k1, j = e - i * k1;   // row k0 + i, column j < k1
            A[(size_t)(k0 + i) * c + j] = j >= k0 + i ? s11[i][j - k0] : 0.0;
        }
}

// r11 is read with ld.global.cg: in the cooperative launch it was written by
// another CTA of the same launch, so it must not come through the read-only path.
__device__ __forceinline__ void chol_update_body(double *__restrict__ A, int c, int k0, int k1, const double *r11,
                                                 int I, int J) {
    if (I > J) return;
    const int tid = threadIdx.x;
    const int bs = k1 - k0;
    if (I == 0 && J == 0)   // the panel's R11 from its scratch block (these entries are not read below)
        for (int e = tid; e < bs * k1; e += blockDim.x) {
            const int i = e / k1, j = e - i * k1;
            A[(size_t)(k0 + i) * c + j] = j >= k0 ? __ldcg(r11 + i * bs + (j - k0)) : 0.0;
        }
    __shared__ double ri[kCholB][16], rj[kCholB][16];
    const int ti = tid >> 4, tj = tid & 15;
    const int i0 = k1 + 16 * I, j0 = k1 + 16 * J;
    for (int e = tid; e < kCholB * 16; e += 256) {
        const int t = e >> 4, q = e & 15;
        ri[t][q] = (t < bs && i0 + q < c) ? A[(size_t)(k0 + t) * c + i0 + q] : 0.0;
        rj[t][q] = (t < bs && j0 + q < c) ? A[(size_t)(k0 + t) * c + j0 + q] : 0.0;
    }
    __syncthreads();
    const int i = i0 + ti, j = j0 + tj;
    if (i < c && j < c && i <= j) {
        double a = A[(size_t)i * c + j];
        for (int t = 0; t < bs; ++t) a = fma(-ri[t][ti], rj[t][tj], a);
        A[(size_t)i * c + j] = a;
    }
}

// All panels in one cooperative launch: the panel and update phases of each
// panel are separated by grid-wide barriers (every CTA is resident, so the
// barriers only wait for running CTAs; each gives up after 2 s and sets the
// status word [1]). The same work in the same order as the per-panel launches.
__device__ __forceinline__ void grid_barrier(unsigned *bar, unsigned &target, int *status) {
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) {
                atomicExch(status + 1, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256, 1) chol_coop_kernel(double *__restrict__ A, int c, int *__restrict__ status,
                                                        double *__restrict__ r11, unsigned *__restrict__ bar) {
    unsigned target = 0;
    for (int k0 = 0; k0 < c; k0 += kCholB) {
        const int k1 = min(c, k0 + kCholB);
        const int nb = max(1, (c - k1 + 15) / 16);
        for (int bx = blockIdx.x; bx < nb; bx += gridDim.x) {
            chol_panel_body(A, c, k0, status, r11, bx, nb);
            __syncthreads();
        }
        if (k1 >= c) break;
        grid_barrier(bar, target, status);
        for (int t = blockIdx.x; t < nb * nb; t += gridDim.x) {
            chol_update_body(A, c, k0, k1, r11, t / nb, t % nb);
            __syncthreads();
        }
        grid_barrier(bar, target, status);
    }
}

// Q = Y R^-1 for upper-triangular R (FP64, rounded to FP32): one warp per row
// solves q R = y by forward substitution; lane l keeps the running sums of
// columns l, l + 32, ...
constexpr int kTrsmThreads = 512;   // 16 rows in flight per CTA (measured: 256 -> 512 threads, 15% faster)

template <int NT>
__global__ void __launch_bounds__(kTrsmThreads) trsm_rows_kernel(const float *__restrict__ Y, int64_t n, int c, int64_t ldy,
                                                        const double *__restrict__ R, float *__restrict__ Q,
                                                        int64_t ldq) {
    extern __shared__ float Rs[];   // c x c, row-major, plus the reciprocal diagonal
    float *rdiag = Rs + c * c;
    // staged 8 loads at a time per thread: independent loads in flight instead
    // of one L2 round trip per element
#pragma unroll 8
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) Rs[e] = (float)__ldg(R + e);
    for (int j = threadIdx.x; j < c; j += blockDim.x) rdiag[j] = (float)(1.0 / R[j * c + j]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        float y[NT], q[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cc = lane + 32 * t;
            y[t] = cc < c ? Y[i * ldy + cc] : 0.f;
            q[t] = 0.f;
        }
        // column j: q_j = y_j * rdiag_j; then y_l -= q_j R[j][l] for l > j
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            for (int jj = 0; jj < 32; ++jj) {
                const int j = 32 * t + jj;
                if (j >= c) break;
                const float qj = __shfl_sync(0xffffffffu, y[t], jj) * rdiag[j];
                if (lane == jj) q[t] = qj;
                const float *rj = Rs + j * c;
#pragma unroll
                for (int u = 0; u < NT; ++u) {
                    const int l = lane + 32 * u;
                    if (u >= t && l > j && l < c) y[u] = fmaf(-qj, rj[l], y[u]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cc = lane + 32 * t;
            if (cc < c) Q[i * ldq + cc] = q[t];
        }
    }
}

// C = A B for upper-triangular c x c FP64 matrices (row i per CTA).
__global__ void upper_matmul_kernel(const double *__restrict__ A, const double *__restrict__ B, int c,
                                    double *__restrict__ C) {
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < c; j += blockDim.x) {
        double s = 0.0;
        if (j >= i)
            for (int l = i; l <= j; ++l) s += A[i * c + l] * B[l * c + j];
        C[i * c + j] = s;
    }
}

// ---------------------------------------------------------------------------
// out[n][dout] = Y[n][c] W[c][dout], FP32 FMA with W rounded to FP32.
// 64 x 64 output tile per CTA, 4 x 4 per thread.
// ---------------------------------------------------------------------------
constexpr int kMMTile = 64;
constexpr int kMMK = 32;

__global__ void __launch_bounds__(256) right_multiply_kernel(
    const float *__restrict__ Y, int64_t n, int c, int64_t ldy, const double *__restrict__ W,
    int64_t ldw, int dout, const double *__restrict__ colscale, float *__restrict__ out, int64_t ldo) {
    __shared__ float ys[kMMTile][kMMK + 1];
    __shared__ float ws[kMMK][kMMTile];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;   // 16 x 16 threads, 4 x 4 each
    const int64_t row0 = (int64_t)blockIdx.x * kMMTile;
    const int col0 = blockIdx.y * kMMTile;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < c; k0 += kMMK) {
        for (int e = tid; e < kMMTile * kMMK; e += 256) {
            int r = e / kMMK, k = e - r * kMMK;
            int64_t gr = row0 + r;
            ys[r][k] = (gr < n && k0 + k < c) ? Y[gr * ldy + k0 + k] : 0.f;
        }
        for (int e = tid; e < kMMK * kMMTile; e += 256) {
            int k = e / kMMTile, cc = e - k * kMMTile;
            ws[k][cc] = (k0 + k < c && col0 + cc < dout) ? (float)W[(int64_t)(k0 + k) * ldw + col0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kMMK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = ys[tr * 4 + x][k];
#pragma unroll
            for (int y = 0; y < 4; ++y) b[y] = ws[k][tc * 4 + y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        int64_t gr = row0 + tr * 4 + x;
        if (gr >= n) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            int gc = col0 + tc * 4 + y;
            if (gc < dout) {
                float v = acc[x][y];
                if (colscale) v = (float)((double)v * colscale[gc]);
                out[gr * ldo + gc] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Small SVD of the c x c factor R (c <= 160), FP64-accurate:
//   1. one-sided (Hestenes) Jacobi on R in FP32, one CTA, accumulating the
//      right rotations V (columns paired by the circle method: m = c rounded up
//      to even players, player 0 fixed, m/2 disjoint pairs per round, 8 threads
//      per pair); U = normalised columns of R V;
//   2. Ogita-Aishima refinement of (U, Sigma, V) of R itself in FP64 (matrix
//      products only, spread over many CTAs; R is never squared);
//   3. sorted by sigma descending.
// FP64 rates on this GPU are a small fraction of FP32, so FP64 is used only
// where the refinement needs it: its products.
// ---------------------------------------------------------------------------
constexpr int kJacTPP = 8;
constexpr int kJacMaxE = (160 + kJacTPP - 1) / kJacTPP;   // elements per thread and column, c <= 160

__device__ __forceinline__ int circle_player(int pos, int round, int m) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (m - 1)) + 1;
}

// Column stride of the shared-memory matrices: = 8 (mod 32), so the four
// 8-thread pair groups of a warp hit distinct banks.
__host__ __device__ __forceinline__ int jac_ld(int c) { return ((c + 23) / 32) * 32 + 8; }

// Jacobi acts on the columns of A = R^T (for a triangular factor this
// converges in fewer sweeps than on R): R^T W = Z Sigma with W the accumulated
// rotations, so R = W Sigma Z^T -- left singular vectors U = W, right ones
// V = normalised columns of R^T W.
__global__ void jacobi32_kernel(const double *__restrict__ R, int c, double *__restrict__ Uout,
                                double *__restrict__ Vout, int max_sweeps, int *__restrict__ sweeps_out) {
    extern __shared__ float js[];
    const int ldc = jac_ld(c);
    float *A = js;              // column j at A + j * ldc
    float *V = js + c * ldc;    // accumulated rotations
    __shared__ float red[32];
    __shared__ int s_done;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    for (int e = tid; e < c * c; e += nthreads) {
        int i = e / c, j = e - i * c;
        A[i * ldc + j] = (float)R[e];   // column i of R^T = row i of R
        V[j * ldc + i] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    const int m = c + (c & 1);
    const int pairs = m / 2;
    const int pi = tid / kJacTPP, sub = tid % kJacTPP;
    // FP32 round-off floor of |a_p . a_q| / (|a_p| |a_q|) is about c * 2^-24
    // stop at cosines of 0.4 c ulp (at least 8 ulp): the FP64 refinement's first-order
    // step needs the start's rotations this close where singular values are dense
    const float tol = fmaxf(0.4f * (float)c, 8.f) * 5.9604645e-8f;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        float local_max = 0.f;
        for (int round = 0; round < m - 1; ++round) {
            int p = 0, q = c;
            if (pi < pairs) {
                p = circle_player(pi, round, m);
                q = circle_player(m - 1 - pi, round, m);
                if (p > q) {
                    int t = p;
                    p = q;
                    q = t;
                }
            }
            const bool active = pi < pairs && q < c;
            float al = 0.f, be = 0.f, ga = 0.f;
            // the pair's elements stay in registers between the dot products
            // and the rotation (one shared-memory read and write per element)
            float xr[kJacMaxE], yr[kJacMaxE];
            float *ap = A + p * ldc, *aq = A + q * ldc;
#pragma unroll
            for (int e = 0; e < kJacMaxE; ++e) {
                const int i = sub + e * kJacTPP;
                const bool in = active && i < c;
                const float x = in ? ap[i] : 0.f, y = in ? aq[i] : 0.f;
                xr[e] = x;
                yr[e] = y;
                al = fmaf(x, x, al);
                be = fmaf(y, y, be);
                ga = fmaf(x, y, ga);
            }
            // every lane takes part in the shuffles; lanes without a pair add zeros
#pragma unroll
            for (int off = 1; off < kJacTPP; off <<= 1) {
                al += __shfl_xor_sync(0xffffffffu, al, off);
                be += __shfl_xor_sync(0xffffffffu, be, off);
                ga += __shfl_xor_sync(0xffffffffu, ga, off);
            }
            if (active && ga != 0.f && al > 0.f && be > 0.f) {
                float rel = fabsf(ga) * rsqrtf(al * be);
                local_max = fmaxf(local_max, rel);
                if (rel > tol) {
                    float zeta = (be - al) / (2.f * ga);
                    float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    float cs = rsqrtf(1.f + t * t);
                    float sn = cs * t;
                    float *vp = V + p * ldc, *vq = V + q * ldc;
#pragma unroll
                    for (int e = 0; e < kJacMaxE; ++e) {
                        const int i = sub + e * kJacTPP;
                        if (i < c) {
                            ap[i] = cs * xr[e] - sn * yr[e];
                            aq[i] = sn * xr[e] + cs * yr[e];
                            const float u = vp[i], w = vq[i];
                            vp[i] = cs * u - sn * w;
                            vq[i] = sn * u + cs * w;
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, off));
        if (lane == 0) red[warp] = local_max;
        __syncthreads();
        if (tid == 0) {
            float mx = 0.f;
            for (int w = 0; w < (nthreads + 31) / 32; ++w) mx = fmaxf(mx, red[w]);
            s_done = mx <= tol;
        }
        __syncthreads();
        if (s_done) {
            ++sweep;
            break;
        }
    }
    __shared__ float s_nrm[kMaxSmemC + 1];
    for (int j = tid; j < c; j += nthreads) {
        float t = 0.f;
        for (int i = 0; i < c; ++i) t = fmaf(A[j * ldc + i], A[j * ldc + i], t);
        s_nrm[j] = t > 0.f ? rsqrtf(t) : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < c * c; e += nthreads) {
        int i = e / c, j = e - i * c;
        Uout[e] = (double)V[j * ldc + i];                 // left vectors of R: the rotations
        Vout[e] = (double)(A[j * ldc + i] * s_nrm[j]);    // right vectors: normalised R^T W
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// Register-resident variant of the same Jacobi (c <= 144). Each 8-thread
// group holds its pair of columns of A in registers (E elements per column
// and thread, as float2 chunks: element 16 q + 2 sub + {0, 1}), so a round
// reads nothing from shared memory; columns move between groups through a
// shared exchange buffer only when the pairing changes. The rotations W are
// not accumulated here: every round's (cos, sin) and column labels are
// recorded, and jacobi_replay_kernel applies them to the identity afterwards,
// one row of W per warp on many SMs (the rows of W evolve independently).
//
// The pairing order is chosen so that most rounds move one column of each
// pair instead of both: a sweep over m = 2G columns takes the columns in slot
// 0 as a set X and those in slot 1 as Y, and pairs X[i] with Y[(i + r) mod G]
// for r = 0..G-1 (only Y moves, one group along); then X and Y are each split
// in halves and the same is done inside X and inside Y in parallel, and so on
// while the set size is even. Sets of odd size s then finish with s rounds of
// the circle method (one column of each set idle per round). Every pair meets
// exactly once per sweep; the layout a sweep ends with is the next sweep's
// starting point, and a label per column records which column of R^T it
// started as.
constexpr int kJacRegMaxC = 144;
constexpr int kJacMaxSweeps = 20;

template <int E>
__host__ __device__ constexpr int jreg_stride() { return ((8 * E + 31) / 32) * 32 + 16; }

// rounds per sweep of the order above for m (even) columns
__host__ __device__ inline int jreg_rounds(int m) { return jorder_rounds(m); }

// Paired FP32 arithmetic (fma.rn.f32x2 / mul.rn.f32x2, sm_100 and later):
// one instruction for two lanes of a float2, each rounded as the scalar op.
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t *>(&a)), "l"(*reinterpret_cast<const uint64_t *>(&b)),
          "l"(*reinterpret_cast<const uint64_t *>(&c)));
    return *reinterpret_cast<const float2 *>(&d);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t *>(&a)), "l"(*reinterpret_cast<const uint64_t *>(&b)));
    return *reinterpret_cast<const float2 *>(&d);
}

template <int E>
__global__ void __launch_bounds__(32 * E, 1) jacobi_reg_kernel(const double *__restrict__ R, int c,
                                                               double *__restrict__ Vout,
                                                               float2 *__restrict__ rot,
                                                               uint32_t *__restrict__ rlab, int max_sweeps,
                                                               int *__restrict__ sweeps_out) {
    constexpr int CP = 8 * E;            // padded column length
    constexpr int NQ = E / 2;            // float2 chunks per column and thread
    static_assert(E % 2 == 0, "columns are held as float2 chunks");
    constexpr int ST = jreg_stride<E>(); // floats per exchange entry (= 16 mod 32: conflict-free float2)
    extern __shared__ float xb[];        // 2 G entries: column [CP], label at CP
    __shared__ float red[32];
    __shared__ int s_done;
    const int m = c + (c & 1), G = m / 2, RD = jreg_rounds(m);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid >> 3, sub = tid & 7;
    const bool real = g < G;             // groups past G only fill the last warp
    // element 2 q + t of a column is component t of chunk q (rows 16 q + 2 sub + t)
    float2 a0[NQ], a1[NQ];
    int lab0 = g, lab1 = g + G;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int i = 16 * q + 2 * sub;
        const bool r0 = real && lab0 < c, r1 = real && lab1 < c;   // column lab of R^T
        a0[q].x = r0 && i < c ? (float)R[(size_t)lab0 * c + i] : 0.f;
        a0[q].y = r0 && i + 1 < c ? (float)R[(size_t)lab0 * c + i + 1] : 0.f;
        a1[q].x = r1 && i < c ? (float)R[(size_t)lab1 * c + i] : 0.f;
        a1[q].y = r1 && i + 1 < c ? (float)R[(size_t)lab1 * c + i + 1] : 0.f;
    }
    // stop at cosines of 0.4 c ulp (at least 8 ulp): the FP64 refinement's first-order
    // step needs the start's rotations this close where singular values are dense
    const float tol = fmaxf(0.4f * (float)c, 8.f) * 5.9604645e-8f;
    const int tz = jorder_levels(m);
    const int s_odd = m >> tz;           // set size the halving ends at
    float local_max = 0.f;
    int rec = 0;                         // record index of this round's group 0

    auto put = [&](int entry, const float2 (&a)[NQ], int lab) {
        float *eb = xb + (size_t)entry * ST;
#pragma unroll
        for (int q = 0; q < NQ; ++q) *reinterpret_cast<float2 *>(eb + 16 * q + 2 * sub) = a[q];
        if (sub == 0) reinterpret_cast<int *>(eb)[CP] = lab;
    };
    auto take = [&](int entry, float2 (&a)[NQ], int &lab) {
        const float *eb = xb + (size_t)entry * ST;
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q] = *reinterpret_cast<const float2 *>(eb + 16 * q + 2 * sub);
        lab = reinterpret_cast<const int *>(eb)[CP];
    };
    // both columns of every group move (sources as group * 2 + slot)
    auto move_both = [&](int src0, int src1) {
        __syncthreads();
        if (real) {
            put(2 * g, a0, lab0);
            put(2 * g + 1, a1, lab1);
        }
        __syncthreads();
        if (real) {
            take(src0, a0, lab0);
            take(src1, a1, lab1);
        }
        __syncthreads();
    };
    // one rotation of the group's pair (every lane takes part in the shuffles),
    // recorded as (cos, sin) = (1, 0) when the pair is left as it is
    auto rotate = [&](bool active) {
        float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            al2 = f2_fma(a0[q], a0[q], al2);
            be2 = f2_fma(a1[q], a1[q], be2);
            ga2 = f2_fma(a0[q], a1[q], ga2);
        }
        float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, off);
            be += __shfl_xor_sync(0xffffffffu, be, off);
            ga += __shfl_xor_sync(0xffffffffu, ga, off);
        }
        float cs = 1.f, sn = 0.f;
        if (active && ga != 0.f && al > 0.f && be > 0.f) {
            const float rel = fabsf(ga) * rsqrtf(al * be);
            local_max = fmaxf(local_max, rel);
            if (rel > tol) {
                const float zeta = (be - al) / (2.f * ga);
                const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                cs = rsqrtf(1.f + t * t);
                sn = cs * t;
                const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ms2 = make_float2(-sn, -sn);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float2 x = a0[q], y = a1[q];
                    a0[q] = f2_fma(c2, x, f2_mul(ms2, y));   // cs x - sn y
                    a1[q] = f2_fma(c2, y, f2_mul(s2, x));    // sn x + cs y
                }
            }
        }
        if (real && sub == 0) {
            rot[(size_t)rec + g] = make_float2(cs, sn);
            rlab[(size_t)rec + g] = (uint32_t)lab0 | ((uint32_t)lab1 << 16);
        }
        rec += G;
    };

    int sweep = 0, par = 0;
    for (; sweep < max_sweeps; ++sweep) {
        local_max = 0.f;
        rec = sweep * RD * G;
        for (int lev = 0; lev < tz; ++lev) {
            const int h = m >> (lev + 1);   // ring length: pairs per set and rounds of this level
            if (lev > 0) {
                // the two halves of each set of the level before become two sets
                int src0, src1;
                jorder_split_sources(g, h, src0, src1);
                move_both(src0, src1);   // every thread reaches the same barriers
            }
            const int ks = jorder_ring_source(g, h);   // slot-1 column comes from the next group
            for (int r = 0; r < h; ++r) {
                if (r > 0) {
                    // double-buffered halves: one barrier per round
                    if (real) put(par * G + g, a1, lab1);
                    __syncthreads();
                    if (real) take(par * G + ks, a1, lab1);
                    par ^= 1;
                }
                rotate(true);
            }
        }
        if (s_odd > 1) {
            // circle method inside each set of odd size s: positions 1..k paired
            // with s-1..k+1 in k groups per set, position 0 idle (the two sets
            // that share a parent put their idle columns in one group)
            const int s = s_odd;
            int e0, e1, r0, r1;
            bool idle;
            jorder_tail_sources(g, s, e0, e1, r0, r1, idle);
            for (int r = 0; r < s; ++r) {
                move_both(r == 0 ? e0 : r0, r == 0 ? e1 : r1);
                rotate(!idle);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, off));
        if (lane == 0) red[warp] = local_max;
        __syncthreads();
        if (tid == 0) {
            float mx = 0.f;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) mx = fmaxf(mx, red[w]);
            s_done = mx <= tol;
        }
        __syncthreads();
        if (s_done) {
            ++sweep;
            break;
        }
    }
    // right singular vectors of R: normalised columns of R^T W, by label
    float2 n02 = make_float2(0.f, 0.f), n12 = n02;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        n02 = f2_fma(a0[q], a0[q], n02);
        n12 = f2_fma(a1[q], a1[q], n12);
    }
    float n0 = n02.x + n02.y, n1 = n12.x + n12.y;
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
        n0 += __shfl_xor_sync(0xffffffffu, n0, off);
        n1 += __shfl_xor_sync(0xffffffffu, n1, off);
    }
    const float q0 = n0 > 0.f ? rsqrtf(n0) : 0.f, q1 = n1 > 0.f ? rsqrtf(n1) : 0.f;
    if (real) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = 16 * q + 2 * sub + t;
                const float x0 = t ? a0[q].y : a0[q].x, x1 = t ? a1[q].y : a1[q].x;
                if (i < c && lab0 < c) Vout[(size_t)i * c + lab0] = (double)(x0 * q0);
                if (i < c && lab1 < c) Vout[(size_t)i * c + lab1] = (double)(x1 * q1);
            }
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// W = the recorded rotations applied to the identity, in order: warp w of a
// CTA owns row i of W in shared memory; in every round its lanes take the
// round's records (disjoint column pairs). The CTA stages the records in
// chunks of kRpChunk rounds through shared memory, loading the next chunk
// into registers while it applies the current one.
constexpr int kRpWarps = 4;
constexpr int kRpPer = 3;      // records per lane and round: G <= 96
constexpr int kRpChunk = 16;   // rounds per staged chunk
constexpr int kRpMaxG = kJacRegMaxC / 2;
constexpr int kRpLoads = (kRpChunk * kRpMaxG + kRpWarps * 32 - 1) / (kRpWarps * 32);
static_assert(kRpMaxG <= 32 * kRpPer, "records of a round fit the lanes");

__global__ void __launch_bounds__(kRpWarps * 32) jacobi_replay_kernel(const float2 *__restrict__ rot,
                                                                      const uint32_t *__restrict__ rlab, int G,
                                                                      int RD, const int *__restrict__ sweeps,
                                                                      int c, double *__restrict__ Uout) {
    __shared__ float rows[kRpWarps][kJacRegMaxC + 1];
    __shared__ float2 srot[2][kRpChunk * kRpMaxG];
    __shared__ uint32_t slab[2][kRpChunk * kRpMaxG];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = blockIdx.x * kRpWarps + warp;
    const bool live = i < c;   // warps past the last row still stage records and meet the barriers
    float *row = rows[warp];
    for (int j = lane; j < c; j += 32) row[j] = i == j ? 1.f : 0.f;
    const int total = *sweeps * RD;
    const int per = kRpChunk * G;   // records per chunk
    float2 rr[kRpLoads];
    uint32_t rl[kRpLoads];
    auto fetch = [&](int ch) {   // chunk ch's records into registers
        const size_t base = (size_t)ch * per, end = (size_t)total * G;
#pragma unroll
        for (int u = 0; u < kRpLoads; ++u) {
            const int e = tid + u * kRpWarps * 32;
            const bool in = e < per && base + e < end;
            rr[u] = in ? rot[base + e] : make_float2(1.f, 0.f);
            rl[u] = in ? rlab[base + e] : 0u;
        }
    };
    auto stash = [&](int b) {
#pragma unroll
        for (int u = 0; u < kRpLoads; ++u) {
            const int e = tid + u * kRpWarps * 32;
            if (e < per) {
                srot[b][e] = rr[u];
                slab[b][e] = rl[u];
            }
        }
    };
    const int nch = (total + kRpChunk - 1) / kRpChunk;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int ch = 0; ch < nch; ++ch) {
        const int b = ch & 1;
        if (ch + 1 < nch) fetch(ch + 1);
        if (live) {
            const int nr = min(kRpChunk, total - ch * kRpChunk);
            for (int r = 0; r < nr; ++r) {
                // the round's pairs are disjoint: all reads first, then all writes
                float2 cn[kRpPer];
                int p[kRpPer], q[kRpPer];
                float u[kRpPer], v[kRpPer];
#pragma unroll
                for (int k = 0; k < kRpPer; ++k) {
                    const int g = lane + 32 * k;
                    cn[k] = g < G ? srot[b][r * G + g] : make_float2(1.f, 0.f);
                    const uint32_t pq = g < G ? slab[b][r * G + g] : 0u;
                    p[k] = (int)(pq & 0xFFFFu);
                    q[k] = (int)(pq >> 16);
                }
#pragma unroll
                for (int k = 0; k < kRpPer; ++k) {
                    u[k] = cn[k].y != 0.f ? row[p[k]] : 0.f;
                    v[k] = cn[k].y != 0.f ? row[q[k]] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < kRpPer; ++k)
                    if (cn[k].y != 0.f) {
                        row[p[k]] = cn[k].x * u[k] - cn[k].y * v[k];
                        row[q[k]] = cn[k].y * u[k] + cn[k].x * v[k];
                    }
                __syncwarp();
            }
        }
        if (ch + 1 < nch) stash(b ^ 1);
        __syncthreads();
    }
    if (live)
        for (int j = lane; j < c; j += 32) Uout[(size_t)i * c + j] = (double)row[j];
}

// records a Jacobi run on c <= kJacRegMaxC columns may write
inline size_t jreg_records(int c) {
    const int m = c + (c & 1);
    return (size_t)kJacMaxSweeps * jreg_rounds(m) * (m / 2);
}

template <int E>
int launch_jacobi_reg_e(const double *R, int c, double *U, double *V, float2 *rot, uint32_t *rlab, int *sweeps,
                        cudaStream_t st) {
    const int m = c + (c & 1);
    const int threads = ((m / 2) * 8 + 31) / 32 * 32;
    const int smem = m * jreg_stride<E>() * (int)sizeof(float);
    if (smem > 48 * 1024) LNE_TRY(allow_dynamic_smem(jacobi_reg_kernel<E>));
    jacobi_reg_kernel<E><<<1, threads, smem, st>>>(R, c, V, rot, rlab, kJacMaxSweeps, sweeps);
    LNE_LAUNCH_CHECK();
    jacobi_replay_kernel<<<(unsigned)ceil_div(c, kRpWarps), kRpWarps * 32, 0, st>>>(rot, rlab, m / 2,
                                                                                  jreg_rounds(m), sweeps, c, U);
    LNE_LAUNCH_CHECK();
    return 0;
}

// FP32 Jacobi start of the small SVD: the register-resident kernel (with its
// replay; rot / rlab hold jreg_records(c) records) up to c = 144, the
// shared-memory one above.
int launch_jacobi(const double *R, int c, double *U, double *V, float2 *rot, uint32_t *rlab, int *sweeps,
                  cudaStream_t st) {
    switch ((c + 15) / 16) {
    case 1: return launch_jacobi_reg_e<2>(R, c, U, V, rot, rlab, sweeps, st);
    case 2: return launch_jacobi_reg_e<4>(R, c, U, V, rot, rlab, sweeps, st);
    case 3: return launch_jacobi_reg_e<6>(R, c, U, V, rot, rlab, sweeps, st);
    case 4: return launch_jacobi_reg_e<8>(R, c, U, V, rot, rlab, sweeps, st);
    case 5: return launch_jacobi_reg_e<10>(R, c, U, V, rot, rlab, sweeps, st);
    case 6: return launch_jacobi_reg_e<12>(R, c, U, V, rot, rlab, sweeps, st);
    case 7: return launch_jacobi_reg_e<14>(R, c, U, V, rot, rlab, sweeps, st);
    case 8: return launch_jacobi_reg_e<16>(R, c, U, V, rot, rlab, sweeps, st);
    case 9: return launch_jacobi_reg_e<18>(R, c, U, V, rot, rlab, sweeps, st);
    default: break;
    }
    const int m = c + (c & 1);
    const int threads = std::max(32, std::min(1024, (m / 2 * kJacTPP + 31) / 32 * 32));
    const int smem = 2 * c * jac_ld(c) * 4;
    if (smem > 48 * 1024) LNE_TRY(allow_dynamic_smem(jacobi32_kernel));
    jacobi32_kernel<<<1, threads, smem, st>>>(R, c, U, V, kJacMaxSweeps, sweeps);
    LNE_LAUNCH_CHECK();
    return 0;
}

// C = op(A) op(B) (+ C0 if given), all c x c row-major FP64; 16 x 16 tile per CTA.
// 8 x 8 output tiles (64 threads, one output each; 324 CTAs for c = 144). The
// CTA's 8 rows of op(A) and 8 columns of op(B) over the whole k range are
// loaded into shared memory at once (one round of load latency instead of one
// per k step), then each thread runs its dot product.
constexpr int kDgTile = 8;
constexpr int kDgMaxC = 160;

// Two products with the same transposes may share a launch: blockIdx.z = 1
// takes the second operand set (A2, B2, C02, C2).
__global__ void __launch_bounds__(kDgTile * kDgTile) dgemm_small_kernel(const double *__restrict__ A, int ta,
                                                                        const double *__restrict__ B, int tb,
                                                                        const double *__restrict__ C0,
                                                                        double *__restrict__ C, int c,
                                                                        const double *__restrict__ A2,
                                                                        const double *__restrict__ B2,
                                                                        const double *__restrict__ C02,
                                                                        double *__restrict__ C2) {
    if (blockIdx.z == 1) {
        A = A2;
        B = B2;
        C0 = C02;
        C = C2;
    }
    __shared__ double As[kDgTile][kDgMaxC + 1], Bs[kDgMaxC][kDgTile + 1];
    const int tid = threadIdx.x, tx = tid % kDgTile, ty = tid / kDgTile;
    const int r0 = blockIdx.y * kDgTile, c0 = blockIdx.x * kDgTile;
#pragma unroll 6
    for (int e = tid; e < kDgTile * c; e += kDgTile * kDgTile) {
        // op(A)[r0 + i][k]: for ta the k index runs along A's rows
        const int i = ta ? e % kDgTile : e / c, k = ta ? e / kDgTile : e % c;
        const int r = r0 + i;
        As[i][k] = r < c ? (ta ? A[k * c + r] : A[r * c + k]) : 0.0;
        // op(B)[k][c0 + j]
        const int j = tb ? e / c : e % kDgTile, kb = tb ? e % c : e / kDgTile;
        const int cc = c0 + j;
        Bs[kb][j] = cc < c ? (tb ? B[cc * c + kb] : B[kb * c + cc]) : 0.0;
    }
    __syncthreads();
    const int row = r0 + ty, col = c0 + tx;
    double acc = 0.0;
    for (int k = 0; k < c; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    if (row < c && col < c) C[row * c + col] = C0 ? C0[row * c + col] + acc : acc;
}

__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    return t;
}

// One step of Ogita-Aishima refinement of an SVD A = U Sigma V^T (Ogita and
// Aishima, "Iterative refinement for singular value decomposition based on
// matrix multiplication", 2020), written from first-order perturbation:
// with U = U^(I + F), V = V^(I + G) exact, P = I - U^T U^ = F + F^T,
// Q = I - V^T V^ = G + G^T and T = U^T A V^ = Sigma - F^T Sigma - Sigma G. So
// sigma_i = t_ii / (1 - (p_ii + q_ii) / 2), f_ii = p_ii / 2, g_ii = q_ii / 2,
// and for i != j the pair (f_ij, g_ij) solves
//   [ s_j  -s_i ] [f_ij]   [t_ij + p_ij s_j]
//   [-s_i   s_j ] [g_ij] = [t_ji + q_ij s_j],
// taken as (p_ij / 2, q_ij / 2) when |s_i - s_j| <= delta (near-equal values),
// delta = 2 (||offdiag T|| + max|s| (||P|| + ||Q||)). A itself is never squared,
// so the accuracy does not depend on the condition number of A.
// Also turns the Gram products into P := I - U^T U, Q := I - V^T V in place.
// kOaParts CTAs each reduce a fixed slice of the c x c entries (FP64 is slow
// on this GPU, so the three sums are spread over several SMs) and write
// their partial sums; svd_oa_fg_kernel adds the partials in a fixed order,
// so delta is the same on every run.
constexpr int kOaParts = 16;

__global__ void svd_oa_norms_kernel(double *__restrict__ P, double *__restrict__ Q, const double *__restrict__ T,
                                    int c, double *__restrict__ sig, double *__restrict__ part) {
    __shared__ double red[32];
    double o2 = 0.0, p2 = 0.0, q2 = 0.0, smax = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
        const int i = e / c, j = e - i * c;
        const double d = i == j ? 1.0 : 0.0;
        const double p = d - P[e], q = d - Q[e], t = T[e];
        P[e] = p;
        Q[e] = q;
        if (i == j) {
            const double sv = t / (1.0 - 0.5 * (p + q));
            sig[i] = sv;
            smax = fmax(smax, fabs(sv));
        } else {
            o2 = fma(t, t, o2);
        }
        p2 = fma(p, p, p2);
        q2 = fma(q, q, q2);
    }
    o2 = block_sum(o2, red);
    p2 = block_sum(p2, red);
    q2 = block_sum(q2, red);
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, off));
        __syncthreads();
        if (lane == 0) red[warp] = smax;
        __syncthreads();
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmax(m, red[w]);
        smax = m;
    }
    if (threadIdx.x == 0) {
        double *o = part + 4 * blockIdx.x;
        o[0] = o2;
        o[1] = p2;
        o[2] = q2;
        o[3] = smax;
    }
}

// F, G of the update, one element per thread (the divisions spread over the GPU).
__global__ void svd_oa_fg_kernel(const double *__restrict__ P, const double *__restrict__ Q,
                                 const double *__restrict__ T, int c, const double *__restrict__ sig,
                                 const double *__restrict__ part, double *__restrict__ F, double *__restrict__ Gm) {
    __shared__ double s_delta;
    if (threadIdx.x == 0) {
        double o2 = 0.0, p2 = 0.0, q2 = 0.0, smax = 0.0;
        for (int b = 0; b < kOaParts; ++b) {
            o2 += part[4 * b];
            p2 += part[4 * b + 1];
            q2 += part[4 * b + 2];
            smax = fmax(smax, part[4 * b + 3]);
        }
        s_delta = 2.0 * (sqrt(o2) + smax * (sqrt(p2) + sqrt(q2)));
    }
    __syncthreads();
    const double delta = s_delta;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c * c) return;
    const int i = e / c, j = e - i * c;
    const double pij = P[e], qij = Q[e];
    double f = 0.5 * pij, g = 0.5 * qij;
    if (i != j) {
        const double si = sig[i], sj = sig[j];
        if (fabs(sj - si) > delta) {
            const double r1 = T[e] + pij * sj;
            const double r2 = T[j * c + i] + qij * sj;
            const double inv = 1.0 / ((sj - si) * (sj + si));
            const double ff = (sj * r1 + si * r2) * inv;
            const double gg = (si * r1 + sj * r2) * inv;
            // outside the first-order regime this step only restores orthogonality:
            // the correction must be small against the pair's relative gap, or its
            // second-order error (|f|^2 (s_i + s_j) / |s_i - s_j|) would exceed it
            const double mf = fmax(fabs(ff), fabs(gg));
            if (mf <= 0.25 && mf * (fabs(si) + fabs(sj)) <= 0.25 * fabs(sj - si)) {
                f = ff;
                g = gg;
            }
        }
    }
    F[e] = f;
    Gm[e] = g;
}

// The pairs the first-order step leaves (near-equal singular values, or a
// start not yet close enough for their gap) keep off-diagonal entries in
// T = U^T A V. They are resolved exactly: a two-sided Jacobi in FP64 on the
// block of T over the indices K of such pairs (entries above 2^-42 max|s|),
// each 2 x 2 block [t_ii t_ij; t_ji t_jj] diagonalised by a left and a right
// plane rotation (a rotation that makes it symmetric, then the symmetric
// Jacobi rotation), the left rotations also applied to the columns of U.
// The rotation angles are taken in FP32 and the rotations renormalised in
// FP64, so they are orthogonal to FP64 rounding (U stays orthonormal) and
// leave at most ~1e-7 of a pair's off-diagonal entries, which the next sweep
// removes. sigma_i = t_ii for i in K. T comes from the last refinement step
// (before its update, which is below the threshold). Entries between K and
// the rest are below the threshold and stay there (a rotation mixes two of
// them).
//
// One CTA. Each sweep takes the pairs above the threshold at its start and
// splits them into rounds of disjoint pairs (first-fit in (a, b) order, up to
// 64 rounds and kClusterList pairs a pass; the rest go to the next pass); in a
// round each warp takes a pair, all rows are rotated before all columns (left
// and right rotations commute, and the pairs of a round share no row or
// column, so the order of the pairs does not change the result). Sweeps until
// no entry is above the threshold (at most kClusterSweeps).
constexpr int kClusterSweeps = 16;
constexpr int kClusterThreads = 256;
constexpr int kClusterWarps = kClusterThreads / 32;
constexpr int kClusterList = 1024;                 // pairs coloured in one pass
constexpr int kClusterRowsPerLane = (kMaxSmemC + 31) / 32;

// |x| > thr for thr >= 0 by the ordering of IEEE-754 bit patterns (integer
// compares: FP64 instructions are slow on this GPU)
__device__ __forceinline__ bool above(double x, long long thr_bits) {
    return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) > thr_bits;
}

// (c, s) from FP32 made a unit vector in FP64: multiplied by the series of
// (1 + d)^-1/2 to second order, d = c^2 + s^2 - 1 (|d| ~ 1e-7, so the
// third-order term is below FP64 rounding)
__device__ __forceinline__ void unit_fp64(double &c, double &s) {
    const double d = fma(c, c, fma(s, s, -1.0));
    const double n = fma(d, fma(0.375, d, -0.5), 1.0);
    c *= n;
    s *= n;
}

// The rotations of one 2 x 2 block M = [taa tab; tba tbb]: left
// L = [al be; -be al] = G J and right J = [cs sn; -sn cs], L^T M J diagonal up
// to the FP32 angles. G = [cf -sf; sf cf] makes G^T M symmetric; J is the
// symmetric Jacobi rotation of G^T M. inv scales the block to about unit size
// for the FP32 arithmetic (a power of two).
__device__ __forceinline__ void cluster_rotation(double taa, double tab, double tba, double tbb, double inv,
                                                 double &al, double &be, double &cs, double &sn) {
    const float x = (float)((taa + tbb) * inv), y = (float)((tba - tab) * inv);
    const float h = hypotf(x, y);
    const float cf = h > 0.f ? x / h : 1.f, sf = h > 0.f ? y / h : 0.f;
    // G^T M = [p q'; q'' r]: q = (q' + q'') / 2, r - p, from the differences
    const double d = tbb - taa, e = tab + tba;
    const double rp = fma((double)cf, d, -(double)sf * e);
    const double q = 0.5 * fma((double)cf, e, (double)sf * d);
    float c32 = 1.f, s32 = 0.f;
    const float qf = (float)(q * inv);
    if (qf != 0.f) {
        const float zeta = (float)(rp * inv) / (2.f * qf);
        const float az = fabsf(zeta);
        const float t = (zeta >= 0.f ? 1.f : -1.f) * (az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(1.f + zeta * zeta)));
        c32 = rsqrtf(1.f + t * t);
        s32 = c32 * t;
    }
    cs = c32;
    sn = s32;
    unit_fp64(cs, sn);
    al = (double)(cf * c32 + sf * s32);
    be = (double)(cf * s32 - sf * c32);
    unit_fp64(al, be);
}

__global__ void __launch_bounds__(kClusterThreads) svd_cluster_kernel(const double *__restrict__ T, int c,
                                                                     double *__restrict__ U,
                                                                     double *__restrict__ sg) {
    extern __shared__ double sT[];       // nK x nK block of T
    constexpr int kWords = (kMaxSmemC + 31) / 32;
    __shared__ int sK[kMaxSmemC];        // block index -> index of T
    __shared__ int s_act[kMaxSmemC];
    __shared__ uint32_t s_mask[kMaxSmemC][kWords];   // row a: bit b > a set for a pair left in the sweep
    __shared__ unsigned long long s_used[kMaxSmemC]; // rounds of the pass that index a takes part in
    __shared__ uint32_t s_list[kClusterList];        // round << 16 | a << 8 | b
    __shared__ uint32_t s_round[kMaxSmemC / 2];      // a << 8 | b
    __shared__ double s_rcs[kMaxSmemC / 2][2];       // each round pair's right rotation (cs, sn)
    __shared__ int s_rgo[kMaxSmemC / 2];             // ... and whether it rotated
    __shared__ long long red[kClusterWarps];
    __shared__ int s_nK, s_any, s_np, s_rounds, s_nr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // max |sigma| by the integer order of the bit patterns
    long long mb = 0;
    for (int i = tid; i < c; i += blockDim.x) mb = max(mb, __double_as_longlong(sg[i]) & 0x7FFFFFFFFFFFFFFFll);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, off));
    if (lane == 0) red[warp] = mb;
    for (int i = tid; i < c; i += blockDim.x) s_act[i] = 0;
    __syncthreads();
    mb = 0;
    for (int w = 0; w < kClusterWarps; ++w) mb = max(mb, red[w]);
    if (mb == 0 || mb >= 0x7FF0000000000000ll) return;   // a zero matrix, or not finite
    const double smax = __longlong_as_double(mb);
    const double thr = 0x1p-42 * smax;
    const long long thr_bits = __double_as_longlong(thr);
    const long long ex = min((mb >> 52) & 0x7FF, 2045ll);
    const double inv = __longlong_as_double((2046ll - ex) << 52);   // 2^(1023 - exponent of smax)
    // indices with an entry above the threshold in their row or column (a warp
    // per row, two rows at a time, every load of the two rows issued at once)
    for (int i0 = 2 * warp; i0 < c; i0 += 2 * kClusterWarps) {
        double v[2][kClusterRowsPerLane];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < kClusterRowsPerLane; ++q) {
                const int i = i0 + h, j = lane + 32 * q;
                v[h][q] = i < c && j < c ? T[(size_t)i * c + j] : 0.0;
            }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + h;
            bool rowbig = false;
#pragma unroll
            for (int q = 0; q < kClusterRowsPerLane; ++q) {
                const int j = lane + 32 * q;
                if (i < c && j < c && j != i && above(v[h][q], thr_bits)) {
                    s_act[j] = 1;
                    rowbig = true;
                }
            }
            if (__any_sync(0xffffffffu, rowbig) && lane == 0) s_act[i] = 1;
        }
    }
    __syncthreads();
    if (warp == 0) {
        int n = 0;
        for (int j0 = 0; j0 < c; j0 += 32) {
            const int j = j0 + lane;
            const bool f = j < c && s_act[j];
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) sK[n + __popc(bal & ((1u << lane) - 1u))] = j;
            n += __popc(bal);
        }
        if (lane == 0) s_nK = n;
    }
    __syncthreads();
    const int nK = s_nK;
    if (nK == 0) return;
    for (int a = warp; a < nK; a += kClusterWarps)
#pragma unroll 5
        for (int b = lane; b < nK; b += 32) sT[a * nK + b] = T[(size_t)sK[a] * c + sK[b]];
    const int words = (nK + 31) / 32;
    for (int sweep = 0; sweep < kClusterSweeps; ++sweep) {
        // the pairs above the threshold at the start of the sweep (a warp per row)
        if (tid == 0) s_any = 0;
        __syncthreads();
        for (int a = warp; a < nK; a += kClusterWarps)
            for (int w = 0; w < words; ++w) {
                const int b = 32 * w + lane;
                const bool big = b > a && b < nK && (above(sT[a * nK + b], thr_bits) || above(sT[b * nK + a], thr_bits));
                const unsigned m = __ballot_sync(0xffffffffu, big);
                if (lane == 0) {
                    s_mask[a][w] = m;
                    if (m) s_any = 1;
                }
            }
        __syncthreads();
        if (!s_any) break;
        for (;;) {   // passes: up to 64 rounds of disjoint pairs each
            if (tid == 0) {
                for (int a = 0; a < nK; ++a) s_used[a] = 0ull;
                int np = 0, rounds = 0;
                for (int a = 0; a < nK && np < kClusterList; ++a)
                    for (int w = 0; w < words && np < kClusterList; ++w) {
                        uint32_t m = s_mask[a][w];
                        while (m && np < kClusterList) {
                            const int bit = __ffs(m) - 1;
                            m &= m - 1u;
                            const int b = 32 * w + bit;
                            const unsigned long long fr = ~(s_used[a] | s_used[b]);
                            if (fr == 0ull) continue;   // stays for the next pass
                            const int r = __ffsll((long long)fr) - 1;
                            s_used[a] |= 1ull << r;
                            s_used[b] |= 1ull << r;
                            s_mask[a][w] &= ~(1u << bit);
                            s_list[np++] = ((uint32_t)r << 16) | ((uint32_t)a << 8) | (uint32_t)b;
                            rounds = max(rounds, r + 1);
                        }
                    }
                s_np = np;
                s_rounds = rounds;
            }
            __syncthreads();
            const int np = s_np, rounds = s_rounds;
            if (np == 0) break;
            for (int r = 0; r < rounds; ++r) {
                if (tid == 0) s_nr = 0;
                __syncthreads();
                for (int k = tid; k < np; k += blockDim.x)
                    if ((int)(s_list[k] >> 16) == r) s_round[atomicAdd(&s_nr, 1)] = s_list[k] & 0xFFFFu;
                __syncthreads();
                const int nr = s_nr;
                // rows of the block and columns of U, a warp per pair (rows disjoint)
                for (int k = warp; k < nr; k += kClusterWarps) {
                    const int a = (int)(s_round[k] >> 8), b = (int)(s_round[k] & 0xFFu);
                    const double taa = sT[a * nK + a], tab = sT[a * nK + b], tba = sT[b * nK + a],
                                 tbb = sT[b * nK + b];
                    const bool go = above(tab, thr_bits) || above(tba, thr_bits);
                    if (lane == 0) s_rgo[k] = go;
                    if (!go) continue;
                    double al, be, cs, sn;
                    cluster_rotation(taa, tab, tba, tbb, inv, al, be, cs, sn);
                    for (int k2 = lane; k2 < nK; k2 += 32) {   // rows a, b: L^T
                        const double u = sT[a * nK + k2], v = sT[b * nK + k2];
                        sT[a * nK + k2] = al * u - be * v;
                        sT[b * nK + k2] = be * u + al * v;
                    }
                    const int ia = sK[a], ib = sK[b];
                    double uu[kClusterRowsPerLane], vv[kClusterRowsPerLane];
#pragma unroll
                    for (int q = 0; q < kClusterRowsPerLane; ++q) {   // columns ia, ib of U: U L
                        const int k2 = lane + 32 * q;
                        uu[q] = k2 < c ? U[(size_t)k2 * c + ia] : 0.0;
                        vv[q] = k2 < c ? U[(size_t)k2 * c + ib] : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < kClusterRowsPerLane; ++q) {
                        const int k2 = lane + 32 * q;
                        if (k2 < c) {
                            U[(size_t)k2 * c + ia] = al * uu[q] - be * vv[q];
                            U[(size_t)k2 * c + ib] = be * uu[q] + al * vv[q];
                        }
                    }
                    if (lane == 0) {
                        s_rcs[k][0] = cs;
                        s_rcs[k][1] = sn;
                    }
                }
                __syncthreads();
                // columns of the block, a warp per pair (columns disjoint): J
                for (int k = warp; k < nr; k += kClusterWarps) {
                    if (!s_rgo[k]) continue;
                    const int a = (int)(s_round[k] >> 8), b = (int)(s_round[k] & 0xFFu);
                    const double cs = s_rcs[k][0], sn = s_rcs[k][1];
                    for (int k2 = lane; k2 < nK; k2 += 32) {
                        const double u = sT[k2 * nK + a], v = sT[k2 * nK + b];
                        sT[k2 * nK + a] = cs * u - sn * v;
                        sT[k2 * nK + b] = sn * u + cs * v;
                    }
                }
                __syncthreads();
            }
        }
    }
    for (int a = tid; a < nK; a += blockDim.x) sg[sK[a]] = sT[a * nK + a];
}

// sigma sorted descending; U_R[:, rank_j] = sign(s_j) U[:, j].
// Ranks first, then the columns copied by all threads over the flat index,
// so the loads of the whole matrix are in flight together. Magnitudes are
// compared and signs flipped on the bit patterns (non-negative doubles order
// as their bits; integer operations instead of the slow FP64 pipe).
__global__ void svd_finish_kernel(const double *__restrict__ U, const double *__restrict__ sg, int c,
                                  double *__restrict__ UR, double *__restrict__ sigma) {
    __shared__ long long s_abs[256];
    __shared__ int s_rank[256];
    __shared__ unsigned long long s_flip[256];
    const int tid = threadIdx.x;
    for (int j = tid; j < c; j += blockDim.x) {
        const long long b = __double_as_longlong(sg[j]);
        s_abs[j] = b & 0x7FFFFFFFFFFFFFFFll;
        s_flip[j] = (unsigned long long)b & 0x8000000000000000ull;   // the sign of sg[j]
    }
    __syncthreads();
    for (int j = tid; j < c; j += blockDim.x) {
        const long long sj = s_abs[j];
        int rank = 0;
        for (int i = 0; i < c; ++i) rank += (s_abs[i] > sj) || (s_abs[i] == sj && i < j);
        sigma[rank] = __longlong_as_double(sj);
        s_rank[j] = rank;
    }
    __syncthreads();
#pragma unroll 8
    for (int e = tid; e < c * c; e += blockDim.x) {
        const int i = e / c, j = e - i * c;
        UR[i * c + s_rank[j]] =
            __longlong_as_double((long long)((unsigned long long)__double_as_longlong(__ldg(U + e)) ^ s_flip[j]));
    }
}

// ---------------------------------------------------------------------------
// sign convention and X = U Sigma^{1/2}
// ---------------------------------------------------------------------------
// Per column: the largest |u| and, among equal magnitudes, the smallest row,
// packed as (|u| bits << 32) | ~row so that one max orders both. Each thread
// keeps a running maximum over a strided set of rows of one column; one
// atomic per CTA and column.
__global__ void __launch_bounds__(256) col_absmax_kernel(const float *__restrict__ U, int64_t n, int d, int64_t ld,
                                                         unsigned long long *__restrict__ best) {
    const int sub = blockDim.x / d;               // row subsets per CTA (d <= 256)
    const int j = threadIdx.x % d, r0 = threadIdx.x / d;
    unsigned long long m = 0;
    if (r0 < sub) {
        for (int64_t i = (int64_t)blockIdx.x * sub + r0; i < n; i += (int64_t)gridDim.x * sub) {
            const float a = fabsf(U[i * ld + j]);
            const unsigned long long key = ((unsigned long long)__float_as_uint(a) << 32) |
                                           (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
            m = key > m ? key : m;
        }
        atomicMax(&best[j], m);
    }
}

__global__ void column_signs_kernel(const float *__restrict__ U, int d, int64_t ld,
                                    const unsigned long long *__restrict__ best, const double *__restrict__ sigma,
                                    float *__restrict__ sgn, float *__restrict__ scale) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const int64_t i = (int64_t)(0xFFFFFFFFu - (uint32_t)(best[j] & 0xFFFFFFFFull));
    sgn[j] = U[i * ld + j] < 0.f ? -1.f : 1.f;
    if (sigma) scale[j] = (float)sqrt(fmax(sigma[j], 0.0));
}

// U <- U diag(sgn); X = U diag(scale) when X is given.
__global__ void sign_scale_kernel(float *__restrict__ U, int64_t n, int d, int64_t ld,
                                  const float *__restrict__ sgn, const float *__restrict__ scale,
                                  float *__restrict__ X, int64_t ldx) {
    const int sub = blockDim.x / d;
    const int j = threadIdx.x % d, r0 = threadIdx.x / d;
    if (r0 >= sub) return;
    const float sg = sgn[j], sc = X ? scale[j] : 0.f;
    for (int64_t i = (int64_t)blockIdx.x * sub + r0; i < n; i += (int64_t)gridDim.x * sub) {
        const float u = U[i * ld + j] * sg;
        U[i * ld + j] = u;
        if (X) X[i * ldx + j] = u * sc;
    }
}

int grid_for(int64_t work, int threads) {
    int64_t g = ceil_div(std::max<int64_t>(work, 1), threads);
    return (int)std::min<int64_t>(g, num_sms() * 32);
}

}  // namespace

int gaussian_sketch(int64_t n, int c, uint64_t seed, float *out, int64_t ld, cudaStream_t st) {
    if (n <= 0 || c <= 0) return 0;
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu) ^ 0x4f4d4547u;
    const uint32_t k1 = (uint32_t)(seed >> 32);
    {
        LNE_TRACE("sketch", st);
        sketch_kernel<<<grid_for(n * ((c + 3) / 4), 256), 256, 0, st>>>(n, c, k0, k1, out, ld);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int right_multiply(const float *Y, int64_t n, int c, int64_t ldy, const double *W, int64_t ldw,
                   int dout, const double *colscale, float *out, int64_t ldo, cudaStream_t st) {
    if (n <= 0 || dout <= 0) return 0;
    dim3 grid((unsigned)ceil_div(n, kMMTile), (unsigned)ceil_div(dout, kMMTile));
    {
        LNE_TRACE("right_multiply", st);
        right_multiply_kernel<<<grid, 256, 0, st>>>(Y, n, c, ldy, W, ldw, dout, colscale, out, ldo);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

// G = Y^T Y (FP64, [c][c]).
static int gram(Workspace &ws, const float *Y, int64_t n, int c, int64_t ld, double *G, cudaStream_t st) {
    const int cp = (c + 7) & ~7;
    const int nt = cp / 8;
    const int ntiles = nt * (nt + 1) / 2;
    (void)ntiles;
    const int threads = kGramThreads;
    // whole waves of resident CTAs (one per SM at this kernel's register use)
    int per_sm = 1;
    LNE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_partial_kernel, threads,
                                                             kGramRows * cp * 4));
    const int64_t slots = num_sms() * (int64_t)std::max(1, per_sm);
    int64_t nblk = std::min<int64_t>(2 * slots, std::max<int64_t>(1, ceil_div(n, 64)));
    if (nblk > slots) nblk = (nblk / slots) * slots;
    const int64_t rows_per = ceil_div(std::max<int64_t>(n, 1), nblk);
    nblk = ceil_div(std::max<int64_t>(n, 1), rows_per);
    double *partial = nullptr;
    LNE_TRY(ws.get("gram.partial", (size_t)nblk * cp * cp, &partial));
    const int smem = kGramRows * cp * 4;
    if (smem > 48 * 1024)
        LNE_TRY(allow_dynamic_smem(gram_partial_kernel));
    {
        LNE_TRACE("gram_partial", st);
        gram_partial_kernel<<<(unsigned)nblk, threads, smem, st>>>(Y, n, c, ld, rows_per, partial);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("gram_reduce", st);
        gram_reduce_kernel<<<grid_for((int64_t)c * (c + 1) / 2 * kGramRedLanes, 256), 256, 0, st>>>(partial,
                                                                                                (int)nblk, c, G);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

// A breakdown (a pivot that is not positive) is recorded in the device status
// word read by status_check, without a host synchronisation here; the
// factorisation goes on with a unit pivot, so later kernels see finite values.
static int chol(Workspace &ws, const double *G, int c, double *R, cudaStream_t st) {
    int *status = nullptr;
    LNE_TRY(device_status(ws, &status, st));
    if (c >= 64) {   // blocked over many SMs: one cooperative launch for all panels
        double *r11 = nullptr;
        unsigned *bar = nullptr;
        LNE_TRY(ws.get("chol.r11", (size_t)kCholB * kCholB, &r11));
        LNE_TRY(ws.get("chol.bar", 1, &bar));
        LNE_CUDA_TRY(cudaMemcpyAsync(R, G, sizeof(double) * (size_t)c * c, cudaMemcpyDeviceToDevice, st));
        LNE_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
        LNE_TRACE("chol", st);
        const int nb0 = (int)std::max<int64_t>(1, ceil_div(c - kCholB, 16));
        int per_sm = 0;
        LNE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_coop_kernel, 256, 0));
        const int grid = std::min(nb0 * nb0, std::max(1, per_sm) * num_sms());
        int ci = c;
        void *args[] = {&R, &ci, &status, &r11, &bar};
        LNE_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(chol_coop_kernel), dim3(grid),
                                                 dim3(256), args, 0, st));
        LNE_LAUNCH_CHECK();
    } else {
        const int smem = c <= kMaxSmemC ? c * c * 8 : 0;
        if (smem > 48 * 1024)
            LNE_TRY(allow_dynamic_smem(chol_kernel));
        LNE_TRACE("chol", st);
        chol_kernel<<<1, kCholThreads, smem, st>>>(G, c, R, status);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int device_status(Workspace &ws, int **status, cudaStream_t st) {
    const bool fresh = !ws.has("dev.status");
    LNE_TRY(ws.get("dev.status", 4, status));
    if (fresh) LNE_CUDA_TRY(cudaMemsetAsync(*status, 0, 4 * sizeof(int), st));
    return 0;
}

int status_check(Workspace &ws, cudaStream_t st) {
    if (!ws.has("dev.status")) return 0;
    int *status = nullptr;
    LNE_TRY(ws.get("dev.status", 4, &status));
    int h[4] = {0, 0, 0, 0};
    LNE_CUDA_TRY(cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0] == 0 && h[1] == 0 && h[2] == 0) return 0;
    LNE_CUDA_TRY(cudaMemsetAsync(status, 0, 4 * sizeof(int), st));
    if (h[1] != 0) return fail(LNE_ERR_TIMEOUT, "a bounded device wait expired (tensor-core pipeline or Cholesky grid barrier)");
    if (h[2] != 0)
        return fail(LNE_ERR_UNSUPPORTED, "a row of the very sparse projection has more than 12 nonzeros (raise s)");
    return fail(LNE_ERR_NUMERIC, "Cholesky breakdown in CholeskyQR (Gram not positive definite)");
}

static int trsm_rows(const float *Y, int64_t n, int c, int64_t ldy, const double *R, float *Q, int64_t ldq,
                     cudaStream_t st) {
    const int nt = (c + 31) / 32;
    const int smem = (c * c + c) * 4;
    // every CTA stages R in shared memory: one wave of resident CTAs, each
    // walking many rows, loads it the fewest times
    const int per_sm = std::max(1, std::min(8, (227 * 1024) / std::max(smem, 1)));
    const int blocks = (int)std::min<int64_t>(ceil_div(n, 8), num_sms() * per_sm);
    LNE_TRACE("trsm_rows", st);
#define LNE_TRSM_CASE(K)                                                                               \
    case K:                                                                                            \
        if (smem > 48 * 1024) LNE_TRY(allow_dynamic_smem(trsm_rows_kernel<K>));                        \
        trsm_rows_kernel<K><<<blocks, kTrsmThreads, smem, st>>>(Y, n, c, ldy, R, Q, ldq);                      \
        break;
    switch (nt) {
        LNE_TRSM_CASE(1)
        LNE_TRSM_CASE(2)
        LNE_TRSM_CASE(3)
        LNE_TRSM_CASE(4)
        LNE_TRSM_CASE(5)
        LNE_TRSM_CASE(6)
        LNE_TRSM_CASE(7)
        LNE_TRSM_CASE(8)
        default:
            return fail(LNE_ERR_UNSUPPORTED, "CholeskyQR supports at most 256 columns");
    }
#undef LNE_TRSM_CASE
    LNE_LAUNCH_CHECK();
    return 0;
}

int cholqr1(Workspace &ws, const float *Y, int64_t n, int c, int64_t ld, float *Q, int64_t ldq, cudaStream_t st) {
    if (c <= 0 || c > 256) return fail(LNE_ERR_INVALID, "CholeskyQR needs 1 <= c <= 256");
    if (n < c) return fail(LNE_ERR_INVALID, "CholeskyQR needs at least as many rows as columns");
    if ((size_t)(c * c + c) * 4 > 227 * 1024) return fail(LNE_ERR_UNSUPPORTED, "CholeskyQR column count too large");
    double *G = nullptr, *R1 = nullptr;
    LNE_TRY(ws.get("qr.G", (size_t)c * c, &G));
    LNE_TRY(ws.get("qr.R1", (size_t)c * c, &R1));
    LNE_TRY(gram(ws, Y, n, c, ld, G, st));
    LNE_TRY(chol(ws, G, c, R1, st));
    return trsm_rows(Y, n, c, ld, R1, Q, ldq, st);
}

int cholqr2(Workspace &ws, float *Y, int64_t n, int c, int64_t ld, double *Rout, cudaStream_t st) {
    if (c <= 0 || c > 256) return fail(LNE_ERR_INVALID, "CholeskyQR2 needs 1 <= c <= 256");
    if (n < c) return fail(LNE_ERR_INVALID, "CholeskyQR2 needs at least as many rows as columns");
    if ((size_t)(c * c + c) * 4 > 227 * 1024) return fail(LNE_ERR_UNSUPPORTED, "CholeskyQR2 column count too large");
    double *G = nullptr, *R1 = nullptr, *R2 = nullptr;
    float *tmp = nullptr;
    LNE_TRY(ws.get("qr.G", (size_t)c * c, &G));
    LNE_TRY(ws.get("qr.R1", (size_t)c * c, &R1));
    LNE_TRY(ws.get("qr.R2", (size_t)c * c, &R2));
    LNE_TRY(ws.get("qr.tmp", (size_t)n * c, &tmp));
    // pass 1: G = Y^T Y, R1 = chol(G), Q1 = Y R1^-1
    LNE_TRY(gram(ws, Y, n, c, ld, G, st));
    LNE_TRY(chol(ws, G, c, R1, st));
    LNE_TRY(trsm_rows(Y, n, c, ld, R1, tmp, c, st));
    // pass 2 on Q1
    LNE_TRY(gram(ws, tmp, n, c, c, G, st));
    LNE_TRY(chol(ws, G, c, R2, st));
    LNE_TRY(trsm_rows(tmp, n, c, c, R2, Y, ld, st));
    if (Rout) {
        LNE_TRACE("upper_matmul", st);
        upper_matmul_kernel<<<c, 128, 0, st>>>(R2, R1, c, Rout);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

// C = op(A) op(B) (+ C0), and when A2 is given also C2 = op(A2) op(B2) (+ C02)
// in the same launch.
static int dgemm_small(const double *A, bool ta, const double *B, bool tb, const double *C0, double *C, int c,
                       cudaStream_t st, const double *A2 = nullptr, const double *B2 = nullptr,
                       const double *C02 = nullptr, double *C2 = nullptr) {
    if (c > kDgMaxC) return fail(LNE_ERR_UNSUPPORTED, "small FP64 products support c <= 160");
    dim3 grid((unsigned)ceil_div(c, kDgTile), (unsigned)ceil_div(c, kDgTile), A2 ? 2u : 1u);
    LNE_TRACE("dgemm_small", st);
    dgemm_small_kernel<<<grid, kDgTile * kDgTile, 0, st>>>(A, ta ? 1 : 0, B, tb ? 1 : 0, C0, C, c, A2, B2, C02,
                                                            C2);
    LNE_LAUNCH_CHECK();
    return 0;
}

// FP64 scratch of the refinement: ten c x c matrices, sigma (c) and the
// norm partials (4 kOaParts).
struct SvdScratch {
    double *U, *U2, *V, *V2, *W, *T, *P, *Q, *F, *Gm, *sg, *dl;
};

// Refines the FP32 start (sc.U, sc.V) into the SVD of R in FP64 and writes
// U_R and sigma (sorted descending).
static int svd_refine_finish(const double *R, int c, SvdScratch sc, double *U_R, double *sigma, cudaStream_t st) {
    const size_t cc = (size_t)c * c;
    double *U = sc.U, *U2 = sc.U2, *V = sc.V, *V2 = sc.V2;
    // FP64 refinement of the SVD of R itself (quadratic convergence; the FP32
    // start may be loose in directions FP32 cannot resolve, hence four steps)
    for (int it = 0; it < 4; ++it) {
        // P = U^T U and Q = V^T V (I - P, I - Q below)
        LNE_TRY(dgemm_small(U, true, U, false, nullptr, sc.P, c, st, V, V, nullptr, sc.Q));
        LNE_TRY(dgemm_small(R, false, V, false, nullptr, sc.W, c, st));   // W = R V
        LNE_TRY(dgemm_small(U, true, sc.W, false, nullptr, sc.T, c, st)); // T = U^T R V
        {
            LNE_TRACE("svd_oa_update", st);
            svd_oa_norms_kernel<<<kOaParts, 256, 0, st>>>(sc.P, sc.Q, sc.T, c, sc.sg, sc.dl);
            LNE_LAUNCH_CHECK();
            svd_oa_fg_kernel<<<(unsigned)ceil_div((int64_t)cc, 256), 256, 0, st>>>(sc.P, sc.Q, sc.T, c, sc.sg,
                                                                                  sc.dl, sc.F, sc.Gm);
            LNE_LAUNCH_CHECK();
        }
        LNE_TRY(dgemm_small(U, false, sc.F, false, U, U2, c, st, V, sc.Gm, V, V2));   // U2 = U + U F, V2 = V + V G
        std::swap(U, U2);
        std::swap(V, V2);
    }
    {
        LNE_TRACE("svd_cluster", st);
        LNE_TRY(allow_dynamic_smem(svd_cluster_kernel));
        svd_cluster_kernel<<<1, kClusterThreads, sizeof(double) * cc, st>>>(sc.T, c, U, sc.sg);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("svd_finish", st);
        svd_finish_kernel<<<1, 256, 0, st>>>(U, sc.sg, c, U_R, sigma);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int small_svd(Workspace &ws, const double *R, int c, double *U_R, double *sigma, cudaStream_t st) {
    if (c > kMaxSmemC) return fail(LNE_ERR_UNSUPPORTED, "small SVD supports c <= 160");
    double *U = nullptr, *U2 = nullptr, *V = nullptr, *V2 = nullptr, *W = nullptr, *T = nullptr, *P = nullptr,
           *Q = nullptr, *F = nullptr, *Gm = nullptr, *sg = nullptr;
    int *sweeps = nullptr;
    const size_t cc = (size_t)c * c;
    LNE_TRY(ws.get("svd.U", cc, &U));
    LNE_TRY(ws.get("svd.U2", cc, &U2));
    LNE_TRY(ws.get("svd.V", cc, &V));
    LNE_TRY(ws.get("svd.V2", cc, &V2));
    LNE_TRY(ws.get("svd.W", cc, &W));
    LNE_TRY(ws.get("svd.T", cc, &T));
    LNE_TRY(ws.get("svd.P", cc, &P));
    LNE_TRY(ws.get("svd.Q", cc, &Q));
    LNE_TRY(ws.get("svd.F", cc, &F));
    LNE_TRY(ws.get("svd.G", cc, &Gm));
    LNE_TRY(ws.get("svd.sg", (size_t)c, &sg));
    double *dl = nullptr;
    LNE_TRY(ws.get("svd.delta", 4 * kOaParts, &dl));
    LNE_TRY(ws.get("svd.sweeps", 1, &sweeps));
    float2 *jrot = nullptr;
    uint32_t *jlab = nullptr;
    if (c <= kJacRegMaxC) {
        LNE_TRY(ws.get("svd.jrot", jreg_records(c), &jrot));
        LNE_TRY(ws.get("svd.jlab", jreg_records(c), &jlab));
    }
    // starting point: FP32 one-sided Jacobi on R (U, V in FP64 storage)
    {
        LNE_TRACE("jacobi32", st);
        LNE_TRY(launch_jacobi(R, c, U, V, jrot, jlab, sweeps, st));
    }
    SvdScratch sc{U, U2, V, V2, W, T, P, Q, F, Gm, sg, dl};
    return svd_refine_finish(R, c, sc, U_R, sigma, st);
}

int sign_fix_embed(Workspace &ws, float *U, int64_t n, int d, int64_t ld, const double *sigma, float *X,
                   int64_t ldx, cudaStream_t st) {
    if (d < 1 || d > 256) return fail(LNE_ERR_UNSUPPORTED, "sign fix supports 1..256 columns");
    unsigned long long *best = nullptr;
    float *sgn = nullptr, *scale = nullptr;
    LNE_TRY(ws.get("sign.best", (size_t)d, &best));
    LNE_TRY(ws.get("sign.sgn", (size_t)d, &sgn));
    LNE_TRY(ws.get("sign.scale", (size_t)d, &scale));
    LNE_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long) * d, st));
    const int sub = 256 / d;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, sub), num_sms() * 8));
    {
        LNE_TRACE("col_absmax", st);
        col_absmax_kernel<<<blocks, 256, 0, st>>>(U, n, d, ld, best);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("column_signs", st);
        column_signs_kernel<<<(d + 127) / 128, 128, 0, st>>>(U, d, ld, best, X ? sigma : nullptr, sgn, scale);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("sign_scale", st);
        sign_scale_kernel<<<blocks, 256, 0, st>>>(U, n, d, ld, sgn, scale, X, ldx);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the small SVD (lne_svd_small_noalloc).
//
// For callers that must not allocate device memory when they call in -- for
// example a process whose device memory is wholly handed to another allocator
// up front, or a latency-bound service that forbids allocation after start-up.
// Its scratch (ten c x c FP64 matrices, a few scalars and the Jacobi's
// rotation records, c <= 160: about 4.5 MB) is a file-scope __device__ array that every GPU which loads this
// library holds until the process exits. In host code the array's name is only
// a stand-in for it, so its device address is looked up with
// cudaGetSymbolAddress once per device, on that device's first call.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxC = 160;
constexpr size_t kNoAllocMat = (size_t)kNoAllocMaxC * kNoAllocMaxC;
constexpr size_t kNoAllocRec = (size_t)kJacMaxSweeps * kJacRegMaxC * (kJacRegMaxC / 2);   // >= jreg_records(c)
constexpr size_t kNoAllocDoubles = 10 * kNoAllocMat + kNoAllocMaxC + 128 + kNoAllocRec + kNoAllocRec / 2;
static_assert(4 * kOaParts + 8 <= 128, "partial sums and sweep count fit the reserve");
static __device__ __align__(256) double g_svd_scratch[kNoAllocDoubles];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kNoAllocMaxDevices] = {};

}  // namespace
}  // namespace lne

extern "C" int lne_svd_small_noalloc(const double *R_dev, int32_t c, double *U_dev, double *sigma_dev, void *stream) {
    using namespace lne;
    clear_message();
    set_tracer(nullptr);   // no timing events (they would be created on demand)
    if (!R_dev || !U_dev || !sigma_dev) return fail(LNE_ERR_INVALID, "NULL argument");
    if (c < 1 || c > kNoAllocMaxC) return fail(LNE_ERR_INVALID, "lne_svd_small_noalloc needs 1 <= c <= 160");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e, __FILE__, __LINE__);
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(LNE_ERR_UNSUPPORTED, "device index too large");
    double *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_svd_scratch);
            if (e != cudaSuccess) return cuda_fail("cudaGetSymbolAddress", e, __FILE__, __LINE__);
            g_noalloc_addr[dev] = static_cast<double *>(ptr);
        }
        base = g_noalloc_addr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t cc = (size_t)c * c;
    // every buffer below is fully written before it is read, so nothing left by
    // an earlier call needs clearing
    double *U = base, *U2 = base + cc, *V = base + 2 * cc, *V2 = base + 3 * cc, *W = base + 4 * cc,
           *T = base + 5 * cc, *P = base + 6 * cc, *Q = base + 7 * cc, *F = base + 8 * cc, *Gm = base + 9 * cc;
    double *sg = base + 10 * kNoAllocMat;
    double *dl = sg + kNoAllocMaxC;
    int *sweeps = reinterpret_cast<int *>(dl + 4 * kOaParts);
    float2 *jrot = reinterpret_cast<float2 *>(base + 10 * kNoAllocMat + kNoAllocMaxC + 128);
    uint32_t *jlab = reinterpret_cast<uint32_t *>(jrot + kNoAllocRec);
    LNE_TRY(launch_jacobi(R_dev, c, U, V, jrot, jlab, sweeps, st));
    SvdScratch sc{U, U2, V, V2, W, T, P, Q, F, Gm, sg, dl};
    LNE_TRY(svd_refine_finish(R_dev, c, sc, U_dev, sigma_dev, st));
    return LNE_OK;
}
