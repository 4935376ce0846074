// Dense stages of the randomized SVD (Algorithm 4) on the GPU:
//
//   sketch         Omega = randn(n, c) from Philox4x32-10 words (Box-Muller).
//   gram           G = Y^T Y in FP64: per-CTA partial Grams over row blocks
//                  (products of FP32 inputs are exact in FP64), summed in a
//                  fixed order so the result is reproducible.
//   chol_inv       G = R^T R (upper Cholesky) and R^-1 in FP64, one CTA.
//   right_multiply out = Y W for a small FP64 W (rounded to FP32), FP32 FMA.
//   cholqr2        Q = Y R1^-1, then again: the orthonormalisation used in
//                  place of eigSVD inside the power iteration (same range).
//   small_svd      one-sided (Hestenes) Jacobi on the c x c factor R in FP64:
//                  R V = U_R Sigma, so Y = Q R gives left singular vectors
//                  Q U_R -- the final eigSVD step of Algorithm 4.
//   sign_fix_embed largest-magnitude entry of each column made positive, and
//                  X = U Sigma^{1/2} (Sec. 3.2).
#include <algorithm>
#include <cmath>

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
// FP64 Gram: thread (ti, tj), ti <= tj, owns an 8x8 tile of the upper half.
// ---------------------------------------------------------------------------
constexpr int kGramRows = 32;   // rows staged per step

constexpr int kGramThreads = 256;

__global__ void __launch_bounds__(kGramThreads) gram_partial_kernel(const float *__restrict__ Y, int64_t n, int c,
                                                                    int64_t ld, int64_t rows_per_cta,
                                                                    double *__restrict__ partial) {
    extern __shared__ float ys[];   // kGramRows x cp
    const int cp = (c + 7) & ~7;
    const int nt = cp / 8;
    const int ntiles = nt * (nt + 1) / 2;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = imin64(n, r0 + rows_per_cta);
    // tiles are processed in groups of kGramThreads (uniform trip count for the barriers)
    for (int g0 = 0; g0 < ntiles; g0 += kGramThreads) {
        const int tile = g0 + tid;
        const bool active = tile < ntiles;
        int ti = 0, tj = 0;
        if (active) {
            int rem = tile;
            while (rem >= nt - ti) {
                rem -= nt - ti;
                ++ti;
            }
            tj = ti + rem;
        }
        double acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
        for (int64_t base = r0; base < r1; base += kGramRows) {
            const int rows = (int)imin64(kGramRows, r1 - base);
            for (int e = tid; e < kGramRows * cp; e += kGramThreads) {
                int rr = e / cp, cc = e - rr * cp;
                ys[e] = (rr < rows && cc < c) ? Y[(base + rr) * ld + cc] : 0.0f;
            }
            __syncthreads();
            if (active) {
                for (int rr = 0; rr < rows; ++rr) {
                    const float *yr = ys + rr * cp;
                    double av[8], bv[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        av[t] = (double)yr[ti * 8 + t];
                        bv[t] = (double)yr[tj * 8 + t];
                    }
#pragma unroll
                    for (int x = 0; x < 8; ++x)
#pragma unroll
                        for (int y = 0; y < 8; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
                }
            }
            __syncthreads();
        }
        if (active) {
            double *P = partial + (int64_t)blockIdx.x * cp * cp;
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) P[(ti * 8 + x) * cp + tj * 8 + y] = acc[x][y];
        }
    }
}

// G[i][j] = sum over CTAs of the partials (fixed order), mirrored to i > j.
__global__ void gram_reduce_kernel(const double *__restrict__ partial, int nblk, int c,
                                   double *__restrict__ G) {
    const int cp = (c + 7) & ~7;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
        int i = e / c, j = e - i * c;
        int a = min(i, j), b = max(i, j);
        // the (a, b) entry lives in tile (a/8, b/8); tiles with a/8 == b/8 hold
        // both orders, tiles above the diagonal only (a, b).
        double s = 0.0;
        for (int k = 0; k < nblk; ++k) s += partial[(int64_t)k * cp * cp + a * cp + b];
        G[e] = s;
    }
}

// ---------------------------------------------------------------------------
// Cholesky (upper, G = R^T R) and R^-1, one CTA, FP64.
// ---------------------------------------------------------------------------
constexpr int kCholThreads = 512;
constexpr int kMaxSmemC = 160;

__global__ void __launch_bounds__(kCholThreads) chol_inv_kernel(const double *__restrict__ G, int c,
                                                                double *__restrict__ R,
                                                                double *__restrict__ Rinv,
                                                                int *__restrict__ status) {
    extern __shared__ double sm[];
    const bool in_smem = c <= kMaxSmemC;
    double *A = in_smem ? sm : R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kCholThreads / 32;
    for (int e = tid; e < c * c; e += kCholThreads) A[e] = G[e];
    __syncthreads();
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < c; ++k) {
        if (tid == 0) {
            double akk = A[k * c + k];
            if (!(akk > 0.0) || !isfinite(akk)) {
                bad = k + 1;
                A[k * c + k] = 1.0;
            } else {
                A[k * c + k] = sqrt(akk);
            }
        }
        __syncthreads();
        const double piv = A[k * c + k];
        for (int j = k + 1 + tid; j < c; j += kCholThreads) A[k * c + j] /= piv;
        __syncthreads();
        for (int i = k + 1 + warp; i < c; i += nw) {
            const double aki = A[k * c + i];
            for (int j = i + lane; j < c; j += 32) A[i * c + j] -= aki * A[k * c + j];
        }
        __syncthreads();
    }
    // R = upper triangle of A
    if (in_smem) {
        for (int e = tid; e < c * c; e += kCholThreads) {
            int i = e / c, j = e - i * c;
            R[e] = j >= i ? A[e] : 0.0;
        }
    } else {
        for (int e = tid; e < c * c; e += kCholThreads) {
            int i = e / c, j = e - i * c;
            if (j < i) R[e] = 0.0;
        }
    }
    __syncthreads();
    // R^-1 row by row from the bottom: Rinv[i][j] = -(sum_{l=i+1..j} R[i][l] Rinv[l][j]) / R[i][i]
    for (int e = tid; e < c * c; e += kCholThreads) Rinv[e] = 0.0;
    __syncthreads();
    for (int i = c - 1; i >= 0; --i) {
        const double rii = R[i * c + i];
        for (int j = i + tid; j < c; j += kCholThreads) {
            double s = (j == i) ? 1.0 : 0.0;
            for (int l = i + 1; l <= j; ++l) s -= R[i * c + l] * Rinv[l * c + j];
            Rinv[i * c + j] = s / rii;
        }
        __syncthreads();
    }
    if (tid == 0) *status = bad;
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
// One-sided Jacobi SVD of a c x c FP64 matrix (c <= 160), one CTA. Columns are
// paired by the circle method (m = c rounded up to even players, player 0
// fixed); every round rotates m/2 disjoint column pairs, 8 threads per pair.
// ---------------------------------------------------------------------------
constexpr int kJacTPP = 8;

__device__ __forceinline__ int circle_player(int pos, int round, int m) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (m - 1)) + 1;
}

__global__ void jacobi_svd_kernel(const double *__restrict__ R, int c, double *__restrict__ UR,
                                  double *__restrict__ sigma, int max_sweeps,
                                  int *__restrict__ sweeps_out) {
    extern __shared__ double A[];   // column-major: A[j * c + i]
    __shared__ double red[32];
    __shared__ double s_sig[kMaxSmemC + 1];
    __shared__ int s_done;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    for (int e = tid; e < c * c; e += nthreads) {
        int i = e / c, j = e - i * c;
        A[j * c + i] = R[e];
    }
    __syncthreads();
    const int m = c + (c & 1);
    const int pairs = m / 2;
    const int pi = tid / kJacTPP, sub = tid % kJacTPP;
    const double tol = 1e-15;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double local_max = 0.0;
        for (int round = 0; round < m - 1; ++round) {
            // every lane takes part in the shuffles; lanes without a pair add zeros
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
            double al = 0.0, be = 0.0, ga = 0.0;
            if (active) {
                const double *ap = A + p * c, *aq = A + q * c;
                for (int i = sub; i < c; i += kJacTPP) {
                    double x = ap[i], y = aq[i];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
            }
#pragma unroll
            for (int off = 1; off < kJacTPP; off <<= 1) {
                al += __shfl_xor_sync(0xffffffffu, al, off);
                be += __shfl_xor_sync(0xffffffffu, be, off);
                ga += __shfl_xor_sync(0xffffffffu, ga, off);
            }
            if (active && ga != 0.0 && al > 0.0 && be > 0.0) {
                double rel = fabs(ga) / sqrt(al * be);
                local_max = fmax(local_max, rel);
                if (rel > tol) {
                    double zeta = (be - al) / (2.0 * ga);
                    double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    double cs = 1.0 / sqrt(1.0 + t * t);
                    double sn = cs * t;
                    double *ap = A + p * c, *aq = A + q * c;
                    for (int i = sub; i < c; i += kJacTPP) {
                        double x = ap[i], y = aq[i];
                        ap[i] = cs * x - sn * y;
                        aq[i] = sn * x + cs * y;
                    }
                }
            }
            __syncthreads();
        }
        // block max of local_max
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, off));
        if (lane == 0) red[warp] = local_max;
        __syncthreads();
        if (tid == 0) {
            double mx = 0.0;
            for (int w = 0; w < (nthreads + 31) / 32; ++w) mx = fmax(mx, red[w]);
            s_done = mx <= tol;
        }
        __syncthreads();
        if (s_done) {
            ++sweep;
            break;
        }
    }
    // singular values = column norms
    for (int j = tid; j < c; j += nthreads) {
        double s = 0.0;
        for (int i = 0; i < c; ++i) s = fma(A[j * c + i], A[j * c + i], s);
        s_sig[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = tid; j < c; j += nthreads) {
        const double sj = s_sig[j];
        int rank = 0;
        for (int i = 0; i < c; ++i) rank += (s_sig[i] > sj) || (s_sig[i] == sj && i < j);
        sigma[rank] = sj;
        const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
        for (int i = 0; i < c; ++i) UR[i * c + rank] = A[j * c + i] * inv;
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// ---------------------------------------------------------------------------
// sign convention and X = U Sigma^{1/2}
// ---------------------------------------------------------------------------
__global__ void col_absmax_kernel(const float *__restrict__ U, int64_t n, int d, int64_t ld,
                                  unsigned long long *__restrict__ best) {
    // thread handles one column for a strided set of rows; packs (|u| bits, ~row)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / d;
        int j = (int)(e - i * d);
        float a = fabsf(U[i * ld + j]);
        unsigned long long key = ((unsigned long long)__float_as_uint(a) << 32) |
                                 (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
        atomicMax(&best[j], key);
    }
}

__global__ void apply_sign_kernel(float *__restrict__ U, int64_t n, int d, int64_t ld,
                                  const float *__restrict__ sgn) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / d;
        int j = (int)(e - i * d);
        U[i * ld + j] *= sgn[j];
    }
}

__global__ void column_signs_kernel(const float *__restrict__ U, int d, int64_t ld,
                                    const unsigned long long *__restrict__ best,
                                    float *__restrict__ sgn) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    int64_t arg = (int64_t)(0xFFFFFFFFu - (uint32_t)(best[j] & 0xFFFFFFFFull));
    sgn[j] = U[arg * ld + j] < 0.f ? -1.f : 1.f;
}

__global__ void embed_scale_kernel(const float *__restrict__ U, int64_t n, int d, int64_t ld,
                                   const double *__restrict__ sigma, float *__restrict__ X,
                                   int64_t ldx) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / d;
        int j = (int)(e - i * d);
        X[i * ldx + j] = (float)((double)U[i * ld + j] * sqrt(fmax(sigma[j], 0.0)));
    }
}

int grid_for(int64_t work, int threads) {
    int64_t g = ceil_div(std::max<int64_t>(work, 1), threads);
    return (int)std::min<int64_t>(g, 152 * 32);
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
    int64_t nblk = std::min<int64_t>(304, std::max<int64_t>(1, ceil_div(n, 64)));
    const int64_t rows_per = ceil_div(std::max<int64_t>(n, 1), nblk);
    nblk = ceil_div(std::max<int64_t>(n, 1), rows_per);
    double *partial = nullptr;
    LNE_TRY(ws.get("gram.partial", (size_t)nblk * cp * cp, &partial));
    const int smem = kGramRows * cp * 4;
    {
        LNE_TRACE("gram_partial", st);
        gram_partial_kernel<<<(unsigned)nblk, threads, smem, st>>>(Y, n, c, ld, rows_per, partial);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("gram_reduce", st);
        gram_reduce_kernel<<<grid_for((int64_t)c * c, 256), 256, 0, st>>>(partial, (int)nblk, c, G);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

static int chol_inv(Workspace &ws, const double *G, int c, double *R, double *Rinv, cudaStream_t st) {
    int *status = nullptr;
    LNE_TRY(ws.get("chol.status", 1, &status));
    const int smem = c <= kMaxSmemC ? c * c * 8 : 0;
    if (smem > 48 * 1024)
        LNE_CUDA_TRY(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    {
        LNE_TRACE("chol_inv", st);
        chol_inv_kernel<<<1, kCholThreads, smem, st>>>(G, c, R, Rinv, status);
        LNE_LAUNCH_CHECK();
    }
    int h = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) return fail(LNE_ERR_NUMERIC, "Cholesky breakdown in CholeskyQR (Gram not positive definite)");
    return 0;
}

int cholqr2(Workspace &ws, float *Y, int64_t n, int c, int64_t ld, double *Rout, cudaStream_t st) {
    if (c <= 0 || c > 256) return fail(LNE_ERR_INVALID, "CholeskyQR2 needs 1 <= c <= 256");
    if (n < c) return fail(LNE_ERR_INVALID, "CholeskyQR2 needs at least as many rows as columns");
    double *G = nullptr, *R1 = nullptr, *R1i = nullptr, *R2 = nullptr, *R2i = nullptr;
    float *tmp = nullptr;
    LNE_TRY(ws.get("qr.G", (size_t)c * c, &G));
    LNE_TRY(ws.get("qr.R1", (size_t)c * c, &R1));
    LNE_TRY(ws.get("qr.R1i", (size_t)c * c, &R1i));
    LNE_TRY(ws.get("qr.R2", (size_t)c * c, &R2));
    LNE_TRY(ws.get("qr.R2i", (size_t)c * c, &R2i));
    LNE_TRY(ws.get("qr.tmp", (size_t)n * c, &tmp));
    // pass 1
    LNE_TRY(gram(ws, Y, n, c, ld, G, st));
    LNE_TRY(chol_inv(ws, G, c, R1, R1i, st));
    LNE_TRY(right_multiply(Y, n, c, ld, R1i, c, c, nullptr, tmp, c, st));
    // pass 2
    LNE_TRY(gram(ws, tmp, n, c, c, G, st));
    LNE_TRY(chol_inv(ws, G, c, R2, R2i, st));
    LNE_TRY(right_multiply(tmp, n, c, c, R2i, c, c, nullptr, Y, ld, st));
    if (Rout) {
        {
            LNE_TRACE("upper_matmul", st);
            upper_matmul_kernel<<<c, 128, 0, st>>>(R2, R1, c, Rout);
            LNE_LAUNCH_CHECK();
        }
    }
    return 0;
}

int small_svd(Workspace &ws, const double *R, int c, double *U_R, double *sigma, cudaStream_t st) {
    if (c > kMaxSmemC) return fail(LNE_ERR_UNSUPPORTED, "small SVD supports c <= 160");
    int *sweeps = nullptr;
    LNE_TRY(ws.get("svd.sweeps", 1, &sweeps));
    const int m = c + (c & 1);
    const int threads = std::max(32, std::min(1024, (m / 2 * kJacTPP + 31) / 32 * 32));
    const int smem = c * c * 8;
    if (smem > 48 * 1024)
        LNE_CUDA_TRY(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    {
        LNE_TRACE("jacobi_svd", st);
        jacobi_svd_kernel<<<1, threads, smem, st>>>(R, c, U_R, sigma, 60, sweeps);
        LNE_LAUNCH_CHECK();
    }
    return 0;
}

int sign_fix_embed(Workspace &ws, float *U, int64_t n, int d, int64_t ld, const double *sigma, float *X,
                   int64_t ldx, cudaStream_t st) {
    unsigned long long *best = nullptr;
    float *sgn = nullptr;
    LNE_TRY(ws.get("sign.best", (size_t)d, &best));
    LNE_TRY(ws.get("sign.sgn", (size_t)d, &sgn));
    LNE_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long) * d, st));
    {
        LNE_TRACE("col_absmax", st);
        col_absmax_kernel<<<grid_for(n * d, 256), 256, 0, st>>>(U, n, d, ld, best);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("column_signs", st);
        column_signs_kernel<<<(d + 127) / 128, 128, 0, st>>>(U, d, ld, best, sgn);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("apply_sign", st);
        apply_sign_kernel<<<grid_for(n * d, 256), 256, 0, st>>>(U, n, d, ld, sgn);
        LNE_LAUNCH_CHECK();
    }
    if (X) {
        {
            LNE_TRACE("embed_scale", st);
            embed_scale_kernel<<<grid_for(n * d, 256), 256, 0, st>>>(U, n, d, ld, sigma, X, ldx);
            LNE_LAUNCH_CHECK();
        }
    }
    return 0;
}

}  // namespace lne
