// Surrogate of the tuning search (Sec. 4.4 tunes the method's hyper-parameters
// by scoring many configurations; a regression network trained on scores of
// full runs ranks candidates so that only the most promising ones are run).
//
// Network: 30 standardised inputs -> 256 ReLU -> 256 ReLU -> 1, trained with
// the mean squared error and Adam. FP32 master weights; every product reads
// the bfloat16 rounding of the weights and accumulates in FP32.
//
// Kernels, one batch of B rows:
//   forward   one CTA per 32 rows, thread j owns hidden unit j of both layers,
//             the batch's activations stay in shared memory;
//   backward  (rows) dL/dz2 and dL/dz1 per row, through W2 read transposed;
//             (weights) one CTA per weight row: fixed-order sums over the
//             batch, so gradients are deterministic;
//   adam      one thread per parameter, also refreshes the bfloat16 copies.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace lne {

namespace {

constexpr int kIn = kSurrogateInputs;
constexpr int kHid = kSurrogateHidden;
constexpr int kRows = 32;   // rows per CTA in the row kernels
constexpr int64_t kW1 = 0, kB1 = kW1 + kIn * kHid, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
                  kB3 = kW3 + kHid;
static_assert(kB3 + 1 == kSurrogateParams, "parameter layout");

__device__ __forceinline__ float bf(__nv_bfloat16 x) { return __bfloat162float(x); }

// He-uniform initial weights (U(-a, a), a = sqrt(6 / fan_in)) from Philox
// (counter = parameter index, key = seed); zero biases.
__global__ void sur_init_kernel(float *__restrict__ w, uint32_t k0, uint32_t k1) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kSurrogateParams;
         i += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f;
        if (i < kB1) a = sqrtf(6.0f / kIn);
        else if (i >= kW2 && i < kB2) a = sqrtf(6.0f / kHid);
        else if (i >= kW3 && i < kB3) a = sqrtf(6.0f / kHid);
        const u32x4 r = philox10(u32x4{(uint32_t)i, 0x5u, 0u, 0u}, k0, k1);
        const float u = ((float)(r.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
        w[i] = (2.0f * u - 1.0f) * a;
    }
}

__device__ __forceinline__ void store_bf16_copies(int64_t i, float wi, __nv_bfloat16 *wb, __nv_bfloat16 *w2t) {
    const __nv_bfloat16 b = __float2bfloat16_rn(wi);
    wb[i] = b;
    if (i >= kW2 && i < kB2) {
        const int64_t e = i - kW2, k = e / kHid, j = e - k * kHid;
        w2t[j * kHid + k] = b;
    }
}

__global__ void sur_cast_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb,
                                __nv_bfloat16 *__restrict__ w2t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kSurrogateParams;
         i += (int64_t)gridDim.x * blockDim.x)
        store_bf16_copies(i, w[i], wb, w2t);
}

// Per-feature mean and population standard deviation (two passes, FP64, one
// CTA per feature, fixed-order reduction); std < 1e-6 becomes 1.
__global__ void __launch_bounds__(256) sur_scaling_kernel(const float *__restrict__ X, int64_t rows,
                                                          float *__restrict__ mean, float *__restrict__ std) {
    __shared__ double red[256];
    const int f = blockIdx.x, tid = threadIdx.x;
    double s = 0.0;
    for (int64_t r = tid; r < rows; r += blockDim.x) s += (double)X[r * kIn + f];
    red[tid] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    const double mu = red[0] / (double)rows;
    __syncthreads();
    double q = 0.0;
    for (int64_t r = tid; r < rows; r += blockDim.x) {
        const double d = (double)X[r * kIn + f] - mu;
        q += d * d;
    }
    red[tid] = q;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        const double sd = sqrt(red[0] / (double)rows);
        mean[f] = (float)mu;
        std[f] = sd < 1e-6 ? 1.0f : (float)sd;
    }
}

// y = w3 . relu(W2^T relu(W1^T x' + b1) + b2) + b3 for rows r0 .. r0 + 31 of
// the batch; row r of the batch is X row idx[r] (or r without idx). Training
// also stores x', h1, h2 of the batch for the backward pass.
__global__ void __launch_bounds__(256) sur_forward_kernel(const float *__restrict__ X, int64_t rows,
                                                          const int32_t *__restrict__ idx,
                                                          const float *__restrict__ mean,
                                                          const float *__restrict__ std,
                                                          const __nv_bfloat16 *__restrict__ wb, float *__restrict__ y,
                                                          float *__restrict__ Xs, float *__restrict__ H1,
                                                          float *__restrict__ H2) {
    extern __shared__ float sm[];
    float *xs = sm;                    // [kRows][32]
    float *h1 = xs + kRows * 32;       // [kRows][kHid]
    float *h2 = h1 + kRows * kHid;     // [kRows][kHid]
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    const int nr = (int)imin64(kRows, rows - r0);
    for (int e = tid; e < kRows * 32; e += blockDim.x) {
        const int r = e >> 5, i = e & 31;
        float v = 0.f;
        if (r < nr && i < kIn) {
            const int64_t row = idx ? (int64_t)idx[r0 + r] : r0 + r;
            v = (X[row * kIn + i] - mean[i]) / std[i];
            if (Xs) Xs[(r0 + r) * kIn + i] = v;
        }
        xs[e] = v;
    }
    __syncthreads();
    const int j = tid;
    float acc[kRows];
    {
        const float b = bf(wb[kB1 + j]);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = b;
        for (int i = 0; i < kIn; ++i) {
            const float w = bf(wb[kW1 + i * kHid + j]);
#pragma unroll
            for (int r = 0; r < kRows; ++r) acc[r] = fmaf(xs[r * 32 + i], w, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float h = fmaxf(acc[r], 0.f);
            h1[r * kHid + j] = h;
            if (H1 && r < nr) H1[(r0 + r) * kHid + j] = h;
        }
    }
    __syncthreads();
    {
        const float b = bf(wb[kB2 + j]);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = b;
        for (int k = 0; k < kHid; ++k) {
            const float w = bf(wb[kW2 + k * kHid + j]);
#pragma unroll
            for (int r = 0; r < kRows; ++r) acc[r] = fmaf(h1[r * kHid + k], w, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float h = fmaxf(acc[r], 0.f);
            h2[r * kHid + j] = h;
            if (H2 && r < nr) H2[(r0 + r) * kHid + j] = h;
        }
    }
    __syncthreads();
    // output: warp w sums rows w, w + 8, w + 16, w + 24 (lanes over units, fixed shuffle tree)
    const int warp = tid >> 5, lane = tid & 31;
    for (int r = warp; r < nr; r += 8) {
        float s = 0.f;
#pragma unroll
        for (int t = 0; t < kHid / 32; ++t) s = fmaf(h2[r * kHid + lane + 32 * t], bf(wb[kW3 + lane + 32 * t]), s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[r0 + r] = s + bf(wb[kB3]);
    }
}

// Per row of the batch: dy = 2 (y - t) / B, dz2 = dy w3 [h2 > 0],
// dz1 = (W2 dz2) [h1 > 0] (W2 read through its transposed bfloat16 copy).
__global__ void __launch_bounds__(256) sur_backward_rows_kernel(
    const float *__restrict__ y, const float *__restrict__ t, const int32_t *__restrict__ idx, int64_t B,
    const float *__restrict__ H1, const float *__restrict__ H2, const __nv_bfloat16 *__restrict__ wb,
    const __nv_bfloat16 *__restrict__ w2t, float *__restrict__ dy, float *__restrict__ dZ2,
    float *__restrict__ dZ1) {
    extern __shared__ float sm[];
    float *dz2 = sm;                   // [kRows][kHid]
    float *dys = dz2 + kRows * kHid;   // [kRows]
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    const int nr = (int)imin64(kRows, B - r0);
    if (tid < kRows) {
        float v = 0.f;
        if (tid < nr) {
            const int64_t row = idx ? (int64_t)idx[r0 + tid] : r0 + tid;
            v = 2.0f * (y[r0 + tid] - t[row]) / (float)B;
            dy[r0 + tid] = v;
        }
        dys[tid] = v;
    }
    __syncthreads();
    const int j = tid;
    const float w3j = bf(wb[kW3 + j]);
    for (int r = 0; r < kRows; ++r) {
        float v = 0.f;
        if (r < nr && H2[(r0 + r) * kHid + j] > 0.f) v = dys[r] * w3j;
        dz2[r * kHid + j] = v;
        if (r < nr) dZ2[(r0 + r) * kHid + j] = v;
    }
    __syncthreads();
    const int k = tid;
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
    for (int jj = 0; jj < kHid; ++jj) {
        const float w = bf(w2t[jj * kHid + k]);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = fmaf(dz2[r * kHid + jj], w, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r)
        if (r < nr) dZ1[(r0 + r) * kHid + k] = H1[(r0 + r) * kHid + k] > 0.f ? acc[r] : 0.f;
}

// Weight gradients, sums over the batch in row order:
// blocks 0..255: dW2[k][:] = sum_r h1[r][k] dz2[r][:]; blocks 256..285:
// dW1[i][:] = sum_r x'[r][i] dz1[r][:]; block 286: db1, db2, dw3, db3.
__global__ void __launch_bounds__(256) sur_weight_grad_kernel(const float *__restrict__ Xs,
                                                              const float *__restrict__ H1,
                                                              const float *__restrict__ H2,
                                                              const float *__restrict__ dy,
                                                              const float *__restrict__ dZ1,
                                                              const float *__restrict__ dZ2, int64_t B,
                                                              float *__restrict__ g) {
    const int b = blockIdx.x, j = threadIdx.x;
    if (b < kHid) {
        float s = 0.f;
        for (int64_t r = 0; r < B; ++r) s = fmaf(H1[r * kHid + b], dZ2[r * kHid + j], s);
        g[kW2 + (int64_t)b * kHid + j] = s;
    } else if (b < kHid + kIn) {
        const int i = b - kHid;
        float s = 0.f;
        for (int64_t r = 0; r < B; ++r) s = fmaf(Xs[r * kIn + i], dZ1[r * kHid + j], s);
        g[kW1 + (int64_t)i * kHid + j] = s;
    } else {
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (int64_t r = 0; r < B; ++r) {
            s1 += dZ1[r * kHid + j];
            s2 += dZ2[r * kHid + j];
            s3 = fmaf(H2[r * kHid + j], dy[r], s3);
        }
        g[kB1 + j] = s1;
        g[kB2 + j] = s2;
        g[kW3 + j] = s3;
        if (j == 0) {
            float s = 0.f;
            for (int64_t r = 0; r < B; ++r) s += dy[r];
            g[kB3] = s;
        }
    }
}

// Adam with bias correction (c1 = 1 - beta1^step, c2 = 1 - beta2^step).
__global__ void sur_adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                                const float *__restrict__ g, float lr, float beta1, float beta2, float eps, float c1,
                                float c2, __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ w2t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kSurrogateParams;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        store_bf16_copies(i, wi, wb, w2t);
    }
}

// Mean squared error of a batch (one CTA, FP64, fixed order); t row r is
// t[idx[r]] (or t[r]).
__global__ void __launch_bounds__(256) sur_mse_kernel(const float *__restrict__ y, const float *__restrict__ t,
                                                      const int32_t *__restrict__ idx, int64_t B,
                                                      double *__restrict__ out) {
    __shared__ double red[256];
    const int tid = threadIdx.x;
    double s = 0.0;
    for (int64_t r = tid; r < B; r += blockDim.x) {
        const double d = (double)y[r] - (double)t[idx ? (int64_t)idx[r] : r];
        s += d * d;
    }
    red[tid] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) *out = red[0] / (double)B;
}

constexpr int kFwdSmem = (kRows * 32 + 2 * kRows * kHid) * 4;
constexpr int kBwdSmem = (kRows * kHid + kRows) * 4;
inline int param_grid() { return 2 * num_sms(); }

}  // namespace

Surrogate::~Surrogate() {
    if (buf) cudaFree(buf);
}

int Surrogate::ensure() {
    if (buf) return 0;
    // master, m, v, grad (FP32), bf16 copy, bf16 W2^T, mean, std
    const size_t f32 = sizeof(float) * (size_t)kSurrogateParams;
    const size_t b16 = sizeof(__nv_bfloat16) * (size_t)kSurrogateParams;
    auto pad = [](size_t n) { return (n + 255) / 256 * 256; };
    const size_t bytes =
        4 * pad(f32) + pad(b16) + pad(sizeof(__nv_bfloat16) * kHid * kHid) + 2 * pad(sizeof(float) * kIn);
    LNE_CUDA_TRY(cudaMalloc(&buf, bytes));
    char *p = static_cast<char *>(buf);
    auto take = [&](size_t n) {
        char *q = p;
        p += pad(n);
        return q;
    };
    w = reinterpret_cast<float *>(take(f32));
    m = reinterpret_cast<float *>(take(f32));
    v = reinterpret_cast<float *>(take(f32));
    g = reinterpret_cast<float *>(take(f32));
    wb = reinterpret_cast<__nv_bfloat16 *>(take(b16));
    w2t = reinterpret_cast<__nv_bfloat16 *>(take(sizeof(__nv_bfloat16) * kHid * kHid));
    mean = reinterpret_cast<float *>(take(sizeof(float) * kIn));
    std = reinterpret_cast<float *>(take(sizeof(float) * kIn));
    return 0;
}

namespace {

int refresh_copies(Surrogate &S, cudaStream_t st) {
    LNE_TRACE("sur_cast", st);
    sur_cast_kernel<<<param_grid(), 256, 0, st>>>(S.w, S.wb, S.w2t);
    LNE_LAUNCH_CHECK();
    return 0;
}

int reset_optimizer(Surrogate &S, cudaStream_t st) {
    LNE_CUDA_TRY(cudaMemsetAsync(S.m, 0, sizeof(float) * kSurrogateParams, st));
    LNE_CUDA_TRY(cudaMemsetAsync(S.v, 0, sizeof(float) * kSurrogateParams, st));
    S.step = 0;
    return 0;
}

struct BatchBufs {
    float *y = nullptr, *xs = nullptr, *h1 = nullptr, *h2 = nullptr, *dy = nullptr, *dz1 = nullptr, *dz2 = nullptr;
};

int batch_bufs(Workspace &ws, int64_t B, BatchBufs *b) {
    LNE_TRY(ws.get("sur.y", (size_t)B, &b->y));
    LNE_TRY(ws.get("sur.xs", (size_t)B * kIn, &b->xs));
    LNE_TRY(ws.get("sur.h1", (size_t)B * kHid, &b->h1));
    LNE_TRY(ws.get("sur.h2", (size_t)B * kHid, &b->h2));
    LNE_TRY(ws.get("sur.dy", (size_t)B, &b->dy));
    LNE_TRY(ws.get("sur.dz1", (size_t)B * kHid, &b->dz1));
    LNE_TRY(ws.get("sur.dz2", (size_t)B * kHid, &b->dz2));
    return 0;
}

int set_smem_attributes() {
    LNE_TRY(allow_dynamic_smem(sur_forward_kernel));
    LNE_TRY(allow_dynamic_smem(sur_backward_rows_kernel));
    return 0;
}

int forward(Surrogate &S, const float *X, int64_t rows, const int32_t *idx, float *y, const BatchBufs *train,
            cudaStream_t st) {
    if (rows <= 0) return 0;
    LNE_TRACE("sur_forward", st);
    sur_forward_kernel<<<(unsigned)ceil_div(rows, kRows), 256, kFwdSmem, st>>>(
        X, rows, idx, S.mean, S.std, S.wb, y, train ? train->xs : nullptr, train ? train->h1 : nullptr,
        train ? train->h2 : nullptr);
    LNE_LAUNCH_CHECK();
    return 0;
}

// gradient of the batch's mean squared error into S.g
int backward(Surrogate &S, const float *t, const int32_t *idx, int64_t B, const BatchBufs &b, cudaStream_t st) {
    LNE_TRACE("sur_backward", st);
    sur_backward_rows_kernel<<<(unsigned)ceil_div(B, kRows), 256, kBwdSmem, st>>>(b.y, t, idx, B, b.h1, b.h2, S.wb,
                                                                                  S.w2t, b.dy, b.dz2, b.dz1);
    LNE_LAUNCH_CHECK();
    sur_weight_grad_kernel<<<kHid + kIn + 1, 256, 0, st>>>(b.xs, b.h1, b.h2, b.dy, b.dz1, b.dz2, B, S.g);
    LNE_LAUNCH_CHECK();
    return 0;
}

int adam(Surrogate &S, float lr, cudaStream_t st) {
    S.step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)S.step));
    const float c2 = (float)(1.0 - std::pow(b2, (double)S.step));
    LNE_TRACE("sur_adam", st);
    sur_adam_kernel<<<param_grid(), 256, 0, st>>>(S.w, S.m, S.v, S.g, lr, (float)b1, (float)b2, 1e-8f, c1, c2, S.wb,
                                                S.w2t);
    LNE_LAUNCH_CHECK();
    return 0;
}

}  // namespace

int surrogate_init(Surrogate &S, uint64_t seed, cudaStream_t st) {
    LNE_TRY(S.ensure());
    LNE_TRY(set_smem_attributes());
    {
        LNE_TRACE("sur_init", st);
        sur_init_kernel<<<param_grid(), 256, 0, st>>>(S.w, (uint32_t)seed, (uint32_t)(seed >> 32));
        LNE_LAUNCH_CHECK();
    }
    const std::vector<float> zero(kIn, 0.f), one(kIn, 1.f);
    LNE_CUDA_TRY(cudaMemcpyAsync(S.mean, zero.data(), sizeof(float) * kIn, cudaMemcpyHostToDevice, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(S.std, one.data(), sizeof(float) * kIn, cudaMemcpyHostToDevice, st));
    LNE_TRY(reset_optimizer(S, st));
    LNE_TRY(refresh_copies(S, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors above go out of scope
    S.ready = true;
    return 0;
}

int surrogate_fit_scaling(Surrogate &S, const float *X, int64_t rows, cudaStream_t st) {
    if (!S.ready) return fail(LNE_ERR_INVALID, "surrogate not initialised");
    LNE_TRACE("sur_scaling", st);
    sur_scaling_kernel<<<kIn, 256, 0, st>>>(X, rows, S.mean, S.std);
    LNE_LAUNCH_CHECK();
    return 0;
}

int surrogate_set(Surrogate &S, const float *w, const float *mean, const float *std, cudaStream_t st) {
    LNE_TRY(S.ensure());
    LNE_TRY(set_smem_attributes());
    LNE_CUDA_TRY(cudaMemcpyAsync(S.w, w, sizeof(float) * kSurrogateParams, cudaMemcpyDefault, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(S.mean, mean, sizeof(float) * kIn, cudaMemcpyDefault, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(S.std, std, sizeof(float) * kIn, cudaMemcpyDefault, st));
    LNE_TRY(reset_optimizer(S, st));
    LNE_TRY(refresh_copies(S, st));
    S.ready = true;
    return 0;
}

int surrogate_get(Surrogate &S, float *w, float *mean, float *std, cudaStream_t st) {
    if (!S.ready) return fail(LNE_ERR_INVALID, "surrogate not initialised");
    if (w) LNE_CUDA_TRY(cudaMemcpyAsync(w, S.w, sizeof(float) * kSurrogateParams, cudaMemcpyDefault, st));
    if (mean) LNE_CUDA_TRY(cudaMemcpyAsync(mean, S.mean, sizeof(float) * kIn, cudaMemcpyDefault, st));
    if (std) LNE_CUDA_TRY(cudaMemcpyAsync(std, S.std, sizeof(float) * kIn, cudaMemcpyDefault, st));
    return 0;
}

int surrogate_predict(Surrogate &S, const float *X, int64_t rows, float *yhat, cudaStream_t st) {
    if (!S.ready) return fail(LNE_ERR_INVALID, "surrogate not initialised");
    return forward(S, X, rows, nullptr, yhat, nullptr, st);
}

int surrogate_grad(Surrogate &S, Workspace &ws, const float *X, const float *t, int64_t rows, float *grad,
                   double *loss, cudaStream_t st) {
    if (!S.ready) return fail(LNE_ERR_INVALID, "surrogate not initialised");
    BatchBufs b;
    LNE_TRY(batch_bufs(ws, rows, &b));
    LNE_TRY(forward(S, X, rows, nullptr, b.y, &b, st));
    LNE_TRY(backward(S, t, nullptr, rows, b, st));
    if (grad) LNE_CUDA_TRY(cudaMemcpyAsync(grad, S.g, sizeof(float) * kSurrogateParams, cudaMemcpyDefault, st));
    if (loss) {
        double *d = nullptr;
        LNE_TRY(ws.get("sur.loss", 1, &d));
        sur_mse_kernel<<<1, 256, 0, st>>>(b.y, t, nullptr, rows, d);
        LNE_LAUNCH_CHECK();
        LNE_CUDA_TRY(cudaMemcpyAsync(loss, d, sizeof(double), cudaMemcpyDeviceToHost, st));
        LNE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return 0;
}

int surrogate_train(Surrogate &S, Workspace &ws, const float *X, const float *t, int64_t rows, int epochs, int batch,
                    float lr, uint64_t seed, double *final_loss, cudaStream_t st) {
    if (!S.ready) return fail(LNE_ERR_INVALID, "surrogate not initialised");
    BatchBufs b;
    LNE_TRY(batch_bufs(ws, std::min<int64_t>(batch, rows), &b));
    int32_t *idx = nullptr;
    LNE_TRY(ws.get("sur.idx", (size_t)rows, &idx));
    std::vector<int32_t> perm((size_t)rows);
    std::mt19937_64 rng(seed);
    for (int e = 0; e < epochs; ++e) {
        // Fisher-Yates shuffle of the row order
        for (int64_t i = 0; i < rows; ++i) perm[i] = (int32_t)i;
        for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[rng() % (uint64_t)(i + 1)]);
        LNE_CUDA_TRY(cudaMemcpyAsync(idx, perm.data(), sizeof(int32_t) * rows, cudaMemcpyHostToDevice, st));
        for (int64_t b0 = 0; b0 < rows; b0 += batch) {
            const int64_t B = std::min<int64_t>(batch, rows - b0);
            LNE_TRY(forward(S, X, B, idx + b0, b.y, &b, st));
            LNE_TRY(backward(S, t, idx + b0, B, b, st));
            LNE_TRY(adam(S, lr, st));
        }
        // the host permutation is rewritten next epoch: the copy must be done
        LNE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (final_loss) {
        float *yh = nullptr;
        double *d = nullptr;
        LNE_TRY(ws.get("sur.yall", (size_t)rows, &yh));
        LNE_TRY(ws.get("sur.loss", 1, &d));
        LNE_TRY(forward(S, X, rows, nullptr, yh, nullptr, st));
        sur_mse_kernel<<<1, 256, 0, st>>>(yh, t, nullptr, rows, d);
        LNE_LAUNCH_CHECK();
        LNE_CUDA_TRY(cudaMemcpyAsync(final_loss, d, sizeof(double), cudaMemcpyDeviceToHost, st));
        LNE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return 0;
}

}  // namespace lne
