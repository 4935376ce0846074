// Downstream objective (Sec. 6.1): one-vs-rest L2-regularised logistic
// regression on the embedding, then Micro/Macro-F1 with the top-k rule (each
// test node predicts its k highest-scoring labels, k = its number of labels).
//
// For each label l: minimise 1/2 |w|^2 + C sum_i log(1 + exp(-y_il w.x_i)),
// y in {-1, +1}, x with a constant-1 bias feature; `iters` Newton steps from
// w = 0, all labels at once:
//   margins   Z = X W                                  (right_multiply)
//   weights   r = C (sigma(yz) - 1) y, D = C sigma (1 - sigma)
//   gradient  G = W + X^T R                            (row blocks, FP32, summed in FP64)
//   Hessians  H_l = I + X^T diag(D_l) X                (row blocks, FP32, summed in FP64)
//   update    W_l -= H_l^-1 G_l                        (batched FP64 Cholesky, one CTA per label)
#include <algorithm>
#include <cmath>
#include <vector>

#include "runtime.h"

namespace lne {
namespace {

constexpr int kEvalRows = 128;   // rows per FP32 partial sum (and per CTA)

// Xa[i] = (X[idx[i]], 1), Ys[i][l] = +1 / -1. A row index outside [0, n) is
// not read: its row becomes zeros (label -1) and status bit 2 is set, which
// the host turns into LNE_ERR_INVALID.
__global__ void gather_rows_kernel(const float *__restrict__ X, int64_t n, int64_t ldx, int d,
                                   const uint8_t *__restrict__ lab, int L, const int32_t *__restrict__ idx, int64_t m,
                                   float *__restrict__ Xa, float *__restrict__ Ys, int *__restrict__ status) {
    const int da = d + 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * da; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / da;
        const int j = (int)(e - i * da);
        const int64_t r = idx[i];
        if (r < 0 || r >= n) {
            if (j == 0) atomicOr(status, 2);
            Xa[e] = 0.0f;
            continue;
        }
        Xa[e] = j < d ? X[r * ldx + j] : 1.0f;
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * L; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / L;
        const int l = (int)(e - i * L);
        const int64_t r = idx[i];
        Ys[e] = (r >= 0 && r < n && lab[r * L + l]) ? 1.0f : -1.0f;
    }
}

// In place: Z -> R = C (sigma(yz) - 1) y; D = C sigma(yz) (1 - sigma(yz)).
__global__ void logistic_weights_kernel(float *__restrict__ Z, const float *__restrict__ Ys, int64_t count, float C,
                                        float *__restrict__ D) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const float y = Ys[e];
        const float sg = 1.0f / (1.0f + expf(-y * Z[e]));
        Z[e] = C * (sg - 1.0f) * y;
        D[e] = C * sg * (1.0f - sg);
    }
}

// partial[b][a][l] = sum over rows of block b of Xa[i][a] R[i][l].
__global__ void grad_partial_kernel(const float *__restrict__ Xa, const float *__restrict__ R, int64_t m, int da, int L,
                                    double *__restrict__ partial) {
    const int64_t r0 = (int64_t)blockIdx.x * kEvalRows;
    const int64_t r1 = imin64(m, r0 + kEvalRows);
    double *out = partial + (int64_t)blockIdx.x * da * L;
    for (int e = threadIdx.x; e < da * L; e += blockDim.x) {
        const int a = e / L, l = e - a * L;
        float acc = 0.f;
        for (int64_t i = r0; i < r1; ++i) acc = fmaf(Xa[i * da + a], R[i * L + l], acc);
        out[e] = acc;
    }
}

// hpart[b][l][a][c] (a <= c) = sum over rows of block b of D[i][l] Xa[i][a] Xa[i][c];
// CTA (row block, label): the block's rows and their D-weighted copies staged in
// shared memory, one thread per entry (a, c) of the upper triangle.
__global__ void __launch_bounds__(256) hess_partial_kernel(const float *__restrict__ Xa, const float *__restrict__ D,
                                                           int64_t m, int da, int L, double *__restrict__ hpart) {
    extern __shared__ float xs[];   // kEvalRows x dp rows, then the weighted rows
    const int dp = (da + 7) & ~7;
    const int l = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * kEvalRows;
    const int rows = (int)imin64(kEvalRows, m - r0);
    float *wx = xs + kEvalRows * dp;
    for (int e = threadIdx.x; e < rows * da; e += blockDim.x) {
        const int r = e / da, a = e - r * da;
        const float x = Xa[(r0 + r) * da + a];
        xs[r * dp + a] = x;
        wx[r * dp + a] = x * D[(r0 + r) * L + l];
    }
    __syncthreads();
    double *out = hpart + ((int64_t)blockIdx.x * L + l) * dp * dp;
    for (int t = threadIdx.x; t < da * da; t += blockDim.x) {
        const int a = t / da, c = t - a * da;
        if (a > c) continue;
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc = fmaf(wx[r * dp + a], xs[r * dp + c], acc);
        out[a * dp + c] = acc;
    }
}

// G = W + sum_b partial[b];  H_l = I + sum_b hpart[b][l] (mirrored), fixed order.
__global__ void newton_reduce_kernel(const double *__restrict__ partial, const double *__restrict__ hpart, int nblk,
                                     int da, int L, const double *__restrict__ W, double *__restrict__ G,
                                     double *__restrict__ H) {
    const int dp = (da + 7) & ~7;
    const int64_t total_h = (int64_t)L * da * da;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total_h + da * L;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < total_h) {
            const int l = (int)(e / ((int64_t)da * da));
            const int rem = (int)(e - (int64_t)l * da * da);
            const int a = rem / da, c = rem - a * da;
            const int lo = min(a, c), hi = max(a, c);
            double s = a == c ? 1.0 : 0.0;
            for (int b = 0; b < nblk; ++b) s += hpart[((int64_t)b * L + l) * dp * dp + lo * dp + hi];
            H[e] = s;
        } else {
            const int64_t f = e - total_h;
            double s = W[f];
            for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * da * L + f];
            G[f] = s;
        }
    }
}

// Per label (one CTA each): Cholesky of H_l (FP64, shared memory), solve
// H_l delta = G[:, l], W[:, l] -= delta.
__global__ void __launch_bounds__(512) newton_solve_kernel(const double *__restrict__ H, const double *__restrict__ G,
                                                           int da, int L, double *__restrict__ W,
                                                           int *__restrict__ status) {
    extern __shared__ double A[];   // da x da, then the right-hand side
    double *rhs = A + da * da;
    const int l = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    __shared__ double s_inv;
    const double *Hl = H + (int64_t)l * da * da;
    for (int e = tid; e < da * da; e += blockDim.x) A[e] = Hl[e];
    for (int a = tid; a < da; a += blockDim.x) rhs[a] = G[a * L + l];
    __syncthreads();
    // upper Cholesky H = R^T R, R in the upper triangle of A
    for (int k = 0; k < da; ++k) {
        if (tid == 0) {
            const double akk = A[k * da + k];
            if (!(akk > 0.0)) {
                atomicOr(status, 1);
                A[k * da + k] = 1.0;
                s_inv = 1.0;
            } else {
                const double dk = sqrt(akk);
                A[k * da + k] = dk;
                s_inv = 1.0 / dk;
            }
        }
        __syncthreads();
        const double inv = s_inv;
        for (int j = k + 1 + tid; j < da; j += blockDim.x) A[k * da + j] *= inv;
        __syncthreads();
        for (int i = k + 1 + warp; i < da; i += nw) {
            const double aki = A[k * da + i];
            for (int j = i + lane; j < da; j += 32) A[i * da + j] = fma(-aki, A[k * da + j], A[i * da + j]);
        }
        __syncthreads();
    }
    // R^T y = rhs (forward), then R delta = y (backward), one thread
    if (tid == 0) {
        for (int i = 0; i < da; ++i) {
            double s = rhs[i];
            for (int k = 0; k < i; ++k) s -= A[k * da + i] * rhs[k];
            rhs[i] = s / A[i * da + i];
        }
        for (int i = da - 1; i >= 0; --i) {
            double s = rhs[i];
            for (int k = i + 1; k < da; ++k) s -= A[i * da + k] * rhs[k];
            rhs[i] = s / A[i * da + i];
        }
    }
    __syncthreads();
    for (int a = tid; a < da; a += blockDim.x) W[a * L + l] -= rhs[a];
}

// Top-k prediction and per-label TP / FP / FN counts.
__global__ void topk_f1_kernel(const float *__restrict__ S, const float *__restrict__ Ys, int64_t m, int L,
                               unsigned long long *__restrict__ counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const float *si = S + i * L;
        const float *yi = Ys + i * L;
        int k = 0;
        for (int l = 0; l < L; ++l) k += yi[l] > 0.f;
        for (int l = 0; l < L; ++l) {
            int rank = 0;
            for (int j = 0; j < L; ++j) rank += (si[j] > si[l]) || (si[j] == si[l] && j < l);
            const bool pred = rank < k, truth = yi[l] > 0.f;
            if (pred && truth) atomicAdd(&counts[3 * l + 0], 1ull);
            if (pred && !truth) atomicAdd(&counts[3 * l + 1], 1ull);
            if (!pred && truth) atomicAdd(&counts[3 * l + 2], 1ull);
        }
    }
}

int egrid(int64_t work) { return (int)std::min<int64_t>(ceil_div(std::max<int64_t>(work, 1), 256), num_sms() * 16); }

}  // namespace

int macro_f1(Workspace &ws, const float *X, int64_t n, int d, int64_t ldx, const uint8_t *labels, int L,
             const int32_t *train_idx, int64_t n_train, const int32_t *test_idx, int64_t n_test, double C, int iters,
             double *macro, double *micro, cudaStream_t st) {
    if (d < 1 || L < 1 || n_train < 1 || n_test < 1 || iters < 0 || !(C > 0.0))
        return fail(LNE_ERR_INVALID, "bad Macro-F1 arguments");
    const int da = d + 1;
    if (da > 160) return fail(LNE_ERR_UNSUPPORTED, "Macro-F1 supports d <= 159");
    const int dp = (da + 7) & ~7;
    const int64_t nblk = ceil_div(n_train, kEvalRows);
    float *Xa = nullptr, *Ys = nullptr, *Z = nullptr, *Dw = nullptr, *Xt = nullptr, *Yt = nullptr, *St = nullptr;
    double *W = nullptr, *G = nullptr, *H = nullptr, *gp = nullptr, *hp = nullptr;
    unsigned long long *cnt = nullptr;
    int *status = nullptr;
    LNE_TRY(ws.get("eval.Xa", (size_t)(n_train * da), &Xa));
    LNE_TRY(ws.get("eval.Ys", (size_t)(n_train * L), &Ys));
    LNE_TRY(ws.get("eval.Z", (size_t)(n_train * L), &Z));
    LNE_TRY(ws.get("eval.D", (size_t)(n_train * L), &Dw));
    LNE_TRY(ws.get("eval.Xt", (size_t)(n_test * da), &Xt));
    LNE_TRY(ws.get("eval.Yt", (size_t)(n_test * L), &Yt));
    LNE_TRY(ws.get("eval.St", (size_t)(n_test * L), &St));
    LNE_TRY(ws.get("eval.W", (size_t)da * L, &W));
    LNE_TRY(ws.get("eval.G", (size_t)da * L, &G));
    LNE_TRY(ws.get("eval.H", (size_t)L * da * da, &H));
    LNE_TRY(ws.get("eval.gp", (size_t)(nblk * da * L), &gp));
    LNE_TRY(ws.get("eval.hp", (size_t)(nblk * L * dp * dp), &hp));
    LNE_TRY(ws.get("eval.cnt", (size_t)3 * L, &cnt));
    LNE_TRY(ws.get("eval.status", 1, &status));
    LNE_CUDA_TRY(cudaMemsetAsync(W, 0, sizeof(double) * da * L, st));
    LNE_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 3 * L, st));
    LNE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    {
        LNE_TRACE("eval_gather", st);
        gather_rows_kernel<<<egrid(n_train * da), 256, 0, st>>>(X, n, ldx, d, labels, L, train_idx, n_train, Xa, Ys,
                                                                status);
        LNE_LAUNCH_CHECK();
        gather_rows_kernel<<<egrid(n_test * da), 256, 0, st>>>(X, n, ldx, d, labels, L, test_idx, n_test, Xt, Yt,
                                                               status);
        LNE_LAUNCH_CHECK();
    }
    const int hsmem = 2 * kEvalRows * dp * 4;
    if (hsmem > 48 * 1024) LNE_TRY(allow_dynamic_smem(hess_partial_kernel));
    const int ssmem = (da * da + da) * 8;
    LNE_TRY(allow_dynamic_smem(newton_solve_kernel));
    for (int it = 0; it < iters; ++it) {
        LNE_TRY(right_multiply(Xa, n_train, da, da, W, L, L, nullptr, Z, L, st));
        {
            LNE_TRACE("logreg_newton", st);
            logistic_weights_kernel<<<egrid(n_train * L), 256, 0, st>>>(Z, Ys, n_train * L, (float)C, Dw);
            LNE_LAUNCH_CHECK();
            grad_partial_kernel<<<(unsigned)nblk, 256, 0, st>>>(Xa, Z, n_train, da, L, gp);
            LNE_LAUNCH_CHECK();
            hess_partial_kernel<<<dim3((unsigned)nblk, (unsigned)L), 256, hsmem, st>>>(Xa, Dw, n_train, da, L, hp);
            LNE_LAUNCH_CHECK();
            newton_reduce_kernel<<<egrid((int64_t)L * da * da + da * L), 256, 0, st>>>(gp, hp, (int)nblk, da, L, W,
                                                                                        G, H);
            LNE_LAUNCH_CHECK();
            newton_solve_kernel<<<L, 512, ssmem, st>>>(H, G, da, L, W, status);
            LNE_LAUNCH_CHECK();
        }
    }
    LNE_TRY(right_multiply(Xt, n_test, da, da, W, L, L, nullptr, St, L, st));
    {
        LNE_TRACE("topk_f1", st);
        topk_f1_kernel<<<egrid(n_test), 256, 0, st>>>(St, Yt, n_test, L, cnt);
        LNE_LAUNCH_CHECK();
    }
    std::vector<unsigned long long> h(3 * L);
    int hs = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(h.data(), cnt, sizeof(unsigned long long) * 3 * L, cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & 2) return fail(LNE_ERR_INVALID, "a train or test row index is outside [0, n)");
    if (hs) return fail(LNE_ERR_NUMERIC, "a logistic-regression Hessian was not positive definite");
    double f1sum = 0.0, tp = 0, fp = 0, fn = 0;
    for (int l = 0; l < L; ++l) {
        const double a = (double)h[3 * l], b = (double)h[3 * l + 1], c = (double)h[3 * l + 2];
        const double den = 2 * a + b + c;
        f1sum += den > 0 ? 2 * a / den : 0.0;
        tp += a;
        fp += b;
        fn += c;
    }
    *macro = f1sum / L;
    *micro = (2 * tp + fp + fn) > 0 ? 2 * tp / (2 * tp + fp + fn) : 0.0;
    return 0;
}

}  // namespace lne
