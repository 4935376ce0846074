// Composition of the stages: fast randomized SVD (Algorithm 4) and spectral
// propagation (Sec. 4.3 / Sec. 5.4).
#include <cmath>
#include <utility>

#include "runtime.h"

namespace lne {
namespace {

__global__ void scale_copy_kernel(const float *__restrict__ X, float a, float *__restrict__ Y, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        Y[i] = a * X[i];
}

__global__ void sub_kernel(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C,
                           int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        C[i] = A[i] - B[i];
}

int elem_grid(int64_t count) {
    return (int)std::min<int64_t>(ceil_div(std::max<int64_t>(count, 1), 256), num_sms() * 16);
}

// I_nu(x) from its power series sum_m (x/2)^(2m+nu) / (m! (m+nu)!).
double bessel_i(int nu, double x) {
    const double h = 0.5 * x;
    double term = 1.0;
    for (int j = 1; j <= nu; ++j) term *= h / (double)j;
    double sum = term;
    for (int m = 1; m < 1000 && term != 0.0; ++m) {
        term *= h * h / ((double)m * (double)(m + nu));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

// SVD of the tall matrix Yq [n][c] (overwritten by its Q factor): left
// singular vectors of the leading dout columns into U [n][dout], sigma [dout].
int tall_svd(Workspace &ws, float *Yq, int64_t n, int c, int dout, float *U, double *sigma,
             cudaStream_t st) {
    double *R = nullptr, *UR = nullptr, *sig = nullptr;
    LNE_TRY(ws.get("tsvd.R", (size_t)c * c, &R));
    LNE_TRY(ws.get("tsvd.UR", (size_t)c * c, &UR));
    LNE_TRY(ws.get("tsvd.sig", (size_t)c, &sig));
    LNE_TRY(cholqr2(ws, Yq, n, c, c, R, st));
    LNE_TRY(small_svd(ws, R, c, UR, sig, st));
    LNE_TRY(right_multiply(Yq, n, c, c, UR, c, dout, nullptr, U, dout, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(sigma, sig, sizeof(double) * dout, cudaMemcpyDeviceToDevice, st));
    return 0;
}

}  // namespace

std::vector<double> chebyshev_coefficients(int k, double theta) {
    std::vector<double> c(std::max(k, 0));
    for (int i = 0; i < k; ++i) {
        double v = bessel_i(i, theta);
        c[i] = i == 0 ? v : 2.0 * ((i & 1) ? -v : v);
    }
    return c;
}

int rsvd(Workspace &ws, const CsrView &M, int d, int oversample, int q, uint64_t seed, int precision, float *U,
         double *sigma, float *X0, cudaStream_t st, const SketchSpec &sketch) {
    const int64_t n = M.n;
    const int c = d + oversample;
    if (d < 1 || oversample < 0) return fail(LNE_ERR_INVALID, "need d >= 1 and oversample >= 0");
    if (c > n) return fail(LNE_ERR_INVALID, "d + oversample must not exceed the number of vertices");
    if (c > 160) return fail(LNE_ERR_UNSUPPORTED, "d + oversample > 160 is not supported by the small SVD");
    if (q < 0) return fail(LNE_ERR_INVALID, "q must be >= 0");
    float *Om = nullptr, *Ya = nullptr, *Yb = nullptr, *Ub = nullptr;
    double *sg = nullptr;
    LNE_TRY(ws.get("rsvd.ya", (size_t)n * c, &Ya));
    LNE_TRY(ws.get("rsvd.yb", (size_t)n * c, &Yb));
    if (!U) LNE_TRY(ws.get("rsvd.u", (size_t)n * d, &Ub));
    if (!sigma) LNE_TRY(ws.get("rsvd.sigma", (size_t)d, &sg));
    float *Uo = U ? U : Ub;
    double *so = sigma ? sigma : sg;
    const bool bf16 = precision == LNE_PREC_BF16_MIXED;
    __nv_bfloat16 *Xh = nullptr;   // BF16 dense operand of the products
    if (bf16) LNE_TRY(ws.get("rsvd.xh", (size_t)n * c, &Xh));
    // FP32 products: the dense table on the tensor cores when the caller
    // supplied it (its TF32 hi / lo parts prepared once for all products)
    const float *a_hi = nullptr, *a_lo = nullptr;
    const bool dense_tc = M.dense && !bf16 && (sketch.kind == LNE_SKETCH_GAUSSIAN || q > 0);
    if (dense_tc) LNE_TRY(dense_tc_prepare(ws, M.dense, M.dense_ld, &a_hi, &a_lo, st));
    // CSR products whose operand does not fit in L2 go by vertex blocks of
    // the columns (built once for the q + 1 products)
    CsrView Mb = M;
    VBlocks vbs;
    if (!dense_tc) {
        const int shift = vblock_shift_for(M.vblock, n, c, bf16 ? 2 : 4);
        bool ok = false;
        if (shift > 0) LNE_TRY(vblocks_build(ws, M, shift, &vbs, &ok, st));
        if (ok) Mb.vb = &vbs;
    }
    auto mprod = [&](const float *X, float *Y) -> int {
        if (dense_tc) return dense_tc_spmm(ws, a_hi, a_lo, M.dense_ld, n, X, c, c, Y, c, st);
        return spmm(ws, Mb, X, c, c, Y, c, st);
    };
    // Algorithm 4: Omega = randn(n, d+s); Y = M Omega. The sparse sign Omega
    // (Sec. 4.2's cheaper alternative) is applied without being formed; its
    // product is exact up to one rounding, in either precision mode.
    if (sketch.kind == LNE_SKETCH_SPARSE_SIGN) {
        const int zeta = sketch.zeta > 0 ? sketch.zeta : std::min(8, c);
        LNE_TRY(sparse_sign_spmm(ws, M, c, zeta, seed, Ya, c, st));
    } else if (sketch.kind == LNE_SKETCH_VERY_SPARSE) {
        LNE_TRY(very_sparse_spmm(ws, M, c, sketch.sparsity, seed, Ya, c, st));
    } else {
        LNE_TRY(ws.get("rsvd.omega", (size_t)n * c, &Om));
        LNE_TRY(gaussian_sketch(n, c, seed, Om, c, st));
        if (bf16) {
            LNE_TRY(to_bf16(Om, Xh, n * c, st));
            LNE_TRY(spmm_bf16(ws, Mb, Xh, c, c, Ya, c, nullptr, st));
        } else {
            LNE_TRY(mprod(Om, Ya));
        }
    }
    // power iterations: Q = orth(Y); Y = M Q (q times). Q only has to span
    // range(Y) well conditioned (the paper's eigSVD Q is FP32 as well): one
    // CholeskyQR pass; the final factorisation below takes two.
    for (int it = 0; it < q; ++it) {
        LNE_TRY(cholqr1(ws, Ya, n, c, c, Yb, c, st));
        if (bf16) {
            LNE_TRY(to_bf16(Yb, Xh, n * c, st));
            LNE_TRY(spmm_bf16(ws, Mb, Xh, c, c, Ya, c, nullptr, st));
        } else {
            LNE_TRY(mprod(Yb, Ya));
        }
    }
    // final eigSVD of Y: U = Q(:, 1:d), Sigma(1:d)
    LNE_TRY(tall_svd(ws, Ya, n, c, d, Uo, so, st));
    LNE_TRY(sign_fix_embed(ws, Uo, n, d, d, so, X0, d, st));
    return status_check(ws, st);
}

int propagate(Workspace &ws, const GraphView &g, int d, int k, double theta, double mu, int precision,
              const float *X0, float *X, float *F, float *P, cudaStream_t st) {
    const int64_t n = g.n;
    const int64_t cnt = n * d;
    if (k <= 0) {
        LNE_CUDA_TRY(cudaMemcpyAsync(X, X0, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st));
        return 0;
    }
    if (d > n) return fail(LNE_ERR_INVALID, "d must not exceed the number of vertices");
    if (d > 160) return fail(LNE_ERR_UNSUPPORTED, "d > 160 is not supported by the small SVD");
    const std::vector<double> cf = chebyshev_coefficients(k, theta);
    float *Fb = F, *Pb = P, *Z = nullptr, *Gb = nullptr, *Ta = nullptr, *Tb = nullptr, *Tc = nullptr,
          *Qb = nullptr, *Ub = nullptr;
    double *sig = nullptr;
    if (!Fb) LNE_TRY(ws.get("prop.F", (size_t)cnt, &Fb));
    if (!Pb) LNE_TRY(ws.get("prop.P", (size_t)cnt, &Pb));
    LNE_TRY(ws.get("prop.Z", (size_t)cnt, &Z));
    LNE_TRY(ws.get("prop.G", (size_t)cnt, &Gb));
    LNE_TRY(ws.get("prop.Ta", (size_t)cnt, &Ta));
    LNE_TRY(ws.get("prop.Tb", (size_t)cnt, &Tb));
    LNE_TRY(ws.get("prop.Tc", (size_t)cnt, &Tc));
    LNE_TRY(ws.get("prop.Q", (size_t)cnt, &Qb));
    LNE_TRY(ws.get("prop.U", (size_t)cnt, &Ub));
    LNE_TRY(ws.get("prop.sig", (size_t)d, &sig));
    const float om = (float)(1.0 - mu);
    // BF16 mode: every gathered operand also lives as a BF16 copy (written by the
    // producing epilogue); the recurrence itself stays FP32.
    const bool bf16 = precision == LNE_PREC_BF16_MIXED;
    __nv_bfloat16 *X0h = nullptr, *Zh = nullptr, *Gh = nullptr, *Th[3] = {nullptr, nullptr, nullptr};
    if (bf16) {
        LNE_TRY(ws.get("prop.X0h", (size_t)cnt, &X0h));
        LNE_TRY(ws.get("prop.Zh", (size_t)cnt, &Zh));
        LNE_TRY(ws.get("prop.Gh", (size_t)cnt, &Gh));
        LNE_TRY(ws.get("prop.Tah", (size_t)cnt, &Th[0]));
        LNE_TRY(ws.get("prop.Tbh", (size_t)cnt, &Th[1]));
        LNE_TRY(ws.get("prop.Tch", (size_t)cnt, &Th[2]));
        LNE_TRY(to_bf16(X0, X0h, cnt, st));
    }
    auto half_of = [&](const float *t) -> __nv_bfloat16 * {
        if (t == X0) return X0h;
        if (t == Z) return Zh;
        if (t == Gb) return Gh;
        if (t == Ta) return Th[0];
        if (t == Tb) return Th[1];
        if (t == Tc) return Th[2];
        return nullptr;
    };
    // Y = op(A) X with X given in FP32; BF16 mode gathers X's BF16 copy and
    // keeps a BF16 copy of the output too
    auto gspmm = [&](const float *Xin, float *Yout, SpmmEpilogue ep) -> int {
        if (!bf16) return graph_spmm(ws, g, Xin, d, d, Yout, d, ep, st);
        ep.Yb = half_of(Yout);
        if (ep.G) ep.Gb = Gh;
        return graph_spmm_bf16(ws, g, half_of(Xin), d, d, Yout, d, ep, st);
    };
    // F = c_0 X0
    {
        LNE_TRACE("scale_copy", st);
        scale_copy_kernel<<<elem_grid(cnt), 256, 0, st>>>(X0, (float)cf[0], Fb, cnt);
        LNE_LAUNCH_CHECK();
    }
    if (k == 1) {
        {
            LNE_TRACE("sub", st);
            sub_kernel<<<elem_grid(cnt), 256, 0, st>>>(X0, Fb, Gb, cnt);
            LNE_LAUNCH_CHECK();
        }
        if (bf16) LNE_TRY(to_bf16(Gb, Gh, cnt, st));
    } else {
        // Z = (Lap - mu I) X0 = (1 - mu) X0 - D^-1 A X0
        SpmmEpilogue e1;
        e1.alpha = -1.f;
        e1.dinv = true;
        e1.E1 = X0;
        e1.b1 = om;
        e1.lde = d;
        LNE_TRY(gspmm(X0, Z, e1));
        // T_1 = Yop X0 = (Lap - mu I) Z / 2 - X0; F += c_1 T_1
        SpmmEpilogue e2;
        e2.alpha = -0.5f;
        e2.dinv = true;
        e2.E1 = Z;
        e2.b1 = 0.5f * om;
        e2.E2 = X0;
        e2.b2 = -1.f;
        e2.lde = d;
        e2.F = Fb;
        e2.gamma = (float)cf[1];
        if (k == 2) {
            e2.X0 = X0;
            e2.G = Gb;
        }
        LNE_TRY(gspmm(Z, Ta, e2));
        // T_{i-2}, T_{i-1} rotate through three buffers; X0 is never written
        float *const bufs[3] = {Ta, Tb, Tc};
        const float *prev = X0;
        float *cur = Ta;
        for (int i = 2; i < k; ++i) {
            float *nxt = nullptr;
            for (float *b : bufs)
                if (b != prev && b != cur) {
                    nxt = b;
                    break;
                }
            // Z = (Lap - mu I) T_{i-1}
            SpmmEpilogue ez;
            ez.alpha = -1.f;
            ez.dinv = true;
            ez.E1 = cur;
            ez.b1 = om;
            ez.lde = d;
            LNE_TRY(gspmm(cur, Z, ez));
            // T_i = 2 Yop T_{i-1} - T_{i-2} = (Lap - mu I) Z - 2 T_{i-1} - T_{i-2}
            SpmmEpilogue e;
            e.alpha = -1.f;
            e.dinv = true;
            e.E1 = Z;
            e.b1 = om;
            e.E2 = cur;
            e.b2 = -2.f;
            e.E3 = prev;
            e.b3 = -1.f;
            e.lde = d;
            e.F = Fb;
            e.gamma = (float)cf[i];
            if (i == k - 1) {
                e.X0 = X0;
                e.G = Gb;
            }
            LNE_TRY(gspmm(Z, nxt, e));
            prev = cur;
            cur = nxt;
        }
    }
    // P = D^-1 A (X0 - F)
    SpmmEpilogue ep;
    ep.alpha = 1.f;
    ep.dinv = true;
    ep.lde = d;
    LNE_TRY(gspmm(Gb, Pb, ep));
    // X = U_P Sigma_P^{1/2} from the SVD of P (economic SVD of the last stage)
    LNE_CUDA_TRY(cudaMemcpyAsync(Qb, Pb, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st));
    LNE_TRY(tall_svd(ws, Qb, n, d, d, Ub, sig, st));
    LNE_TRY(sign_fix_embed(ws, Ub, n, d, d, sig, X, d, st));
    return status_check(ws, st);
}

}  // namespace lne

// ---------------------------------------------------------------------------
// Batched propagation: ncand candidates (k_j, theta_j, mu_j) on the same graph
// run as column blocks of one wide product -- Lap is shared, so each column
// evolves independently and every column gets exactly the arithmetic of a
// single-candidate run. Per-column coefficients live in device memory, so the
// chain can be captured once in a CUDA graph and replayed for new candidates.
// ---------------------------------------------------------------------------
namespace lne {
namespace {

__global__ void scale_cols_kernel(const float *__restrict__ X, const float *__restrict__ s, int64_t n, int C,
                                  float *__restrict__ Y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * C; e += (int64_t)gridDim.x * blockDim.x)
        Y[e] = s[e % C] * X[e];
}

}  // namespace

struct PropBatchGraph {
    bool valid = false;
    int seen = 0;
    int64_t kernels = 0;
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;   // the chain is captured here (the caller's stream may be the legacy one)
    ~PropBatchGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture) cudaStreamDestroy(capture);
    }
};

static int prop_batch_chain(Workspace &ws, const GraphView &g, int C, int kmax, const float *X0, float *F, float *Z,
                            float *Tbuf[3], float *G, float *P, const float *om, const float *hom, const float *gam,
                            SpmmTile tile, cudaStream_t st) {
    const int64_t cnt = g.n * C;
    {
        LNE_TRACE("scale_cols", st);
        scale_cols_kernel<<<elem_grid(cnt), 256, 0, st>>>(X0, gam, g.n, C, F);
        LNE_LAUNCH_CHECK();
    }
    if (kmax >= 2) {
        SpmmEpilogue e1;
        e1.alpha = -1.f;
        e1.dinv = true;
        e1.E1 = X0;
        e1.b1_col = om;
        e1.lde = C;
        e1.threads = tile.threads;
        e1.col_block = tile.col_block;
        e1.carry_tag = "pb.carry";
        LNE_TRY(graph_spmm(ws, g, X0, C, C, Z, C, e1, st));
        SpmmEpilogue e2;
        e2.alpha = -0.5f;
        e2.dinv = true;
        e2.E1 = Z;
        e2.b1_col = hom;
        e2.E2 = X0;
        e2.b2 = -1.f;
        e2.lde = C;
        e2.F = F;
        e2.gamma_col = gam + C;
        e2.threads = tile.threads;
        e2.col_block = tile.col_block;
        e2.carry_tag = "pb.carry";
        LNE_TRY(graph_spmm(ws, g, Z, C, C, Tbuf[0], C, e2, st));
        const float *prev = X0;
        float *cur = Tbuf[0];
        for (int i = 2; i < kmax; ++i) {
            float *nxt = nullptr;
            for (int b = 0; b < 3; ++b)
                if (Tbuf[b] != prev && Tbuf[b] != cur) {
                    nxt = Tbuf[b];
                    break;
                }
            SpmmEpilogue ez;
            ez.alpha = -1.f;
            ez.dinv = true;
            ez.E1 = cur;
            ez.b1_col = om;
            ez.lde = C;
            ez.threads = tile.threads;
        ez.col_block = tile.col_block;
            ez.carry_tag = "pb.carry";
            LNE_TRY(graph_spmm(ws, g, cur, C, C, Z, C, ez, st));
            SpmmEpilogue e;
            e.alpha = -1.f;
            e.dinv = true;
            e.E1 = Z;
            e.b1_col = om;
            e.E2 = cur;
            e.b2 = -2.f;
            e.E3 = prev;
            e.b3 = -1.f;
            e.lde = C;
            e.F = F;
            e.gamma_col = gam + (int64_t)i * C;
            e.threads = tile.threads;
        e.col_block = tile.col_block;
            e.carry_tag = "pb.carry";
            LNE_TRY(graph_spmm(ws, g, Z, C, C, nxt, C, e, st));
            prev = cur;
            cur = nxt;
        }
    }
    {
        LNE_TRACE("sub", st);
        sub_kernel<<<elem_grid(cnt), 256, 0, st>>>(X0, F, G, cnt);
        LNE_LAUNCH_CHECK();
    }
    SpmmEpilogue ep;
    ep.alpha = 1.f;
    ep.dinv = true;
    ep.lde = C;
    ep.threads = tile.threads;
    ep.col_block = tile.col_block;
    ep.carry_tag = "pb.carry";
    return graph_spmm(ws, g, G, C, C, P, C, ep, st);
}

int propagate_batch(Workspace &ws, PropBatchGraph *cache, const GraphView &g, int d, int ncand, const int *k,
                    const double *theta, const double *mu, const float *X0, float *P, SpmmTile tile,
                    cudaStream_t st) {
    const int C = d * ncand;
    if (C % 4 != 0 || C > 1024) return fail(LNE_ERR_UNSUPPORTED, "batched propagation needs d * ncand <= 1024, % 4");
    int kmax = 1;
    for (int j = 0; j < ncand; ++j) {
        if (k[j] < 1) return fail(LNE_ERR_INVALID, "batched propagation needs k >= 1 for every candidate");
        kmax = std::max(kmax, k[j]);
    }
    // per-column coefficient tables: om = 1 - mu, hom = (1 - mu) / 2, gam[i] = c_i(theta) for i < k
    std::vector<float> h((size_t)(2 + kmax) * C, 0.f);
    for (int j = 0; j < ncand; ++j) {
        const std::vector<double> cf = chebyshev_coefficients(k[j], theta[j]);
        for (int t = 0; t < d; ++t) {
            const int col = j * d + t;
            h[col] = (float)(1.0 - mu[j]);
            h[C + col] = (float)(0.5 * (1.0 - mu[j]));
            for (int i = 0; i < k[j]; ++i) h[(size_t)(2 + i) * C + col] = (float)cf[i];
        }
    }
    float *coef = nullptr, *F = nullptr, *Z = nullptr, *G = nullptr, *Tb[3] = {nullptr, nullptr, nullptr};
    const int64_t cnt = g.n * C;
    LNE_TRY(ws.get("pb.coef", h.size(), &coef));
    LNE_TRY(ws.get("pb.F", (size_t)cnt, &F));
    LNE_TRY(ws.get("pb.Z", (size_t)cnt, &Z));
    LNE_TRY(ws.get("pb.G", (size_t)cnt, &G));
    LNE_TRY(ws.get("pb.Ta", (size_t)cnt, &Tb[0]));
    LNE_TRY(ws.get("pb.Tb", (size_t)cnt, &Tb[1]));
    LNE_TRY(ws.get("pb.Tc", (size_t)cnt, &Tb[2]));
    LNE_CUDA_TRY(cudaMemcpyAsync(coef, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st));
    float4 *carry = nullptr;
    int64_t *carry_row = nullptr;
    LNE_TRY(merge_carry(ws, "pb.carry", g.nnz, g.n, C, &carry, &carry_row));
    const float *om = coef, *hom = coef + C, *gam = coef + 2 * C;
    if (!cache) return prop_batch_chain(ws, g, C, kmax, X0, F, Z, Tb, G, P, om, hom, gam, tile, st);
    // graph key: everything the captured launches depend on
    std::vector<uintptr_t> key = {(uintptr_t)g.indptr, (uintptr_t)g.indices, (uintptr_t)g.n,  (uintptr_t)g.nnz,
                                  (uintptr_t)C,        (uintptr_t)kmax,      (uintptr_t)X0,   (uintptr_t)P,
                                  (uintptr_t)coef,     (uintptr_t)F,         (uintptr_t)Z,    (uintptr_t)G,
                                  (uintptr_t)Tb[0],    (uintptr_t)Tb[1],     (uintptr_t)Tb[2], (uintptr_t)tile.threads,
                                  (uintptr_t)tile.col_block,
                                  (uintptr_t)carry,    (uintptr_t)carry_row, (uintptr_t)g.wf, (uintptr_t)g.dinv};
    if (cache->valid && cache->key == key) {
        LNE_TRACE("propagate_batch_graph", st);
        LNE_CUDA_TRY(cudaGraphLaunch(cache->exec, st));
        add_launches(cache->kernels);
        return 0;
    }
    if (cache->key != key) {
        cache->key = key;
        cache->seen = 0;
        cache->valid = false;
    }
    if (cache->seen == 0) {   // first run: eager (allocates every buffer the chain needs)
        cache->seen = 1;
        return prop_batch_chain(ws, g, C, kmax, X0, F, Z, Tb, G, P, om, hom, gam, tile, st);
    }
    // second run with the same key: capture, instantiate, launch
    if (cache->exec) {
        cudaGraphExecDestroy(cache->exec);
        cache->exec = nullptr;
    }
    // launches counted while capturing are the kernels the graph runs (once
    // now, then once per replay)
    Tracer *const tracer = get_tracer();
    set_tracer(nullptr);
    cudaGraph_t graph = nullptr;
    if (!cache->capture) LNE_CUDA_TRY(cudaStreamCreateWithFlags(&cache->capture, cudaStreamNonBlocking));
    const int64_t before = launches_now();
    LNE_CUDA_TRY(cudaStreamBeginCapture(cache->capture, cudaStreamCaptureModeThreadLocal));
    int rc = prop_batch_chain(ws, g, C, kmax, X0, F, Z, Tb, G, P, om, hom, gam, tile, cache->capture);
    cudaError_t e = cudaStreamEndCapture(cache->capture, &graph);
    set_tracer(tracer);
    cache->kernels = launches_now() - before;
    if (rc != 0) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail("cudaStreamEndCapture", e, __FILE__, __LINE__);
    e = cudaGraphInstantiate(&cache->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail("cudaGraphInstantiate", e, __FILE__, __LINE__);
    cache->valid = true;
    LNE_TRACE("propagate_batch_graph", st);
    LNE_CUDA_TRY(cudaGraphLaunch(cache->exec, st));
    return 0;
}

void destroy_prop_cache(PropBatchGraph *c) { delete c; }
PropBatchGraph *new_prop_cache() { return new PropBatchGraph(); }

}  // namespace lne
