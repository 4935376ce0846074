// Internal host-side API of the library: device workspace and the stage
// functions that the C ABI (capi.cu) composes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"

namespace lne {

// Named, grow-only device buffers owned by a context. A buffer keeps its
// contents until it is re-requested with a larger size.
class Workspace {
public:
    ~Workspace() { release(); }
    // Returns 0 and sets *ptr, or LNE_ERR_OOM / LNE_ERR_CUDA.
    int get(const std::string &name, size_t bytes, void **ptr);
    template <typename T>
    int get(const std::string &name, size_t count, T **ptr) {
        return get(name, count * sizeof(T), reinterpret_cast<void **>(ptr));
    }
    void release();
    // Whether a buffer of that name exists.
    bool has(const std::string &name) const { return bufs_.count(name) != 0; }
    // Frees one named buffer (no-op if absent).
    void release(const std::string &name);
    int64_t bytes() const;

private:
    struct Buf {
        void *p = nullptr;
        size_t bytes = 0;
    };
    std::map<std::string, Buf> bufs_;
};

struct GraphView {
    int64_t n = 0;
    int64_t nnz = 0;
    const int64_t *indptr = nullptr;
    const int32_t *indices = nullptr;
    // weighted graphs (w = NULL: unweighted); the rest is derived from w by
    // prepare_weighted
    const uint32_t *w = nullptr;      // [nnz] positive integer arc weights, symmetric
    const uint32_t *wdeg = nullptr;   // [n] weighted degrees d_u (< 2^31)
    const float *wf = nullptr;        // [nnz] the weights as float (graph products)
    const float *dinv = nullptr;      // [n] 1 / d_u as float (graph products)
    double vol = 0.0;                 // sum of all arc weights
    uint32_t wmax = 0;                // largest arc weight
};
// Weighted degrees, volume and the float copies of a weighted graph into the
// workspace ("wg.*"); no-op for unweighted graphs. Synchronises.
int prepare_weighted(Workspace &ws, GraphView *g, cudaStream_t st);

// Column blocks of a CSR matrix (columns sorted within rows) by vertex ranges
// [b << shift, (b + 1) << shift): row i's nonzeros in block b are positions
// seg[b n + i] .. seg[(b + 1) n + i] of the row; V[b (n + 1) + i] is the
// exclusive prefix sum of those segment lengths over rows (V[b (n + 1) + n]
// = nnz[b]). Built by vblocks_build; products with a CSR view that carries it
// go block by block, so the operand rows a block gathers are a bounded region.
struct VBlocks {
    int shift = 0, nb = 0;
    const uint32_t *seg = nullptr;   // (nb + 1) x n
    const int64_t *V = nullptr;      // nb x (n + 1)
    std::vector<int64_t> nnz;        // per block
};

struct CsrView {
    int64_t n = 0;
    int64_t nnz = 0;
    const int64_t *indptr = nullptr;
    const int32_t *indices = nullptr;
    const float *data = nullptr;
    // the same matrix as a dense upper triangle (row-major, leading dimension
    // dense_ld), when the products should use it instead of the CSR
    const float *dense = nullptr;
    int64_t dense_ld = 0;
    // column blocking of the CSR products: 0 = when the operand does not fit
    // in L2, -1 = never, s > 0 = blocks of 2^s vertices; vb = the blocks in use
    int vblock = 0;
    const VBlocks *vb = nullptr;
};
// the block shift for a product with n x c operand rows of elem_bytes each
// (0 = no blocking) and the block structure of M (ok = false when M has
// unsorted rows or a single block)
int vblock_shift_for(int mode, int64_t n, int c, int elem_bytes);
int vblocks_build(Workspace &ws, const CsrView &M, int shift, VBlocks *vb, bool *ok, cudaStream_t st);

// Host-derived constants of the sampler (Algorithm 3 with the readings of the
// window draw, the per-arc Bernoulli and the Philox stream layout).
struct SamplerSpec {
    uint32_t k0 = 0, k1 = 0;      // Philox key = (seed_lo, seed_hi)
    uint32_t base = 0;            // floor(S / 2m)
    uint32_t thr_frac = 0;        // floor(frac(S / 2m) * 2^32)
    int T = 1;
    uint64_t thr[16] = {0};       // thr_1..thr_{T-1}
    int B = 1;                    // bits per endpoint in a pair key
    double alpha_off = 0, alpha_diag = 0;
    float off_hi = 0, off_lo = 0, diag_hi = 0, diag_lo = 0;   // alpha as float pairs
    int aggregation = 0;          // LNE_AGG_* (0 = automatic)
    double ds_C = 0.0;            // edge downsampling constant C (0 = off)
    // the arguments the spec was built from (window-stratified sampling
    // samples with uniform s and applies these weights afterwards)
    double s_raw[16] = {0};
    double S = 0.0, b = 1.0;
    uint64_t seed = 0;
    int stratified = 0;           // 1: M from window-stratified counts
    const uint32_t *wdeg = nullptr;   // weighted degrees for Eq. 1 (weighted graphs)
};

int make_sampler_spec(const GraphView &g, int T, const double *s, double S, double b, uint64_t seed,
                      SamplerSpec *out);

// ---- sparsifier (sampler.cu) ------------------------------------------------
int sample_pairs(Workspace &ws, const GraphView &g, const SamplerSpec &sp, int64_t a0, int64_t a1,
                 int32_t *u1, int32_t *v1, int64_t capacity, int64_t *count, cudaStream_t st);

struct CountsResult {
    int64_t nnz = 0;
    int64_t total_samples = 0;
    int32_t *x = nullptr;
    int32_t *y = nullptr;
    uint32_t *cnt = nullptr;      // multiplicities (no downsampling)
    uint64_t *weight = nullptr;   // summed 1/p_e in 2^-32 units (edge downsampling)
    uint8_t *window = nullptr;    // window length r of each entry (stratified counts)
};
int sparsifier_counts(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CountsResult *out,
                      cudaStream_t st);

struct CsrResult {
    int64_t n = 0, nnz = 0;
    int64_t *indptr = nullptr;
    int32_t *indices = nullptr;
    float *data = nullptr;
    const float *dense = nullptr;   // the count table after Eq. 1 (table aggregation only)
    int64_t dense_ld = 0;
};
// The view the randomized SVD's products use: the dense table when there is
// one and mode allows (0 = when at least a fraction 8 / c of all pairs is
// present, c the products' width; 1 = never; 2 = always), else the CSR.
CsrView product_view(const CsrResult &M, int dense_mode, int c);
int sparsifier_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CsrResult *out,
                   cudaStream_t st);

// ---- dense and sparse linear algebra (dense.cu, spmm.cu) -------------------
int gaussian_sketch(int64_t n, int c, uint64_t seed, float *out, int64_t ld, cudaStream_t st);
int spmm(Workspace &ws, const CsrView &M, const float *X, int64_t ldx, int c, float *Y, int64_t ldy,
         cudaStream_t st);
// Y := Q in place; R (optional, device FP64 [c][c]) receives the upper factor.
int cholqr2(Workspace &ws, float *Y, int64_t n, int c, int64_t ld, double *R, cudaStream_t st);
// One CholeskyQR pass: Q = Y chol(Y^T Y)^-1 (FP64 Gram and Cholesky, FP32 Q).
int cholqr1(Workspace &ws, const float *Y, int64_t n, int c, int64_t ld, float *Q, int64_t ldq, cudaStream_t st);
// SVD of an upper-triangular c x c FP64 R: U_R [c][c] FP64, sigma [c] descending.
int small_svd(Workspace &ws, const double *R, int c, double *U_R, double *sigma, cudaStream_t st);
// out[n][dout] = Y[n][c] * W[c][dout] (W FP64 row-major with leading dim ldw),
// optionally scaled per output column by colscale (FP64, length dout).
int right_multiply(const float *Y, int64_t n, int c, int64_t ldy, const double *W, int64_t ldw,
                   int dout, const double *colscale, float *out, int64_t ldo, cudaStream_t st);
// Flip columns of U [n][d] so that each column's largest-magnitude entry is
// positive; if X is not NULL also writes X = U diag(sqrt(sigma)).
int sign_fix_embed(Workspace &ws, float *U, int64_t n, int d, int64_t ld, const double *sigma,
                   float *X, int64_t ldx, cudaStream_t st);

// Epilogue of the graph products (see spmm.cu).
struct SpmmEpilogue {
    float alpha = 1.f;
    bool dinv = false;                  // multiply (A X)_i by 1 / deg(i)
    const float *dinv_w = nullptr;      // with dinv: per-row 1 / d_i (weighted graphs) instead
    const float *E1 = nullptr;
    float b1 = 0.f;
    const float *E2 = nullptr;
    float b2 = 0.f;
    const float *E3 = nullptr;
    float b3 = 0.f;
    int64_t lde = 0;                    // leading dimension of E*, F, X0, G
    float *F = nullptr;                 // F += gamma * out
    float gamma = 0.f;
    const float *X0 = nullptr;          // with G: G = X0 - F (after the update)
    float *G = nullptr;
    bool store = true;                  // write out to Y
    __nv_bfloat16 *Yb = nullptr;        // BF16 copy of out (leading dimension ldy)
    __nv_bfloat16 *Gb = nullptr;        // BF16 copy of G (leading dimension lde)
    // per-column coefficients (device, length c); when set they replace b1 / gamma
    const float *b1_col = nullptr;
    const float *gamma_col = nullptr;
    int threads = 0;                    // CTA size of the merge kernel (0 = default)
    int col_block = 0;                  // merge products of more columns run in blocks of this many (0 = one)
    const char *carry_tag = nullptr;    // workspace name of the merge carry buffers (NULL = shared)
};
// Device status words of the context (workspace "dev.status", zeroed when
// created): [0] the first Cholesky breakdown, [1] a tensor-core pipeline wait
// that expired, [2] a very sparse projection row with more than 12 nonzeros.
// Kernels only ever set them; status_check reads them once (one host
// synchronisation), clears them and returns LNE_ERR_TIMEOUT /
// LNE_ERR_UNSUPPORTED / LNE_ERR_NUMERIC if one was set.
int device_status(Workspace &ws, int **status, cudaStream_t st);
int status_check(Workspace &ws, cudaStream_t st);
// Partial products of ks k-slices (P[z][n][c]) added in slice order into Y.
int slice_sum(const float *P, int ks, int64_t n, int c, float *Y, int64_t ldy, cudaStream_t st);
// The tensor-core (tcgen05) dense product: dense_tc_prepare splits the
// upper-triangle table into the full symmetric matrix's TF32 hi / lo parts
// (workspace "tc.ahi" / "tc.alo"); dense_tc_spmm computes Y = M X from them.
int dense_tc_prepare(Workspace &ws, const float *T, int64_t ld, const float **hi, const float **lo,
                     cudaStream_t st);
int dense_tc_spmm(Workspace &ws, const float *Ahi, const float *Alo, int64_t ld, int64_t n, const float *X,
                  int64_t ldx, int c, float *Y, int64_t ldy, cudaStream_t st);
// Carry buffers of the merge SpMM for nnz nonzeros over n rows and c columns, under the
// workspace names tag + ".c" / tag + ".r" (tag NULL = "spmm.carry").
int merge_carry(Workspace &ws, const char *tag, int64_t nnz, int64_t n, int c, float4 **carry,
                int64_t **carry_row);
int graph_spmm(Workspace &ws, const GraphView &g, const float *X, int64_t ldx, int c, float *Y, int64_t ldy,
               const SpmmEpilogue &ep, cudaStream_t st);
// The same products with a BF16 dense operand (FP32 accumulation); c % 4 == 0.
int spmm_bf16(Workspace &ws, const CsrView &M, const __nv_bfloat16 *X, int64_t ldx, int c, float *Y, int64_t ldy,
              __nv_bfloat16 *Yb, cudaStream_t st);
int graph_spmm_bf16(Workspace &ws, const GraphView &g, const __nv_bfloat16 *X, int64_t ldx, int c, float *Y,
                    int64_t ldy, const SpmmEpilogue &ep, cudaStream_t st);
// out[i] = bf16(in[i]) for count elements.
int to_bf16(const float *in, __nv_bfloat16 *out, int64_t count, cudaStream_t st);

// Sparse sign test matrix (sketch.cu): zeta nonzeros +-1 per row, each row
// packed in 16 bytes (column bytes, then sign bits) in the workspace.
constexpr int kMaxSketchZeta = 12;
struct SketchSpec {
    int kind = LNE_SKETCH_GAUSSIAN;
    int zeta = 0;             // nonzeros per row of the sparse sign sketch; 0 = min(8, c)
    double sparsity = 0.0;    // s of the very sparse projection; 0 = sqrt(n)
};
// Very sparse projection (sketch.cu): entries +-1 with probability 1/(2s)
// each, packed like the sparse sign rows (at most 12 nonzeros a row; more
// sets device status word 2). s <= 0 means sqrt(n).
double very_sparse_s(int64_t n, double s);
int very_sparse_sketch(Workspace &ws, int64_t n, int c, double s, uint64_t seed, const uint4 **packed,
                       cudaStream_t st);
int very_sparse_dense(Workspace &ws, int64_t n, int c, double s, uint64_t seed, float *out, int64_t ld,
                      cudaStream_t st);
int very_sparse_spmm(Workspace &ws, const CsrView &M, int c, double s, uint64_t seed, float *Y, int64_t ldy,
                     cudaStream_t st);
int sparse_sign_sketch(Workspace &ws, int64_t n, int c, int zeta, uint64_t seed, const uint4 **packed,
                       cudaStream_t st);
// The sketch written out densely (out[n][ld], ld >= c).
int sparse_sign_dense(Workspace &ws, int64_t n, int c, int zeta, uint64_t seed, float *out, int64_t ld,
                      cudaStream_t st);
// Y = M Omega for the sparse sign Omega (exact 64-bit fixed-point sums).
int sparse_sign_spmm(Workspace &ws, const CsrView &M, int c, int zeta, uint64_t seed, float *Y, int64_t ldy,
                     cudaStream_t st);

// Randomized SVD (Algorithm 4) and propagation (Sec. 4.3).
int rsvd(Workspace &ws, const CsrView &M, int d, int oversample, int q, uint64_t seed, int precision,
         float *U, double *sigma, float *X0, cudaStream_t st, const SketchSpec &sketch = SketchSpec());
int propagate(Workspace &ws, const GraphView &g, int d, int k, double theta, double mu, int precision,
              const float *X0, float *X, float *F, float *P, cudaStream_t st);

// Batched propagation of ncand candidates as column blocks (pipeline.cu);
// with a cache the chain is captured in a CUDA graph and replayed.
struct PropBatchGraph;
PropBatchGraph *new_prop_cache();
void destroy_prop_cache(PropBatchGraph *c);
// Tile shape of the batched merge SpMM: CTA size (0 = 256) and column-block
// width (0 = all columns at once). Neither changes any column's arithmetic.
struct SpmmTile {
    int threads = 0;
    int col_block = 0;
};
int propagate_batch(Workspace &ws, PropBatchGraph *cache, const GraphView &g, int d, int ncand, const int *k,
                    const double *theta, const double *mu, const float *X0, float *P, SpmmTile tile,
                    cudaStream_t st);
std::vector<double> chebyshev_coefficients(int k, double theta);

// The batched merge SpMM's tile shape, picked by timing every candidate
// (CTA size 64 / 128 / 256 x column blocks of 128 / 256 / 512 / all columns)
// once per (row-length bucket, nnz bucket, width) and cached; `forced` fixes
// the CTA size. Results do not depend on the choice.
struct SpmmTune {
    int forced = 0;         // CTA size (0 = tuned)
    int forced_block = 0;   // column-block width (0 = tuned, -1 = all columns at once)
    std::map<uint64_t, SpmmTile> best;
};
// Returns 0 and sets *tile, or an error code.
int spmm_tile_for(SpmmTune &tc, Workspace &ws, const GraphView &g, const float *X, int C, float *Y, SpmmTile *tile,
                  cudaStream_t st);
// Batched tuning over ncand candidate parameter sets (tune.cu).
// stratified: the candidates' sparsifiers come from window-stratified counts,
// sampled once per (T, S, seed) and shared.
int tune_batch(Workspace &ws, PropBatchGraph *cache, SpmmTune &tc, int aggregation, int dense_mode, int stratified,
               const GraphView &g,
               const lne_params *cands, int ncand, const uint8_t *labels, int L, const int32_t *train,
               int64_t n_train, const int32_t *test, int64_t n_test, double Creg, int iters, double *macro,
               double *micro, float *X_out, cudaStream_t st);

// Independent tuning tasks run by host worker threads, each with its own
// workspace and stream (tune.cu).
struct TuneWorker {
    Workspace ws;
    SpmmTune tune;
    cudaStream_t st = nullptr;
    ~TuneWorker();
};
struct TuneTask {
    GraphView g;
    const uint8_t *labels = nullptr;
    int L = 0;
    const int32_t *train = nullptr;
    int64_t n_train = 0;
    const int32_t *test = nullptr;
    int64_t n_test = 0;
};
int tune_tasks(std::vector<std::unique_ptr<TuneWorker>> &workers, int nworkers, int device, int forced_threads,
               int forced_block,
               int aggregation, int dense_mode, int stratified, const TuneTask *tasks, int ntasks,
               const lne_params *cands, int ncand, double Creg, int iters, double *macro, double *micro);

// Surrogate regression network of the tuning search (surrogate.cu):
// 30 -> 256 ReLU -> 256 ReLU -> 1, FP32 master weights, bfloat16 copies.
constexpr int kSurrogateInputs = 30;
constexpr int kSurrogateHidden = 256;
constexpr int64_t kSurrogateParams = 30 * 256 + 256 + 256 * 256 + 256 + 256 + 1;
struct Surrogate {
    void *buf = nullptr;   // one allocation holding everything below
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *mean = nullptr, *std = nullptr;
    __nv_bfloat16 *wb = nullptr, *w2t = nullptr;
    int64_t step = 0;
    bool ready = false;
    ~Surrogate();
    int ensure();
};
int surrogate_init(Surrogate &S, uint64_t seed, cudaStream_t st);
int surrogate_fit_scaling(Surrogate &S, const float *X, int64_t rows, cudaStream_t st);
int surrogate_set(Surrogate &S, const float *w, const float *mean, const float *std, cudaStream_t st);
int surrogate_get(Surrogate &S, float *w, float *mean, float *std, cudaStream_t st);
int surrogate_predict(Surrogate &S, const float *X, int64_t rows, float *yhat, cudaStream_t st);
int surrogate_grad(Surrogate &S, Workspace &ws, const float *X, const float *t, int64_t rows, float *grad,
                   double *loss, cudaStream_t st);
int surrogate_train(Surrogate &S, Workspace &ws, const float *X, const float *t, int64_t rows, int epochs, int batch,
                    float lr, uint64_t seed, double *final_loss, cudaStream_t st);

// One-vs-rest logistic regression + Micro/Macro-F1 (eval.cu).
int macro_f1(Workspace &ws, const float *X, int64_t n, int d, int64_t ldx, const uint8_t *labels, int L,
             const int32_t *train_idx, int64_t n_train, const int32_t *test_idx, int64_t n_test, double C, int iters,
             double *macro, double *micro, cudaStream_t st);

// Exclusive scan helpers (scan.cu).
int scan_exclusive_u32_to_i64(const uint32_t *in, int64_t *out, int64_t n, cudaStream_t st);
int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st);
// In place, per row: data[r][0..n) -> exclusive prefix, data[r][n] = row total
// (rows of n + 1 entries).
int scan_exclusive_rows_i64(int64_t *data, int64_t rows, int64_t n, cudaStream_t st);

// Sorting of 64-bit keys (sort.cu). Stable LSD radix sort over the low `bits`
// bits with an optional 32-bit payload (vals may be NULL); the result lands in
// keys_alt / vals_alt when *in_alt is true, else in keys / vals.
int radix_sort_u64(Workspace &ws, uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                   int64_t n, int bits, bool *in_alt, cudaStream_t st);
// Unique keys of a sorted array and their multiplicities.
int run_length(Workspace &ws, const uint64_t *keys, int64_t n, uint64_t *ukeys, uint32_t *counts,
               int64_t *nunique, cudaStream_t st);
// Window-stratified counts (sampler.cu): draws take r ~ U{1..T}; per distinct
// pair its (r, count) entries. One sampling pass serves every weighting s: a
// candidate's matrix uses K_s = sum_r w_r C_r, w_r = floor(T s_r / sum(s)
// 2^24 + 1/2) (2^-24 units). Buffers live in the workspace ("strat.*").
struct Strata {
    int64_t total = 0;                 // draws
    int64_t U = 0;                     // distinct (pair, r)
    int64_t P = 0;                     // distinct pairs
    const uint64_t *pair = nullptr;    // [P] (x << B) | y, ascending
    const int64_t *seg = nullptr;      // [P + 1] entries of pair p: seg[p] .. seg[p + 1] - 1
    const uint8_t *r = nullptr;        // [U] window length of each entry
    const uint32_t *cnt = nullptr;     // [U] its count
    int T = 0, B = 0;
    double S = 0.0;
    uint64_t seed = 0;
    const int64_t *g_indptr = nullptr;   // the graph the strata belong to
    int64_t g_n = 0, g_nnz = 0;
};
// Samples the strata for sp's (T, S, seed) (the window weights of sp are
// ignored; the draw of r is uniform).
int stratified_sample(Workspace &ws, const GraphView &g, const SamplerSpec &sp, Strata *out, cudaStream_t st);
// The candidate sp's sparsifier (its s, b) from the strata.
int stratified_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, const Strata &S, CsrResult *out,
                   cudaStream_t st);
void stratified_release(Workspace &ws);

// Number of keys of a sorted array below `key` (synchronises).
int count_below(Workspace &ws, const uint64_t *keys, int64_t n, uint64_t key, int64_t *count, cudaStream_t st);
// Unique keys of a sorted array and, per run, the sum of w[arcs[i]] over it.
int run_length_weighted(Workspace &ws, const uint64_t *keys, const uint32_t *arcs, const uint64_t *w, int64_t n,
                        uint64_t *ukeys, uint64_t *wsum, int64_t *nunique, cudaStream_t st);

}  // namespace lne
