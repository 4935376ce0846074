/*
 * lne.h -- C ABI of the GB300 (sm_103a) LightNE 2.0 hot path.
 *
 * The method (Qiu et al., "Towards Lightweight and Automated Representation
 * Learning System for Networks", LightNE 2.0):
 *   1. sparsifier construction: per-edge PathSampling (Algorithms 1 and 3,
 *      Sec. 5.2) aggregated into exact pair counts, scaled and passed through
 *      the truncated logarithm of Eq. 1;
 *   2. fast randomized SVD of that sparse matrix (Algorithm 4) giving the
 *      initial embedding X0 = U Sigma^{1/2} (Sec. 4.2);
 *   3. spectral propagation of X0 by a Chebyshev filter in the normalised
 *      Laplacian I - D^-1 A, followed by an economic SVD (Sec. 4.3, Sec. 6.3).
 *
 * Conventions shared by every entry point:
 *   - Every pointer named *_dev is CUDA device memory on the context's device;
 *     every other pointer is host memory. The caller owns what it passes in.
 *     Buffers handed back through lne_counts / lne_csr are owned by the context
 *     and stay valid until the next call on the same context or lne_destroy.
 *   - Dense matrices are row-major float32 with the stated leading dimension.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) unless they return a host scalar, which implies a synchronise.
 *     A context may be used by one host thread at a time.
 *   - Every call returns LNE_OK (0) or a negative LNE_ERR_* code; the message of
 *     the last failure is returned by lne_last_error. A failed call leaves the
 *     context usable.
 *   - Graphs are undirected and unweighted: symmetric CSR, no self-loops, no
 *     duplicate edges, rows sorted. Every call that takes an lne_graph checks
 *     its structure on the device first (one pass over indptr and indices):
 *     indptr starts at 0, ends at nnz and never decreases, and every index
 *     lies in [0, n); otherwise it returns LNE_ERR_INVALID before any kernel
 *     walks the graph. Symmetry, self-loops, duplicates and row order are not
 *     checked: a graph that breaks them gives undefined results.
 *   - A CSR matrix handed to lne_spmm / lne_rsvd (lne_csr) is not checked (the
 *     calls stay asynchronous): its indptr must be non-decreasing from 0 to
 *     nnz and its indices must lie in [0, n).
 */
#ifndef LNE_H
#define LNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LNE_OK               0
#define LNE_ERR_INVALID     -1   /* bad argument or size */
#define LNE_ERR_OOM         -2   /* device allocation failed */
#define LNE_ERR_CUDA        -3   /* CUDA runtime error (message says which) */
#define LNE_ERR_TIMEOUT     -4   /* a bounded device wait ran out */
#define LNE_ERR_UNSUPPORTED -5   /* valid input outside what this build handles */
#define LNE_ERR_NUMERIC     -6   /* Cholesky breakdown or non-finite values */

/* Precision of the dense operand of the sparse products (the products of
 * Algorithm 4, the propagation products). Accumulation is FP32 in both; the Gram,
 * Cholesky and small SVD are FP64 in both. With LNE_PREC_BF16_MIXED the sketch,
 * the power-iteration bases and the propagation operands are gathered as
 * bfloat16 copies (the recurrences themselves stay FP32); d and d + oversample
 * must be multiples of 4. */
#define LNE_PREC_FP32        0
#define LNE_PREC_BF16_MIXED  1

/* Test matrix Omega of the randomized SVD (Algorithm 4). */
#define LNE_SKETCH_GAUSSIAN     0   /* randn(n, c), the paper's default */
#define LNE_SKETCH_SPARSE_SIGN  1   /* zeta nonzeros +-1 per row (Sec. 4.2's sparse sign alternative) */
#define LNE_SKETCH_VERY_SPARSE  2   /* entries +-1 with probability 1/(2s) each (Sec. 4.2's very
                                       sparse random projection); s = sketch_zeta, 0 = sqrt(n) */

typedef struct {
    int64_t n;                 /* vertices */
    int64_t nnz;               /* arcs = 2m = indptr[n] */
    const int64_t *indptr;     /* device, [n+1] */
    const int32_t *indices;    /* device, [nnz] */
    const uint32_t *weights;   /* device, [nnz] positive integer arc weights A_uv (equal on both arcs of
                                  an edge; weighted degrees below 2^31), or NULL for an unweighted
                                  graph. Weighted: arc a draws S A_a / vol samples in expectation
                                  (rate fl(fl(S A_a) / vol)), a walk step takes arc j of x for words
                                  below floor(2^32 (A_0 + .. + A_j) / d_x) (inverse CDF), and Eq. 1,
                                  edge downsampling (p_e = min(1, A_uv (C (1/d_u + 1/d_v)))) and the
                                  propagation (D^-1 A) use the weighted degrees and volume. */
} lne_graph;

/* Parameters in the paper's notation (notation table of Sec. 3). */
typedef struct {
    int32_t T;                 /* window size, 1..16 */
    const double *s;           /* host, [T] window weights s_1..s_T (>= 0, sum > 0; normalised) */
    double samples;            /* S: total expected edge samples; S/(2m) per arc (Algorithm 3) */
    double b;                  /* negative samples b of Eq. 1 (1 if <= 0) */
    int32_t d;                 /* embedding dimension */
    int32_t oversample;        /* oversampling s of Algorithm 4 (16 if < 0) */
    int32_t q;                 /* power iterations of Algorithm 4, >= 0 */
    int32_t k;                 /* Chebyshev terms of the propagation; 0 = no propagation */
    double theta;              /* filter width theta */
    double mu;                 /* filter centre mu */
    uint64_t seed;             /* Philox key for sampling and the sketch */
    int32_t precision;         /* LNE_PREC_* */
    double downsample_C;       /* edge downsampling (Sec. 4.1): 0 = off; C > 0 keeps a draw of arc
                                  u -> v with probability p_e = min(1, C (1/d_u + 1/d_v)) and
                                  weighs it 1/p_e; finite, >= 0 */
    int32_t sketch;            /* LNE_SKETCH_* */
    int32_t sketch_zeta;       /* LNE_SKETCH_SPARSE_SIGN: nonzeros per row, 1..min(12, c),
                                  0 = min(8, c); LNE_SKETCH_VERY_SPARSE: the sparsity s >= 1,
                                  0 = sqrt(n) */
} lne_params;

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t *indptr;           /* device [n+1] */
    int32_t *indices;          /* device [nnz], sorted within each row */
    float *data;               /* device [nnz] */
} lne_csr;

typedef struct {
    int64_t nnz;               /* distinct sampled unordered pairs */
    int32_t *x;                /* device [nnz], x <= y, sorted by (x, y) */
    int32_t *y;                /* device [nnz] */
    uint32_t *count;           /* device [nnz], exact multiplicities; NULL with edge downsampling */
    int64_t total_samples;     /* sum of all per-arc sample counts (dropped draws included) */
    uint64_t *weight;          /* device [nnz], with edge downsampling: sum of 1/p_e over the pair's
                                  kept draws in units of 2^-32, each 1/p_e rounded to
                                  floor(2^32/p_e + 1/2) (exact integer sums); else NULL */
    uint8_t *window;           /* device [nnz], with LNE_OPT_STRATIFIED: the window length r of
                                  each (x, y, r) entry (sorted by x, y, r); else NULL */
} lne_counts;

typedef struct lne_ctx lne_ctx;

/* Options of a context (lne_set_option). */
#define LNE_OPT_AGGREGATION  1   /* how sampled pairs are counted: */
#define LNE_AGG_AUTO         0   /*   dense table when n <= 65536 and it is the cheaper, else sort */
#define LNE_AGG_TABLE        1   /*   dense n x n count table, atomic increments (n <= 65536) */
#define LNE_AGG_BUCKET       2   /*   keys bucketed by row block, shared-memory counting (n <= 65536) */
#define LNE_AGG_SORT         3   /*   64-bit keys, radix sort and run lengths (any n < 2^31) */
#define LNE_OPT_SPMM_THREADS 2   /* CTA size of the batched-tuning SpMM: 0 = picked by timing
                                    (default), or 64 / 128 / 256; results do not depend on it */
#define LNE_OPT_SPMM_COLBLOCK 6  /* column-block width of the batched-tuning SpMM: 0 = picked by
                                    timing together with the CTA size (default), -1 = all columns
                                    in one pass, or a multiple of 4 up to 1024; results do not
                                    depend on it */
#define LNE_OPT_DENSE_PRODUCT 4  /* products of the randomized SVD (FP32) on the dense count table
                                    instead of the CSR, when the table aggregation ran: 0 = when at
                                    least a fraction 8 / (d + oversample) of all pairs is present
                                    (default), 1 = never,
                                    2 = always. The dense product runs on the tcgen05 tensor cores
                                    (TF32 hi / lo split, three MMAs per product: FP32 accuracy);
                                    same values as the CSR product, summed in another order */
#define LNE_OPT_TUNE_WORKERS 3   /* host worker threads (each with its own stream and workspace)
                                    of lne_tune_tasks, 1..16 (default 4) */
#define LNE_OPT_STRATIFIED   5   /* 1: window-stratified sampling (not in the paper): draws take
                                    r ~ U{1..T} and pair counts C_r are kept per r; a parameter
                                    set's matrix uses K = sum_r w_r C_r 2^-24 with
                                    w_r = floor(T (s_r / sum(s)) 2^24 + 1/2), an unbiased
                                    estimate of its count, so lne_tune_batch / lne_tune_tasks
                                    sample once per (T, S, seed) for all window weightings.
                                    lne_sparsifier_counts then returns (x, y, r, count) entries.
                                    Any n with 2 ceil(log2 n) + 4 <= 64; no edge downsampling.
                                    0 (default): the paper's sampler */
#define LNE_OPT_SPMM_VBLOCK  7   /* column blocking of the CSR products with the sparsifier
                                    (lne_rsvd, lne_embed, lne_spmm): the columns are taken in
                                    vertex blocks [b 2^s, (b + 1) 2^s), one block's partial
                                    product added to Y at a time in block order, so the dense
                                    operand rows one block gathers are a bounded region.
                                    0 (default): when the operand (n x c) does not fit in L2,
                                    with blocks of at most 2.5 times L2 (the measured best on
                                    a 10M-vertex graph: 10% off its products); -1: never;
                                    s in 1..30: blocks of 2^s
                                    vertices. Needs columns sorted within rows (a matrix with
                                    unsorted rows is multiplied unblocked). The sum order per
                                    entry differs from the unblocked product (block by block):
                                    both are within the FP32 bound */

/* Create a context on CUDA device `device`. The context owns its workspace. */
int lne_create(lne_ctx **out, int device);
void lne_destroy(lne_ctx *ctx);
const char *lne_last_error(const lne_ctx *ctx);
/* Bytes of device workspace the context currently holds. */
int64_t lne_workspace_bytes(const lne_ctx *ctx);
/* Release all workspace (the next call re-allocates). */
int lne_trim(lne_ctx *ctx);
/* Set a context option (LNE_OPT_*); the three aggregation methods give
 * identical (exact) counts, they differ in memory use and speed. An unknown
 * option or a value outside its range fails with LNE_ERR_INVALID. */
int lne_set_option(lne_ctx *ctx, int option, int64_t value);

/*
 * Raw PathSampling draws of arcs [arc_begin, arc_end) (Algorithm 1 driven per
 * arc as in Algorithm 3), in (arc, sample) order: u1_dev[i] is the end of the
 * walk from the arc's source, v1_dev[i] the end of the walk from its target.
 * `capacity` is the length of the two output arrays; *count_out receives the
 * number of draws (synchronises). Fails with LNE_ERR_INVALID if capacity is too
 * small (nothing is written then). With edge downsampling a draw whose coin
 * drops it keeps its slot and reads (-1, -1).
 */
int lne_sample_pairs(lne_ctx *ctx, const lne_graph *g, const lne_params *p,
                     int64_t arc_begin, int64_t arc_end, int32_t *u1_dev, int32_t *v1_dev,
                     int64_t capacity, int64_t *count_out, void *stream);

/*
 * Exact multiplicity of every sampled unordered pair (x <= y) over all arcs --
 * the aggregation step of Sec. 5.2 ("sparse parallel hashing"). Output buffers
 * are context-owned. Synchronises. With edge downsampling the pairs are those
 * of the kept draws and `weight` replaces `count` (table or sort aggregation;
 * LNE_AGG_BUCKET fails with LNE_ERR_UNSUPPORTED).
 */
int lne_sparsifier_counts(lne_ctx *ctx, const lne_graph *g, const lne_params *p,
                          lne_counts *out, void *stream);

/*
 * The sparse NetMF estimate M (Eq. 1): entry v = K * alpha / (d_x d_y) with
 * alpha = vol^2 / (2 S b) off the diagonal and vol^2 / (S b) on it (K the
 * unordered count), kept iff v > 1 (decided exactly as fl(fl(K alpha) /
 * fl(d_x d_y)) > 1 in FP64), value log(v) in float32. Symmetric CSR, both
 * triangles, rows sorted; context-owned. Synchronises. With edge downsampling K
 * is the pair's summed weight times 2^-32 (converted to FP64 exactly up to one
 * rounding) in place of the count.
 */
int lne_sparsifier_csr(lne_ctx *ctx, const lne_graph *g, const lne_params *p,
                       lne_csr *out, void *stream);

/*
 * Gaussian sketch Omega = randn(n, c) (Algorithm 4), Box-Muller from
 * Philox4x32-10 words: row i, column block j/4 uses counter (i, j/4, 0, 0) and
 * key (seed_lo ^ 0x4f4d4547, seed_hi). out_dev is [n][ld], ld >= c.
 */
int lne_gaussian_sketch(lne_ctx *ctx, int64_t n, int32_t c, uint64_t seed, float *out_dev,
                        int64_t ld, void *stream);

/*
 * Sparse sign test matrix (the cheaper alternative to the Gaussian Omega that
 * Sec. 4.2 names; construction of Tropp et al., SISC 2019): row i of out_dev
 * ([n][ld], ld >= c, float) has exactly zeta entries +-1 at distinct columns,
 * zeros elsewhere. Columns by Floyd's subset sampling: with words w_0.. of
 * Philox4x32-10 counters (i, b, 0, 0x53505253), b = 0, 1, .., key
 * (seed_lo ^ 0x4f4d4547, seed_hi), step k = 0..zeta-1 takes j = c - zeta + k,
 * t = w_k mod (j + 1) and adds t unless already chosen, else j; the k-th
 * chosen column is -1 iff bit k of w_zeta is set. 1 <= zeta <= min(12, c),
 * c <= 255; LNE_ERR_INVALID otherwise.
 */
int lne_sparse_sign_sketch(lne_ctx *ctx, int64_t n, int32_t c, int32_t zeta, uint64_t seed, float *out_dev,
                           int64_t ld, void *stream);

/*
 * Y_dev = M Omega for the sparse sign Omega of lne_sparse_sign_sketch (never
 * formed): each entry is the exact sum of its terms (M's values rounded to
 * multiples of 2^-32, summed in 64-bit fixed point) rounded once to float.
 * Needs |row sums of M| < 2^31. Y_dev is [n][ldy], ldy >= c, row-major.
 */
int lne_sparse_sign_spmm(lne_ctx *ctx, const lne_csr *M, int32_t c, int32_t zeta, uint64_t seed, float *Y_dev,
                         int64_t ldy, void *stream);

/*
 * Very sparse random projection (Sec. 4.2 names it beside the sparse sign
 * matrix as a cheaper Omega for Algorithm 4; construction of Li, Hastie and
 * Church, KDD 2006, at scale 1): out_dev ([n][ld], ld >= c, float) gets entry
 * (i, j) = +1 if word j mod 4 of Philox4x32-10 counter (i, j / 4, 0,
 * 0x56535250) under key (seed_lo ^ 0x4f4d4547, seed_hi) is below
 * thr = floor(2^32 / (2 s)), -1 if it is in [thr, 2 thr), else 0. s >= 1
 * (s <= 0 means sqrt(n), the "very sparse" choice); c <= 255. A row with more
 * than 12 nonzeros is refused with LNE_ERR_UNSUPPORTED (raise s);
 * LNE_ERR_INVALID for other bad arguments. Synchronises the stream.
 */
int lne_very_sparse_sketch(lne_ctx *ctx, int64_t n, int32_t c, double s, uint64_t seed, float *out_dev, int64_t ld,
                           void *stream);

/*
 * Y_dev = M Omega for the very sparse Omega of lne_very_sparse_sketch (never
 * formed), exact in 64-bit fixed point as lne_sparse_sign_spmm, then rounded
 * once to float. Y_dev is [n][ldy], ldy >= c, row-major. Synchronises the
 * stream (the row-count check).
 */
int lne_very_sparse_spmm(lne_ctx *ctx, const lne_csr *M, int32_t c, double s, uint64_t seed, float *Y_dev,
                         int64_t ldy, void *stream);

/* Y = M X for CSR M (n x n) and X [n][ldx] (c columns), Y [n][ldy] FP32,
 * accumulated in FP32 (Algorithm 4). X_dev is float
 * (precision LNE_PREC_FP32) or bfloat16 (LNE_PREC_BF16_MIXED; c and ldx must then
 * be multiples of 4). */
int lne_spmm(lne_ctx *ctx, const lne_csr *M, const void *X_dev, int64_t ldx, int32_t c,
             float *Y_dev, int64_t ldy, int32_t precision, void *stream);

/*
 * CholeskyQR2 of Y [n][ld] (c columns, c <= 256) in place: Y := Q with Q^T Q = I,
 * and R_dev (optional, [c][c] FP64 row-major, upper triangular) such that
 * Y_in = Q R. Gram and Cholesky in FP64. Returns LNE_ERR_NUMERIC when the
 * Gram is not numerically positive definite.
 */
int lne_cholqr2(lne_ctx *ctx, float *Y_dev, int64_t n, int32_t c, int64_t ld, double *R_dev,
                void *stream);

/*
 * SVD of a c x c FP64 matrix R (c <= 160; in the method R is the triangular
 * factor of the last sketch, so that Y = Q R gives Y's SVD as Q U_R) -- the
 * eig step of eigSVD (Algorithm 2). U_dev [c][c] row-major FP64 (column j = j-th
 * left singular vector), sigma_dev [c] FP64 descending. FP64-accurate: FP32
 * one-sided Jacobi start, then Ogita-Aishima refinement of the SVD of R in FP64,
 * then an exact FP64 two-sided Jacobi on the pairs of close singular values
 * the refinement leaves coupled.
 */
int lne_svd_small(lne_ctx *ctx, const double *R_dev, int32_t c, double *U_dev, double *sigma_dev,
                  void *stream);

/*
 * lne_svd_small without any device allocation. The paper has no counterpart:
 * this entry point serves callers that must not allocate device memory when
 * they call in (for example a process whose device memory is handed wholly to
 * another allocator up front, or a service that forbids allocation after
 * start-up). It needs no context: same arguments and results as lne_svd_small,
 * c <= 160 (larger c returns LNE_ERR_INVALID and does nothing).
 * Scratch: a fixed ~4.5 MB array in device memory that every GPU which loads the
 * library holds until the process exits; its device address is looked up on
 * the first call on each device, so make that first call before any stream
 * capture. All calls on a device share the array: calls that overlap on the GPU
 * (different streams, or different host threads) race and give wrong results.
 * Returns LNE_OK or a negative LNE_ERR_* code (no message is kept).
 */
int lne_svd_small_noalloc(const double *R_dev, int32_t c, double *U_dev, double *sigma_dev, void *stream);

/*
 * Fast randomized SVD (Algorithm 4) of the symmetric CSR M with the Gaussian
 * sketch of lne_gaussian_sketch(seed = p->seed): U_dev [n][d] (left singular
 * vectors, largest-magnitude entry of each column positive), sigma_dev [d]
 * (FP64, descending), X0_dev [n][d] = U Sigma^{1/2}. Any output may be NULL.
 */
int lne_rsvd(lne_ctx *ctx, const lne_csr *M, const lne_params *p, float *U_dev,
             double *sigma_dev, float *X0_dev, void *stream);

/*
 * Spectral propagation (Sec. 4.3): with Lap = I - D^-1 A and
 * Yop = (Lap - mu I)^2 / 2 - I, F = sum_{i<k} c_i T_i(Yop) X0 where
 * c_0 = I_0(theta), c_i = 2 (-1)^i I_i(theta); P = D^-1 A (X0 - F); X = U_P
 * Sigma_P^{1/2} from the SVD of P (Sec. 6.3). X0_dev and X_dev are [n][d]. With
 * k = 0, X = X0. F_dev / P_dev, when not NULL, receive F and P ([n][d]).
 */
int lne_propagate(lne_ctx *ctx, const lne_graph *g, const lne_params *p, const float *X0_dev,
                  float *X_dev, float *F_dev, float *P_dev, void *stream);

/*
 * Downstream objective of the embedding (Sec. 6.1): one-vs-rest L2-regularised
 * logistic regression (the LIBLINEAR model: for each label minimise
 * 1/2 |w|^2 + C sum log(1 + exp(-y w.x)), x with a constant-1 bias feature),
 * trained by `iters` Newton steps from w = 0 on the rows train_dev[0..n_train),
 * then each row of test_dev predicts its k highest-scoring labels (k = its
 * number of true labels). X_dev [n][ldx] float (d columns used, d <= 159);
 * labels_dev [n][L] uint8 0/1; train/test row indices int32 on the device.
 * *macro_f1 = mean over labels of 2TP / (2TP + FP + FN) (0 for a label with no
 * positives or predictions), *micro_f1 = the same on pooled counts. A train
 * or test index outside [0, n) is not read: the call returns LNE_ERR_INVALID.
 * Host outputs: synchronises.
 */
int lne_macro_f1(lne_ctx *ctx, const float *X_dev, int64_t n, int32_t d, int64_t ldx, const uint8_t *labels_dev,
                 int32_t L, const int32_t *train_dev, int64_t n_train, const int32_t *test_dev, int64_t n_test,
                 double C, int32_t iters, double *macro_f1, double *micro_f1, void *stream);

/* The whole method: sparsifier -> randomized SVD -> propagation. X_dev [n][d]. */
int lne_embed(lne_ctx *ctx, const lne_graph *g, const lne_params *p, float *X_dev, void *stream);

/*
 * Batched hyper-parameter tuning (Sec. 4.4: the method's parameters are tuned
 * per data set by scoring many configurations on the downstream task). Each of
 * the ncand host candidates cands[j] is a full parameter set; the result for
 * candidate j equals lne_embed(cands[j]) followed by lne_macro_f1 on the given
 * split (macro_f1[j] / micro_f1[j], host arrays of ncand). Candidates that
 * agree on T, s, S, b, d, oversample, q and seed share one sparsifier and one
 * randomized SVD; the propagation of all candidates with k >= 1 runs as column
 * blocks of one product (up to 1024 / d candidates per block), captured in a
 * CUDA graph on the second call of a given shape and replayed afterwards.
 * Requirements: every candidate has the same d (a multiple of 4, <= 160) and
 * precision LNE_PREC_FP32 (else LNE_ERR_UNSUPPORTED / LNE_ERR_INVALID). X_dev,
 * when not NULL, receives the embeddings, [ncand][n][d]. The evaluation
 * arguments are those of lne_macro_f1 (with ldx = d). Host outputs:
 * synchronises. Not to be called while `stream` is being captured.
 */
int lne_tune_batch(lne_ctx *ctx, const lne_graph *g, const lne_params *cands, int32_t ncand,
                   const uint8_t *labels_dev, int32_t L, const int32_t *train_dev, int64_t n_train,
                   const int32_t *test_dev, int64_t n_test, double C, int32_t iters, double *macro_f1,
                   double *micro_f1, float *X_dev, void *stream);

/*
 * Many independent tuning tasks (Sec. 4.4 tuning, repeated over data sets):
 * task t is a graph with its labels and split (the evaluation arguments of
 * lne_macro_f1); its ncand candidates are cands[t * ncand .. t * ncand + ncand)
 * and its scores land in macro_f1 / micro_f1[t * ncand + j] (host). Each task is
 * lne_tune_batch on that graph, with results identical to it. Host worker
 * threads (LNE_OPT_TUNE_WORKERS), each with its own stream and workspace, take
 * tasks in turn so the kernels of different graphs overlap. The call first
 * synchronises `stream` (inputs written there are complete), and returns when
 * every score is on the host. The first failing task's error is returned.
 */
typedef struct {
    lne_graph graph;
    const uint8_t *labels_dev;   /* [n][L] 0/1 */
    int32_t L;
    const int32_t *train_dev;    /* [n_train] row indices */
    int64_t n_train;
    const int32_t *test_dev;     /* [n_test] row indices */
    int64_t n_test;
} lne_task;

int lne_tune_tasks(lne_ctx *ctx, const lne_task *tasks, int32_t ntasks, const lne_params *cands, int32_t ncand,
                   double C, int32_t iters, double *macro_f1, double *micro_f1, void *stream);

/*
 * Surrogate of the tuning search. The paper tunes its hyper-parameters per data
 * set with an AutoML search over full runs (Sec. 4.4); this regression network
 * predicts a candidate's downstream score from 30 features (s_1..s_10, k,
 * theta, mu, q and 16 graph statistics) so that the search runs only the
 * candidates it ranks highest. One network per context:
 * 30 standardised inputs -> 256 ReLU -> 256 ReLU -> 1; loss = mean squared
 * error; Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected). FP32 master
 * weights; products use their bfloat16 roundings with FP32 accumulation.
 * Parameters, flat FP32 (73,985): W1 [30][256], b1 [256], W2 [256][256],
 * b2 [256], w3 [256], b3 [1] (W[i][j] = weight from input i to unit j).
 * Features are row-major [rows][30] FP32 on the device; targets [rows].
 *
 * lne_surrogate_init: He-uniform weights from Philox(seed), zero biases,
 *   mean 0 / std 1 scaling, Adam state cleared.
 * lne_surrogate_fit_scaling: per-feature mean and population std of the rows
 *   (std < 1e-6 -> 1), used by every later call.
 * lne_surrogate_set_params / get_params: copy the weights and the scaling in
 *   or out (host or device pointers; synchronises); set clears Adam state.
 * lne_surrogate_train: `epochs` passes over the rows in a fresh seeded order
 *   per pass, mini-batches of `batch` rows (the last one shorter), one Adam
 *   step per batch; *final_loss (host, may be NULL) = MSE over all rows after
 *   training (synchronises).
 * lne_surrogate_predict: yhat_dev [rows] = network output.
 * lne_surrogate_grad: gradient of the MSE over all `rows` at the current
 *   weights into grad_dev [73,985] (may be NULL), *loss (host, may be NULL).
 */
int lne_surrogate_init(lne_ctx *ctx, uint64_t seed, void *stream);
int lne_surrogate_fit_scaling(lne_ctx *ctx, const float *X_dev, int64_t rows, void *stream);
int lne_surrogate_set_params(lne_ctx *ctx, const float *theta, const float *mean, const float *std, void *stream);
int lne_surrogate_get_params(lne_ctx *ctx, float *theta, float *mean, float *std, void *stream);
int lne_surrogate_train(lne_ctx *ctx, const float *X_dev, const float *y_dev, int64_t rows, int32_t epochs,
                        int32_t batch, float lr, uint64_t seed, double *final_loss, void *stream);
int lne_surrogate_predict(lne_ctx *ctx, const float *X_dev, int64_t rows, float *yhat_dev, void *stream);
int lne_surrogate_grad(lne_ctx *ctx, const float *X_dev, const float *y_dev, int64_t rows, float *grad_dev,
                       double *loss, void *stream);

/*
 * Instrumentation (no counterpart in the paper, which reports wall-clock time
 * per stage only, Table "time distribution" of Sec. 6.3).
 *
 * lne_kernel_launches: kernels launched by this library in this process so far.
 * lne_trace_enable: start (on != 0) or stop recording named regions; clears
 *   earlier records. While on, each region (one kernel or one stage) records a
 *   CUDA event pair on the stream its kernels are launched on.
 * lne_trace_read: waits for the recorded events and returns one entry per
 *   region name, in order of first appearance (regions = times the region ran,
 *   launches = kernels launched inside it, total_ms = summed event time); at
 *   most `capacity` entries are written and *count receives how many exist.
 *   Clears the records.
 */
typedef struct {
    char name[40];
    int64_t regions;
    int64_t launches;
    double total_ms;
} lne_trace_entry;

int64_t lne_kernel_launches(void);
int lne_trace_enable(lne_ctx *ctx, int on);
int lne_trace_read(lne_ctx *ctx, lne_trace_entry *out, int capacity, int *count);

#ifdef __cplusplus
}
#endif

#endif /* LNE_H */
