// Batched parameter tuning (Sec. 4.4: the hyper-parameters of the method --
// window weights, sample count, filter k / theta / mu -- are tuned by running
// many candidate configurations on one graph and keeping the best downstream
// Macro-F1).
//
// The GPU-side batching:
//   * candidates that agree on everything the sparsifier and the randomized SVD
//     read (T, s, S, b, d, oversample, q, seed) share one sparsifier and one
//     randomized SVD;
//   * the spectral propagation of every candidate with k >= 1 runs as one
//     column block of a single wide product [n][m d] -- the normalized
//     Laplacian is the same matrix for all of them, so each column evolves on
//     its own with exactly the arithmetic of a one-candidate run; the per-column
//     (1 - mu) and c_i(theta) live in a device table, and the chain of
//     products is captured once in a CUDA graph and replayed for the next
//     candidate set of the same shape;
//   * the merge SpMM's CTA size is picked by timing (results do not depend on
//     it: every warp owns the same nonzero slice whatever the CTA size).
// Each candidate then gets its own final SVD (Sec. 6.3: eigSVD as the economic SVD of P) and
// its own Macro-F1.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace lne {

namespace {

bool same_rsvd_inputs(const lne_params &a, const lne_params &b, int osa, int osb) {
    if (a.T != b.T || a.samples != b.samples || a.b != b.b || a.d != b.d || osa != osb || a.q != b.q ||
        a.seed != b.seed || a.downsample_C != b.downsample_C || a.sketch != b.sketch ||
        a.sketch_zeta != b.sketch_zeta)
        return false;
    for (int i = 0; i < a.T; ++i)
        if (a.s[i] != b.s[i]) return false;
    return true;
}

}  // namespace

int spmm_tile_for(SpmmTune &tc, Workspace &ws, const GraphView &g, const float *X, int C, float *Y, SpmmTile *tile,
                  cudaStream_t st) {
    const int64_t avg = g.n > 0 ? std::max<int64_t>(1, g.nnz / g.n) : 1;
    int dbucket = 0;
    while ((int64_t(1) << (dbucket + 1)) <= avg) ++dbucket;
    int nbucket = 0;
    while ((int64_t(1) << (nbucket + 1)) <= std::max<int64_t>(1, g.nnz)) ++nbucket;
    const uint64_t key = (uint64_t)dbucket | ((uint64_t)nbucket << 8) | ((uint64_t)C << 16) |
                         ((uint64_t)tc.forced << 32) | ((uint64_t)(tc.forced_block + 1) << 44);
    auto it = tc.best.find(key);
    if (it != tc.best.end()) {
        *tile = it->second;
        return 0;
    }
    // candidates: CTA sizes x column-block widths (0 = all columns at once)
    std::vector<int> ts, bs;
    if (tc.forced > 0) ts = {tc.forced};
    else ts = {64, 128, 256};
    if (tc.forced_block < 0) bs = {0};
    else if (tc.forced_block > 0) bs = {tc.forced_block < C ? tc.forced_block : 0};
    else {
        bs = {0};
        for (int b : {512, 256, 128})
            if (b < C) bs.push_back(b);
    }
    std::vector<SpmmTile> cands;
    for (int t : ts)
        for (int b : bs) cands.push_back(SpmmTile{t, b});
    cudaEvent_t e0, e1;
    LNE_CUDA_TRY(cudaEventCreate(&e0));
    LNE_CUDA_TRY(cudaEventCreate(&e1));
    SpmmTile best = cands.front();
    float best_ms = 1e30f;
    int rc = 0;
    for (const SpmmTile &cand : cands) {
        SpmmEpilogue ep;
        ep.alpha = 1.f;
        ep.dinv = true;
        ep.lde = C;
        ep.threads = cand.threads;
        ep.col_block = cand.col_block;
        if ((rc = graph_spmm(ws, g, X, C, C, Y, C, ep, st)) != 0) break;   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && rc == 0; ++r) rc = graph_spmm(ws, g, X, C, C, Y, C, ep, st);
        cudaEventRecord(e1, st);
        if (rc != 0) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail("cudaEventSynchronize", e, __FILE__, __LINE__);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != 0) return rc;
    tc.best[key] = best;
    *tile = best;
    return 0;
}

int tune_batch(Workspace &ws, PropBatchGraph *cache, SpmmTune &tc, int aggregation, int dense_mode, int stratified,
               const GraphView &g,
               const lne_params *cands, int ncand, const uint8_t *labels, int L, const int32_t *train,
               int64_t n_train, const int32_t *test, int64_t n_test, double Creg, int iters, double *macro,
               double *micro, float *X_out, cudaStream_t st) {
    if (ncand < 1) return fail(LNE_ERR_INVALID, "need at least one candidate");
    const int d = cands[0].d;
    const int64_t n = g.n;
    for (int j = 0; j < ncand; ++j) {
        const lne_params &p = cands[j];
        if (p.d != d) return fail(LNE_ERR_INVALID, "all candidates must share the embedding dimension d");
        if (p.precision != LNE_PREC_FP32) return fail(LNE_ERR_UNSUPPORTED, "batched tuning runs in FP32 only");
        if (p.k < 0 || p.q < 0) return fail(LNE_ERR_INVALID, "need q >= 0 and k >= 0");
    }
    if (d < 4 || d % 4 != 0) return fail(LNE_ERR_UNSUPPORTED, "batched tuning needs d to be a multiple of 4");
    if (d > 160) return fail(LNE_ERR_UNSUPPORTED, "d > 160 is not supported by the small SVD");
    if (d > n) return fail(LNE_ERR_INVALID, "d must not exceed the number of vertices");
    auto os_of = [](const lne_params &p) { return p.oversample < 0 ? 16 : p.oversample; };
    // groups of candidates sharing the sparsifier and the randomized SVD
    std::vector<int> group(ncand), leader;
    for (int j = 0; j < ncand; ++j) {
        int gid = -1;
        for (int q = 0; q < (int)leader.size() && gid < 0; ++q)
            if (same_rsvd_inputs(cands[leader[q]], cands[j], os_of(cands[leader[q]]), os_of(cands[j]))) gid = q;
        if (gid < 0) {
            gid = (int)leader.size();
            leader.push_back(j);
        }
        group[j] = gid;
    }
    float *X0s = nullptr;
    LNE_TRY(ws.get("tune.x0", (size_t)leader.size() * n * d, &X0s));
    Strata strata;   // shared by the candidates with the same (T, S, seed)
    bool have_strata = false;
    for (int q = 0; q < (int)leader.size(); ++q) {
        const lne_params &p = cands[leader[q]];
        SamplerSpec sp;
        LNE_TRY(make_sampler_spec(g, p.T, p.s, p.samples, p.b, p.seed, &sp));
        sp.aggregation = aggregation;
        sp.ds_C = p.downsample_C;
        CsrResult M;
        if (stratified) {
            if (!have_strata || strata.T != sp.T || strata.S != sp.S || strata.seed != sp.seed) {
                LNE_TRY(stratified_sample(ws, g, sp, &strata, st));
                have_strata = true;
            }
            LNE_TRY(stratified_csr(ws, g, sp, strata, &M, st));
        } else {
            LNE_TRY(sparsifier_csr(ws, g, sp, &M, st));
        }
        SketchSpec sk;
        sk.kind = p.sketch;
        sk.zeta = p.sketch_zeta;
        LNE_TRY(rsvd(ws, product_view(M, dense_mode, d + os_of(p)), d, os_of(p), p.q, p.seed, p.precision, nullptr, nullptr,
                     X0s + (size_t)q * n * d, st, sk));
    }
    if (have_strata) stratified_release(ws);
    float *X = nullptr, *U = nullptr;
    double *R = nullptr, *UR = nullptr, *sig = nullptr;
    LNE_TRY(ws.get("tune.x", (size_t)n * d, &X));
    LNE_TRY(ws.get("tune.u", (size_t)n * d, &U));
    LNE_TRY(ws.get("tune.r", (size_t)d * d, &R));
    LNE_TRY(ws.get("tune.ur", (size_t)d * d, &UR));
    LNE_TRY(ws.get("tune.sig", (size_t)d, &sig));
    auto score = [&](int j, const float *Xj) -> int {
        if (X_out)
            LNE_CUDA_TRY(cudaMemcpyAsync(X_out + (size_t)j * n * d, Xj, sizeof(float) * n * d,
                                         cudaMemcpyDeviceToDevice, st));
        return macro_f1(ws, Xj, n, d, d, labels, L, train, n_train, test, n_test, Creg, iters, &macro[j], &micro[j],
                        st);
    };
    // k = 0: the embedding is X0 itself
    std::vector<int> prop;
    for (int j = 0; j < ncand; ++j) {
        if (cands[j].k == 0)
            LNE_TRY(score(j, X0s + (size_t)group[j] * n * d));
        else
            prop.push_back(j);
    }
    const int per_chunk = std::max(1, 1024 / d);
    for (size_t b0 = 0; b0 < prop.size(); b0 += per_chunk) {
        const int m = (int)std::min<size_t>(per_chunk, prop.size() - b0);
        const int C = m * d;
        float *X0r = nullptr, *P = nullptr;
        LNE_TRY(ws.get("tune.x0rep", (size_t)n * C, &X0r));
        LNE_TRY(ws.get("tune.p", (size_t)n * C, &P));
        std::vector<int> ks(m);
        std::vector<double> th(m), mu(m);
        for (int t = 0; t < m; ++t) {
            const lne_params &p = cands[prop[b0 + t]];
            ks[t] = p.k;
            th[t] = p.theta;
            mu[t] = p.mu;
            LNE_CUDA_TRY(cudaMemcpy2DAsync(X0r + (size_t)t * d, sizeof(float) * C,
                                           X0s + (size_t)group[prop[b0 + t]] * n * d, sizeof(float) * d,
                                           sizeof(float) * d, n, cudaMemcpyDeviceToDevice, st));
        }
        SpmmTile tile;
        LNE_TRY(spmm_tile_for(tc, ws, g, X0r, C, P, &tile, st));
        LNE_TRY(propagate_batch(ws, cache, g, d, m, ks.data(), th.data(), mu.data(), X0r, P, tile, st));
        // per candidate: X = U_P Sigma_P^{1/2} from the economic SVD of its block of P
        for (int t = 0; t < m; ++t) {
            float *Pj = P + (size_t)t * d;
            LNE_TRY(cholqr2(ws, Pj, n, d, C, R, st));
            LNE_TRY(small_svd(ws, R, d, UR, sig, st));
            LNE_TRY(right_multiply(Pj, n, d, C, UR, d, d, nullptr, U, d, st));
            LNE_TRY(sign_fix_embed(ws, U, n, d, d, sig, X, d, st));
            LNE_TRY(score(prop[b0 + t], X));
        }
        LNE_TRY(status_check(ws, st));
    }
    return 0;
}

}  // namespace lne

// ---------------------------------------------------------------------------
// Many independent tuning tasks (one graph + its labelled split each): host
// worker threads, each with its own workspace and non-blocking stream, take
// tasks in turn, so the small kernels of different graphs overlap on the GPU.
// ---------------------------------------------------------------------------
namespace lne {

TuneWorker::~TuneWorker() {
    if (st) cudaStreamDestroy(st);
}

int tune_tasks(std::vector<std::unique_ptr<TuneWorker>> &workers, int nworkers, int device, int forced_threads,
               int forced_block, int aggregation, int dense_mode, int stratified, const TuneTask *tasks, int ntasks,
               const lne_params *cands, int ncand, double Creg, int iters, double *macro, double *micro) {
    nworkers = std::max(1, std::min(nworkers, ntasks));
    while ((int)workers.size() < nworkers) {
        auto w = std::make_unique<TuneWorker>();
        LNE_CUDA_TRY(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking));
        workers.push_back(std::move(w));
    }
    std::atomic<int> next{0};
    std::atomic<bool> stop{false};
    std::mutex mu;
    int err = 0;
    std::string msg;
    auto run = [&](TuneWorker *w) {
        clear_message();
        set_tracer(nullptr);
        cudaError_t e = cudaSetDevice(device);
        int rc = e == cudaSuccess ? 0 : cuda_fail("cudaSetDevice", e, __FILE__, __LINE__);
        if (w->tune.forced != forced_threads || w->tune.forced_block != forced_block) w->tune.best.clear();
        w->tune.forced = forced_threads;
        w->tune.forced_block = forced_block;
        for (int t; rc == 0 && !stop.load() && (t = next.fetch_add(1)) < ntasks;) {
            const TuneTask &k = tasks[t];
            GraphView gk = k.g;
            rc = prepare_weighted(w->ws, &gk, w->st);
            if (rc == 0)
                rc = tune_batch(w->ws, nullptr, w->tune, aggregation, dense_mode, stratified, gk,
                            cands + (size_t)t * ncand, ncand, k.labels,
                            k.L, k.train, k.n_train, k.test, k.n_test, Creg, iters, macro + (size_t)t * ncand,
                            micro + (size_t)t * ncand, nullptr, w->st);
        }
        if (rc == 0) {
            e = cudaStreamSynchronize(w->st);
            if (e != cudaSuccess) rc = cuda_fail("cudaStreamSynchronize", e, __FILE__, __LINE__);
        }
        if (rc != 0) {
            stop.store(true);
            std::lock_guard<std::mutex> lock(mu);
            if (err == 0) {
                err = rc;
                msg = last_message();
            }
        }
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < nworkers; ++i) pool.emplace_back(run, workers[i].get());
    run(workers[0].get());
    for (auto &th : pool) th.join();
    if (err != 0) return fail(err, "tuning task failed: " + msg);
    return 0;
}

}  // namespace lne
