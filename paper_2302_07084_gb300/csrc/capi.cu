// C ABI of the library (declared in include/lne.h): argument checks, device
// selection, error reporting, and the composition of the stages.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "lne.h"
#include "runtime.h"

namespace lne {

namespace {
thread_local std::string g_msg;
}

int fail(int code, const std::string &msg) {
    g_msg = msg;
    return code;
}

int cuda_fail(const char *what, cudaError_t e, const char *file, int line) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_msg = buf;
    return (e == cudaErrorMemoryAllocation) ? LNE_ERR_OOM : LNE_ERR_CUDA;
}

const std::string &last_message() { return g_msg; }
void clear_message() { g_msg.clear(); }

namespace {
std::atomic<int64_t> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_sm_count[kMaxDevices];   // 0 = not queried yet
}  // namespace

int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    int v = g_sm_count[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int q = 0;
    if (cudaDeviceGetAttribute(&q, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || q <= 0) q = 1;
    g_sm_count[dev].store(q, std::memory_order_relaxed);
    return q;
}

namespace {
std::mutex g_smem_mu;
std::set<std::pair<const void *, int>> g_smem_raised;
}  // namespace

bool smem_limit_raised(const void *kernel, int dev) {
    std::lock_guard<std::mutex> lock(g_smem_mu);
    return g_smem_raised.count({kernel, dev}) != 0;
}

void mark_smem_limit_raised(const void *kernel, int dev) {
    std::lock_guard<std::mutex> lock(g_smem_mu);
    g_smem_raised.insert({kernel, dev});
}

// Per-context record of timed regions (CUDA event pairs).
struct Tracer {
    bool on = false;
    struct Rec {
        std::string name;
        cudaEvent_t a = nullptr, b = nullptr;
        int64_t launches = 0;
        bool closed = false;
    };
    std::vector<Rec> recs;
    std::vector<size_t> open;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    void recycle() {
        for (auto &r : recs) {
            if (r.a) pool.push_back(r.a);
            if (r.b) pool.push_back(r.b);
        }
        recs.clear();
        open.clear();
    }
    ~Tracer() {
        recycle();
        for (auto e : pool) cudaEventDestroy(e);
    }
};

namespace {
thread_local Tracer *g_tracer = nullptr;
}

void set_tracer(Tracer *t) { g_tracer = t; }
Tracer *get_tracer() { return g_tracer; }
int64_t launches_now() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void trace_begin(const char *name, cudaStream_t st) {
    Tracer *t = g_tracer;
    if (!t || !t->on) return;
    Tracer::Rec r;
    r.name = name;
    r.a = t->take();
    r.b = t->take();
    r.launches = g_launches.load(std::memory_order_relaxed);
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    t->open.push_back(t->recs.size());
    t->recs.push_back(r);
}

void trace_end(cudaStream_t st) {
    Tracer *t = g_tracer;
    if (!t || !t->on || t->open.empty()) return;
    Tracer::Rec &r = t->recs[t->open.back()];
    t->open.pop_back();
    cudaEventRecord(r.b, st);
    r.launches = g_launches.load(std::memory_order_relaxed) - r.launches;
    r.closed = true;
}

int Workspace::get(const std::string &name, size_t bytes, void **ptr) {
    if (bytes == 0) bytes = 1;
    Buf &b = bufs_[name];
    if (b.bytes < bytes) {
        if (b.p) {
            cudaError_t e = cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
            if (e != cudaSuccess) return cuda_fail("cudaFree", e, __FILE__, __LINE__);
        }
        // round up to limit regrowth
        size_t want = bytes + std::min(bytes / 8, (size_t)1 << 28);
        want = (want + 255) & ~(size_t)255;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            char buf[256];
            std::snprintf(buf, sizeof(buf), "device allocation of %zu bytes for '%s' failed: %s", want,
                          name.c_str(), cudaGetErrorString(e));
            g_msg = buf;
            return LNE_ERR_OOM;
        }
        b.bytes = want;
    }
    *ptr = b.p;
    return 0;
}

void Workspace::release() {
    for (auto &kv : bufs_)
        if (kv.second.p) cudaFree(kv.second.p);
    bufs_.clear();
}

void Workspace::release(const std::string &name) {
    auto it = bufs_.find(name);
    if (it == bufs_.end()) return;
    if (it->second.p) cudaFree(it->second.p);
    bufs_.erase(it);
}

int64_t Workspace::bytes() const {
    int64_t t = 0;
    for (auto &kv : bufs_) t += (int64_t)kv.second.bytes;
    return t;
}

}  // namespace lne

struct lne_ctx {
    int device = 0;
    int aggregation = LNE_AGG_AUTO;
    std::string err;
    lne::Workspace ws;
    lne::Tracer tracer;
    lne::SpmmTune spmm_tune;
    lne::PropBatchGraph *prop_graph = nullptr;
    int tune_workers = 4;
    int dense_mode = 0;
    int vblock = 0;   // LNE_OPT_SPMM_VBLOCK
    int stratified = 0;
    std::vector<std::unique_ptr<lne::TuneWorker>> workers;
    lne::Surrogate surrogate;
};

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

int finish(lne_ctx *ctx, int rc) {
    if (rc != 0) {
        ctx->err = lne::last_message();
        if (ctx->err.empty()) ctx->err = "unknown error";
    }
    return rc;
}

int enter(lne_ctx *ctx) {
    lne::clear_message();
    lne::set_tracer(&ctx->tracer);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return lne::cuda_fail("cudaSetDevice", e, __FILE__, __LINE__);
    return 0;
}

int check_graph(const lne_graph *g) {
    if (!g) return lne::fail(LNE_ERR_INVALID, "graph is NULL");
    if (g->n < 1) return lne::fail(LNE_ERR_INVALID, "graph needs n >= 1");
    if (g->n > 2147483647LL) return lne::fail(LNE_ERR_UNSUPPORTED, "more than 2^31 - 1 vertices");
    if (g->nnz < 0) return lne::fail(LNE_ERR_INVALID, "graph nnz < 0");
    if (!g->indptr || (g->nnz > 0 && !g->indices)) return lne::fail(LNE_ERR_INVALID, "graph arrays are NULL");
    return 0;
}

lne::GraphView view(const lne_graph *g) {
    lne::GraphView v;
    v.n = g->n;
    v.nnz = g->nnz;
    v.indptr = g->indptr;
    v.indices = g->indices;
    v.w = g->weights;
    return v;
}

int check_params(const lne_params *p, bool sampling) {
    if (!p) return lne::fail(LNE_ERR_INVALID, "params is NULL");
    if (sampling) {
        if (p->T < 1 || p->T > 16) return lne::fail(LNE_ERR_INVALID, "T must be in 1..16");
        if (!p->s) return lne::fail(LNE_ERR_INVALID, "s is NULL");
        if (!(p->samples > 0.0) || !std::isfinite(p->samples))
            return lne::fail(LNE_ERR_INVALID, "samples must be a finite value > 0");
    }
    if (p->precision != LNE_PREC_FP32 && p->precision != LNE_PREC_BF16_MIXED)
        return lne::fail(LNE_ERR_INVALID, "unknown precision");
    if (!(p->downsample_C >= 0.0) || !std::isfinite(p->downsample_C))
        return lne::fail(LNE_ERR_INVALID, "downsample_C must be a finite value >= 0");
    if (p->sketch != LNE_SKETCH_GAUSSIAN && p->sketch != LNE_SKETCH_SPARSE_SIGN && p->sketch != LNE_SKETCH_VERY_SPARSE)
        return lne::fail(LNE_ERR_INVALID, "unknown sketch");
    if (p->sketch == LNE_SKETCH_SPARSE_SIGN && (p->sketch_zeta < 0 || p->sketch_zeta > lne::kMaxSketchZeta))
        return lne::fail(LNE_ERR_INVALID, "sketch_zeta must be in 0..12");
    if (p->sketch == LNE_SKETCH_VERY_SPARSE && p->sketch_zeta < 0)
        return lne::fail(LNE_ERR_INVALID, "the very sparse projection's s (sketch_zeta) must be >= 0");
    return 0;
}

int oversample_of(const lne_params *p) { return p->oversample < 0 ? 16 : p->oversample; }

lne::SketchSpec sketch_of(const lne_params *p) {
    lne::SketchSpec s;
    s.kind = p->sketch;
    s.zeta = p->sketch == LNE_SKETCH_SPARSE_SIGN ? p->sketch_zeta : 0;
    s.sparsity = p->sketch == LNE_SKETCH_VERY_SPARSE ? (double)p->sketch_zeta : 0.0;
    return s;
}

lne::CsrView csr_view(const lne_csr *M) {
    lne::CsrView v;
    v.n = M->n;
    v.nnz = M->nnz;
    v.indptr = M->indptr;
    v.indices = M->indices;
    v.data = M->data;
    return v;
}

// The CSR structure of a graph: bit 1 of *bad for an indptr entry below its
// predecessor, bit 2 for a column index outside [0, n). Reads indptr[0..n]
// and indices[0..nnz) only. With indptr[0] = 0 and indptr[n] = nnz (checked
// on the host), a non-decreasing indptr keeps every row inside [0, nnz).
__global__ void csr_structure_kernel(const int64_t *__restrict__ indptr, int64_t n,
                                     const int32_t *__restrict__ indices, int64_t nnz, int *__restrict__ bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    for (int64_t i = t0; i < n; i += stride)
        if (indptr[i + 1] < indptr[i]) f |= 1;
    for (int64_t e = t0; e < nnz; e += stride) {
        const int32_t v = indices[e];
        if (v < 0 || (int64_t)v >= n) f |= 2;
    }
    if (f) atomicOr(bad, f);
}

// Checks the graph on the device before any kernel walks it: indptr starts at
// 0, ends at nnz and never decreases, and every index lies in [0, n).
int check_graph_device(lne_ctx *ctx, const lne_graph *g, cudaStream_t st) {
    int64_t ends[2] = {0, 0};
    int bad = 0;
    int *bad_dev = nullptr;
    LNE_TRY(ctx->ws.get("graph.check", 1, &bad_dev));
    LNE_CUDA_TRY(cudaMemsetAsync(bad_dev, 0, sizeof(int), st));
    {
        const int64_t work = std::max<int64_t>(std::max<int64_t>(g->n, g->nnz), 1);
        const unsigned blocks = (unsigned)std::min<int64_t>(lne::ceil_div(work, (int64_t)256), lne::num_sms() * 8);
        csr_structure_kernel<<<blocks, 256, 0, st>>>(g->indptr, g->n, g->indices, g->nnz, bad_dev);
        LNE_LAUNCH_CHECK();
    }
    LNE_CUDA_TRY(cudaMemcpyAsync(&ends[0], g->indptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(&ends[1], g->indptr + g->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(&bad, bad_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (ends[0] != 0 || ends[1] != g->nnz)
        return lne::fail(LNE_ERR_INVALID, "graph indptr must start at 0 and end at nnz");
    if (bad & 1) return lne::fail(LNE_ERR_INVALID, "graph indptr decreases");
    if (bad & 2) return lne::fail(LNE_ERR_INVALID, "a graph index is outside [0, n)");
    return 0;
}

}  // namespace

extern "C" {

int lne_create(lne_ctx **out, int device) {
    if (!out) return LNE_ERR_INVALID;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return LNE_ERR_CUDA;
    }
    lne_ctx *ctx = new lne_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return LNE_ERR_CUDA;
    }
    *out = ctx;
    return LNE_OK;
}

void lne_destroy(lne_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    lne::set_tracer(nullptr);
    if (ctx->prop_graph) lne::destroy_prop_cache(ctx->prop_graph);
    ctx->workers.clear();
    ctx->ws.release();
    delete ctx;
}

int64_t lne_kernel_launches(void) { return lne::g_launches.load(); }

int lne_set_option(lne_ctx *ctx, int option, int64_t value) {
    if (!ctx) return LNE_ERR_INVALID;
    lne::clear_message();
    if (option == LNE_OPT_AGGREGATION) {
        if (value != LNE_AGG_AUTO && value != LNE_AGG_TABLE && value != LNE_AGG_BUCKET && value != LNE_AGG_SORT)
            return finish(ctx, lne::fail(LNE_ERR_INVALID, "unknown aggregation method"));
        ctx->aggregation = (int)value;
        return LNE_OK;
    }
    if (option == LNE_OPT_SPMM_THREADS) {
        if (value != 0 && value != 64 && value != 128 && value != 256)
            return finish(ctx, lne::fail(LNE_ERR_INVALID, "SpMM CTA size must be 0 (timed), 64, 128 or 256"));
        ctx->spmm_tune.forced = (int)value;
        return LNE_OK;
    }
    if (option == LNE_OPT_SPMM_COLBLOCK) {
        if (value != 0 && value != -1 && !(value > 0 && value <= 1024 && value % 4 == 0))
            return finish(ctx, lne::fail(LNE_ERR_INVALID,
                                         "SpMM column block must be 0 (timed), -1 (none) or a multiple of 4 up to 1024"));
        ctx->spmm_tune.forced_block = (int)value;
        ctx->spmm_tune.best.clear();
        return LNE_OK;
    }
    if (option == LNE_OPT_SPMM_VBLOCK) {
        if (value < -1 || value > 30)
            return finish(ctx, lne::fail(LNE_ERR_INVALID, "vertex block must be 0 (auto), -1 (off) or a shift 1..30"));
        ctx->vblock = (int)value;
        return LNE_OK;
    }
    if (option == LNE_OPT_DENSE_PRODUCT) {
        if (value < 0 || value > 2) return finish(ctx, lne::fail(LNE_ERR_INVALID, "dense product mode must be 0..2"));
        ctx->dense_mode = (int)value;
        return LNE_OK;
    }
    if (option == LNE_OPT_STRATIFIED) {
        if (value != 0 && value != 1) return finish(ctx, lne::fail(LNE_ERR_INVALID, "stratified must be 0 or 1"));
        ctx->stratified = (int)value;
        return LNE_OK;
    }
    if (option == LNE_OPT_TUNE_WORKERS) {
        if (value < 1 || value > 16) return finish(ctx, lne::fail(LNE_ERR_INVALID, "tuning workers must be 1..16"));
        ctx->tune_workers = (int)value;
        return LNE_OK;
    }
    return finish(ctx, lne::fail(LNE_ERR_INVALID, "unknown option"));
}

int lne_trace_enable(lne_ctx *ctx, int on) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) {
        cudaDeviceSynchronize();
        ctx->tracer.recycle();
        ctx->tracer.on = on != 0;
    }
    return finish(ctx, rc);
}

int lne_trace_read(lne_ctx *ctx, lne_trace_entry *out, int capacity, int *count) {
    if (!ctx || !count || (capacity > 0 && !out)) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc != 0) return finish(ctx, rc);
    // aggregate closed regions by name, in order of first appearance
    std::vector<lne_trace_entry> agg;
    for (auto &r : ctx->tracer.recs) {
        if (!r.closed) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return finish(ctx, lne::cuda_fail("cudaEventSynchronize", e, __FILE__, __LINE__));
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return finish(ctx, lne::cuda_fail("cudaEventElapsedTime", e, __FILE__, __LINE__));
        lne_trace_entry *hit = nullptr;
        for (auto &a : agg)
            if (std::strncmp(a.name, r.name.c_str(), sizeof(a.name)) == 0) hit = &a;
        if (!hit) {
            lne_trace_entry z;
            std::memset(&z, 0, sizeof(z));
            std::strncpy(z.name, r.name.c_str(), sizeof(z.name) - 1);
            agg.push_back(z);
            hit = &agg.back();
        }
        hit->regions += 1;
        hit->launches += r.launches;
        hit->total_ms += ms;
    }
    ctx->tracer.recycle();
    *count = (int)agg.size();
    for (int i = 0; i < (int)agg.size() && i < capacity; ++i) out[i] = agg[i];
    return finish(ctx, 0);
}

const char *lne_last_error(const lne_ctx *ctx) { return ctx ? ctx->err.c_str() : "context is NULL"; }

int64_t lne_workspace_bytes(const lne_ctx *ctx) { return ctx ? ctx->ws.bytes() : 0; }

int lne_trim(lne_ctx *ctx) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) {
        cudaDeviceSynchronize();
        if (ctx->prop_graph) lne::destroy_prop_cache(ctx->prop_graph);
        ctx->prop_graph = nullptr;
        ctx->workers.clear();
        ctx->ws.release();
    }
    return finish(ctx, rc);
}

int lne_sample_pairs(lne_ctx *ctx, const lne_graph *g, const lne_params *p, int64_t arc_begin,
                     int64_t arc_end, int32_t *u1_dev, int32_t *v1_dev, int64_t capacity,
                     int64_t *count_out, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = check_graph(g);
    if (rc == 0) rc = check_params(p, true);
    if (rc == 0 && (!count_out || (capacity > 0 && (!u1_dev || !v1_dev))))
        rc = lne::fail(LNE_ERR_INVALID, "NULL output");
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = check_graph_device(ctx, g, st);
    lne::GraphView gv = view(g);
    if (rc == 0) rc = lne::prepare_weighted(ctx->ws, &gv, st);
    lne::SamplerSpec sp;
    if (rc == 0) rc = lne::make_sampler_spec(gv, p->T, p->s, p->samples, p->b, p->seed, &sp);
    sp.aggregation = ctx->aggregation;
    sp.ds_C = p->downsample_C;
    sp.stratified = ctx->stratified;
    if (rc == 0) rc = lne::sample_pairs(ctx->ws, gv, sp, arc_begin, arc_end, u1_dev, v1_dev, capacity,
                                        count_out, st);
    return finish(ctx, rc);
}

int lne_sparsifier_counts(lne_ctx *ctx, const lne_graph *g, const lne_params *p, lne_counts *out,
                          void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = check_graph(g);
    if (rc == 0) rc = check_params(p, true);
    if (rc == 0 && !out) rc = lne::fail(LNE_ERR_INVALID, "NULL output");
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = check_graph_device(ctx, g, st);
    lne::GraphView gv = view(g);
    if (rc == 0) rc = lne::prepare_weighted(ctx->ws, &gv, st);
    lne::SamplerSpec sp;
    if (rc == 0) rc = lne::make_sampler_spec(gv, p->T, p->s, p->samples, p->b, p->seed, &sp);
    sp.aggregation = ctx->aggregation;
    sp.ds_C = p->downsample_C;
    sp.stratified = ctx->stratified;
    lne::CountsResult r;
    if (rc == 0) rc = lne::sparsifier_counts(ctx->ws, gv, sp, &r, st);
    if (rc == 0) {
        out->nnz = r.nnz;
        out->x = r.x;
        out->y = r.y;
        out->count = r.cnt;
        out->total_samples = r.total_samples;
        out->weight = r.weight;
        out->window = r.window;
    }
    return finish(ctx, rc);
}

int lne_sparsifier_csr(lne_ctx *ctx, const lne_graph *g, const lne_params *p, lne_csr *out, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = check_graph(g);
    if (rc == 0) rc = check_params(p, true);
    if (rc == 0 && !out) rc = lne::fail(LNE_ERR_INVALID, "NULL output");
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = check_graph_device(ctx, g, st);
    lne::GraphView gv = view(g);
    if (rc == 0) rc = lne::prepare_weighted(ctx->ws, &gv, st);
    lne::SamplerSpec sp;
    if (rc == 0) rc = lne::make_sampler_spec(gv, p->T, p->s, p->samples, p->b, p->seed, &sp);
    sp.aggregation = ctx->aggregation;
    sp.ds_C = p->downsample_C;
    sp.stratified = ctx->stratified;
    lne::CsrResult r;
    if (rc == 0) rc = lne::sparsifier_csr(ctx->ws, gv, sp, &r, st);
    if (rc == 0) {
        out->n = r.n;
        out->nnz = r.nnz;
        out->indptr = r.indptr;
        out->indices = r.indices;
        out->data = r.data;
    }
    return finish(ctx, rc);
}

int lne_gaussian_sketch(lne_ctx *ctx, int64_t n, int32_t c, uint64_t seed, float *out_dev, int64_t ld,
                        void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (n < 0 || c < 0 || ld < c || (n > 0 && c > 0 && !out_dev)))
        rc = lne::fail(LNE_ERR_INVALID, "bad sketch arguments");
    if (rc == 0) rc = lne::gaussian_sketch(n, c, seed, out_dev, ld, as_stream(stream));
    return finish(ctx, rc);
}

int lne_sparse_sign_sketch(lne_ctx *ctx, int64_t n, int32_t c, int32_t zeta, uint64_t seed, float *out_dev,
                           int64_t ld, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (n < 0 || (n > 0 && !out_dev))) rc = lne::fail(LNE_ERR_INVALID, "bad sketch arguments");
    if (rc == 0) rc = lne::sparse_sign_dense(ctx->ws, n, c, zeta, seed, out_dev, ld, as_stream(stream));
    return finish(ctx, rc);
}

int lne_very_sparse_sketch(lne_ctx *ctx, int64_t n, int32_t c, double s, uint64_t seed, float *out_dev, int64_t ld,
                           void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (n < 0 || (n > 0 && !out_dev))) rc = lne::fail(LNE_ERR_INVALID, "bad sketch arguments");
    if (rc == 0) rc = lne::very_sparse_dense(ctx->ws, n, c, s, seed, out_dev, ld, as_stream(stream));
    return finish(ctx, rc);
}

int lne_very_sparse_spmm(lne_ctx *ctx, const lne_csr *M, int32_t c, double s, uint64_t seed, float *Y_dev,
                         int64_t ldy, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!M || M->n < 0 || !M->indptr || (M->n > 0 && !Y_dev)))
        rc = lne::fail(LNE_ERR_INVALID, "bad very sparse product arguments");
    if (rc == 0) rc = lne::very_sparse_spmm(ctx->ws, csr_view(M), c, s, seed, Y_dev, ldy, as_stream(stream));
    if (rc == 0) rc = lne::status_check(ctx->ws, as_stream(stream));
    return finish(ctx, rc);
}

int lne_sparse_sign_spmm(lne_ctx *ctx, const lne_csr *M, int32_t c, int32_t zeta, uint64_t seed, float *Y_dev,
                         int64_t ldy, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!M || M->n < 0 || !M->indptr || (M->n > 0 && !Y_dev)))
        rc = lne::fail(LNE_ERR_INVALID, "bad sparse sign product arguments");
    if (rc == 0) rc = lne::sparse_sign_spmm(ctx->ws, csr_view(M), c, zeta, seed, Y_dev, ldy, as_stream(stream));
    return finish(ctx, rc);
}

int lne_spmm(lne_ctx *ctx, const lne_csr *M, const void *X_dev, int64_t ldx, int32_t c, float *Y_dev,
             int64_t ldy, int32_t precision, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!M || M->n < 0 || c < 1 || ldx < c || ldy < c || !X_dev || !Y_dev || !M->indptr))
        rc = lne::fail(LNE_ERR_INVALID, "bad SpMM arguments");
    if (rc == 0 && precision != LNE_PREC_FP32 && precision != LNE_PREC_BF16_MIXED)
        rc = lne::fail(LNE_ERR_INVALID, "unknown precision");
    if (rc == 0) {
        lne::CsrView v;
        v.n = M->n;
        v.nnz = M->nnz;
        v.indptr = M->indptr;
        v.indices = M->indices;
        v.data = M->data;
        // column blocks by vertex ranges when the operand does not fit in L2
        // (or as the option forces); matrices with unsorted rows go unblocked
        lne::VBlocks vbs;
        const int shift = lne::vblock_shift_for(ctx->vblock, v.n, c, precision == LNE_PREC_BF16_MIXED ? 2 : 4);
        bool ok = false;
        if (shift > 0 && v.nnz > 0) rc = lne::vblocks_build(ctx->ws, v, shift, &vbs, &ok, as_stream(stream));
        if (ok) v.vb = &vbs;
        if (rc == 0 && precision == LNE_PREC_BF16_MIXED)
            rc = lne::spmm_bf16(ctx->ws, v, static_cast<const __nv_bfloat16 *>(X_dev), ldx, c, Y_dev, ldy, nullptr,
                                as_stream(stream));
        else if (rc == 0)
            rc = lne::spmm(ctx->ws, v, static_cast<const float *>(X_dev), ldx, c, Y_dev, ldy, as_stream(stream));
    }
    return finish(ctx, rc);
}

int lne_cholqr2(lne_ctx *ctx, float *Y_dev, int64_t n, int32_t c, int64_t ld, double *R_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!Y_dev || ld < c)) rc = lne::fail(LNE_ERR_INVALID, "bad CholeskyQR2 arguments");
    if (rc == 0) rc = lne::cholqr2(ctx->ws, Y_dev, n, c, ld, R_dev, as_stream(stream));
    if (rc == 0) rc = lne::status_check(ctx->ws, as_stream(stream));
    return finish(ctx, rc);
}

int lne_svd_small(lne_ctx *ctx, const double *R_dev, int32_t c, double *U_dev, double *sigma_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!R_dev || !U_dev || !sigma_dev || c < 1)) rc = lne::fail(LNE_ERR_INVALID, "bad small SVD arguments");
    if (rc == 0) rc = lne::small_svd(ctx->ws, R_dev, c, U_dev, sigma_dev, as_stream(stream));
    return finish(ctx, rc);
}

int lne_rsvd(lne_ctx *ctx, const lne_csr *M, const lne_params *p, float *U_dev, double *sigma_dev,
             float *X0_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!M || !M->indptr || M->n < 1)) rc = lne::fail(LNE_ERR_INVALID, "bad matrix");
    if (rc == 0) rc = check_params(p, false);
    if (rc == 0) {
        lne::CsrView v;
        v.n = M->n;
        v.nnz = M->nnz;
        v.indptr = M->indptr;
        v.indices = M->indices;
        v.data = M->data;
        v.vblock = ctx->vblock;
        rc = lne::rsvd(ctx->ws, v, p->d, oversample_of(p), p->q, p->seed, p->precision, U_dev, sigma_dev, X0_dev,
                       as_stream(stream), sketch_of(p));
    }
    return finish(ctx, rc);
}

int lne_propagate(lne_ctx *ctx, const lne_graph *g, const lne_params *p, const float *X0_dev, float *X_dev,
                  float *F_dev, float *P_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = check_graph(g);
    if (rc == 0) rc = check_params(p, false);
    if (rc == 0 && (!X0_dev || !X_dev)) rc = lne::fail(LNE_ERR_INVALID, "NULL embedding buffer");
    if (rc == 0 && (p->k < 0 || !std::isfinite(p->theta) || !std::isfinite(p->mu)))
        rc = lne::fail(LNE_ERR_INVALID, "need k >= 0 and finite theta, mu");
    if (rc == 0 && p->d < 1) rc = lne::fail(LNE_ERR_INVALID, "need d >= 1");
    lne::GraphView gv = view(g);
    if (rc == 0) rc = lne::prepare_weighted(ctx->ws, &gv, as_stream(stream));
    if (rc == 0)
        rc = lne::propagate(ctx->ws, gv, p->d, p->k, p->theta, p->mu, p->precision, X0_dev, X_dev, F_dev,
                            P_dev, as_stream(stream));
    return finish(ctx, rc);
}

int lne_macro_f1(lne_ctx *ctx, const float *X_dev, int64_t n, int32_t d, int64_t ldx, const uint8_t *labels_dev,
                 int32_t L, const int32_t *train_dev, int64_t n_train, const int32_t *test_dev, int64_t n_test,
                 double C, int32_t iters, double *macro_f1, double *micro_f1, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!X_dev || !labels_dev || !train_dev || !test_dev || !macro_f1 || !micro_f1 || ldx < d || n < 1))
        rc = lne::fail(LNE_ERR_INVALID, "bad Macro-F1 arguments");
    if (rc == 0)
        rc = lne::macro_f1(ctx->ws, X_dev, n, d, ldx, labels_dev, L, train_dev, n_train, test_dev, n_test, C, iters,
                           macro_f1, micro_f1, as_stream(stream));
    return finish(ctx, rc);
}

int lne_embed(lne_ctx *ctx, const lne_graph *g, const lne_params *p, float *X_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = check_graph(g);
    if (rc == 0) rc = check_params(p, true);
    if (rc == 0 && !X_dev) rc = lne::fail(LNE_ERR_INVALID, "NULL embedding buffer");
    if (rc == 0 && (p->k < 0 || p->q < 0 || p->d < 1)) rc = lne::fail(LNE_ERR_INVALID, "need d >= 1, q >= 0, k >= 0");
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = check_graph_device(ctx, g, st);
    lne::GraphView gv = view(g);
    if (rc == 0) rc = lne::prepare_weighted(ctx->ws, &gv, st);
    lne::SamplerSpec sp;
    if (rc == 0) rc = lne::make_sampler_spec(gv, p->T, p->s, p->samples, p->b, p->seed, &sp);
    sp.aggregation = ctx->aggregation;
    sp.ds_C = p->downsample_C;
    sp.stratified = ctx->stratified;
    lne::CsrResult M;
    if (rc == 0) rc = lne::sparsifier_csr(ctx->ws, gv, sp, &M, st);
    float *X0 = nullptr;
    if (rc == 0) rc = ctx->ws.get("embed.x0", (size_t)g->n * p->d, &X0);
    if (rc == 0) {
        lne::CsrView mv = lne::product_view(M, ctx->dense_mode, p->d + oversample_of(p));
        mv.vblock = ctx->vblock;
        rc = lne::rsvd(ctx->ws, mv, p->d, oversample_of(p), p->q, p->seed, p->precision, nullptr, nullptr, X0, st,
                       sketch_of(p));
    }
    if (rc == 0)
        rc = lne::propagate(ctx->ws, gv, p->d, p->k, p->theta, p->mu, p->precision, X0, X_dev, nullptr, nullptr,
                            st);
    return finish(ctx, rc);
}

int lne_tune_batch(lne_ctx *ctx, const lne_graph *g, const lne_params *cands, int32_t ncand,
                   const uint8_t *labels_dev, int32_t L, const int32_t *train_dev, int64_t n_train,
                   const int32_t *test_dev, int64_t n_test, double C, int32_t iters, double *macro_f1,
                   double *micro_f1, float *X_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = check_graph(g);
    if (rc == 0 && (!cands || ncand < 1)) rc = lne::fail(LNE_ERR_INVALID, "need at least one candidate");
    for (int j = 0; rc == 0 && j < ncand; ++j) rc = check_params(&cands[j], true);
    if (rc == 0 && (!macro_f1 || !micro_f1)) rc = lne::fail(LNE_ERR_INVALID, "NULL score outputs");
    if (rc == 0 && (!labels_dev || L < 1 || !train_dev || n_train < 1 || !test_dev || n_test < 1 || iters < 0))
        rc = lne::fail(LNE_ERR_INVALID, "bad evaluation split or labels");
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = check_graph_device(ctx, g, st);
    lne::GraphView gv = view(g);
    if (rc == 0) rc = lne::prepare_weighted(ctx->ws, &gv, st);
    if (rc == 0 && !ctx->prop_graph) ctx->prop_graph = lne::new_prop_cache();
    if (rc == 0)
        rc = lne::tune_batch(ctx->ws, ctx->prop_graph, ctx->spmm_tune, ctx->aggregation, ctx->dense_mode,
                             ctx->stratified, gv,
                             cands, ncand,
                             labels_dev, L, train_dev, n_train, test_dev, n_test, C, iters, macro_f1, micro_f1,
                             X_dev, st);
    return finish(ctx, rc);
}

int lne_tune_tasks(lne_ctx *ctx, const lne_task *tasks, int32_t ntasks, const lne_params *cands, int32_t ncand,
                   double C, int32_t iters, double *macro_f1, double *micro_f1, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!tasks || ntasks < 1 || !cands || ncand < 1))
        rc = lne::fail(LNE_ERR_INVALID, "need at least one task and one candidate per task");
    if (rc == 0 && (!macro_f1 || !micro_f1)) rc = lne::fail(LNE_ERR_INVALID, "NULL score outputs");
    if (rc == 0 && iters < 0) rc = lne::fail(LNE_ERR_INVALID, "iters must be >= 0");
    cudaStream_t st = as_stream(stream);
    std::vector<lne::TuneTask> tt(rc == 0 ? ntasks : 0);
    for (int t = 0; rc == 0 && t < ntasks; ++t) {
        const lne_task &k = tasks[t];
        rc = check_graph(&k.graph);
        if (rc == 0 && (!k.labels_dev || k.L < 1 || !k.train_dev || k.n_train < 1 || !k.test_dev || k.n_test < 1))
            rc = lne::fail(LNE_ERR_INVALID, "bad evaluation split or labels");
        for (int j = 0; rc == 0 && j < ncand; ++j) rc = check_params(&cands[(size_t)t * ncand + j], true);
        if (rc == 0) rc = check_graph_device(ctx, &k.graph, st);
        if (rc == 0) {
            tt[t].g = view(&k.graph);
            tt[t].labels = k.labels_dev;
            tt[t].L = k.L;
            tt[t].train = k.train_dev;
            tt[t].n_train = k.n_train;
            tt[t].test = k.test_dev;
            tt[t].n_test = k.n_test;
        }
    }
    if (rc == 0) {   // inputs written on `stream` are complete before the workers start
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = lne::cuda_fail("cudaStreamSynchronize", e, __FILE__, __LINE__);
    }
    if (rc == 0)
        rc = lne::tune_tasks(ctx->workers, ctx->tune_workers, ctx->device, ctx->spmm_tune.forced,
                             ctx->spmm_tune.forced_block, ctx->aggregation,
                             ctx->dense_mode, ctx->stratified, tt.data(), ntasks, cands, ncand, C, iters, macro_f1,
                             micro_f1);
    return finish(ctx, rc);
}

int lne_surrogate_init(lne_ctx *ctx, uint64_t seed, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0) rc = lne::surrogate_init(ctx->surrogate, seed, as_stream(stream));
    return finish(ctx, rc);
}

int lne_surrogate_fit_scaling(lne_ctx *ctx, const float *X_dev, int64_t rows, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!X_dev || rows < 1)) rc = lne::fail(LNE_ERR_INVALID, "need rows >= 1 features");
    if (rc == 0) rc = lne::surrogate_fit_scaling(ctx->surrogate, X_dev, rows, as_stream(stream));
    return finish(ctx, rc);
}

int lne_surrogate_set_params(lne_ctx *ctx, const float *theta, const float *mean, const float *std, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!theta || !mean || !std)) rc = lne::fail(LNE_ERR_INVALID, "NULL parameter array");
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = lne::surrogate_set(ctx->surrogate, theta, mean, std, st);
    if (rc == 0) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = lne::cuda_fail("cudaStreamSynchronize", e, __FILE__, __LINE__);
    }
    return finish(ctx, rc);
}

int lne_surrogate_get_params(lne_ctx *ctx, float *theta, float *mean, float *std, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    cudaStream_t st = as_stream(stream);
    if (rc == 0) rc = lne::surrogate_get(ctx->surrogate, theta, mean, std, st);
    if (rc == 0) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = lne::cuda_fail("cudaStreamSynchronize", e, __FILE__, __LINE__);
    }
    return finish(ctx, rc);
}

int lne_surrogate_train(lne_ctx *ctx, const float *X_dev, const float *y_dev, int64_t rows, int32_t epochs,
                        int32_t batch, float lr, uint64_t seed, double *final_loss, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!X_dev || !y_dev || rows < 1 || rows > 2147483647LL))
        rc = lne::fail(LNE_ERR_INVALID, "need 1 <= rows < 2^31 and non-NULL data");
    if (rc == 0 && (epochs < 0 || batch < 1 || !(lr > 0.f)))
        rc = lne::fail(LNE_ERR_INVALID, "need epochs >= 0, batch >= 1, lr > 0");
    if (rc == 0)
        rc = lne::surrogate_train(ctx->surrogate, ctx->ws, X_dev, y_dev, rows, epochs, batch, lr, seed, final_loss,
                                  as_stream(stream));
    return finish(ctx, rc);
}

int lne_surrogate_predict(lne_ctx *ctx, const float *X_dev, int64_t rows, float *yhat_dev, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (rows < 0 || (rows > 0 && (!X_dev || !yhat_dev))))
        rc = lne::fail(LNE_ERR_INVALID, "need rows >= 0 and non-NULL buffers");
    if (rc == 0) rc = lne::surrogate_predict(ctx->surrogate, X_dev, rows, yhat_dev, as_stream(stream));
    return finish(ctx, rc);
}

int lne_surrogate_grad(lne_ctx *ctx, const float *X_dev, const float *y_dev, int64_t rows, float *grad_dev,
                       double *loss, void *stream) {
    if (!ctx) return LNE_ERR_INVALID;
    int rc = enter(ctx);
    if (rc == 0 && (!X_dev || !y_dev || rows < 1)) rc = lne::fail(LNE_ERR_INVALID, "need rows >= 1 and data");
    if (rc == 0)
        rc = lne::surrogate_grad(ctx->surrogate, ctx->ws, X_dev, y_dev, rows, grad_dev, loss, as_stream(stream));
    return finish(ctx, rc);
}

}  // extern "C"
