// Y = M X on the 5th-generation tensor cores (tcgen05, TMEM accumulators,
// TMA-staged operands), for M held as the dense table of Eq. 1 values (the
// randomized SVD's products, Algorithm 4, when the sparsifier keeps a large
// fraction of all pairs).
//
// FP32 accuracy from TF32 products: every operand value a is split as
// a = a_hi + a_lo with a_hi = a with its 13 low mantissa bits cleared (exactly
// representable in TF32) and a_lo = a - a_hi (exact in FP32), and
// a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi, three MMAs accumulating in FP32
// (the dropped a_lo b_lo and the TF32 truncation of the lo parts are ~2^-22 of
// a b).
//
// Operands, prepared once per table / per product:
//   A_hi, A_lo: the full symmetric n_pad x n_pad matrix (the table holds only
//               its upper triangle), row-major, so a row block of M is a
//               K-major operand;
//   B_hi, B_lo: X transposed, N_pad x n_pad (N_pad = c rounded up to 16),
//               K-major, zero beyond n rows / c columns.
//
// Kernel: one CTA (128 threads) per (128-row block of Y, slice of the k range).
// Warp 0 lane 0 streams 32-wide k chunks of A_hi, A_lo, B_hi, B_lo into a
// 3-stage shared-memory ring by TMA (128-byte swizzle); warp 1 lane 0 issues,
// per chunk, 4 k-steps x 3 tcgen05.mma (M = 128, N = N_pad, K = 8) into one
// TMEM accumulator of 128 lanes x N_pad columns and releases the stage with
// tcgen05.commit; at the end all four warps read their 32 TMEM lanes
// (tcgen05.ld) and write the slice's partial product, which slice_sum adds in
// slice order (deterministic). Every mbarrier wait is bounded: on expiry the
// kernel sets the context's device status word (read by status_check) instead
// of hanging.
#include <cuda.h>

#include <utility>

#include "runtime.h"
#include "tc_desc.h"

namespace lne {
namespace {

constexpr int kTcRows = 128;          // MMA M: rows of Y per CTA
constexpr int kTcKc = 32;             // k per stage: one 128-byte row of FP32
constexpr int kTcStages = 3;
constexpr int kTcEpiWarps = 4;                 // warps 2..5 (one per TMEM lane quadrant)
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);   // warp 0: TMA, warp 1: MMA, then the epilogue
constexpr int kTcATile = kTcRows * kTcKc * 4;   // 16 KB
constexpr uint64_t kTcWaitNs = 2000000000ull;   // a pipeline wait gives up after 2 s

__host__ __device__ constexpr int tc_npad(int c) { return (c + 15) / 16 * 16; }
__host__ __device__ constexpr int tc_stage_bytes(int npad) { return 2 * kTcATile + 2 * npad * kTcKc * 4; }
__host__ __device__ constexpr int tc_smem_bytes(int npad) { return kTcStages * tc_stage_bytes(npad) + 1024; }
__host__ __device__ constexpr uint32_t tc_tmem_cols(int npad) {
    return npad <= 32 ? 32u : npad <= 64 ? 64u : npad <= 128 ? 128u : 256u;
}

__host__ __device__ constexpr uint32_t tc_idesc(int npad) { return tc_idesc_tf32(kTcRows, npad); }
__host__ __device__ constexpr uint64_t tc_sdesc(uint32_t saddr) { return tc_sdesc_sw128(saddr); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the phase of `bar` with the given parity has completed; false
// (and *err set) if it has not after kTcWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0) {
            const uint64_t t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > kTcWaitNs) break;
        }
    }
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes: thread t gets lane
// 32 (warp % 4) + t.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent: one CTA per SM walks the work items t = blockIdx.x, + gridDim.x,
// ... (item t = k-slice t / rbs of row block t % rbs). The TMA producer and the
// MMA issuer run ahead across items through the shared-memory ring; two TMEM
// accumulators let the epilogue of one item overlap the MMAs of the next.
__global__ void __launch_bounds__(kTcThreads, 1) dense_tc_kernel(
    const __grid_constant__ CUtensorMap tm_ahi, const __grid_constant__ CUtensorMap tm_alo,
    const __grid_constant__ CUtensorMap tm_bhi, const __grid_constant__ CUtensorMap tm_blo, int64_t n,
    int nchunks, int slice_chunks, int rbs, int items, int npad, int c, float *__restrict__ P,
    int *__restrict__ err) {
    extern __shared__ uint8_t tc_smem_raw[];
    __shared__ __align__(8) uint64_t s_full[kTcStages], s_empty[kTcStages], s_accf[2], s_acce[2];
    __shared__ uint32_t s_tmem;
    // stage tiles at 1024-byte boundaries of the shared window (the swizzle atom)
    uint8_t *smem = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t acc_cols = tc_tmem_cols(npad);   // columns of one accumulator
    const uint32_t ncols = 2 * acc_cols;
    const int stage_bytes = tc_stage_bytes(npad);
    const int b_tile = npad * kTcKc * 4;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(smem_u32(&s_full[s]), 1);
            mbar_init(smem_u32(&s_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&s_accf[b]), 1);                  // tcgen05.commit of the item's MMAs
            mbar_init(smem_u32(&s_acce[b]), kTcEpiWarps);        // one lane of each epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tc_idesc(npad);
    auto item_range = [&](int t, int &r0, int &z, int &c0, int &nk) {
        const int rb = t % rbs;
        z = t / rbs;
        r0 = rb * kTcRows;
        c0 = z * slice_chunks;
        nk = max(0, min(nchunks, c0 + slice_chunks) - c0);
    };
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {   // producer: TMA loads of every item's k chunks into the ring
            uint32_t g = 0;
            for (int t = blockIdx.x; t < items && ok; t += gridDim.x) {
                int r0, z, c0, nk;
                item_range(t, r0, z, c0, nk);
                for (int i = 0; i < nk; ++i, ++g) {
                    const uint32_t s = g % kTcStages;
                    if (g >= kTcStages) ok = mbar_wait(smem_u32(&s_empty[s]), (g / kTcStages + 1) & 1u, err);
                    if (!ok) break;
                    uint8_t *st = smem + (size_t)s * stage_bytes;
                    const uint32_t bar = smem_u32(&s_full[s]);
                    mbar_expect_tx(bar, (uint32_t)stage_bytes);
                    const int k = (c0 + i) * kTcKc;
                    tma_load_2d(smem_u32(st), &tm_ahi, k, r0, bar);
                    tma_load_2d(smem_u32(st + kTcATile), &tm_alo, k, r0, bar);
                    tma_load_2d(smem_u32(st + 2 * kTcATile), &tm_bhi, k, 0, bar);
                    tma_load_2d(smem_u32(st + 2 * kTcATile + b_tile), &tm_blo, k, 0, bar);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            uint32_t g = 0, j = 0;
            for (int t = blockIdx.x; t < items && ok; t += gridDim.x, ++j) {
                int r0, z, c0, nk;
                item_range(t, r0, z, c0, nk);
                const uint32_t b = j & 1u;
                // the epilogue has drained this accumulator's previous item
                if (j >= 2) ok = mbar_wait(smem_u32(&s_acce[b]), ((j >> 1) + 1) & 1u, err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t acc = tmem + b * acc_cols;
                for (int i = 0; i < nk; ++i, ++g) {
                    const uint32_t s = g % kTcStages;
                    ok = mbar_wait(smem_u32(&s_full[s]), (g / kTcStages) & 1u, err);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_hi = smem_u32(smem + (size_t)s * stage_bytes);
                    const uint32_t a_lo = a_hi + kTcATile, b_hi = a_hi + 2 * kTcATile, b_lo = b_hi + b_tile;
#pragma unroll
                    for (int kk = 0; kk < kTcKc / 8; ++kk) {   // K = 8 TF32 = 32 bytes per MMA
                        const uint32_t off = 32u * kk;
                        tc_mma(acc, tc_sdesc(a_lo + off), tc_sdesc(b_hi + off), idesc, (i > 0 || kk > 0) ? 1u : 0u);
                        tc_mma(acc, tc_sdesc(a_hi + off), tc_sdesc(b_lo + off), idesc, 1u);
                        tc_mma(acc, tc_sdesc(a_hi + off), tc_sdesc(b_hi + off), idesc, 1u);
                    }
                    tc_commit(smem_u32(&s_empty[s]));   // the stage is free once these MMAs have read it
                }
                tc_commit(smem_u32(&s_accf[b]));        // the item's accumulator is complete
            }
        }
        __syncwarp();
    } else {
        // epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, rows r0 + 32 (w % 4) + lane
        const int q = warp & 3;
        uint32_t j = 0;
        for (int t = blockIdx.x; t < items; t += gridDim.x, ++j) {
            int r0, z, c0, nk;
            item_range(t, r0, z, c0, nk);
            const uint32_t b = j & 1u;
            bool acc_ok = mbar_wait(smem_u32(&s_accf[b]), (j >> 1) & 1u, err);
            acc_ok = __all_sync(0xffffffffu, acc_ok);   // tcgen05.ld is warp-collective
            if (!acc_ok) break;
            tc_fence_after();
            const int64_t row = (int64_t)r0 + 32 * q + lane;
            float *out = P + ((int64_t)z * n + row) * c;
            const uint32_t base = tmem + b * acc_cols + ((uint32_t)(32 * q) << 16);
            for (int col0 = 0; col0 < npad; col0 += 16) {
                float v[16];
                tc_ld16(base + (uint32_t)col0, v);
                if (row < n) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (col0 + i < c) out[col0 + i] = v[i];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&s_acce[b]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// The full symmetric matrix from the upper-triangle table, split into TF32
// hi / lo parts: one CTA per 64 x 64 tile on or above the diagonal reads it
// once (16-byte loads) and writes it and its mirror below the diagonal
// (16-byte stores, the mirror through a shared-memory transpose); a diagonal
// tile takes its lower half from its upper half.
__device__ __forceinline__ void split_store4(float *hi, float *lo, float4 v) {
    float4 h;
    h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
    h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
    h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
    h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
    *reinterpret_cast<float4 *>(hi) = h;
    *reinterpret_cast<float4 *>(lo) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

__global__ void __launch_bounds__(256) table_split_kernel(const float *__restrict__ T, int64_t ld,
                                                          float *__restrict__ hi, float *__restrict__ lo) {
    __shared__ float S[64][65];
    const int bi = blockIdx.y, bk = blockIdx.x;
    if (bi > bk) return;   // the mirror of an upper tile is written by that tile's CTA
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)bi * 64, c0 = (int64_t)bk * 64;
    for (int y = ty; y < 64; y += 16) {
        const float4 v = *reinterpret_cast<const float4 *>(T + (r0 + y) * ld + c0 + 4 * tx);
        S[y][4 * tx] = v.x;
        S[y][4 * tx + 1] = v.y;
        S[y][4 * tx + 2] = v.z;
        S[y][4 * tx + 3] = v.w;
    }
    __syncthreads();
    if (bi == bk) {   // only the upper half of a diagonal tile is in the table
        for (int e = threadIdx.x; e < 64 * 64; e += 256) {
            const int y = e >> 6, x = e & 63;
            if (y > x) S[y][x] = S[x][y];
        }
        __syncthreads();
    }
    for (int y = ty; y < 64; y += 16) {
        const int64_t at = (r0 + y) * ld + c0 + 4 * tx;
        split_store4(hi + at, lo + at, make_float4(S[y][4 * tx], S[y][4 * tx + 1], S[y][4 * tx + 2], S[y][4 * tx + 3]));
    }
    if (bi == bk) return;
    for (int y = ty; y < 64; y += 16) {   // row c0 + y of the mirror tile = column y of this one
        const int64_t at = (c0 + y) * ld + r0 + 4 * tx;
        split_store4(hi + at, lo + at,
                     make_float4(S[4 * tx][y], S[4 * tx + 1][y], S[4 * tx + 2][y], S[4 * tx + 3][y]));
    }
}

// X (n x c, row-major) transposed into N_pad x n_pad hi / lo parts, zero beyond.
__global__ void __launch_bounds__(256) x_split_kernel(const float *__restrict__ X, int64_t ldx, int64_t n, int c,
                                                      int npad, int64_t npk, float *__restrict__ hi,
                                                      float *__restrict__ lo) {
    __shared__ float S[32][33];
    const int bj = blockIdx.y, bk = blockIdx.x;   // 32 columns of X x 32 rows of X
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int y = ty; y < 32; y += 8) {
        const int64_t k = (int64_t)bk * 32 + y;
        const int j = bj * 32 + tx;
        S[y][tx] = (k < n && j < c) ? X[k * ldx + j] : 0.f;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int64_t j = (int64_t)bj * 32 + y, k = (int64_t)bk * 32 + tx;
        if (j >= npad) break;
        const float v = S[tx][y];
        const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        hi[j * npk + k] = h;
        lo[j * npk + k] = v - h;
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiled *fn) {
    // resolved once per process (thread-safe static initialisation)
    static const std::pair<EncodeTiled, cudaError_t> entry = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e == cudaSuccess && (q != cudaDriverEntryPointSuccess || !p)) e = cudaErrorSymbolNotFound;
        return std::make_pair(reinterpret_cast<EncodeTiled>(p), e);
    }();
    if (entry.second != cudaSuccess)
        return cuda_fail("cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled)", entry.second, __FILE__, __LINE__);
    *fn = entry.first;
    return 0;
}

// 2-D FP32 tensor map of a rows x cols row-major array (row pitch `pitch`
// elements), boxes of 32 columns x box_rows rows in the 128-byte swizzle.
int encode_map(CUtensorMap *m, const float *base, int64_t rows, int64_t cols, int64_t pitch, int box_rows) {
    EncodeTiled enc = nullptr;
    LNE_TRY(get_encoder(&enc));
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTcKc, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LNE_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return 0;
}

}  // namespace

int dense_tc_prepare(Workspace &ws, const float *T, int64_t ld, const float **hi, const float **lo,
                     cudaStream_t st) {
    if (ld % 64 != 0) return fail(LNE_ERR_INVALID, "dense table leading dimension must be a multiple of 64");
    float *h = nullptr, *l = nullptr;
    LNE_TRY(ws.get("tc.ahi", (size_t)(ld * ld), &h));
    LNE_TRY(ws.get("tc.alo", (size_t)(ld * ld), &l));
    LNE_TRACE("table_split", st);
    const dim3 grid((unsigned)(ld / 64), (unsigned)(ld / 64));
    table_split_kernel<<<grid, 256, 0, st>>>(T, ld, h, l);
    LNE_LAUNCH_CHECK();
    *hi = h;
    *lo = l;
    return 0;
}

int dense_tc_spmm(Workspace &ws, const float *Ahi, const float *Alo, int64_t ld, int64_t n, const float *X,
                  int64_t ldx, int c, float *Y, int64_t ldy, cudaStream_t st) {
    if (n <= 0) return 0;
    if (c < 1 || c > 160) return fail(LNE_ERR_UNSUPPORTED, "dense-table product supports 1..160 columns");
    if (ld % 64 != 0 || ld < n) return fail(LNE_ERR_INVALID, "bad dense table leading dimension");
    const int npad = tc_npad(c);
    float *bhi = nullptr, *blo = nullptr;
    LNE_TRY(ws.get("tc.bhi", (size_t)npad * ld, &bhi));
    LNE_TRY(ws.get("tc.blo", (size_t)npad * ld, &blo));
    {
        LNE_TRACE("x_split", st);
        const dim3 grid((unsigned)(ld / 32), (unsigned)(npad + 31) / 32);
        x_split_kernel<<<grid, 256, 0, st>>>(X, ldx, n, c, npad, ld, bhi, blo);
        LNE_LAUNCH_CHECK();
    }
    CUtensorMap m_ahi, m_alo, m_bhi, m_blo;
    LNE_TRY(encode_map(&m_ahi, Ahi, ld, ld, ld, kTcRows));
    LNE_TRY(encode_map(&m_alo, Alo, ld, ld, ld, kTcRows));
    LNE_TRY(encode_map(&m_bhi, bhi, npad, ld, ld, npad));
    LNE_TRY(encode_map(&m_blo, blo, npad, ld, ld, npad));
    const int smem = tc_smem_bytes(npad);
    LNE_CUDA_TRY(cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int rb = (int)ceil_div(n, (int64_t)kTcRows);
    const int nchunks = (int)(ld / kTcKc);
    // k-slices: row blocks x slices, as items of the persistent CTAs, give every
    // SM the same number of items (slices of equal length)
    const int64_t slots = num_sms();
    int ks = 1;
    double best = 1e300;
    for (int cand = 1; cand <= 16 && cand <= nchunks; ++cand) {
        const double t = (double)ceil_div((int64_t)rb * cand, slots) / cand;
        if (t < best - 1e-12) {
            best = t;
            ks = cand;
        }
    }
    const int slice_chunks = (int)ceil_div(nchunks, ks);
    ks = (int)ceil_div(nchunks, slice_chunks);
    const int items = rb * ks;
    float *part = nullptr;
    int *status = nullptr;
    LNE_TRY(ws.get("tc.part", (size_t)ks * n * c, &part));
    LNE_TRY(device_status(ws, &status, st));
    {
        LNE_TRACE("dense_tc", st);
        const unsigned grid = (unsigned)std::min<int64_t>(items, slots);
        dense_tc_kernel<<<grid, kTcThreads, smem, st>>>(m_ahi, m_alo, m_bhi, m_blo, n, nchunks, slice_chunks, rb,
                                                         items, npad, c, part, status + 1);
        LNE_LAUNCH_CHECK();
    }
    // a wait that expired is reported by the caller's status_check
    return slice_sum(part, ks, n, c, Y, ldy, st);
}

}  // namespace lne
