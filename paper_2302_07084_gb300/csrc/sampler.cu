// Sparsifier construction on the GPU (Sec. 5.2 of the paper, re-designed):
//
//   1. tile_counts     per-arc sample counts n_a = floor(S/2m) + Bernoulli
//                      (Algorithm 3) summed per tile of arcs; scanned
//                      into tile offsets.
//   2. walk_emit       one thread per sample: window r ~ Multinomial(s)
//                      (Algorithm 3), split sigma ~ U{0..r-1} and the
//                      two walks of PathSampling (Algorithm 1), each step
//                      x <- nbr(x)[word mod deg(x)] (Sec. 5.2). Emits the
//                      canonical pair key (min << B | max) and a shared-memory
//                      histogram of key buckets.
//   3. bucket_scatter  moves keys into their bucket's region (CTA-aggregated
//                      cursors; order inside a bucket does not matter).
//   4. bucket_reduce   one CTA per bucket counts its keys in a dense 2^15-entry
//                      shared-memory histogram and writes the distinct keys in
//                      key order with their exact counts -- the integer
//                      aggregation the paper does with a concurrent hash table.
//   5. trunclog        Eq. 1 value v = K alpha / (d_x d_y), kept iff v > 1 (an
//                      exact decision), log(v) as float32.
//   6. csr_fill/sort   symmetric CSR of the kept entries, rows sorted.
//
// For graphs whose pair space fits a dense table (n <= 65536) the counting is
// direct instead: the walk adds each sample into an n x n table of counters
// (upper triangle, fire-and-forget atomics), one pass turns counts into Eq. 1
// values in place, and 64 x 64 tiles of the symmetric matrix (the lower half
// read through a shared-memory transpose) give row counts and then the CSR in
// column order -- no key buffers, no sort.
//
// Every integer result (counts, keep decisions, CSR structure) is independent of
// scheduling, so it equals the CPU oracle bit for bit.
#include <cstring>

#include "runtime.h"

namespace lne {
namespace {

constexpr int kBucketBits = 15;                 // keys per reduce bucket = 2^15
constexpr int kMaxSmemBuckets = 12288;          // walk/scatter histogram capacity
constexpr int kWalkThreads = 128;
constexpr int kWalkWarps = kWalkThreads / 32;
constexpr int kChunk = 512;                     // samples ranked by window length at a time
static_assert(kChunk <= 2048 && kChunk % kWalkThreads == 0, "a chunk index fits the 11 low bits of a packed sample");

struct WalkArgs {
    const int64_t *indptr;
    const int32_t *indices;
    const uint4 *vinfo;           // per-vertex walk record (see build_vinfo_kernel)
    const uint4 *arcrec;          // per-arc record of the arc's head vertex
    int64_t n;
    int64_t n_arcs;
    uint32_t k0, k1;
    uint32_t base;
    uint32_t thr_frac;
    int T;
    int B;
    uint64_t thr[16];
    // derived on the host
    uint32_t rk[20];              // Philox round keys (k0 + i W0, k1 + i W1), i = 0..9
    uint32_t thr32[16];           // thresholds below 2^32, ascending
    int T_eff;                    // how many thresholds are below 2^32
    const uint8_t *rlut;          // window-length table (build_rlut_kernel), 4096 entries
    uint64_t base_magic;          // ceil(2^64 / base): s / base by a high multiply
    uint32_t rmod[17];            // barrett_mod multipliers for r = 1..16 (index r)
    // edge downsampling (NULL = off): per arc, the coin keeps a draw iff its
    // coin word < ds_thr[arc]; a kept draw weighs ds_w[arc] (2^-32 units)
    const uint64_t *ds_thr;
    const uint64_t *ds_w;
    int strat;                    // MODE 3 keys carry r - 1 in 4 low bits
    // weighted graphs (w = NULL: unweighted): arc a draws S w_a / vol samples
    // in expectation, and a step takes arc j of x with probability w_j / d_x
    // (first j with word < cum[off + j], cum = floor(2^32 prefix_j / d_x))
    const uint32_t *w;
    const uint32_t *cum;
    const uint32_t *guide;        // per arc b of x: the answer for the smallest word of bucket b
    double S, vol;
    uint32_t wmax;                // host copy of the largest weight (tile size bounds)
};

__device__ __forceinline__ uint32_t arc_count(const WalkArgs &A, int64_t arc) {
    uint32_t base = A.base, thr = A.thr_frac;
    if (A.w) {   // rate = fl(fl(S w_a) / vol): floor and Bernoulli threshold of the fraction
        const double rate = __ddiv_rn(__dmul_rn(A.S, (double)__ldg(A.w + arc)), A.vol);
        const double b = floor(rate);
        base = (uint32_t)b;
        thr = (uint32_t)floor(__dmul_rn(__dsub_rn(rate, b), 4294967296.0));
    }
    if (thr == 0) return base;
    u32x4 c = {0xFFFFFFFFu, (uint32_t)((uint64_t)arc & 0xFFFFFFFFu), (uint32_t)((uint64_t)arc >> 32),
               0xFFFFFFFFu};
    u32x4 w = philox10(c, A.k0, A.k1);
    return base + (w.x < thr ? 1u : 0u);
}

// Philox4x32-10 with precomputed round keys; each 32 x 32 -> 64 product is one
// wide multiply.
__device__ __forceinline__ u32x4 philox_rk(u32x4 c, const uint32_t *rk) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        u32x4 n;
        n.x = (uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * round];
        n.y = (uint32_t)p1;
        n.z = (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * round + 1];
        n.w = (uint32_t)p0;
        c = n;
    }
    return c;
}

// a / d for 32-bit a and d >= 1 with M = ceil(2^64 / d): the high 64 bits of
// M a are the quotient (Lemire, Kaser and Kurz, "Faster remainder by direct
// computation", 2019).
__device__ __forceinline__ uint32_t fastdiv32(uint32_t a, uint64_t M) {
    return (uint32_t)__umul64hi(M, (uint64_t)a);
}

// Per-vertex walk record {offset bits 0..31, offset bits 32..39 | degree << 8,
// m, the vertex} with m = floor(2^32 / degree) for degree >= 2, m = 2^32 - 1 for
// degree 1 (then the Barrett step below yields 0 without a special case) and
// 0 for degree 0. Degrees of 2^24 and more are marked 0xFFFFFF and read from
// indptr.
__global__ void build_vinfo_kernel(const int64_t *__restrict__ indptr, int64_t n, uint4 *__restrict__ vinfo) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t off = indptr[x];
        const int64_t deg = indptr[x + 1] - off;
        const uint32_t dfield = deg >= 0xFFFFFF ? 0xFFFFFFu : (uint32_t)deg;
        const uint32_t m = (deg >= 2 && deg < 0xFFFFFF) ? (uint32_t)((1ull << 32) / (uint64_t)deg)
                           : deg == 1 ? 0xFFFFFFFFu : 0u;
        vinfo[x] = make_uint4((uint32_t)off, (uint32_t)((off >> 32) & 0xFF) | (dfield << 8), m, (uint32_t)x);
    }
}

// Per-arc record (16 bytes): for arc p -> v, {v, v's offset bits 0..31,
// v's offset bits 32..39 | degree << 8, v's m}. A walk step reads the record of
// the arc it takes and so learns the next vertex's offset, degree and
// reciprocal in one 16-byte load: one dependent load per step.
__global__ void build_arcrec_kernel(const int32_t *__restrict__ indices, int64_t nnz, const uint4 *__restrict__ vinfo,
                                    uint4 *__restrict__ arcrec) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = indices[p];
        const uint4 r = vinfo[v];
        arcrec[p] = make_uint4((uint32_t)v, r.x, r.y, r.z);
    }
}

// Window-length table over the top 12 bits of a word: entry b holds
// r = 1 + #{i : thr_i <= b 2^20} (Algorithm 3's multinomial draw by
// thresholds), with bit 7 set when a threshold falls inside the bucket
// (b 2^20, b 2^20 + 2^20 - 1], where the draw counts thresholds itself.
__global__ void build_rlut_kernel(WalkArgs A, uint8_t *__restrict__ lut) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= 4096) return;
    const uint32_t lo = (uint32_t)b << 20, hi = lo | 0xFFFFFu;
    int r = 1;
    bool amb = false;
    for (int i = 0; i < A.T_eff; ++i) {
        r += lo >= A.thr32[i] ? 1 : 0;
        amb |= (A.thr32[i] > lo) && (A.thr32[i] <= hi);
    }
    lut[b] = (uint8_t)(r | (amb ? 0x80 : 0));
}

// Weighted graphs: per arc j of vertex x the walk threshold
// floor(2^32 (w_0 + .. + w_j) / d_x) (exact: prefix < 2^31, so prefix 2^32
// fits 64 bits). A warp per vertex; its lanes scan the prefix in chunks of 32.
__global__ void build_cum_kernel(const int64_t *__restrict__ indptr, const uint32_t *__restrict__ w,
                                 const uint32_t *__restrict__ wdeg, int64_t n, uint32_t *__restrict__ cum) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
        const int64_t a0 = indptr[x], a1 = indptr[x + 1];
        const uint64_t d = __ldg(wdeg + x);
        uint64_t carry = 0;
        for (int64_t base = a0; base < a1; base += 32) {
            const int64_t a = base + lane;
            uint64_t v = a < a1 ? (uint64_t)__ldg(w + a) : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            const uint64_t prefix = carry + v;
            // the last arc's threshold would be 2^32: it is never read
            const uint64_t t = (prefix << 32) / d;
            if (a < a1) cum[a] = t > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)t;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// Guide of the weighted step: for bucket b of vertex x (words w with
// floor(w deg / 2^32) = b) the answer for the bucket's smallest word
// ceil(b 2^32 / deg); the inverse CDF is monotone in w, so a word of bucket b
// takes an arc between guide[b] and guide[b + 1] (or the last arc).
__global__ void build_guide_kernel(const int64_t *__restrict__ indptr, const uint32_t *__restrict__ cum, int64_t n,
                                   uint32_t *__restrict__ guide) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
        const int64_t a0 = indptr[x];
        const uint64_t deg = (uint64_t)(indptr[x + 1] - a0);
        for (uint64_t b = lane; b < deg; b += 32) {
            const uint64_t w0 = ((b << 32) + deg - 1) / deg;   // ceil(b 2^32 / deg) < 2^32
            uint32_t lo = 0, hi = (uint32_t)deg - 1;           // first j with w0 < cum[j], else the last
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (w0 < (uint64_t)cum[a0 + mid]) hi = mid; else lo = mid + 1;
            }
            guide[a0 + (int64_t)b] = lo;
        }
    }
}

__device__ __forceinline__ int32_t arc_source(const int64_t *__restrict__ indptr, int64_t n,
                                              int64_t a) {
    int64_t lo = 0, hi = n;   // indptr[lo] <= a < indptr[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(indptr + mid) <= a) lo = mid; else hi = mid;
    }
    return (int32_t)lo;
}

// Walk state: the current vertex and its walk record.
struct WalkCur {
    int32_t x;
    uint32_t off_lo, hidg, m;   // offset bits 0..31, offset bits 32..39 | degree << 8, floor(2^32 / degree)
};

__device__ __forceinline__ WalkCur walk_start(const WalkArgs &A, int32_t x) {
    const uint4 r = __ldg(A.vinfo + x);
    return WalkCur{x, r.x, r.y, r.z};
}

// w mod d for 2 <= d < 2^24 with m = floor(2^32 / d) (Barrett reduction):
// q = floor(w m / 2^32) is the true quotient or one less, so one conditional
// subtraction finishes the remainder. d = 1 takes m = 2^32 - 1 (q = w - 1 for
// w >= 1, then one subtraction; q = 0 for w = 0): the remainder is 0.
__device__ __forceinline__ uint32_t barrett_mod(uint32_t w, uint32_t m, uint32_t d) {
    const uint32_t q = __umulhi(w, m);
    uint32_t r = w - q * d;
    return r >= d ? r - d : r;
}

// One walk step: x <- nbr(x)[w mod deg(x)] (Sec. 5.2), reading the taken
// arc's record. GEN: the variant that also handles weighted graphs.
template <bool GEN>
__device__ __forceinline__ void walk_step(const WalkArgs &A, WalkCur &c, uint32_t w) {
    uint32_t deg = c.hidg >> 8;
    const int64_t off = (int64_t)c.off_lo | ((int64_t)(c.hidg & 0xFF) << 32);
    if (deg == 0) return;   // only on graphs that break the contract
    uint32_t j;
    if (deg == 0xFFFFFFu) deg = (uint32_t)(__ldg(A.indptr + c.x + 1) - __ldg(A.indptr + c.x));
    if (GEN && A.cum) {
        // weighted: inverse CDF over the vertex's thresholds (the last is
        // 2^32). The word's bucket b = floor(w deg / 2^32) brackets the
        // answer between the guides of buckets b and b + 1, usually one arc.
        const uint32_t b = __umulhi(w, deg);
        uint32_t lo = __ldg(A.guide + off + b);
        uint32_t hi = b + 1 < deg ? __ldg(A.guide + off + b + 1) : deg - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (w < __ldg(A.cum + off + mid)) hi = mid; else lo = mid + 1;
        }
        j = lo;
    } else if ((c.hidg >> 8) == 0xFFFFFFu) {
        j = w % deg;
    } else {
        j = deg == 1 ? 0u : barrett_mod(w, c.m, deg);
    }
    const uint4 ra = __ldg(A.arcrec + off + j);
    c = WalkCur{(int32_t)ra.x, ra.y, ra.z, ra.w};
}

// One PathSampling draw (Algorithm 1) of sample j on arc a = (u -> v), as a
// small state machine. Words of counter
// (j, a_lo, a_hi, blk): word 0 picks the window r (Algorithm 3), word 1 the
// split sigma, word 2 is the reserved coin, words 3.. drive the walk steps,
// sigma from u first, then r - 1 - sigma from v.
struct Draw {
    uint32_t j, c1, c2;
    int steps, sigma;
    u32x4 nb;            // current Philox block
    WalkCur cur;
    int32_t v, uend;
};

// Block 0 of the sample's stream: the window r, the split sigma, the
// downsampling coin and word 3.
__device__ __forceinline__ void draw_head(const WalkArgs &A, const uint8_t *__restrict__ rlut,
                                          const uint32_t *__restrict__ rmod, int64_t arc, uint32_t j, int *r_out,
                                          int *sigma_out, uint32_t *coin_out, uint32_t *w3_out) {
    const u32x4 b0 = philox_rk(u32x4{j, (uint32_t)((uint64_t)arc & 0xFFFFFFFFu), (uint32_t)((uint64_t)arc >> 32), 0u},
                               A.rk);
    // r = 1 + #{i : thr_i <= w0}; the table gives it unless a threshold falls
    // inside the word's 2^20-wide bucket
    const uint8_t e = rlut[b0.x >> 20];
    int r = e & 31;
    if (e & 0x80) {
        r = 1;
        for (int i = 0; i < A.T_eff; ++i) r += b0.x >= A.thr32[i] ? 1 : 0;
    }
    *r_out = r;
    *sigma_out = (int)barrett_mod(b0.y, rmod[r], (uint32_t)r);
    *coin_out = b0.z;
    *w3_out = b0.w;
}

// The draw's walk state from its head.
__device__ __forceinline__ void draw_begin(const WalkArgs &A, int64_t arc, uint32_t j, int r, int sigma, uint32_t w3,
                                           int32_t u, int32_t v, Draw &d) {
    d.j = j;
    d.c1 = (uint32_t)((uint64_t)arc & 0xFFFFFFFFu);
    d.c2 = (uint32_t)((uint64_t)arc >> 32);
    d.nb = u32x4{0u, 0u, 0u, w3};
    d.steps = r - 1;
    d.sigma = sigma;
    d.v = v;
    d.uend = u;
    d.cur = walk_start(A, sigma == 0 && d.steps > 0 ? v : u);
}

// Step k (word 3 + k) of the draw, if it has one.
template <int K, bool GEN>
__device__ __forceinline__ void draw_step(const WalkArgs &A, Draw &d) {
    if (K >= d.steps) return;
    constexpr int widx = 3 + K;
    if ((widx & 3) == 0) d.nb = philox_rk(u32x4{d.j, d.c1, d.c2, (uint32_t)(widx >> 2)}, A.rk);
    const uint32_t w = (widx & 3) == 0 ? d.nb.x : (widx & 3) == 1 ? d.nb.y : (widx & 3) == 2 ? d.nb.z : d.nb.w;
    walk_step<GEN>(A, d.cur, w);
    if (K + 1 == d.sigma && K + 1 < d.steps) {   // u side done: continue from v
        d.uend = d.cur.x;
        d.cur = walk_start(A, d.v);
    }
}

__device__ __forceinline__ void draw_end(const Draw &d, int32_t *pu, int32_t *pv) {
    if (d.sigma >= d.steps) {   // every step on the u side (or none at all)
        *pu = d.steps > 0 ? d.cur.x : d.uend;
        *pv = d.v;
    } else {
        *pu = d.uend;
        *pv = d.cur.x;
    }
}

template <int K, bool GEN>
struct StepAll {
    __device__ __forceinline__ static void run(const WalkArgs &A, Draw &a, Draw &b, int kmax) {
        if (K >= kmax) return;
        draw_step<K, GEN>(A, a);
        draw_step<K, GEN>(A, b);
        StepAll<K + 1, GEN>::run(A, a, b, kmax);
    }
};
template <bool GEN>
struct StepAll<15, GEN> {
    __device__ __forceinline__ static void run(const WalkArgs &, Draw &, Draw &, int) {}
};

// In-place exclusive scan of s[0..n) in shared memory by one CTA; returns total.
template <int BLOCK>
__device__ uint32_t block_exclusive_scan(uint32_t *s, int n) {
    __shared__ uint32_t warp_tot[BLOCK / 32];
    __shared__ uint32_t total_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + BLOCK - 1) / BLOCK;
    const int i0 = tid * per;
    uint32_t local = 0;
    for (int j = 0; j < per; ++j)
        if (i0 + j < n) local += s[i0 + j];
    uint32_t x = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < BLOCK / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < BLOCK / 32) warp_tot[lane] = w;
        if (lane == BLOCK / 32 - 1) total_s = w;
    }
    __syncthreads();
    uint32_t run = (warp > 0 ? warp_tot[warp - 1] : 0) + x - local;
    for (int j = 0; j < per; ++j) {
        if (i0 + j < n) {
            uint32_t t = s[i0 + j];
            s[i0 + j] = run;
            run += t;
        }
    }
    __syncthreads();
    uint32_t t = total_s;
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kWalkThreads) tile_counts_kernel(WalkArgs A, int64_t a_begin,
                                                                   int64_t a_end, int tile_arcs,
                                                                   uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t red[kWalkThreads / 32];
    const int64_t a0 = a_begin + (int64_t)blockIdx.x * tile_arcs;
    const int64_t a1 = min(a0 + tile_arcs, a_end);
    uint32_t c = 0;
    for (int64_t a = a0 + threadIdx.x; a < a1; a += kWalkThreads) c += arc_count(A, a);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kWalkThreads / 32; ++w) t += red[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// MODE 0: write ordered endpoint pairs (u1, v1). MODE 1: write canonical keys
// and count key buckets. MODE 2: add the pair into the dense count table
// table[x * ld + y] (x <= y); `keys` is the table, ld = nb_smem. MODE 3: write
// the canonical key at the sample's position (no counting). GEN = false is the
// variant for unweighted graphs without downsampling or window strata (the
// checks for those compiled out); GEN = true handles everything.
template <typename KeyT, int MODE, bool GEN>
__global__ void __launch_bounds__(kWalkThreads, MODE == 2 ? 10 : 8) walk_emit_kernel(
    WalkArgs A, int64_t a_begin, int64_t a_end, int tile_arcs, const int64_t *__restrict__ tile_off,
    KeyT *__restrict__ keys, int32_t *__restrict__ u1, int32_t *__restrict__ v1,
    uint32_t *__restrict__ bucket_cnt, int nb_smem) {
    extern __shared__ uint32_t smem[];
    __shared__ __align__(16) uint8_t s_rlut[4096];
    __shared__ uint32_t s_rmod[17];
    // s_upack: per chunk sample its index, r, sigma and rank; s_uw3: its word 3
    // (phase 2 reads it through the index, so no permuted copy takes shared
    // memory that the L1 cache can use); s_pack: the samples in r order
    __shared__ uint32_t s_upack[kChunk], s_uw3[kChunk], s_pack[kChunk];
    __shared__ uint16_t s_lo[kChunk];   // arc within the tile of each chunk sample (phase 1 -> phase 2)
    __shared__ uint32_t s_wcnt[17 * kWalkWarps];

    uint32_t *s_off = smem;                                      // tile_arcs + 1
    int32_t *s_src = reinterpret_cast<int32_t *>(s_off + tile_arcs + 1);
    int32_t *s_dst = s_src + tile_arcs;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_dst + tile_arcs);
    const int tid = threadIdx.x;
    // window-length table (built once per launch)
    for (int b = tid; b < 4096 / 16; b += kWalkThreads)
        reinterpret_cast<uint4 *>(s_rlut)[b] = __ldg(reinterpret_cast<const uint4 *>(A.rlut) + b);
    if (tid < 17) s_rmod[tid] = A.rmod[tid];
    const int64_t a0 = a_begin + (int64_t)blockIdx.x * tile_arcs;
    const int na = (int)imin64(tile_arcs, a_end - a0);
    if (MODE == 1 && nb_smem > 0)
        for (int i = tid; i < nb_smem; i += kWalkThreads) s_hist[i] = 0;
    for (int i = tid; i < na; i += kWalkThreads) {
        s_off[i] = arc_count(A, a0 + i);
        s_src[i] = arc_source(A.indptr, A.n, a0 + i);
        s_dst[i] = __ldg(A.indices + a0 + i);
    }
    __syncthreads();
    const uint32_t total = block_exclusive_scan<kWalkThreads>(s_off, na);
    if (tid == 0) s_off[na] = total;
    __syncthreads();
    const int64_t out0 = tile_off ? tile_off[blockIdx.x] : 0;
    const bool uniform = A.thr_frac == 0 && !(GEN && A.w);
    // sample s of the tile -> (arc within the tile, sample index j on that arc)
    auto locate = [&](uint32_t s, int &lo, uint32_t &j) {
        if (uniform) {
            // every arc draws `base` samples (ceil(2^64 / 1) wraps to 0, hence the case)
            lo = A.base == 1 ? (int)s : (int)fastdiv32(s, A.base_magic);
        } else {
            lo = 0;
            int hi = na;   // s_off[lo] <= s < s_off[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] <= s) lo = mid; else hi = mid;
            }
        }
        j = s - s_off[lo];
    };
    // a draw the downsampling coin drops leaves a marker at its position:
    // (-1, -1) for raw draws, a key above every pair key for the sort
    auto emit_dropped = [&](uint32_t s, int64_t arc) {
        if (MODE == 0) {
            u1[out0 + s] = -1;
            v1[out0 + s] = -1;
        } else if (MODE == 3) {
            keys[out0 + s] = ~(KeyT)0;
            if (u1) reinterpret_cast<uint32_t *>(u1)[out0 + s] = (uint32_t)arc;
        }
    };
    auto emit = [&](uint32_t s, int64_t arc, int32_t pu, int32_t pv, uint32_t r) {
        if (MODE == 0) {
            u1[out0 + s] = pu;
            v1[out0 + s] = pv;
        } else if (MODE == 2) {
            const uint32_t x = (uint32_t)min(pu, pv), y = (uint32_t)max(pu, pv);
            const size_t at = (size_t)x * (uint32_t)nb_smem + y;
            if (sizeof(KeyT) == 8)   // downsampled: weights, 2^-32 fixed point
                atomicAdd(reinterpret_cast<unsigned long long *>(keys) + at, (unsigned long long)A.ds_w[arc]);
            else
                atomicAdd(reinterpret_cast<uint32_t *>(keys) + at, 1u);
        } else if (MODE == 3) {
            const uint32_t x = (uint32_t)min(pu, pv), y = (uint32_t)max(pu, pv);
            const KeyT key = ((KeyT)x << A.B) | (KeyT)y;
            keys[out0 + s] = (GEN && A.strat) ? (key << 4) | (KeyT)(r - 1u) : key;
            if (u1) reinterpret_cast<uint32_t *>(u1)[out0 + s] = (uint32_t)arc;   // the draw's arc
        } else {
            const uint32_t x = (uint32_t)min(pu, pv), y = (uint32_t)max(pu, pv);
            const KeyT key = ((KeyT)x << A.B) | (KeyT)y;
            keys[out0 + s] = key;
            const uint32_t b = (uint32_t)(key >> kBucketBits);
            if (nb_smem > 0) atomicAdd(&s_hist[b], 1u);
            else atomicAdd(&bucket_cnt[b], 1u);
        }
    };
    // Chunks of kChunk samples. Phase 1 draws each sample's head and ranks the
    // chunk by window length r: __match_any groups equal r within a warp, the
    // group leader adds to the warp's row of a (warp x r) histogram, and one
    // scan turns the histogram into positions. Phase 2 walks the samples in
    // r order, so the lanes of a warp take the same number of steps.
    const int lane = tid & 31, warp = tid >> 5;
    for (uint32_t cb = 0; cb < total; cb += kChunk) {
        const uint32_t cn = min((uint32_t)kChunk, total - cb);
        for (int e = tid; e < 17 * kWalkWarps; e += kWalkThreads) s_wcnt[e] = 0;
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < kChunk / kWalkThreads; ++t) {
            const uint32_t idx = (uint32_t)t * kWalkThreads + tid;
            int r = 0, sg = 0;
            uint32_t w3 = 0;
            if (idx < cn) {
                int lo;
                uint32_t j, coin;
                locate(cb + idx, lo, j);
                s_lo[idx] = (uint16_t)lo;
                draw_head(A, s_rlut, s_rmod, a0 + lo, j, &r, &sg, &coin, &w3);
                // edge downsampling (Algorithm 3): the draw walks only if its coin comes up heads
                if (GEN && A.ds_thr && (uint64_t)coin >= __ldg(A.ds_thr + a0 + lo)) {
                    emit_dropped(cb + idx, a0 + lo);
                    r = 0;
                }
            }
            const unsigned grp = __match_any_sync(0xffffffffu, r);
            const int leader = __ffs(grp) - 1;
            uint32_t base = 0;
            if (lane == leader) {
                base = s_wcnt[r * kWalkWarps + warp];
                s_wcnt[r * kWalkWarps + warp] = base + (uint32_t)__popc(grp);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            const uint32_t lpos = base + (uint32_t)__popc(grp & ((1u << lane) - 1u));
            s_upack[idx] = idx | ((uint32_t)r << 11) | ((uint32_t)sg << 16) | (lpos << 20);
            s_uw3[idx] = w3;
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive scan over (r, warp) in r-major order; r = 0 marks empty slots
            uint32_t carry = 0;
            for (int e0 = 0; e0 < 17 * kWalkWarps; e0 += 32) {
                const int e = e0 + lane;
                const uint32_t v = e < 17 * kWalkWarps ? s_wcnt[e] : 0u;
                uint32_t x = v;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
                    if (lane >= off) x += y;
                }
                if (e < 17 * kWalkWarps) s_wcnt[e] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < kChunk / kWalkThreads; ++t) {
            const uint32_t idx = (uint32_t)t * kWalkThreads + tid;
            const uint32_t pk = s_upack[idx];
            const uint32_t r = (pk >> 11) & 31;
            const uint32_t pos = s_wcnt[r * kWalkWarps + warp] + (pk >> 20);
            s_pack[pos] = pk;
        }
        __syncthreads();
        // empty slots (r = 0) sort first: skip them. Two draws per thread,
        // interleaved step by step (same r in a warp, two chains in flight).
        const uint32_t first = s_wcnt[1 * kWalkWarps];
        for (uint32_t q0 = first + tid; q0 < kChunk; q0 += 2 * kWalkThreads) {
            const uint32_t q1 = q0 + kWalkThreads;
            const bool has1 = q1 < kChunk;
            const uint32_t pk0 = s_pack[q0], pk1 = s_pack[has1 ? q1 : q0];
            const uint32_t s0 = cb + (pk0 & 0x7FFu), s1 = cb + (pk1 & 0x7FFu);
            int lo0, lo1;
            uint32_t j0, j1;
            lo0 = s_lo[pk0 & 0x7FFu];
            lo1 = s_lo[pk1 & 0x7FFu];
            j0 = s0 - s_off[lo0];
            j1 = s1 - s_off[lo1];
            Draw d0, d1;
            draw_begin(A, a0 + lo0, j0, (int)((pk0 >> 11) & 31), (int)((pk0 >> 16) & 15), s_uw3[pk0 & 0x7FFu], s_src[lo0],
                       s_dst[lo0], d0);
            draw_begin(A, a0 + lo1, j1, (int)((pk1 >> 11) & 31), (int)((pk1 >> 16) & 15), s_uw3[pk1 & 0x7FFu],
                       s_src[lo1], s_dst[lo1], d1);
            if (!has1) d1.steps = 0;
            StepAll<0, GEN>::run(A, d0, d1, max(d0.steps, d1.steps));
            int32_t pu, pv;
            draw_end(d0, &pu, &pv);
            emit(s0, a0 + lo0, pu, pv, (pk0 >> 11) & 31);
            if (has1) {
                draw_end(d1, &pu, &pv);
                emit(s1, a0 + lo1, pu, pv, (pk1 >> 11) & 31);
            }
        }
        __syncthreads();
    }
    if (MODE == 1 && nb_smem > 0) {
        __syncthreads();
        for (int i = tid; i < nb_smem; i += kWalkThreads) {
            uint32_t c = s_hist[i];
            if (c) atomicAdd(&bucket_cnt[i], c);
        }
    }
}

// ---------------------------------------------------------------------------
// The dense-table walk of unweighted graphs without downsampling or window
// strata (the benchmark's case). Same draws as walk_emit_kernel<.., 2, false>
// (Algorithms 1 and 3, the same Philox words), organised for fewer
// instructions and less DRAM traffic per draw:
//
// * each warp works alone on batches of kTabBatch consecutive samples of the
//   CTA's arc tile: it draws the heads (block 0: r, sigma, word 3), ranks the
//   batch by window length r in warp-private shared memory (__match_any
//   groups, one 17-bin scan), then walks the batch in r order with two draws
//   per lane taken from adjacent ranked positions, so a lane's two chains and
//   the lanes of a warp take nearly the same number of steps; no CTA barrier
//   after the tile set-up;
// * the target vertex's record is loaded with the source's when a draw
//   starts, so switching from the u side to the v side is a register move;
// * n <= 65536: arc offsets fit 32 bits and degrees 16, so a step is a
//   Barrett reduction, one 32-bit add and one 16-byte load;
// * counts go into narrow counters packed 32 / BITS to a 32-bit word (8 bits:
//   a quarter of the table's bytes, so it stays in L2): every increment is a
//   returning atomic add, and the rare add that wraps a field records the wrap
//   (and those of the fields its carry runs into) in the 32-bit table;
//   table_decode_kernel turns fields and wraps into exact 32-bit counts.
// ---------------------------------------------------------------------------
constexpr int kTabThreads = 128;
constexpr int kTabWarps = kTabThreads / 32;
constexpr int kTabBatch = 256;
constexpr int kTabMaxTileArcs = 128;   // arcs per CTA tile (their walk records: 32 B each in shared memory)
constexpr int kTabMinBlocks = 9;       // CTAs per SM (56 registers a thread; 10 CTAs: 48 with spills, 1% slower)
constexpr int kTabBits = 8;            // bits per packed counter (measured: 8 bits 12.6 ms, 16 bits 13.3 ms)
static_assert(kTabBatch == 256, "ranks and batch indices are packed in 8 bits");

struct TabDraw {
    uint32_t j, arc;            // Philox counter words 0 and 1 (arc < 2^32)
    int steps, sigma;
    u32x4 nb;                   // current Philox block
    uint32_t cx, coff, chd, cm; // current vertex: id, arc offset, degree << 8, Barrett m
    uint32_t v, voff, vhd, vm;  // the arc's target and its record
    uint32_t uend;
};

// ru, rv: the walk records of the arc's source u and target v (vertex in .w).
__device__ __forceinline__ void tab_begin(uint32_t arc, uint32_t j, int r, int sigma, uint32_t w3, uint4 ru,
                                          uint4 rv, TabDraw &d) {
    d.j = j;
    d.arc = arc;
    d.steps = r - 1;
    d.sigma = sigma;
    d.nb = u32x4{0u, 0u, 0u, w3};
    d.v = rv.w;
    d.voff = rv.x;
    d.vhd = rv.y;
    d.vm = rv.z;
    d.uend = ru.w;
    const bool from_v = sigma == 0 && d.steps > 0;
    d.cx = from_v ? rv.w : ru.w;
    d.coff = from_v ? rv.x : ru.x;
    d.chd = from_v ? rv.y : ru.y;
    d.cm = from_v ? rv.z : ru.z;
}

// Step K (word 3 + K) of the draw, if it has one.
template <int K>
__device__ __forceinline__ void tab_step(const WalkArgs &A, TabDraw &d) {
    if (K >= d.steps) return;
    constexpr int widx = 3 + K;
    if ((widx & 3) == 0) d.nb = philox_rk(u32x4{d.j, d.arc, 0u, (uint32_t)(widx >> 2)}, A.rk);
    const uint32_t w = (widx & 3) == 0 ? d.nb.x : (widx & 3) == 1 ? d.nb.y : (widx & 3) == 2 ? d.nb.z : d.nb.w;
    const uint32_t deg = d.chd >> 8;
    if (deg != 0) {   // degree 0 only on graphs that break the symmetry contract: stay
        // w mod deg by Barrett (m = floor(2^32 / deg), 2^32 - 1 for deg = 1):
        // the estimate is the remainder or the remainder + deg
        const uint32_t q = __umulhi(w, d.cm);
        const uint32_t rr = w - q * deg;
        const uint32_t jj = min(rr, rr - deg);
        const uint4 ra = __ldg(A.arcrec + (d.coff + jj));
        d.cx = ra.x;
        d.coff = ra.y;
        d.chd = ra.z;
        d.cm = ra.w;
    }
    if (K + 1 == d.sigma && K + 1 < d.steps) {   // u side done: continue from v
        d.uend = d.cx;
        d.cx = d.v;
        d.coff = d.voff;
        d.chd = d.vhd;
        d.cm = d.vm;
    }
}

template <int K>
struct TabSteps {
    __device__ __forceinline__ static void run(const WalkArgs &A, TabDraw &a, TabDraw &b, int kmax) {
        if (K >= kmax) return;
        tab_step<K>(A, a);
        tab_step<K>(A, b);
        TabSteps<K + 1>::run(A, a, b, kmax);
    }
};
template <>
struct TabSteps<15> {
    __device__ __forceinline__ static void run(const WalkArgs &, TabDraw &, TabDraw &, int) {}
};

__device__ __forceinline__ void tab_end(const TabDraw &d, uint32_t *x, uint32_t *y) {
    uint32_t pu, pv;
    if (d.sigma >= d.steps) {   // every step on the u side (or none at all)
        pu = d.steps > 0 ? d.cx : d.uend;
        pv = d.v;
    } else {
        pu = d.uend;
        pv = d.cx;
    }
    *x = min(pu, pv);
    *y = max(pu, pv);
}

// Packed narrow counters: 32 / BITS counters per 32-bit word, counter i in
// bits [BITS (i mod P), BITS (i mod P) + BITS) of word i / P.
template <int BITS>
struct TabPack {
    static constexpr int P = 32 / BITS;
    static constexpr uint32_t mask = (1u << BITS) - 1u;
};

// Counts one draw of counter `at` (= x ld + y) into the packed table; returns
// the word's previous value for tab_wraps (checked later, so that the atomic's
// round trip overlaps the next draws' walks).
template <int BITS>
__device__ __forceinline__ uint32_t tab_count(uint32_t *__restrict__ tp, uint32_t at) {
    constexpr int P = TabPack<BITS>::P;
    return atomicAdd(tp + at / P, 1u << (BITS * (at % P)));
}

// Records the wraps caused by the increment of counter `at` that found `old`:
// the counter's field wraps when it held all ones, its carry then moves into
// the next field of the word, which wraps in turn if it held all ones, and so
// on (a carry out of the word's top bit is lost). carry[i] counts the wraps of
// counter i's field.
template <int BITS>
__device__ __forceinline__ void tab_wraps(uint32_t *__restrict__ carry, uint32_t at, uint32_t old) {
    constexpr int P = TabPack<BITS>::P;
    constexpr uint32_t mask = TabPack<BITS>::mask;
    const uint32_t f = at % P;
    if (((old >> (BITS * f)) & mask) != mask) return;
    const uint32_t base = at - f;
    for (uint32_t i = f; i < (uint32_t)P; ++i) {
        if (((old >> (BITS * i)) & mask) != mask) break;
        atomicAdd(carry + base + i, 1u);
    }
}

template <int BITS>
__global__ void __launch_bounds__(kTabThreads, kTabMinBlocks) walk_table_kernel(WalkArgs A, int tile_arcs,
                                                                     uint32_t *__restrict__ tp,
                                                                     uint32_t *__restrict__ carry, uint32_t ld) {
    extern __shared__ uint4 smem4[];
    __shared__ __align__(16) uint8_t s_rlut[4096];
    __shared__ uint32_t s_rmod[17];
    __shared__ uint32_t s_ent[kTabWarps][kTabBatch];    // arc in tile | r << 12 | sigma << 17 | rank << 21
    __shared__ uint32_t s_w3[kTabWarps][kTabBatch];     // word 3 of each draw
    __shared__ uint8_t s_sorted[kTabWarps][kTabBatch];  // batch index at each ranked position
    __shared__ uint32_t s_hist[kTabWarps][32];          // draws per r so far in the batch

    uint4 *s_rec = smem4;                                        // 2 tile_arcs: records of u and v
    uint32_t *s_off = reinterpret_cast<uint32_t *>(smem4 + 2 * tile_arcs);   // tile_arcs + 1
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b < 4096 / 16; b += kTabThreads)
        reinterpret_cast<uint4 *>(s_rlut)[b] = __ldg(reinterpret_cast<const uint4 *>(A.rlut) + b);
    if (tid < 17) s_rmod[tid] = A.rmod[tid];
    s_hist[warp][lane] = 0;
    const int64_t a0 = (int64_t)blockIdx.x * tile_arcs;
    const int na = (int)imin64(tile_arcs, A.n_arcs - a0);
    for (int i = tid; i < na; i += kTabThreads) {
        s_off[i] = arc_count(A, a0 + i);
        s_rec[2 * i] = __ldg(A.vinfo + arc_source(A.indptr, A.n, a0 + i));
        s_rec[2 * i + 1] = __ldg(A.vinfo + __ldg(A.indices + a0 + i));
    }
    __syncthreads();
    const uint32_t total = block_exclusive_scan<kTabThreads>(s_off, na);
    if (tid == 0) s_off[na] = total;
    __syncthreads();
    const bool uniform = A.thr_frac == 0;
    uint32_t *ent = s_ent[warp];
    uint32_t *w3s = s_w3[warp];
    uint8_t *sorted = s_sorted[warp];
    uint32_t *hist = s_hist[warp];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t nbatch = (total + kTabBatch - 1) / kTabBatch;
    for (uint32_t bt = warp; bt < nbatch; bt += kTabWarps) {
        const uint32_t bbase = bt * kTabBatch;
        // heads and ranks by r (r = 0: past the tile's last sample)
#pragma unroll 2   // two heads' Philox chains interleaved (1% off the walk)
        for (int t = 0; t < kTabBatch / 32; ++t) {
            const uint32_t idx = (uint32_t)t * 32 + lane;
            const uint32_t s = bbase + idx;
            int r = 0, sg = 0, lo = 0;
            uint32_t w3 = 0;
            if (s < total) {
                if (uniform) {
                    lo = A.base == 1 ? (int)s : (int)fastdiv32(s, A.base_magic);
                } else {
                    int hi = na;   // s_off[lo] <= s < s_off[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_off[mid] <= s) lo = mid; else hi = mid;
                    }
                }
                uint32_t coin;
                draw_head(A, s_rlut, s_rmod, a0 + lo, s - s_off[lo], &r, &sg, &coin, &w3);
            }
            const unsigned grp = __match_any_sync(0xffffffffu, r);
            const int leader = __ffs(grp) - 1;
            uint32_t base = 0;
            if (lane == leader) {
                base = hist[r];
                hist[r] = base + (uint32_t)__popc(grp);
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            const uint32_t rank = base + (uint32_t)__popc(grp & lt_mask);
            ent[idx] = (uint32_t)lo | ((uint32_t)r << 12) | ((uint32_t)sg << 17) | (rank << 21);
            w3s[idx] = w3;
            __syncwarp();   // the next group leader reads what this one wrote
        }
        // exclusive scan of the 17 bins: lane r holds the first position of r
        const uint32_t h = lane < 17 ? hist[lane] : 0u;
        uint32_t incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t start = incl - h;
        hist[lane] = 0;
#pragma unroll 1
        for (int t = 0; t < kTabBatch / 32; ++t) {
            const uint32_t idx = (uint32_t)t * 32 + lane;
            const uint32_t e = ent[idx];
            const uint32_t pos = __shfl_sync(0xffffffffu, start, (e >> 12) & 31) + (e >> 21);
            sorted[pos] = (uint8_t)idx;
        }
        __syncwarp();
        // walks in r order, two adjacent ranked draws per lane
        const uint32_t first = __shfl_sync(0xffffffffu, start, 1);
        // the previous pair's counters and the words their increments found
        uint32_t at0 = 0, at1 = 0, old0 = 0, old1 = 0;
        bool pend0 = false, pend1 = false;
#pragma unroll 1
        for (uint32_t q = first + 2 * (uint32_t)lane; q < (uint32_t)kTabBatch; q += 64) {
            const bool has1 = q + 1 < (uint32_t)kTabBatch;
            const uint32_t i0 = sorted[q], i1 = sorted[has1 ? q + 1 : q];
            const uint32_t e0 = ent[i0], e1 = ent[i1];
            const uint32_t lo0 = e0 & 0xFFFu, lo1 = e1 & 0xFFFu;
            TabDraw d0, d1;
            tab_begin((uint32_t)(a0 + lo0), bbase + i0 - s_off[lo0], (int)((e0 >> 12) & 31), (int)((e0 >> 17) & 15),
                      w3s[i0], s_rec[2 * lo0], s_rec[2 * lo0 + 1], d0);
            tab_begin((uint32_t)(a0 + lo1), bbase + i1 - s_off[lo1], (int)((e1 >> 12) & 31), (int)((e1 >> 17) & 15),
                      w3s[i1], s_rec[2 * lo1], s_rec[2 * lo1 + 1], d1);
            if (!has1) d1.steps = 0;
            TabSteps<0>::run(A, d0, d1, max(d0.steps, d1.steps));
            if (pend0) tab_wraps<BITS>(carry, at0, old0);
            if (pend1) tab_wraps<BITS>(carry, at1, old1);
            uint32_t x, y;
            tab_end(d0, &x, &y);
            at0 = x * ld + y;   // < 2^32: ld <= 65536
            old0 = tab_count<BITS>(tp, at0);
            pend0 = true;
            pend1 = has1;
            if (has1) {
                tab_end(d1, &x, &y);
                at1 = x * ld + y;
                old1 = tab_count<BITS>(tp, at1);
            }
        }
        if (pend0) tab_wraps<BITS>(carry, at0, old0);
        if (pend1) tab_wraps<BITS>(carry, at1, old1);
        __syncwarp();
    }
}

// Exact 32-bit counts from the packed table and its wrap records, in place in
// the 32-bit table (upper triangle only: nothing else was counted). Field i
// of a word received its counter's c_i increments plus one carry per wrap of
// field i - 1 (none for i = 0), and wrapped carry[i] times, so
// c_i = field_i + 2^BITS carry[i] - carry[i - 1].
template <int BITS>
__global__ void table_decode_kernel(const uint32_t *__restrict__ tp, uint32_t *__restrict__ tab, int n, int64_t ld) {
    constexpr int P = TabPack<BITS>::P;
    constexpr uint32_t mask = TabPack<BITS>::mask;
    for (int x = blockIdx.x; x < n; x += gridDim.x) {
        const int64_t k0 = ((int64_t)x * ld + x) / P, k1 = ((int64_t)x * ld + ld) / P;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const uint32_t w = tp[k];
            uint32_t prev = 0;
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const uint32_t wr = tab[P * k + i];
                tab[P * k + i] = ((w >> (BITS * i)) & mask) + (wr << BITS) - prev;
                prev = wr;
            }
        }
    }
}

constexpr int kScatterThreads = 512;
constexpr int kScatterItems = 16;

template <typename KeyT>
__global__ void __launch_bounds__(kScatterThreads) bucket_scatter_kernel(
    const KeyT *__restrict__ in, int64_t nkeys, KeyT *__restrict__ out,
    unsigned long long *__restrict__ cursor, int nb) {
    extern __shared__ unsigned long long s_base[];                 // nb
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_base + nb);  // nb
    const int tid = threadIdx.x;
    for (int i = tid; i < nb; i += kScatterThreads) s_cnt[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kScatterThreads * kScatterItems;
    KeyT k[kScatterItems];
    uint32_t rank[kScatterItems];
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        int64_t idx = base + (int64_t)i * kScatterThreads + tid;
        if (idx < nkeys) {
            k[i] = in[idx];
            rank[i] = atomicAdd(&s_cnt[(uint32_t)(k[i] >> kBucketBits)], 1u);
        }
    }
    __syncthreads();
    for (int i = tid; i < nb; i += kScatterThreads) {
        uint32_t c = s_cnt[i];
        if (c) s_base[i] = atomicAdd(&cursor[i], (unsigned long long)c);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        int64_t idx = base + (int64_t)i * kScatterThreads + tid;
        if (idx < nkeys) out[s_base[(uint32_t)(k[i] >> kBucketBits)] + rank[i]] = k[i];
    }
}

// Global-atomic fallback when the bucket count does not fit shared memory.
template <typename KeyT>
__global__ void bucket_scatter_global_kernel(const KeyT *__restrict__ in, int64_t nkeys,
                                             KeyT *__restrict__ out,
                                             unsigned long long *__restrict__ cursor) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nkeys;
         i += (int64_t)gridDim.x * blockDim.x) {
        KeyT k = in[i];
        out[atomicAdd(&cursor[(uint32_t)(k >> kBucketBits)], 1ull)] = k;
    }
}

constexpr int kReduceThreads = 1024;

// One CTA per bucket: dense shared-memory histogram over the bucket's 2^15
// keys, then the distinct keys in key order with their counts.
template <typename KeyT>
__global__ void __launch_bounds__(kReduceThreads) bucket_reduce_kernel(
    const KeyT *__restrict__ keys, const int64_t *__restrict__ bucket_off, KeyT *__restrict__ out_key,
    uint32_t *__restrict__ out_cnt, uint32_t *__restrict__ distinct) {
    extern __shared__ uint32_t hist[];   // 2^kBucketBits
    constexpr int W = 1 << kBucketBits;
    constexpr int PER = W / kReduceThreads;
    __shared__ uint32_t warp_tot[kReduceThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int64_t lo = bucket_off[b], hi = bucket_off[b + 1];
    if (lo == hi) {
        if (tid == 0) distinct[b] = 0;
        return;
    }
    for (int i = tid; i < W; i += kReduceThreads) hist[i] = 0;
    __syncthreads();
    for (int64_t i = lo + tid; i < hi; i += kReduceThreads)
        atomicAdd(&hist[(uint32_t)(keys[i] & (KeyT)(W - 1))], 1u);
    __syncthreads();
    // each thread owns PER consecutive histogram slots
    uint32_t nz = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) nz += hist[tid * PER + j] != 0;
    uint32_t x = nz;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    uint32_t pos = (warp > 0 ? warp_tot[warp - 1] : 0) + x - nz;
    const KeyT kbase = (KeyT)b << kBucketBits;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        uint32_t c = hist[tid * PER + j];
        if (c) {
            out_key[lo + pos] = kbase | (KeyT)(tid * PER + j);
            out_cnt[lo + pos] = c;
            ++pos;
        }
    }
    if (tid == kReduceThreads - 1) distinct[b] = pos;
}

// Copies every bucket's distinct entries to contiguous (x, y, count) arrays.
template <typename KeyT>
__global__ void compact_kernel(const KeyT *__restrict__ rkey, const uint32_t *__restrict__ rcnt,
                               const int64_t *__restrict__ bucket_off,
                               const int64_t *__restrict__ dst_off, int B, int32_t *__restrict__ x,
                               int32_t *__restrict__ y, uint32_t *__restrict__ cnt) {
    const int b = blockIdx.x;
    const int64_t src = bucket_off[b];
    const int64_t dst = dst_off[b];
    const int64_t m = dst_off[b + 1] - dst;
    const KeyT mask = ((KeyT)1 << B) - 1;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        KeyT k = rkey[src + i];
        x[dst + i] = (int32_t)(k >> B);
        y[dst + i] = (int32_t)(k & mask);
        cnt[dst + i] = rcnt[src + i];
    }
}

struct NetmfConst {
    double a_off, a_diag;              // alpha = vol^2 / (2 S b), vol^2 / (S b)
    float off_hi, off_lo, diag_hi, diag_lo;
    const uint32_t *wdeg;              // weighted degrees (weighted graphs), else NULL
};

// The degree of Eq. 1: weighted when the graph is, else the arc count.
__device__ __forceinline__ int64_t eq1_degree(const NetmfConst &k, const int64_t *__restrict__ indptr, int64_t x) {
    return k.wdeg ? (int64_t)__ldg(k.wdeg + x) : __ldg(indptr + x + 1) - __ldg(indptr + x);
}

// Eq. 1 entry with the truncated log for count K of pair (x, y):
// v = fl(fl(K alpha) / fl(d_x d_y)), kept iff v > 1, value log(v) as float32
// (0 means dropped; log v > 0 for every kept entry).
// Fast path: D = K alpha - q (q = d_x d_y) in FP32 with alpha split into a
// float pair; fmaf makes the product exact, so D carries a relative error of
// ~1e-7. Whenever |D| > 1e-5 q its sign is the FP64 decision and
// log1p(D / q) is accurate to a few ulp. Otherwise (v within 1e-5 of 1, or
// operands beyond 2^24) the exact FP64 rule decides: a correctly rounded
// quotient exceeds 1 iff p >= 2q or (p > q and (p - q) 2^53 > q), with p - q
// exact there (Sterbenz), so no division is needed.
__device__ __forceinline__ float netmf_value(uint32_t cnt, int64_t dx, int64_t dy, bool diag,
                                             const NetmfConst &k) {
    const int64_t q64 = dx * dy;
    if (cnt < (1u << 24) && q64 < (1ll << 24)) {
        const float cf = (float)cnt, qf = (float)q64;
        const float hi = diag ? k.diag_hi : k.off_hi, lo = diag ? k.diag_lo : k.off_lo;
        const float dq = fmaf(cf, hi, -qf) + cf * lo;
        if (fabsf(dq) > 1e-5f * qf) return dq > 0.f ? log1pf(__fdiv_rn(dq, qf)) : 0.f;
    }
    const double p = __dmul_rn((double)cnt, diag ? k.a_diag : k.a_off);
    const double q = __ll2double_rn(q64);
    if (!(p > q)) return 0.f;
    const double q2 = __dmul_rn(2.0, q);
    if (p < q2) {
        const double dd = __dsub_rn(p, q);
        if (!(__dmul_rn(dd, 9007199254740992.0) > q)) return 0.f;
        return log1pf(__fdiv_rn((float)dd, (float)q));
    }
    if (p < 1e30) return logf(__fdiv_rn((float)p, (float)q));
    return (float)(log(p) - log(q));
}

// Eq. 1 entry from a fixed-point count: K = wsum * unit (2^-32 for summed
// downsampling weights 1/p_e, 2^-24 for stratified estimates),
// v = fl(fl(K alpha) / fl(d_x d_y)) in FP64, kept iff v > 1, value log v as
// float32. Fast path as for counts: the 64-bit sum is split into a float pair
// (kh + kl, exact to 2^-48 relative), D = K alpha - q in FP32 with fmaf, so D
// carries an error of ~1e-7 |D| + 1e-14 q; when |D| > 1e-5 q its sign is the
// FP64 decision. Otherwise the exact FP64 rule (no division) decides.
// unit_f / unit_d: the power of two that one unit of wsum stands for.
__device__ __forceinline__ float netmf_value_fixed(uint64_t wsum, float unit_f, double unit_d, int64_t dx,
                                                   int64_t dy, bool diag, const NetmfConst &k) {
    const int64_t q64 = dx * dy;
    if (q64 < (1ll << 24)) {
        const float kh = __ull2float_rn(wsum);
        // kh is an integer below 2^64 (unless wsum rounds up to 2^64): the
        // residual wsum - kh is exact in 64-bit arithmetic
        const float kl = kh < 1.8446744e19f ? (float)(int64_t)(wsum - __float2ull_rn(kh)) : 0.f;
        const float khs = kh * unit_f, kls = kl * unit_f;
        const float qf = (float)q64;
        const float hi = diag ? k.diag_hi : k.off_hi, lo = diag ? k.diag_lo : k.off_lo;
        const float dq = fmaf(khs, hi, -qf) + fmaf(khs, lo, kls * hi);
        if (fabsf(dq) > 1e-5f * qf) return dq > 0.f ? log1pf(__fdiv_rn(dq, qf)) : 0.f;
    }
    const double K = __dmul_rn(__ull2double_rn(wsum), unit_d);
    const double p = __dmul_rn(K, diag ? k.a_diag : k.a_off);
    const double q = __ll2double_rn(q64);
    if (!(p > q)) return 0.f;
    const double q2 = __dmul_rn(2.0, q);
    if (p < q2) {
        const double dd = __dsub_rn(p, q);
        if (!(__dmul_rn(dd, 9007199254740992.0) > q)) return 0.f;
        return log1pf(__fdiv_rn((float)dd, (float)q));
    }
    if (p < 1e30) return logf(__fdiv_rn((float)p, (float)q));
    return (float)(log(p) - log(q));
}

__device__ __forceinline__ float netmf_value_w(uint64_t wsum, int64_t dx, int64_t dy, bool diag,
                                               const NetmfConst &k) {
    return netmf_value_fixed(wsum, 2.3283064e-10f, 2.3283064365386963e-10, dx, dy, diag, k);   // 2^-32
}

// Weighted table -> the float-bits value table (upper triangle).
__global__ void table_values_w_kernel(const uint64_t *__restrict__ W, uint32_t *__restrict__ T, int64_t ld, int n,
                                      const int64_t *__restrict__ indptr, NetmfConst kc) {
    const int x = blockIdx.x;
    const int64_t dx = eq1_degree(kc, indptr, x);
    for (int y = x + threadIdx.x; y < n; y += blockDim.x) {
        const uint64_t w = W[(size_t)x * ld + y];
        if (w == 0) continue;
        const int64_t dy = eq1_degree(kc, indptr, y);
        T[(size_t)x * ld + y] = __float_as_uint(netmf_value_w(w, dx, dy, x == y, kc));
    }
}

// Per arc u -> v: the coin threshold min(2^32, floor(p 2^32)) and the weight
// floor(2^32 / p + 1/2) of p = min(1, C (1/d_u + 1/d_v)), each FP64 step one
// IEEE rounding (Sec. 4.1, degree sampling). A warp per source vertex, its
// lanes over the vertex's arcs (degrees are skewed).
__global__ void downsample_arcs_kernel(const int64_t *__restrict__ indptr, const int32_t *__restrict__ indices,
                                       const uint32_t *__restrict__ aw, const uint32_t *__restrict__ wdeg,
                                       int64_t n, double C, uint64_t *__restrict__ thr, uint64_t *__restrict__ w) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const int64_t a0 = indptr[u], a1 = indptr[u + 1];
        if (a1 == a0) continue;
        const double iu = __ddiv_rn(1.0, wdeg ? (double)__ldg(wdeg + u) : (double)(a1 - a0));
        for (int64_t a = a0 + lane; a < a1; a += 32) {
            const int32_t v = __ldg(indices + a);
            const double dv = wdeg ? (double)__ldg(wdeg + v) : (double)(__ldg(indptr + v + 1) - __ldg(indptr + v));
            const double iv = __ddiv_rn(1.0, dv);
            double p = __dmul_rn(C, __dadd_rn(iu, iv));
            if (aw) p = __dmul_rn((double)__ldg(aw + a), p);   // p_e = min(1, A_uv (C (1/d_u + 1/d_v)))
            if (p >= 1.0) p = 1.0;
            thr[a] = p >= 1.0 ? (1ull << 32) : (uint64_t)floor(__dmul_rn(p, 4294967296.0));
            w[a] = (uint64_t)floor(__dadd_rn(__ddiv_rn(4294967296.0, p), 0.5));
        }
    }
}

__global__ void trunclog_kernel(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                                const uint32_t *__restrict__ cnt, int64_t nnz,
                                const int64_t *__restrict__ indptr, NetmfConst kc,
                                float *__restrict__ val, uint8_t *__restrict__ keep,
                                uint32_t *__restrict__ rowcnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t xi = x[i], yi = y[i];
        const int64_t dx = eq1_degree(kc, indptr, xi);
        const int64_t dy = eq1_degree(kc, indptr, yi);
        const float v = netmf_value(cnt[i], dx, dy, xi == yi, kc);
        const bool k = v > 0.f;
        if (k) {
            atomicAdd(&rowcnt[xi], 1u);
            if (xi != yi) atomicAdd(&rowcnt[yi], 1u);
        }
        keep[i] = k;
        val[i] = v;
    }
}

__global__ void csr_fill_kernel(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                                const float *__restrict__ val, const uint8_t *__restrict__ keep,
                                int64_t nnz, const int64_t *__restrict__ rowptr,
                                uint32_t *__restrict__ cursor, int32_t *__restrict__ col,
                                float *__restrict__ data) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[i]) continue;
        const int32_t xi = x[i], yi = y[i];
        const float v = val[i];
        int64_t p = rowptr[xi] + atomicAdd(&cursor[xi], 1u);
        col[p] = yi;
        data[p] = v;
        if (xi != yi) {
            p = rowptr[yi] + atomicAdd(&cursor[yi], 1u);
            col[p] = xi;
            data[p] = v;
        }
    }
}

constexpr int kSortThreads = 512;
constexpr int kSortMax = 16384;   // entries of one row sorted in shared memory

// Bitonic sort of every row by column (columns in a row are distinct). Rows are
// packed as (col << 32 | float bits) so the sort key is the column.
__global__ void __launch_bounds__(kSortThreads) csr_row_sort_kernel(const int64_t *__restrict__ rowptr,
                                                                    int32_t *__restrict__ col,
                                                                    float *__restrict__ data,
                                                                    int *__restrict__ too_long) {
    extern __shared__ unsigned long long e[];
    const int64_t r0 = rowptr[blockIdx.x], r1 = rowptr[blockIdx.x + 1];
    const int L = (int)(r1 - r0);
    if (L <= 1) return;
    if (L > kSortMax) {
        if (threadIdx.x == 0) atomicMax(too_long, L);
        return;
    }
    int P = 1;
    while (P < L) P <<= 1;
    for (int i = threadIdx.x; i < P; i += kSortThreads) {
        if (i < L)
            e[i] = ((unsigned long long)(uint32_t)col[r0 + i] << 32) |
                   (unsigned long long)__float_as_uint(data[r0 + i]);
        else
            e[i] = ~0ull;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += kSortThreads) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long a = e[i], b = e[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        e[i] = b;
                        e[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < L; i += kSortThreads) {
        col[r0 + i] = (int32_t)(e[i] >> 32);
        data[r0 + i] = __uint_as_float((uint32_t)(e[i] & 0xFFFFFFFFull));
    }
}

// ---------------------------------------------------------------------------
// dense-table aggregation (n <= 65536)
// ---------------------------------------------------------------------------
constexpr int kTile = 64;

// Counts -> Eq. 1 values in place (float bits; 0 = not kept). One CTA per row
// x of the upper triangle (y >= x).
__global__ void table_values_kernel(uint32_t *__restrict__ T, int64_t ld, int n,
                                    const int64_t *__restrict__ indptr, NetmfConst kc) {
    const int x = blockIdx.x;
    const int64_t dx = eq1_degree(kc, indptr, x);
    uint32_t *row = T + (size_t)x * ld;
    for (int y = x + threadIdx.x; y < n; y += blockDim.x) {
        const uint32_t c = row[y];
        if (c == 0) continue;
        const int64_t dy = eq1_degree(kc, indptr, y);
        row[y] = __float_as_uint(netmf_value(c, dx, dy, x == y, kc));
    }
}

// table_decode_kernel and table_values_kernel in one pass, for the CSR: the
// exact count of each upper-triangle counter from its packed field and wrap
// records (see table_decode_kernel), then its Eq. 1 value written as float
// bits in place of the wrap record (which is 0 where nothing was counted).
template <int BITS>
__global__ void table_decode_values_kernel(const uint32_t *__restrict__ tp, uint32_t *__restrict__ T, int64_t ld,
                                           int n, const int64_t *__restrict__ indptr, NetmfConst kc) {
    constexpr int P = TabPack<BITS>::P;
    constexpr uint32_t mask = TabPack<BITS>::mask;
    const int x = blockIdx.x;
    const int64_t dx = eq1_degree(kc, indptr, x);
    const int64_t k0 = ((int64_t)x * ld + x) / P, k1 = ((int64_t)x * ld + ld) / P;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const uint32_t w = tp[k];
        uint32_t wr[P];
#pragma unroll
        for (int i = 0; i < P; ++i) wr[i] = T[P * k + i];
        uint32_t prev = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const uint32_t cnt = ((w >> (BITS * i)) & mask) + (wr[i] << BITS) - prev;
            prev = wr[i];
            const int64_t y = P * k + i - (int64_t)x * ld;
            // left of the diagonal, padding, or nothing counted: value 0. The
            // record is 0 there unless the field took the carries of a
            // neighbour that wrapped 2^BITS times and wrapped itself (a
            // neighbour past 2^16 counts): clear it
            if (y < x || y >= n || cnt == 0) {
                if (wr[i] != 0u) T[P * k + i] = 0u;
                continue;
            }
            T[P * k + i] = __float_as_uint(netmf_value(cnt, dx, eq1_degree(kc, indptr, y), x == y, kc));
        }
    }
}

// table_decode_values_kernel for sparse tables: a warp decodes 32
// consecutive words at a time and queues the counted (index, count) pairs in
// shared memory; the values are taken 32 at a time, one per lane, so a sparse
// row does not run the value arithmetic with most lanes idle (each value is
// independent: the order does not matter).
constexpr int kDvThreads = 256;
constexpr int kDvQueue = 160;   // 31 left over + 4 x 32 new

template <int BITS>
__global__ void __launch_bounds__(kDvThreads) table_decode_values_sparse_kernel(const uint32_t *__restrict__ tp,
                                                                        uint32_t *__restrict__ T, int64_t ld, int n,
                                                                        const int64_t *__restrict__ indptr,
                                                                        NetmfConst kc) {
    constexpr int P = TabPack<BITS>::P;
    constexpr uint32_t mask = TabPack<BITS>::mask;
    static_assert(P * 32 + 31 <= kDvQueue, "queue holds a chunk's counters and the leftovers");
    __shared__ uint32_t s_qi[kDvThreads / 32][kDvQueue], s_qc[kDvThreads / 32][kDvQueue];
    const int x = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t dx = eq1_degree(kc, indptr, x);
    const int64_t k0 = ((int64_t)x * ld + x) / P, k1 = ((int64_t)x * ld + ld) / P;
    uint32_t *qi = s_qi[warp], *qc = s_qc[warp];
    int qn = 0;   // queued entries (the same in every lane)
    // values of queued entries [q0, q0 + cnt), cnt <= 32, one per lane
    auto values = [&](int q0, int cnt) {
        if (lane < cnt) {
            const uint32_t idx = qi[q0 + lane], c = qc[q0 + lane];
            const int64_t y = (int64_t)idx - (int64_t)x * ld;
            T[idx] = __float_as_uint(netmf_value(c, dx, eq1_degree(kc, indptr, y), x == y, kc));
        }
    };
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t kb = k0 + 32 * warp; kb < k1; kb += kDvThreads) {
        const int64_t k = kb + lane;
        const bool valid = k < k1;
        const uint32_t w = valid ? tp[k] : 0u;
        uint32_t wr[P];
#pragma unroll
        for (int i = 0; i < P; ++i) wr[i] = valid ? T[P * k + i] : 0u;
        uint32_t prev = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const uint32_t cnt = ((w >> (BITS * i)) & mask) + (wr[i] << BITS) - prev;
            prev = wr[i];
            const int64_t y = P * k + i - (int64_t)x * ld;
            // left of the diagonal, padding, or nothing counted: value 0. The
            // record is 0 there unless the field took the carries of a
            // neighbour that wrapped 2^BITS times and wrapped itself (a
            // neighbour past 2^16 counts): clear it
            const bool keep = valid && y >= x && y < n && cnt != 0u;
            if (valid && !keep && wr[i] != 0u) T[P * k + i] = 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = qn + __popc(bal & lt);
                qi[pos] = (uint32_t)(P * k + i);
                qc[pos] = cnt;
            }
            qn += __popc(bal);
        }
        __syncwarp();
        while (qn >= 32) {   // the last 32 queued
            values(qn - 32, 32);
            qn -= 32;
            __syncwarp();
        }
    }
    values(0, qn);
}

// Distinct pairs per upper-triangle row (for the counts output).
template <typename E>
__global__ void table_row_nnz_kernel(const E *__restrict__ T, int64_t ld, int n, uint32_t *__restrict__ cnt) {
    __shared__ uint32_t red[32];
    const int x = blockIdx.x;
    const E *row = T + (size_t)x * ld;
    uint32_t c = 0;
    for (int y = x + threadIdx.x; y < n; y += blockDim.x) c += row[y] != 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
        cnt[x] = t;
    }
}

// (x, y, count) of the upper triangle in (x, y) order: one CTA per row, the
// row is walked in chunks of blockDim with a block-wide ballot scan.
template <typename E>
__global__ void table_compact_kernel(const E *__restrict__ T, int64_t ld, int n, const int64_t *__restrict__ off,
                                     int32_t *__restrict__ ox, int32_t *__restrict__ oy, E *__restrict__ oc) {
    __shared__ uint32_t warp_cnt[32];
    __shared__ uint32_t base_s;
    const int x = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const E *row = T + (size_t)x * ld;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    const int64_t o = off[x];
    for (int y0 = x; y0 < n; y0 += blockDim.x) {
        const int y = y0 + threadIdx.x;
        const E c = y < n ? row[y] : (E)0;
        const unsigned bal = __ballot_sync(0xffffffffu, c != 0);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = base_s;
        for (int w = 0; w < warp; ++w) before += warp_cnt[w];
        if (c != 0) {
            const int64_t pos = o + before + __popc(bal & ((1u << lane) - 1u));
            ox[pos] = x;
            oy[pos] = y;
            oc[pos] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < nw; ++w) t += warp_cnt[w];
            base_s += t;
        }
        __syncthreads();
    }
}

// The upper tile (u, v), u <= v, of the stored upper triangle, once: S[i][j]
// = T(u kTile + i, v kTile + j); on the diagonal tile the lower half is the
// mirror of the upper. Its rows give the tile (u, v) of the symmetric matrix
// and its columns (u < v) the tile (v, u), so each stored tile is read once.
__device__ __forceinline__ void load_upper_tile(const uint32_t *__restrict__ T, int64_t ld, int u, int v,
                                                uint32_t (*S)[kTile + 1]) {
    const uint32_t *base = T + (size_t)u * kTile * ld + (size_t)v * kTile;
    if (u < v) {
        for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
            const int i = e / kTile, j = e % kTile;
            S[i][j] = base[(size_t)i * ld + j];
        }
    } else {
        for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
            const int i = e / kTile, j = e % kTile;
            S[i][j] = base[(size_t)min(i, j) * ld + max(i, j)];
        }
    }
}

// Kept entries per (row, column tile) of the symmetric matrix: a CTA per
// upper tile (the grid's other half returns at once) counts the tile's rows
// for (u, v) and, off the diagonal, its columns for (v, u).
__global__ void __launch_bounds__(256) tile_count_kernel(const uint32_t *__restrict__ T, int64_t ld, int n, int nt,
                                                         uint32_t *__restrict__ rowtile) {
    __shared__ uint32_t S[kTile][kTile + 1];
    const int u = blockIdx.y, v = blockIdx.x;
    if (u > v) return;
    load_upper_tile(T, ld, u, v, S);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < kTile; i += 8) {
        const int r = u * kTile + i;
        if (r < n) {
            const unsigned b0 = __ballot_sync(0xffffffffu, S[i][lane] != 0u);
            const unsigned b1 = __ballot_sync(0xffffffffu, S[i][lane + 32] != 0u);
            if (lane == 0) rowtile[(size_t)r * nt + v] = __popc(b0) + __popc(b1);
        }
        const int rt = v * kTile + i;   // row i of the tile (v, u): column i of S
        if (u < v && rt < n) {
            const unsigned b0 = __ballot_sync(0xffffffffu, S[lane][i] != 0u);
            const unsigned b1 = __ballot_sync(0xffffffffu, S[lane + 32][i] != 0u);
            if (lane == 0) rowtile[(size_t)rt * nt + u] = __popc(b0) + __popc(b1);
        }
    }
}

// Per row: exclusive scan of its tile counts (in place) and the row total.
__global__ void row_tile_scan_kernel(uint32_t *__restrict__ rowtile, int n, int nt,
                                     uint32_t *__restrict__ rowcnt) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    uint32_t *rt = rowtile + (size_t)r * nt;
    uint32_t carry = 0;
    for (int t0 = 0; t0 < nt; t0 += 32) {
        const int t = t0 + lane;
        const uint32_t v = t < nt ? rt[t] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (t < nt) rt[t] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) rowcnt[r] = carry;
}

// Writes every kept entry of the upper tile at its sorted position in the
// CSR: the tile's rows into (u, v) and, off the diagonal, its columns into
// (v, u) (a row of the tile (v, u) takes S's column in row order, which is
// its column order).
__device__ __forceinline__ void fill_row(int64_t base, uint32_t v0, uint32_t v1, int col0, int lane,
                                         int32_t *__restrict__ col, float *__restrict__ data) {
    const unsigned b0 = __ballot_sync(0xffffffffu, v0 != 0u);
    const unsigned b1 = __ballot_sync(0xffffffffu, v1 != 0u);
    const unsigned below = (1u << lane) - 1u;
    if (v0) {
        const int64_t pos = base + __popc(b0 & below);
        col[pos] = col0 + lane;
        data[pos] = __uint_as_float(v0);
    }
    if (v1) {
        const int64_t pos = base + __popc(b0) + __popc(b1 & below);
        col[pos] = col0 + 32 + lane;
        data[pos] = __uint_as_float(v1);
    }
}

__global__ void __launch_bounds__(256) tile_fill_kernel(const uint32_t *__restrict__ T, int64_t ld, int n, int nt,
                                                        const uint32_t *__restrict__ rowtile,
                                                        const int64_t *__restrict__ indptr,
                                                        int32_t *__restrict__ col, float *__restrict__ data) {
    __shared__ uint32_t S[kTile][kTile + 1];
    const int u = blockIdx.y, v = blockIdx.x;
    if (u > v) return;
    load_upper_tile(T, ld, u, v, S);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < kTile; i += 8) {
        const int r = u * kTile + i;
        if (r < n) fill_row(indptr[r] + rowtile[(size_t)r * nt + v], S[i][lane], S[i][lane + 32], v * kTile, lane,
                            col, data);
        const int rt = v * kTile + i;
        if (u < v && rt < n)
            fill_row(indptr[rt] + rowtile[(size_t)rt * nt + u], S[lane][i], S[lane + 32][i], u * kTile, lane, col,
                     data);
    }
}

// ---------------------------------------------------------------------------
// Sort path (any n < 2^31): 64-bit keys, radix sort, run lengths, then the
// symmetric CSR assembled from the sorted unique pairs. Every entry u of the
// unique list is handled by a thread owning kSortRun consecutive entries, so
// the kept / mirrored indices of an entry come from one block scan per tile.
// ---------------------------------------------------------------------------
constexpr int kPathThreads = 256;
constexpr int kPathRun = 32;
constexpr int kPathTile = kPathThreads * kPathRun;

__device__ __forceinline__ int64_t path_block_scan(int64_t v, int64_t *s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    __syncthreads();
    return before + x - v;
}

__global__ void decode_keys_kernel(const uint64_t *__restrict__ uk, int64_t u, int B, int32_t *__restrict__ x,
                                   int32_t *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < u; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = uk[i];
        x[i] = (int32_t)(k >> B);
        y[i] = (int32_t)(k & ((1ull << B) - 1ull));
    }
}

__global__ void degree_kernel(const int64_t *__restrict__ indptr, int64_t n, uint32_t *__restrict__ deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        deg[i] = (uint32_t)(indptr[i + 1] - indptr[i]);
}

// Eq. 1 value of every unique pair, written over its count (float bits; 0 =
// dropped), and per tile the number of kept and of kept off-diagonal pairs.
// With edge downsampling the value comes from the pair's summed weight wsum.
__global__ void __launch_bounds__(kPathThreads) path_value_kernel(const uint64_t *__restrict__ uk,
                                                                  uint32_t *__restrict__ cnt_val,
                                                                  const uint64_t *__restrict__ wsum, int64_t U, int B,
                                                                  const uint32_t *__restrict__ deg, NetmfConst kc,
                                                                  uint32_t *__restrict__ tile_kept,
                                                                  uint32_t *__restrict__ tile_mir) {
    __shared__ uint32_t s_k, s_m;
    if (threadIdx.x == 0) s_k = s_m = 0;
    __syncthreads();
    uint32_t ck = 0, cm = 0;
    const int64_t t0 = (int64_t)blockIdx.x * kPathTile;
    for (int j = threadIdx.x; j < kPathTile; j += kPathThreads) {   // coalesced here: counts only
        const int64_t u = t0 + j;
        if (u >= U) break;
        const uint64_t k = uk[u];
        const uint32_t x = (uint32_t)(k >> B), y = (uint32_t)(k & ((1ull << B) - 1ull));
        const float v = wsum ? netmf_value_w(wsum[u], __ldg(deg + x), __ldg(deg + y), x == y, kc)
                             : netmf_value(cnt_val[u], __ldg(deg + x), __ldg(deg + y), x == y, kc);
        cnt_val[u] = __float_as_uint(v);
        if (v > 0.f) {
            ++ck;
            cm += x != y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ck += __shfl_xor_sync(0xffffffffu, ck, o);
        cm += __shfl_xor_sync(0xffffffffu, cm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_k, ck);
        atomicAdd(&s_m, cm);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tile_kept[blockIdx.x] = s_k;
        tile_mir[blockIdx.x] = s_m;
    }
}

// Kept entries compacted in unique-list order (= grouped by row, columns
// ascending): their columns and values, and per row how many and where they
// start (runs of equal rows within a thread's entries share one atomic); the
// mirrored entries (key (y << B) | x, value bits) in the same order.
__global__ void __launch_bounds__(kPathThreads) path_rows_kernel(
    const uint64_t *__restrict__ uk, const uint32_t *__restrict__ val, int64_t U, int B,
    const int64_t *__restrict__ kept_off, const int64_t *__restrict__ mir_off, uint32_t *__restrict__ dlen,
    unsigned long long *__restrict__ dstart, int32_t *__restrict__ dcol, uint32_t *__restrict__ dval,
    uint64_t *__restrict__ mkey, uint32_t *__restrict__ mval) {
    __shared__ int64_t s_warp[kPathThreads / 32];
    const int64_t i0 = (int64_t)blockIdx.x * kPathTile + (int64_t)threadIdx.x * kPathRun;
    uint32_t ck = 0, cm = 0;
    for (int j = 0; j < kPathRun; ++j) {
        const int64_t u = i0 + j;
        if (u >= U) break;
        if (__uint_as_float(val[u]) > 0.f) {
            ++ck;
            const uint64_t k = uk[u];
            cm += (k >> B) != (k & ((1ull << B) - 1ull));
        }
    }
    int64_t k = kept_off[blockIdx.x] + path_block_scan(ck, s_warp);
    int64_t m = mir_off[blockIdx.x] + path_block_scan(cm, s_warp);
    int64_t run_x = -1, run_k = 0;
    uint32_t run_n = 0;
    for (int j = 0; j < kPathRun; ++j) {
        const int64_t u = i0 + j;
        if (u >= U) break;
        const uint32_t vb = val[u];
        if (!(__uint_as_float(vb) > 0.f)) continue;
        const uint64_t key = uk[u];
        const int64_t x = (int64_t)(key >> B), y = (int64_t)(key & ((1ull << B) - 1ull));
        if (x != run_x) {
            if (run_n) {
                atomicAdd(&dlen[run_x], run_n);
                atomicMin(&dstart[run_x], (unsigned long long)run_k);
            }
            run_x = x;
            run_k = k;
            run_n = 0;
        }
        ++run_n;
        dcol[k] = (int32_t)y;
        dval[k] = vb;
        if (x != y) {
            mkey[m] = ((uint64_t)y << B) | (uint64_t)x;
            mval[m] = vb;
            ++m;
        }
        ++k;
    }
    if (run_n) {
        atomicAdd(&dlen[run_x], run_n);
        atomicMin(&dstart[run_x], (unsigned long long)run_k);
    }
}

// Over the mirrored entries sorted by (row, column): where each row's run
// starts (first) and ends (end, exclusive; 0 = no mirrored entries).
__global__ void path_mirror_rows_kernel(const uint64_t *__restrict__ mk, int64_t M, int B,
                                        int64_t *__restrict__ first, int64_t *__restrict__ end) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < M; f += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = mk[f] >> B;
        if (f == 0 || (mk[f - 1] >> B) != r) first[r] = f;
        if (f + 1 == M || (mk[f + 1] >> B) != r) end[r] = f + 1;
    }
}

__global__ void path_row_total_kernel(const uint32_t *__restrict__ dlen, const int64_t *__restrict__ end,
                                      const int64_t *__restrict__ first, int64_t n, uint32_t *__restrict__ total) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        total[r] = dlen[r] + (end[r] ? (uint32_t)(end[r] - first[r]) : 0u);
}

// Row x of the CSR: its mirrored entries (columns < x) first, then its direct
// ones (columns >= x), copied from the compacted kept list (a warp per row).
__global__ void path_direct_fill_kernel(const int32_t *__restrict__ dcol, const uint32_t *__restrict__ dval,
                                        const uint32_t *__restrict__ dlen,
                                        const unsigned long long *__restrict__ dstart,
                                        const int64_t *__restrict__ rowptr, int64_t n, int32_t *__restrict__ col,
                                        float *__restrict__ data) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const uint32_t len = dlen[x];
        if (len == 0) continue;
        const int64_t src = (int64_t)dstart[x], dst = rowptr[x + 1] - len;
        for (uint32_t i = lane; i < len; i += 32) {
            col[dst + i] = dcol[src + i];
            data[dst + i] = __uint_as_float(dval[src + i]);
        }
    }
}

__global__ void path_mirror_fill_kernel(const uint64_t *__restrict__ mk, const uint32_t *__restrict__ mv,
                                        int64_t M, int B, const int64_t *__restrict__ rowptr,
                                        const int64_t *__restrict__ first, int32_t *__restrict__ col,
                                        float *__restrict__ data) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < M; f += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = mk[f];
        const int64_t r = (int64_t)(k >> B);
        const int64_t pos = rowptr[r] + (f - first[r]);
        col[pos] = (int32_t)(k & ((1ull << B) - 1ull));
        data[pos] = __uint_as_float(mv[f]);
    }
}

WalkArgs make_walk_args(const GraphView &g, const SamplerSpec &sp) {
    WalkArgs A;
    A.indptr = g.indptr;
    A.indices = g.indices;
    A.n = g.n;
    A.n_arcs = g.nnz;
    A.k0 = sp.k0;
    A.k1 = sp.k1;
    A.base = sp.base;
    A.thr_frac = sp.thr_frac;
    A.T = sp.T;
    A.B = sp.B;
    A.vinfo = nullptr;
    A.rlut = nullptr;
    for (int i = 0; i < 16; ++i) A.thr[i] = sp.thr[i];
    uint32_t k0 = sp.k0, k1 = sp.k1;
    for (int r = 0; r < 10; ++r) {
        A.rk[2 * r] = k0;
        A.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    A.T_eff = 0;
    for (int i = 0; i + 1 < sp.T; ++i)
        if (sp.thr[i] < (1ull << 32)) A.thr32[A.T_eff++] = (uint32_t)sp.thr[i];
    for (int i = A.T_eff; i < 16; ++i) A.thr32[i] = 0xFFFFFFFFu;
    A.ds_thr = nullptr;
    A.ds_w = nullptr;
    A.strat = sp.stratified;
    A.w = g.w;
    A.cum = nullptr;
    A.guide = nullptr;
    A.S = sp.S;
    A.vol = g.vol;
    A.wmax = g.wmax;
    A.base_magic = sp.base > 0 ? (~0ull) / sp.base + 1ull : 0ull;
    A.rmod[0] = 0;
    A.rmod[1] = 0xFFFFFFFFu;
    for (int r = 2; r <= 16; ++r) A.rmod[r] = (uint32_t)((1ull << 32) / (uint64_t)r);
    return A;
}

// Builds the per-vertex walk records into the workspace.
int attach_vinfo(Workspace &ws, const GraphView &g, WalkArgs *A, cudaStream_t st) {
    uint4 *vi = nullptr;
    LNE_TRY(ws.get("walk.vinfo", (size_t)std::max<int64_t>(g.n, 1), &vi));
    LNE_TRACE("build_vinfo", st);
    build_vinfo_kernel<<<(unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(g.n, 1), 256), num_sms() * 8), 256, 0, st>>>(
        g.indptr, g.n, vi);
    LNE_LAUNCH_CHECK();
    A->vinfo = vi;
    uint4 *ar = nullptr;
    LNE_TRY(ws.get("walk.arcrec", (size_t)std::max<int64_t>(g.nnz, 1), &ar));
    {
        LNE_TRACE("build_arcrec", st);
        build_arcrec_kernel<<<(unsigned)std::min<int64_t>(ceil_div(std::max<int64_t>(g.nnz, 1), 256), num_sms() * 16), 256, 0,
                              st>>>(g.indices, g.nnz, vi, ar);
        LNE_LAUNCH_CHECK();
    }
    A->arcrec = ar;
    uint8_t *lut = nullptr;
    LNE_TRY(ws.get("walk.rlut", 4096, &lut));
    build_rlut_kernel<<<16, 256, 0, st>>>(*A, lut);
    LNE_LAUNCH_CHECK();
    A->rlut = lut;
    if (g.w) {
        uint32_t *cum = nullptr;
        LNE_TRY(ws.get("walk.cum", (size_t)std::max<int64_t>(g.nnz, 1), &cum));
        LNE_TRACE("build_vinfo", st);
        build_cum_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g.n, 8), num_sms() * 16)), 256, 0,
                           st>>>(g.indptr, g.w, g.wdeg, g.n, cum);
        LNE_LAUNCH_CHECK();
        uint32_t *guide = nullptr;
        LNE_TRY(ws.get("walk.guide", (size_t)std::max<int64_t>(g.nnz, 1), &guide));
        build_guide_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g.n, 8), num_sms() * 16)), 256, 0,
                             st>>>(g.indptr, cum, g.n, guide);
        LNE_LAUNCH_CHECK();
        A->cum = cum;
        A->guide = guide;
    }
    return 0;
}

// Edge downsampling's per-arc coin thresholds and weights (when C > 0).
int attach_downsample(Workspace &ws, const GraphView &g, const SamplerSpec &sp, WalkArgs *A, cudaStream_t st) {
    if (!(sp.ds_C > 0.0)) return 0;
    uint64_t *thr = nullptr, *w = nullptr;
    LNE_TRY(ws.get("walk.ds_thr", (size_t)std::max<int64_t>(g.nnz, 1), &thr));
    LNE_TRY(ws.get("walk.ds_w", (size_t)std::max<int64_t>(g.nnz, 1), &w));
    LNE_TRACE("downsample_arcs", st);
    downsample_arcs_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g.n, 8), num_sms() * 16)), 256, 0,
                             st>>>(
        g.indptr, g.indices, g.w, g.wdeg, g.n, sp.ds_C, thr, w);
    LNE_LAUNCH_CHECK();
    A->ds_thr = thr;
    A->ds_w = w;
    return 0;
}

// Tile size: aim for ~32k samples per CTA but at least ~8 CTAs per SM overall.
int choose_tile_arcs(int64_t n_arcs, double rate) {
    double per_arc = rate < 1.0 ? 1.0 : rate;
    double total = per_arc * (double)n_arcs;
    double want = total / ((double)num_sms() * 8.0);
    if (want > 32768.0) want = 32768.0;
    if (want < 2048.0) want = 2048.0;
    int64_t t = (int64_t)(want / per_arc);
    if (t < 1) t = 1;
    if (t > 4096) t = 4096;
    return (int)t;
}

NetmfConst netmf_const(const SamplerSpec &sp) {
    NetmfConst k;
    k.a_off = sp.alpha_off;
    k.a_diag = sp.alpha_diag;
    k.off_hi = sp.off_hi;
    k.off_lo = sp.off_lo;
    k.diag_hi = sp.diag_hi;
    k.diag_lo = sp.diag_lo;
    k.wdeg = sp.wdeg;
    return k;
}

int walk_smem_bytes(int tile_arcs, int nb_smem) {
    return (tile_arcs + 1) * 4 + 2 * tile_arcs * 4 + nb_smem * 4;
}

// Per-tile offsets of arcs [a0, a1): returns the total number of samples.
// Launches the walk kernel variant the arguments need (see walk_emit_kernel).
template <typename KeyT, int MODE>
int launch_walk_emit(const WalkArgs &A, unsigned grid, int smem, cudaStream_t st, int64_t a_begin, int64_t a_end,
                     int tile_arcs, const int64_t *tile_off, KeyT *keys, int32_t *u1, int32_t *v1,
                     uint32_t *bucket_cnt, int nb_smem) {
    if (A.ds_thr || A.cum || A.w || A.strat) {
        LNE_TRY(allow_dynamic_smem(walk_emit_kernel<KeyT, MODE, true>));
        walk_emit_kernel<KeyT, MODE, true><<<grid, kWalkThreads, smem, st>>>(A, a_begin, a_end, tile_arcs, tile_off,
                                                                            keys, u1, v1, bucket_cnt, nb_smem);
    } else {
        LNE_TRY(allow_dynamic_smem(walk_emit_kernel<KeyT, MODE, false>));
        walk_emit_kernel<KeyT, MODE, false><<<grid, kWalkThreads, smem, st>>>(A, a_begin, a_end, tile_arcs, tile_off,
                                                                             keys, u1, v1, bucket_cnt, nb_smem);
    }
    LNE_LAUNCH_CHECK();
    return 0;
}

int tile_offsets(Workspace &ws, const WalkArgs &A, int64_t a0, int64_t a1, int tile_arcs,
                 int64_t **tile_off, int64_t *total, cudaStream_t st) {
    if (A.w) {   // a tile's sample count is a 32-bit sum: bound it by the heaviest arc
        const double max_rate = A.S * (double)A.wmax / A.vol;
        if ((max_rate + 1.0) * (double)tile_arcs >= 2147483648.0)
            return fail(LNE_ERR_UNSUPPORTED, "an arc's weight share of S is too large for the sample tiles");
    }
    const int64_t ntiles = ceil_div(a1 - a0, tile_arcs);
    uint32_t *tile_cnt = nullptr;
    LNE_TRY(ws.get("walk.tile_cnt", (size_t)ntiles, &tile_cnt));
    LNE_TRY(ws.get("walk.tile_off", (size_t)ntiles + 1, tile_off));
    {
        LNE_TRACE("tile_counts", st);
        tile_counts_kernel<<<(unsigned)ntiles, kWalkThreads, 0, st>>>(A, a0, a1, tile_arcs, tile_cnt);
        LNE_LAUNCH_CHECK();
    }
    LNE_TRY(scan_exclusive_u32_to_i64(tile_cnt, *tile_off, ntiles, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(total, *tile_off + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

}  // namespace

int make_sampler_spec(const GraphView &g, int T, const double *s, double S, double b, uint64_t seed,
                      SamplerSpec *out) {
    if (T < 1 || T > 16) return fail(LNE_ERR_INVALID, "T must be in 1..16");
    if (!s) return fail(LNE_ERR_INVALID, "window weights s are NULL");
    if (g.nnz <= 0) return fail(LNE_ERR_INVALID, "graph has no edges");
    if (!(S > 0.0)) return fail(LNE_ERR_INVALID, "sample count S must be > 0");
    SamplerSpec sp;
    sp.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    sp.k1 = (uint32_t)(seed >> 32);
    sp.T = T;
    for (int t = 0; t < T; ++t) sp.s_raw[t] = s[t];
    sp.S = S;
    sp.b = b;
    sp.seed = seed;
    double total = 0.0;
    for (int t = 0; t < T; ++t) {
        if (!(s[t] >= 0.0)) return fail(LNE_ERR_INVALID, "window weights must be >= 0");
        total += s[t];
    }
    if (!(total > 0.0)) return fail(LNE_ERR_INVALID, "window weights must not all be zero");
    // thr_i = min(2^32, floor(2^32 * (s_1 + .. + s_i) / (s_1 + .. + s_T)))
    double cum = 0.0;
    for (int i = 0; i + 1 < T; ++i) {
        cum += s[i];
        double p = cum / total;
        double x = std::floor(p * 4294967296.0);
        sp.thr[i] = x >= 4294967296.0 ? (1ull << 32) : x <= 0.0 ? 0ull : (uint64_t)x;
    }
    double rate = S / (double)g.nnz;
    if (rate >= 4294967295.0) return fail(LNE_ERR_UNSUPPORTED, "more than 2^32 samples per arc");
    double fl = std::floor(rate);
    sp.base = (uint32_t)fl;
    sp.thr_frac = (uint32_t)std::floor((rate - fl) * 4294967296.0);
    int B = 1;
    while (((int64_t)1 << B) < g.n) ++B;
    sp.B = B;
    if (b <= 0.0) b = 1.0;
    const double vol = g.w ? g.vol : (double)g.nnz;
    sp.wdeg = g.wdeg;
    const double vv = vol * vol;
    sp.alpha_off = vv / ((2.0 * S) * b);
    sp.alpha_diag = vv / (S * b);
    sp.off_hi = (float)sp.alpha_off;
    sp.off_lo = (float)(sp.alpha_off - (double)sp.off_hi);
    sp.diag_hi = (float)sp.alpha_diag;
    sp.diag_lo = (float)(sp.alpha_diag - (double)sp.diag_hi);
    *out = sp;
    return 0;
}

int sample_pairs(Workspace &ws, const GraphView &g, const SamplerSpec &sp, int64_t a0, int64_t a1,
                 int32_t *u1, int32_t *v1, int64_t capacity, int64_t *count, cudaStream_t st) {
    if (a0 < 0 || a1 > g.nnz || a0 > a1) return fail(LNE_ERR_INVALID, "arc range out of bounds");
    *count = 0;
    if (a0 == a1) return 0;
    WalkArgs A = make_walk_args(g, sp);
    LNE_TRY(attach_vinfo(ws, g, &A, st));
    LNE_TRY(attach_downsample(ws, g, sp, &A, st));
    const int tile_arcs = choose_tile_arcs(a1 - a0, (double)sp.base + 0.5);
    int64_t *tile_off = nullptr;
    int64_t total = 0;
    LNE_TRY(tile_offsets(ws, A, a0, a1, tile_arcs, &tile_off, &total, st));
    *count = total;
    if (total > capacity) return fail(LNE_ERR_INVALID, "output capacity too small for the sampled pairs");
    const int64_t ntiles = ceil_div(a1 - a0, tile_arcs);
    const int smem = walk_smem_bytes(tile_arcs, 0);
    // dynamic shared memory comes on top of the kernel's static tables
    {
        LNE_TRACE("walk_emit", st);
        LNE_TRY((launch_walk_emit<uint32_t, 0>(A, (unsigned)ntiles, smem, st, a0, a1, tile_arcs, tile_off, nullptr, u1,
                                              v1, nullptr, 0)));
    }
    return 0;
}

namespace {

// Sample, bucket and reduce: distinct keys with counts in per-bucket regions.
struct Reduced {
    int64_t total = 0;
    int nb = 0;
    int64_t *bucket_off = nullptr;   // [nb+1], region of bucket b in rkey/rcnt
    uint32_t *distinct = nullptr;    // [nb]
    uint32_t *rkey = nullptr;
    uint32_t *rcnt = nullptr;
};

int sample_and_reduce(Workspace &ws, const GraphView &g, const SamplerSpec &sp, Reduced *R,
                      cudaStream_t st) {
    if (2 * sp.B > 32)
        return fail(LNE_ERR_UNSUPPORTED, "graphs with more than 65536 vertices need 64-bit pair keys (not in this build)");
    WalkArgs A = make_walk_args(g, sp);
    LNE_TRY(attach_vinfo(ws, g, &A, st));
    const int tile_arcs = choose_tile_arcs(g.nnz, (double)sp.base + 0.5);
    int64_t *tile_off = nullptr;
    int64_t total = 0;
    LNE_TRY(tile_offsets(ws, A, 0, g.nnz, tile_arcs, &tile_off, &total, st));
    R->total = total;
    const uint64_t max_key = ((uint64_t)(g.n - 1) << sp.B) | (uint64_t)(g.n - 1);
    const int nb = (int)((max_key >> kBucketBits) + 1);
    R->nb = nb;
    uint32_t *keys0 = nullptr, *keys1 = nullptr, *bucket_cnt = nullptr;
    unsigned long long *cursor = nullptr;
    LNE_TRY(ws.get("spars.keys0", (size_t)std::max<int64_t>(total, 1), &keys0));
    LNE_TRY(ws.get("spars.keys1", (size_t)std::max<int64_t>(total, 1), &keys1));
    LNE_TRY(ws.get("spars.bucket_cnt", (size_t)nb, &bucket_cnt));
    LNE_TRY(ws.get("spars.bucket_off", (size_t)nb + 1, &R->bucket_off));
    LNE_TRY(ws.get("spars.cursor", (size_t)nb, &cursor));
    LNE_TRY(ws.get("spars.distinct", (size_t)nb, &R->distinct));
    LNE_CUDA_TRY(cudaMemsetAsync(bucket_cnt, 0, sizeof(uint32_t) * nb, st));
    const int64_t ntiles = ceil_div(g.nnz, tile_arcs);
    const int nb_smem = nb <= kMaxSmemBuckets ? nb : 0;
    const int smem = walk_smem_bytes(tile_arcs, nb_smem);
    // dynamic shared memory comes on top of the kernel's static tables
    {
        LNE_TRACE("walk_emit", st);
        LNE_TRY((launch_walk_emit<uint32_t, 1>(A, (unsigned)ntiles, smem, st, 0, g.nnz, tile_arcs, tile_off, keys0,
                                              nullptr, nullptr, bucket_cnt, nb_smem)));
    }
    LNE_TRY(scan_exclusive_u32_to_i64(bucket_cnt, R->bucket_off, nb, st));
    static_assert(sizeof(unsigned long long) == sizeof(int64_t), "cursor layout");
    LNE_CUDA_TRY(cudaMemcpyAsync(cursor, R->bucket_off, sizeof(int64_t) * nb,
                                 cudaMemcpyDeviceToDevice, st));
    if (total > 0) {
        if (nb <= kMaxSmemBuckets) {
            const int sm = nb * (8 + 4);
            if (sm > 48 * 1024)
                LNE_TRY(allow_dynamic_smem(bucket_scatter_kernel<uint32_t>));
            const int64_t grid = ceil_div(total, (int64_t)kScatterThreads * kScatterItems);
            LNE_TRACE("bucket_scatter", st);
            bucket_scatter_kernel<uint32_t><<<(unsigned)grid, kScatterThreads, sm, st>>>(
                keys0, total, keys1, cursor, nb);
            LNE_LAUNCH_CHECK();
        } else {
            LNE_TRACE("bucket_scatter", st);
            bucket_scatter_global_kernel<uint32_t><<<(unsigned)num_sms() * 8, 256, 0, st>>>(keys0, total, keys1, cursor);
            LNE_LAUNCH_CHECK();
        }
    }
    // reduce into keys0 (reused) and a count array of the same size
    uint32_t *rcnt = nullptr;
    LNE_TRY(ws.get("spars.rcnt", (size_t)std::max<int64_t>(total, 1), &rcnt));
    const int rsmem = (1 << kBucketBits) * 4;
    LNE_TRY(allow_dynamic_smem(bucket_reduce_kernel<uint32_t>));
    {
        LNE_TRACE("bucket_reduce", st);
        bucket_reduce_kernel<uint32_t><<<nb, kReduceThreads, rsmem, st>>>(keys1, R->bucket_off, keys0,
                                                                          rcnt, R->distinct);
        LNE_LAUNCH_CHECK();
    }
    R->rkey = keys0;
    R->rcnt = rcnt;
    return 0;
}

int compact_counts(Workspace &ws, const SamplerSpec &sp, const Reduced &R, CountsResult *out,
                   cudaStream_t st) {
    int64_t *dst_off = nullptr;
    LNE_TRY(ws.get("spars.dst_off", (size_t)R.nb + 1, &dst_off));
    LNE_TRY(scan_exclusive_u32_to_i64(R.distinct, dst_off, R.nb, st));
    int64_t nnz = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&nnz, dst_off + R.nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    LNE_TRY(ws.get("counts.x", (size_t)std::max<int64_t>(nnz, 1), &out->x));
    LNE_TRY(ws.get("counts.y", (size_t)std::max<int64_t>(nnz, 1), &out->y));
    LNE_TRY(ws.get("counts.cnt", (size_t)std::max<int64_t>(nnz, 1), &out->cnt));
    {
        LNE_TRACE("compact", st);
        compact_kernel<uint32_t><<<R.nb, 256, 0, st>>>(R.rkey, R.rcnt, R.bucket_off, dst_off, sp.B,
                                                       out->x, out->y, out->cnt);
        LNE_LAUNCH_CHECK();
    }
    out->nnz = nnz;
    out->total_samples = R.total;
    return 0;
}

}  // namespace

int bucket_counts(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CountsResult *out,
                  cudaStream_t st) {
    Reduced R;
    LNE_TRY(sample_and_reduce(ws, g, sp, &R, st));
    LNE_TRY(compact_counts(ws, sp, R, out, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int bucket_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CsrResult *out,
               cudaStream_t st) {
    Reduced R;
    LNE_TRY(sample_and_reduce(ws, g, sp, &R, st));
    CountsResult C;
    LNE_TRY(compact_counts(ws, sp, R, &C, st));
    const int64_t nnz_c = C.nnz;
    float *val = nullptr;
    uint8_t *keep = nullptr;
    uint32_t *rowcnt = nullptr;
    LNE_TRY(ws.get("csr.val_c", (size_t)std::max<int64_t>(nnz_c, 1), &val));
    LNE_TRY(ws.get("csr.keep", (size_t)std::max<int64_t>(nnz_c, 1), &keep));
    LNE_TRY(ws.get("csr.rowcnt", (size_t)g.n, &rowcnt));
    LNE_TRY(ws.get("csr.indptr", (size_t)g.n + 1, &out->indptr));
    LNE_CUDA_TRY(cudaMemsetAsync(rowcnt, 0, sizeof(uint32_t) * g.n, st));
    const int grid = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(nnz_c, 1), 256), num_sms() * 16);
    {
        LNE_TRACE("trunclog", st);
        trunclog_kernel<<<grid, 256, 0, st>>>(C.x, C.y, C.cnt, nnz_c, g.indptr, netmf_const(sp), val, keep,
                                              rowcnt);
        LNE_LAUNCH_CHECK();
    }
    LNE_TRY(scan_exclusive_u32_to_i64(rowcnt, out->indptr, g.n, st));
    int64_t nnz = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&nnz, out->indptr + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    LNE_TRY(ws.get("csr.indices", (size_t)std::max<int64_t>(nnz, 1), &out->indices));
    LNE_TRY(ws.get("csr.data", (size_t)std::max<int64_t>(nnz, 1), &out->data));
    LNE_CUDA_TRY(cudaMemsetAsync(rowcnt, 0, sizeof(uint32_t) * g.n, st));
    {
        LNE_TRACE("csr_fill", st);
        csr_fill_kernel<<<grid, 256, 0, st>>>(C.x, C.y, val, keep, nnz_c, out->indptr, rowcnt,
                                              out->indices, out->data);
        LNE_LAUNCH_CHECK();
    }
    int *too_long = nullptr;
    LNE_TRY(ws.get("csr.too_long", 1, &too_long));
    LNE_CUDA_TRY(cudaMemsetAsync(too_long, 0, sizeof(int), st));
    const int ssmem = kSortMax * 8;
    LNE_TRY(allow_dynamic_smem(csr_row_sort_kernel));
    {
        LNE_TRACE("csr_row_sort", st);
        csr_row_sort_kernel<<<(unsigned)g.n, kSortThreads, ssmem, st>>>(out->indptr, out->indices,
                                                                       out->data, too_long);
        LNE_LAUNCH_CHECK();
    }
    int tl = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&tl, too_long, sizeof(int), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (tl > 0) return fail(LNE_ERR_UNSUPPORTED, "a sparsifier row is longer than the in-shared-memory row sort handles");
    out->n = g.n;
    out->nnz = nnz;
    return 0;
}


namespace {

struct Table {
    uint32_t *T = nullptr;    // counts, then the float bits of the Eq. 1 values
    uint64_t *W = nullptr;    // summed weights (edge downsampling only)
    uint32_t *packed = nullptr;   // packed narrow counters not yet decoded into T (plain walks)
    int64_t ld = 0;
    int nt = 0;
};

// ---- sort path: host side ----------------------------------------------------

// Samples of every arc as 64-bit keys, sorted, as unique keys with counts.
// On return the unique keys are in *uk ("sort.k0" or "sort.k1"), counts in
// "sort.cnt"; the other key buffer and the run starts are released. With edge
// downsampling each key carries its arc, a dropped draw's key is all ones
// (sorted past every pair: the sort takes one more bit when n = 2^B, where the
// all-ones pair of B-bit halves is a real vertex pair), and *w gets the summed
// weights ("sort.w"); "sort.cnt" is then only sized for the values.
struct SortRaw {
    int64_t total = 0, U = 0;
    uint64_t *uk = nullptr;
    uint32_t *cnt = nullptr;
    uint64_t *w = nullptr;
    const char *uk_name = nullptr, *spare_name = nullptr;
};

int sort_raw(Workspace &ws, const GraphView &g, const SamplerSpec &sp, SortRaw *R, cudaStream_t st) {
    if (2 * sp.B > 64) return fail(LNE_ERR_UNSUPPORTED, "pair keys need 2 ceil(log2 n) <= 64 bits");
    WalkArgs A = make_walk_args(g, sp);
    LNE_TRY(attach_vinfo(ws, g, &A, st));
    LNE_TRY(attach_downsample(ws, g, sp, &A, st));
    const bool ds = A.ds_thr != nullptr;
    const int bits = 2 * sp.B + ((ds && ((int64_t)1 << sp.B) == g.n) ? 1 : 0);
    if (bits > 64) return fail(LNE_ERR_UNSUPPORTED, "downsampled pair keys need 2 ceil(log2 n) + 1 <= 64 bits");
    if (ds && g.nnz > (int64_t)UINT32_MAX)
        return fail(LNE_ERR_UNSUPPORTED, "edge downsampling on the sort path needs fewer than 2^32 arcs");
    const int tile_arcs = choose_tile_arcs(g.nnz, (double)sp.base + 0.5);
    int64_t *tile_off = nullptr;
    int64_t total = 0;
    LNE_TRY(tile_offsets(ws, A, 0, g.nnz, tile_arcs, &tile_off, &total, st));
    R->total = total;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    LNE_TRY(ws.get("sort.k0", (size_t)std::max<int64_t>(total, 1), &k0));
    LNE_TRY(ws.get("sort.k1", (size_t)std::max<int64_t>(total, 1), &k1));
    uint32_t *arc0 = nullptr, *arc1 = nullptr;
    if (ds) {
        LNE_TRY(ws.get("sort.a0", (size_t)std::max<int64_t>(total, 1), &arc0));
        LNE_TRY(ws.get("sort.a1", (size_t)std::max<int64_t>(total, 1), &arc1));
    }
    const int64_t ntiles = ceil_div(g.nnz, tile_arcs);
    const int smem = walk_smem_bytes(tile_arcs, 0);
    {
        LNE_TRACE("walk_keys", st);
        LNE_TRY((launch_walk_emit<uint64_t, 3>(A, (unsigned)ntiles, smem, st, 0, g.nnz, tile_arcs, tile_off, k0,
                                              reinterpret_cast<int32_t *>(arc0), nullptr, nullptr, 0)));
    }
    bool in_alt = false;
    LNE_TRY(radix_sort_u64(ws, k0, k1, arc0, arc1, total, bits, &in_alt, st));
    uint64_t *sorted = in_alt ? k1 : k0, *spare = in_alt ? k0 : k1;
    ws.release("sort.offs");
    if (ds) {
        // the dropped draws sort last: run lengths over the kept ones only
        int64_t kept = 0;
        LNE_TRY(count_below(ws, sorted, total, ~0ull, &kept, st));
        LNE_TRY(ws.get("sort.w", (size_t)std::max<int64_t>(kept, 1), &R->w));
        LNE_TRY(run_length_weighted(ws, sorted, in_alt ? arc1 : arc0, A.ds_w, kept, spare, R->w, &R->U, st));
        ws.release("sort.a0");
        ws.release("sort.a1");
        LNE_TRY(ws.get("sort.cnt", (size_t)std::max<int64_t>(R->U, 1), &R->cnt));
    } else {
        LNE_TRY(ws.get("sort.cnt", (size_t)std::max<int64_t>(total, 1), &R->cnt));
        LNE_TRY(run_length(ws, sorted, total, spare, R->cnt, &R->U, st));
    }
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    R->uk = spare;
    R->uk_name = in_alt ? "sort.k0" : "sort.k1";
    R->spare_name = in_alt ? "sort.k1" : "sort.k0";
    ws.release(R->spare_name);
    return 0;
}

void sort_release(Workspace &ws) {
    for (const char *n : {"sort.k0", "sort.k1", "sort.cnt", "sort.w", "sort.a0", "sort.a1", "sort.bound", "sort.offs",
                          "sort.mk", "sort.mv",
                          "path.dcol", "path.dval", "path.tk", "path.tm", "path.ko", "path.mo", "path.deg",
                          "path.dlen", "path.rowlen", "path.dstart", "path.first", "path.end"})
        ws.release(n);
}

int sort_counts(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CountsResult *out, cudaStream_t st) {
    SortRaw R;
    LNE_TRY(sort_raw(ws, g, sp, &R, st));
    const int64_t u = R.U;
    LNE_TRY(ws.get("counts.x", (size_t)std::max<int64_t>(u, 1), &out->x));
    LNE_TRY(ws.get("counts.y", (size_t)std::max<int64_t>(u, 1), &out->y));
    if (R.w) LNE_TRY(ws.get("counts.w", (size_t)std::max<int64_t>(u, 1), &out->weight));
    else LNE_TRY(ws.get("counts.cnt", (size_t)std::max<int64_t>(u, 1), &out->cnt));
    if (u > 0) {
        LNE_TRACE("decode_keys", st);
        decode_keys_kernel<<<(unsigned)std::min<int64_t>(ceil_div(u, 256), num_sms() * 16), 256, 0, st>>>(
            R.uk, u, sp.B, out->x, out->y);
        LNE_LAUNCH_CHECK();
        if (R.w)
            LNE_CUDA_TRY(cudaMemcpyAsync(out->weight, R.w, sizeof(uint64_t) * u, cudaMemcpyDeviceToDevice, st));
        else
            LNE_CUDA_TRY(cudaMemcpyAsync(out->cnt, R.cnt, sizeof(uint32_t) * u, cudaMemcpyDeviceToDevice, st));
    }
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    sort_release(ws);
    out->nnz = u;
    out->total_samples = R.total;
    return 0;
}

// Symmetric CSR from U ascending unique pair keys uk and their Eq. 1 value
// bits val (0 = dropped), with per-tile (kPathTile) kept / kept off-diagonal
// counts tk / tm. uk and val (workspace buffers uk_name / val_name) serve as
// spare buffers of the mirrored sort and are released.
int assemble_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, uint64_t *uk, uint32_t *val, int64_t U,
                 const uint32_t *tk, const uint32_t *tm, const char *uk_name, const char *val_name, CsrResult *out,
                 cudaStream_t st) {
    const int64_t n = g.n;
    const int64_t ntiles = std::max<int64_t>(1, ceil_div(U, (int64_t)kPathTile));
    const unsigned egrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 16));
    uint32_t *dlen = nullptr, *rowlen = nullptr;
    int64_t *ko = nullptr, *mo = nullptr, *first = nullptr, *end = nullptr;
    unsigned long long *dstart = nullptr;
    LNE_TRY(ws.get("path.ko", (size_t)ntiles + 1, &ko));
    LNE_TRY(ws.get("path.mo", (size_t)ntiles + 1, &mo));
    LNE_TRY(ws.get("path.dlen", (size_t)n, &dlen));
    LNE_TRY(ws.get("path.rowlen", (size_t)n, &rowlen));
    LNE_TRY(ws.get("path.dstart", (size_t)n, &dstart));
    LNE_TRY(ws.get("path.first", (size_t)n, &first));
    LNE_TRY(ws.get("path.end", (size_t)n, &end));
    LNE_TRY(ws.get("csr.indptr", (size_t)n + 1, &out->indptr));
    LNE_CUDA_TRY(cudaMemsetAsync(dlen, 0, sizeof(uint32_t) * n, st));
    LNE_CUDA_TRY(cudaMemsetAsync(end, 0, sizeof(int64_t) * n, st));
    LNE_CUDA_TRY(cudaMemsetAsync(dstart, 0xFF, sizeof(unsigned long long) * n, st));
    LNE_TRY(scan_exclusive_u32_to_i64(tk, ko, ntiles, st));
    LNE_TRY(scan_exclusive_u32_to_i64(tm, mo, ntiles, st));
    int64_t nk = 0, nm = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&nk, ko + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaMemcpyAsync(&nm, mo + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t *dcol = nullptr;
    uint32_t *dval = nullptr, *mv = nullptr;
    uint64_t *mk = nullptr;
    LNE_TRY(ws.get("path.dcol", (size_t)std::max<int64_t>(nk, 1), &dcol));
    LNE_TRY(ws.get("path.dval", (size_t)std::max<int64_t>(nk, 1), &dval));
    LNE_TRY(ws.get("sort.mk", (size_t)std::max<int64_t>(nm, 1), &mk));
    LNE_TRY(ws.get("sort.mv", (size_t)std::max<int64_t>(nm, 1), &mv));
    {
        LNE_TRACE("path_rows", st);
        path_rows_kernel<<<(unsigned)ntiles, kPathThreads, 0, st>>>(uk, val, U, sp.B, ko, mo, dlen, dstart, dcol,
                                                                   dval, mk, mv);
        LNE_LAUNCH_CHECK();
    }
    // mirrored entries sorted by (row y, column x); the unique keys and the
    // values are no longer needed and serve as the sort's spare buffers
    bool in_alt = false;
    LNE_TRY(radix_sort_u64(ws, mk, uk, mv, val, nm, 2 * sp.B, &in_alt, st));
    const uint64_t *smk = in_alt ? uk : mk;
    const uint32_t *smv = in_alt ? val : mv;
    const unsigned mgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nm, 256), num_sms() * 16));
    {
        LNE_TRACE("path_rows", st);
        if (nm > 0) {
            path_mirror_rows_kernel<<<mgrid, 256, 0, st>>>(smk, nm, sp.B, first, end);
            LNE_LAUNCH_CHECK();
        }
        path_row_total_kernel<<<egrid, 256, 0, st>>>(dlen, end, first, n, rowlen);
        LNE_LAUNCH_CHECK();
    }
    LNE_TRY(scan_exclusive_u32_to_i64(rowlen, out->indptr, n, st));
    int64_t nnz = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&nnz, out->indptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    // the buffers not holding the sorted mirrored entries are free now
    if (in_alt) {
        ws.release("sort.mk");
        ws.release("sort.mv");
    } else {
        ws.release(uk_name);
        ws.release(val_name);
    }
    LNE_TRY(ws.get("csr.indices", (size_t)std::max<int64_t>(nnz, 1), &out->indices));
    LNE_TRY(ws.get("csr.data", (size_t)std::max<int64_t>(nnz, 1), &out->data));
    {
        LNE_TRACE("path_fill", st);
        path_direct_fill_kernel<<<egrid, 256, 0, st>>>(dcol, dval, dlen, dstart, out->indptr, n, out->indices,
                                                       out->data);
        LNE_LAUNCH_CHECK();
        if (nm > 0) {
            path_mirror_fill_kernel<<<mgrid, 256, 0, st>>>(smk, smv, nm, sp.B, out->indptr, first, out->indices,
                                                          out->data);
            LNE_LAUNCH_CHECK();
        }
    }
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    sort_release(ws);
    ws.release(uk_name);
    ws.release(val_name);
    out->n = n;
    out->nnz = nnz;
    return 0;
}

int sort_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CsrResult *out, cudaStream_t st) {
    // a previous sparsifier's arrays are rebuilt below: free them before the
    // sort's peak (tens of GB for billions of samples)
    ws.release("csr.indices");
    ws.release("csr.data");
    SortRaw R;
    LNE_TRY(sort_raw(ws, g, sp, &R, st));
    const int64_t U = R.U, n = g.n;
    const int64_t ntiles = std::max<int64_t>(1, ceil_div(U, (int64_t)kPathTile));
    const unsigned egrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 16));
    uint32_t *tk = nullptr, *tm = nullptr, *deg = nullptr;
    LNE_TRY(ws.get("path.tk", (size_t)ntiles, &tk));
    LNE_TRY(ws.get("path.tm", (size_t)ntiles, &tm));
    LNE_TRY(ws.get("path.deg", (size_t)n, &deg));
    {
        LNE_TRACE("path_value", st);
        if (!g.wdeg) {
            degree_kernel<<<egrid, 256, 0, st>>>(g.indptr, n, deg);
            LNE_LAUNCH_CHECK();
        }
        // values overwrite the counts (the counts are not needed afterwards)
        path_value_kernel<<<(unsigned)ntiles, kPathThreads, 0, st>>>(R.uk, R.cnt, R.w, U, sp.B,
                                                                    g.wdeg ? g.wdeg : deg, netmf_const(sp), tk, tm);
        LNE_LAUNCH_CHECK();
    }
    return assemble_csr(ws, g, sp, R.uk, R.cnt, U, tk, tm, R.uk_name, "sort.cnt", out, st);
}

bool use_table(const GraphView &g, const SamplerSpec &sp) {
    if (sp.aggregation == LNE_AGG_TABLE) return true;
    if (sp.aggregation != LNE_AGG_AUTO) return false;
    if (g.n > 65536) return false;
    // measured on GB300: the table's passes cost ~4e-12 s per counter of the
    // n_pad^2 table, the sort path ~1.9e-10 s per sample -- the table when it
    // is the cheaper of the two
    const double ld = (double)ceil_div(g.n, (int64_t)kTile) * kTile;
    const double samples = (double)g.nnz * ((double)sp.base + (double)sp.thr_frac / 4294967296.0);
    return ld * ld <= 40.0 * samples;
}

// Walk every arc's samples and count them into the dense upper-triangle table.
// decode = false leaves the plain walk's packed counters in tb->packed for
// table_decode_values_kernel (otherwise T holds the exact counts on return).
int sample_table(Workspace &ws, const GraphView &g, const SamplerSpec &sp, Table *tb, cudaStream_t st,
                 bool decode = true) {
    if (g.n > 65536) return fail(LNE_ERR_UNSUPPORTED, "the dense count table needs n <= 65536");
    const int nt = (int)ceil_div(g.n, kTile);
    const int64_t ld = (int64_t)nt * kTile;
    LNE_TRY(ws.get("table.T", (size_t)(ld * ld), &tb->T));
    tb->ld = ld;
    tb->nt = nt;
    LNE_CUDA_TRY(cudaMemsetAsync(tb->T, 0, sizeof(uint32_t) * (size_t)(ld * ld), st));
    WalkArgs A = make_walk_args(g, sp);
    LNE_TRY(attach_vinfo(ws, g, &A, st));
    LNE_TRY(attach_downsample(ws, g, sp, &A, st));
    const int tile_arcs = choose_tile_arcs(g.nnz, (double)sp.base + 0.5);
    const int64_t ntiles = ceil_div(g.nnz, tile_arcs);
    const int smem = walk_smem_bytes(tile_arcs, 0);
    if (!A.ds_thr && !A.w && !A.strat) {
        // tiles of at most kTabMaxTileArcs arcs, whose walk records sit in shared memory
        const int tab_arcs = std::min(tile_arcs, kTabMaxTileArcs);
        const int64_t tab_tiles = ceil_div(g.nnz, tab_arcs);
        const int tab_smem = tab_arcs * 32 + (tab_arcs + 1) * 4;
        // packed narrow counters, decoded into the 32-bit table afterwards
        constexpr int BITS = kTabBits;
        constexpr int P = TabPack<BITS>::P;
        uint32_t *tp = nullptr;
        LNE_TRY(ws.get("table.packed", (size_t)(ld * ld / P), &tp));
        LNE_CUDA_TRY(cudaMemsetAsync(tp, 0, sizeof(uint32_t) * (size_t)(ld * ld / P), st));
        {
            LNE_TRACE("walk_count", st);
            LNE_TRY(allow_dynamic_smem(walk_table_kernel<BITS>));
            walk_table_kernel<BITS><<<(unsigned)tab_tiles, kTabThreads, tab_smem, st>>>(A, tab_arcs, tp, tb->T,
                                                                                         (uint32_t)ld);
            LNE_LAUNCH_CHECK();
        }
        if (!decode) {
            tb->packed = tp;
            return 0;
        }
        LNE_TRACE("table_decode", st);
        table_decode_kernel<BITS><<<(unsigned)std::min<int64_t>(g.n, num_sms() * 8), 256, 0, st>>>(tp, tb->T,
                                                                                                    (int)g.n, ld);
        LNE_LAUNCH_CHECK();
        return 0;
    }
    LNE_TRACE("walk_count", st);
    if (A.ds_thr) {   // downsampled: 64-bit weight sums
        LNE_TRY(ws.get("table.W", (size_t)(ld * ld), &tb->W));
        LNE_CUDA_TRY(cudaMemsetAsync(tb->W, 0, sizeof(uint64_t) * (size_t)(ld * ld), st));
        LNE_TRY((launch_walk_emit<uint64_t, 2>(A, (unsigned)ntiles, smem, st, 0, g.nnz, tile_arcs, nullptr, tb->W,
                                              nullptr, nullptr, nullptr, (int)ld)));
    } else {
        LNE_TRY((launch_walk_emit<uint32_t, 2>(A, (unsigned)ntiles, smem, st, 0, g.nnz, tile_arcs, nullptr, tb->T,
                                              nullptr, nullptr, nullptr, (int)ld)));
    }
    return 0;
}

int total_samples(Workspace &ws, const GraphView &g, const SamplerSpec &sp, int64_t *total, cudaStream_t st) {
    WalkArgs A = make_walk_args(g, sp);
    const int tile_arcs = choose_tile_arcs(g.nnz, (double)sp.base + 0.5);
    int64_t *tile_off = nullptr;
    return tile_offsets(ws, A, 0, g.nnz, tile_arcs, &tile_off, total, st);
}

int table_counts(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CountsResult *out, cudaStream_t st) {
    Table tb;
    LNE_TRY(sample_table(ws, g, sp, &tb, st));
    uint32_t *rc = nullptr;
    int64_t *off = nullptr;
    LNE_TRY(ws.get("table.rownnz", (size_t)g.n, &rc));
    LNE_TRY(ws.get("table.rowoff", (size_t)g.n + 1, &off));
    {
        LNE_TRACE("table_row_nnz", st);
        if (tb.W) table_row_nnz_kernel<uint64_t><<<(unsigned)g.n, 256, 0, st>>>(tb.W, tb.ld, (int)g.n, rc);
        else table_row_nnz_kernel<uint32_t><<<(unsigned)g.n, 256, 0, st>>>(tb.T, tb.ld, (int)g.n, rc);
        LNE_LAUNCH_CHECK();
    }
    LNE_TRY(scan_exclusive_u32_to_i64(rc, off, g.n, st));
    int64_t nnz = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&nnz, off + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    LNE_TRY(ws.get("counts.x", (size_t)std::max<int64_t>(nnz, 1), &out->x));
    LNE_TRY(ws.get("counts.y", (size_t)std::max<int64_t>(nnz, 1), &out->y));
    {
        LNE_TRACE("table_compact", st);
        if (tb.W) {
            LNE_TRY(ws.get("counts.w", (size_t)std::max<int64_t>(nnz, 1), &out->weight));
            table_compact_kernel<uint64_t><<<(unsigned)g.n, 256, 0, st>>>(tb.W, tb.ld, (int)g.n, off, out->x,
                                                                          out->y, out->weight);
        } else {
            LNE_TRY(ws.get("counts.cnt", (size_t)std::max<int64_t>(nnz, 1), &out->cnt));
            table_compact_kernel<uint32_t><<<(unsigned)g.n, 256, 0, st>>>(tb.T, tb.ld, (int)g.n, off, out->x,
                                                                          out->y, out->cnt);
        }
        LNE_LAUNCH_CHECK();
    }
    out->nnz = nnz;
    LNE_TRY(total_samples(ws, g, sp, &out->total_samples, st));
    return 0;
}

int table_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CsrResult *out, cudaStream_t st) {
    Table tb;
    LNE_TRY(sample_table(ws, g, sp, &tb, st, false));
    const int n = (int)g.n;
    // the samples bound the counted pairs: below ~15% of all pairs the value
    // pass queues its counters (measured: 2.02 -> 1.09 ms at 3% on a
    // 39k-vertex graph, 0.18 -> 0.21 ms at 41% on the benchmark's)
    const double samples = (double)g.nnz * ((double)sp.base + (double)sp.thr_frac / 4294967296.0);
    const bool sparse = 2.0 * samples < 0.15 * (double)n * (double)n;
    {
        LNE_TRACE("table_values", st);
        if (tb.W) table_values_w_kernel<<<(unsigned)n, 256, 0, st>>>(tb.W, tb.T, tb.ld, n, g.indptr, netmf_const(sp));
        else if (tb.packed && sparse)
            table_decode_values_sparse_kernel<kTabBits><<<(unsigned)n, kDvThreads, 0, st>>>(
                tb.packed, tb.T, tb.ld, n, g.indptr, netmf_const(sp));
        else if (tb.packed)
            table_decode_values_kernel<kTabBits><<<(unsigned)n, 256, 0, st>>>(tb.packed, tb.T, tb.ld, n, g.indptr,
                                                                             netmf_const(sp));
        else table_values_kernel<<<(unsigned)n, 256, 0, st>>>(tb.T, tb.ld, n, g.indptr, netmf_const(sp));
        LNE_LAUNCH_CHECK();
    }
    uint32_t *rowtile = nullptr, *rowcnt = nullptr;
    LNE_TRY(ws.get("table.rowtile", (size_t)n * tb.nt, &rowtile));
    LNE_TRY(ws.get("table.rowcnt", (size_t)n, &rowcnt));
    LNE_TRY(ws.get("csr.indptr", (size_t)n + 1, &out->indptr));
    dim3 grid((unsigned)tb.nt, (unsigned)tb.nt);
    {
        LNE_TRACE("tile_count", st);
        tile_count_kernel<<<grid, 256, 0, st>>>(tb.T, tb.ld, n, tb.nt, rowtile);
        LNE_LAUNCH_CHECK();
    }
    {
        LNE_TRACE("row_tile_scan", st);
        row_tile_scan_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(rowtile, n, tb.nt, rowcnt);
        LNE_LAUNCH_CHECK();
    }
    LNE_TRY(scan_exclusive_u32_to_i64(rowcnt, out->indptr, n, st));
    int64_t nnz = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&nnz, out->indptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    LNE_TRY(ws.get("csr.indices", (size_t)std::max<int64_t>(nnz, 1), &out->indices));
    LNE_TRY(ws.get("csr.data", (size_t)std::max<int64_t>(nnz, 1), &out->data));
    {
        LNE_TRACE("tile_fill", st);
        tile_fill_kernel<<<grid, 256, 0, st>>>(tb.T, tb.ld, n, tb.nt, rowtile, out->indptr, out->indices, out->data);
        LNE_LAUNCH_CHECK();
    }
    out->n = g.n;
    out->nnz = nnz;
    out->dense = reinterpret_cast<const float *>(tb.T);
    out->dense_ld = tb.ld;
    return 0;
}

// ---- weighted graphs ----------------------------------------------------------

// A warp per vertex: d_u = sum of its arc weights (exact, 64-bit), 1 / d_u and
// the float weights for the graph products, d_u added into the volume. flags
// bit 0: a zero weight, bit 1: a degree of 2^31 or more.
__global__ void weighted_prep_kernel(const int64_t *__restrict__ indptr, const uint32_t *__restrict__ w, int64_t n,
                                     uint32_t *__restrict__ wdeg, float *__restrict__ dinv, float *__restrict__ wf,
                                     unsigned long long *__restrict__ vol, unsigned int *__restrict__ flags,
                                     unsigned int *__restrict__ wmax) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
        const int64_t a0 = indptr[x], a1 = indptr[x + 1];
        uint64_t d = 0;
        bool zero = false;
        uint32_t mx = 0;
        for (int64_t a = a0 + lane; a < a1; a += 32) {
            const uint32_t v = __ldg(w + a);
            zero |= v == 0u;
            d += v;
            mx = v > mx ? v : mx;
            wf[a] = (float)v;
        }
        if (mx) atomicMax(wmax, mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        zero = __any_sync(0xffffffffu, zero);
        if (lane == 0) {
            const bool big = d >= (1ull << 31);
            wdeg[x] = big ? 0u : (uint32_t)d;
            dinv[x] = d > 0 ? 1.f / (float)d : 0.f;
            atomicAdd(vol, (unsigned long long)d);
            if (zero) atomicOr(flags, 1u);
            if (big) atomicOr(flags, 2u);
        }
    }
}

// ---- window-stratified counts --------------------------------------------

struct StratW {
    uint32_t w[16];   // w_r for r = 1..T (index r - 1), 2^-24 units
};

// Sorted unique (pair << 4 | r - 1) keys -> pair keys (for the run lengths of
// the pairs) and window lengths.
__global__ void strat_split_kernel(const uint64_t *__restrict__ ukr, int64_t U, uint64_t *__restrict__ pairkey,
                                   uint8_t *__restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < U; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ukr[i];
        pairkey[i] = k >> 4;
        r[i] = (uint8_t)((k & 15u) + 1u);
    }
}

// Stratified counts as (x, y, r, count) entries.
__global__ void strat_decode_kernel(const uint64_t *__restrict__ ukr, int64_t U, int B, int32_t *__restrict__ x,
                                    int32_t *__restrict__ y, uint8_t *__restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < U; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ukr[i];
        x[i] = (int32_t)(k >> (B + 4));
        y[i] = (int32_t)((k >> 4) & ((1ull << B) - 1ull));
        r[i] = (uint8_t)((k & 15u) + 1u);
    }
}

// K_s = sum over the pair's entries of w_r C_r (exact 64-bit sum), its Eq. 1
// value bits, and per tile the kept and kept off-diagonal pair counts (the
// layout path_value_kernel gives the CSR assembly).
__global__ void __launch_bounds__(kPathThreads) strat_value_kernel(
    const uint64_t *__restrict__ pair, const int64_t *__restrict__ seg, const uint8_t *__restrict__ rr,
    const uint32_t *__restrict__ cnt, int64_t P, int B, const uint32_t *__restrict__ deg, NetmfConst kc, StratW w,
    uint32_t *__restrict__ val, uint32_t *__restrict__ tile_kept, uint32_t *__restrict__ tile_mir) {
    __shared__ uint32_t s_k, s_m;
    if (threadIdx.x == 0) s_k = s_m = 0;
    __syncthreads();
    uint32_t ck = 0, cm = 0;
    const int64_t t0 = (int64_t)blockIdx.x * kPathTile;
    for (int j = threadIdx.x; j < kPathTile; j += kPathThreads) {
        const int64_t u = t0 + j;
        if (u >= P) break;
        uint64_t K = 0;
        for (int64_t e = seg[u]; e < seg[u + 1]; ++e) K += (uint64_t)w.w[rr[e] - 1] * cnt[e];
        const uint64_t k = pair[u];
        const uint32_t x = (uint32_t)(k >> B), y = (uint32_t)(k & ((1ull << B) - 1ull));
        const float v = netmf_value_fixed(K, 5.9604645e-8f, 5.9604644775390625e-08, __ldg(deg + x), __ldg(deg + y),
                                          x == y, kc);   // 2^-24
        val[u] = __float_as_uint(v);
        if (v > 0.f) {
            ++ck;
            cm += x != y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ck += __shfl_xor_sync(0xffffffffu, ck, o);
        cm += __shfl_xor_sync(0xffffffffu, cm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_k, ck);
        atomicAdd(&s_m, cm);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tile_kept[blockIdx.x] = s_k;
        tile_mir[blockIdx.x] = s_m;
    }
}

// Draws with r ~ U{1..T} as keys (pair << 4 | r - 1), sorted, as unique keys
// ("sort.k0"/"sort.k1", named in *uk_name) with counts ("sort.cnt").
int strat_keys(Workspace &ws, const GraphView &g, const SamplerSpec &sp, int64_t *total_out, uint64_t **ukr,
               uint64_t **spare, uint32_t **cnt, int64_t *U, cudaStream_t st) {
    if (2 * sp.B + 4 > 64) return fail(LNE_ERR_UNSUPPORTED, "stratified keys need 2 ceil(log2 n) + 4 <= 64 bits");
    if (sp.ds_C > 0.0) return fail(LNE_ERR_UNSUPPORTED, "stratified counts do not combine with edge downsampling");
    SamplerSpec su;
    std::vector<double> ones((size_t)sp.T, 1.0);
    LNE_TRY(make_sampler_spec(g, sp.T, ones.data(), sp.S, sp.b, sp.seed, &su));
    su.stratified = 1;
    WalkArgs A = make_walk_args(g, su);
    LNE_TRY(attach_vinfo(ws, g, &A, st));
    const int tile_arcs = choose_tile_arcs(g.nnz, (double)su.base + 0.5);
    int64_t *tile_off = nullptr;
    int64_t total = 0;
    LNE_TRY(tile_offsets(ws, A, 0, g.nnz, tile_arcs, &tile_off, &total, st));
    uint64_t *k0 = nullptr, *k1 = nullptr;
    LNE_TRY(ws.get("sort.k0", (size_t)std::max<int64_t>(total, 1), &k0));
    LNE_TRY(ws.get("sort.k1", (size_t)std::max<int64_t>(total, 1), &k1));
    const int64_t ntiles = ceil_div(g.nnz, tile_arcs);
    {
        LNE_TRACE("walk_keys", st);
        LNE_TRY((launch_walk_emit<uint64_t, 3>(A, (unsigned)ntiles, walk_smem_bytes(tile_arcs, 0), st, 0, g.nnz,
                                              tile_arcs, tile_off, k0, nullptr, nullptr, nullptr, 0)));
    }
    bool in_alt = false;
    LNE_TRY(radix_sort_u64(ws, k0, k1, nullptr, nullptr, total, 2 * su.B + 4, &in_alt, st));
    uint64_t *sorted = in_alt ? k1 : k0, *other = in_alt ? k0 : k1;
    ws.release("sort.offs");
    LNE_TRY(ws.get("sort.cnt", (size_t)std::max<int64_t>(total, 1), cnt));
    LNE_TRY(run_length(ws, sorted, total, other, *cnt, U, st));
    *total_out = total;
    *ukr = other;
    *spare = sorted;
    return 0;
}

uint32_t strat_weight(const SamplerSpec &sp, int r) {
    // w_r = floor(T (s_r / sum(s)) 2^24 + 1/2), the sum left to right
    double tot = 0.0;
    for (int t = 0; t < sp.T; ++t) tot += sp.s_raw[t];
    return (uint32_t)std::floor((double)sp.T * (sp.s_raw[r] / tot) * 16777216.0 + 0.5);
}

}  // namespace

CsrView product_view(const CsrResult &M, int dense_mode, int c) {
    CsrView v;
    v.n = M.n;
    v.nnz = M.nnz;
    v.indptr = M.indptr;
    v.indices = M.indices;
    v.data = M.data;
    // the CSR product gathers c values per nonzero, the tensor-core product
    // streams 8 bytes per table entry (plus its hi / lo split): measured on
    // GB300, the table is the faster once the density reaches ~8 / c (c = 48:
    // CSR faster at 0.11, table at 0.23; c = 144: table at 0.41)
    const double dens = M.n > 0 ? (double)M.nnz / ((double)M.n * (double)M.n) : 0.0;
    if (M.dense && (dense_mode == 2 || (dense_mode == 0 && dens >= 8.0 / std::max(c, 1)))) {
        v.dense = M.dense;
        v.dense_ld = M.dense_ld;
    }
    return v;
}

int prepare_weighted(Workspace &ws, GraphView *g, cudaStream_t st) {
    if (!g->w) return 0;
    uint32_t *wdeg = nullptr;
    float *dinv = nullptr, *wf = nullptr;
    unsigned long long *acc = nullptr;
    LNE_TRY(ws.get("wg.deg", (size_t)std::max<int64_t>(g->n, 1), &wdeg));
    LNE_TRY(ws.get("wg.dinv", (size_t)std::max<int64_t>(g->n, 1), &dinv));
    LNE_TRY(ws.get("wg.wf", (size_t)std::max<int64_t>(g->nnz, 1), &wf));
    LNE_TRY(ws.get("wg.acc", 3, &acc));   // [0] volume, [1] flags, [2] largest weight
    LNE_CUDA_TRY(cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), st));
    if (g->n > 0) {
        LNE_TRACE("build_vinfo", st);
        weighted_prep_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->n, 8), num_sms() * 16)), 256, 0,
                               st>>>(g->indptr, g->w, g->n, wdeg, dinv, wf, acc,
                                     reinterpret_cast<unsigned int *>(acc + 1),
                                     reinterpret_cast<unsigned int *>(acc + 2));
        LNE_LAUNCH_CHECK();
    }
    unsigned long long h[3] = {0, 0, 0};
    LNE_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[1] & 1ull) return fail(LNE_ERR_INVALID, "arc weights must be positive integers");
    if (h[1] & 2ull) return fail(LNE_ERR_UNSUPPORTED, "weighted degrees must stay below 2^31");
    g->wdeg = wdeg;
    g->dinv = dinv;
    g->wf = wf;
    g->vol = (double)h[0];
    g->wmax = (uint32_t)h[2];
    return 0;
}

int stratified_sample(Workspace &ws, const GraphView &g, const SamplerSpec &sp, Strata *out, cudaStream_t st) {
    stratified_release(ws);
    int64_t total = 0, U = 0, P = 0;
    uint64_t *ukr = nullptr, *spare = nullptr;
    uint32_t *cnt = nullptr;
    LNE_TRY(strat_keys(ws, g, sp, &total, &ukr, &spare, &cnt, &U, st));
    uint8_t *r = nullptr;
    uint32_t *scnt = nullptr, *seglen = nullptr;
    uint64_t *pair = nullptr;
    int64_t *seg = nullptr;
    LNE_TRY(ws.get("strat.r", (size_t)std::max<int64_t>(U, 1), &r));
    LNE_TRY(ws.get("strat.cnt", (size_t)std::max<int64_t>(U, 1), &scnt));
    if (U > 0) {
        LNE_TRACE("strat_split", st);
        strat_split_kernel<<<(unsigned)std::min<int64_t>(ceil_div(U, 256), num_sms() * 16), 256, 0, st>>>(ukr, U, spare,
                                                                                                      r);
        LNE_LAUNCH_CHECK();
        LNE_CUDA_TRY(cudaMemcpyAsync(scnt, cnt, sizeof(uint32_t) * U, cudaMemcpyDeviceToDevice, st));
    }
    // the pair keys are sorted with their windows: pairs are runs of them
    LNE_TRY(ws.get("strat.pair", (size_t)std::max<int64_t>(U, 1), &pair));
    LNE_TRY(ws.get("strat.seglen", (size_t)std::max<int64_t>(U, 1), &seglen));
    LNE_TRY(run_length(ws, spare, U, pair, seglen, &P, st));
    LNE_TRY(ws.get("strat.seg", (size_t)P + 1, &seg));
    LNE_TRY(scan_exclusive_u32_to_i64(seglen, seg, P, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    for (const char *nm : {"sort.k0", "sort.k1", "sort.cnt", "strat.seglen", "rle.tile_cnt", "rle.tile_off"})
        ws.release(nm);
    out->total = total;
    out->U = U;
    out->P = P;
    out->pair = pair;
    out->seg = seg;
    out->r = r;
    out->cnt = scnt;
    out->T = sp.T;
    out->B = sp.B;
    out->S = sp.S;
    out->seed = sp.seed;
    out->g_indptr = g.indptr;
    out->g_n = g.n;
    out->g_nnz = g.nnz;
    return 0;
}

int stratified_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, const Strata &S, CsrResult *out,
                   cudaStream_t st) {
    if (S.T != sp.T || S.B != sp.B || S.g_n != g.n || S.g_nnz != g.nnz)
        return fail(LNE_ERR_INVALID, "strata belong to another graph or window size");
    ws.release("csr.indices");
    ws.release("csr.data");
    StratW w = {};
    for (int r = 0; r < sp.T; ++r) w.w[r] = strat_weight(sp, r);
    const int64_t P = S.P, n = g.n;
    const int64_t ntiles = std::max<int64_t>(1, ceil_div(P, (int64_t)kPathTile));
    const unsigned egrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 16));
    uint32_t *tk = nullptr, *tm = nullptr, *deg = nullptr, *val = nullptr;
    uint64_t *uk = nullptr;
    LNE_TRY(ws.get("path.tk", (size_t)ntiles, &tk));
    LNE_TRY(ws.get("path.tm", (size_t)ntiles, &tm));
    LNE_TRY(ws.get("path.deg", (size_t)n, &deg));
    LNE_TRY(ws.get("strat.cuk", (size_t)std::max<int64_t>(P, 1), &uk));
    LNE_TRY(ws.get("strat.cval", (size_t)std::max<int64_t>(P, 1), &val));
    if (P > 0) LNE_CUDA_TRY(cudaMemcpyAsync(uk, S.pair, sizeof(uint64_t) * P, cudaMemcpyDeviceToDevice, st));
    {
        LNE_TRACE("path_value", st);
        if (!g.wdeg) {
            degree_kernel<<<egrid, 256, 0, st>>>(g.indptr, n, deg);
            LNE_LAUNCH_CHECK();
        }
        strat_value_kernel<<<(unsigned)ntiles, kPathThreads, 0, st>>>(S.pair, S.seg, S.r, S.cnt, P, sp.B,
                                                                     g.wdeg ? g.wdeg : deg, netmf_const(sp), w,
                                                                     val, tk, tm);
        LNE_LAUNCH_CHECK();
    }
    return assemble_csr(ws, g, sp, uk, val, P, tk, tm, "strat.cuk", "strat.cval", out, st);
}

void stratified_release(Workspace &ws) {
    for (const char *nm : {"strat.r", "strat.cnt", "strat.pair", "strat.seglen", "strat.seg", "strat.cuk",
                           "strat.cval"})
        ws.release(nm);
}

namespace {

// (x, y, r, count) of every distinct (pair, window) entry, sorted.
int strat_counts(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CountsResult *out, cudaStream_t st) {
    int64_t total = 0, U = 0;
    uint64_t *ukr = nullptr, *spare = nullptr;
    uint32_t *cnt = nullptr;
    LNE_TRY(strat_keys(ws, g, sp, &total, &ukr, &spare, &cnt, &U, st));
    LNE_TRY(ws.get("counts.x", (size_t)std::max<int64_t>(U, 1), &out->x));
    LNE_TRY(ws.get("counts.y", (size_t)std::max<int64_t>(U, 1), &out->y));
    LNE_TRY(ws.get("counts.cnt", (size_t)std::max<int64_t>(U, 1), &out->cnt));
    LNE_TRY(ws.get("counts.r", (size_t)std::max<int64_t>(U, 1), &out->window));
    if (U > 0) {
        LNE_TRACE("decode_keys", st);
        strat_decode_kernel<<<(unsigned)std::min<int64_t>(ceil_div(U, 256), num_sms() * 16), 256, 0, st>>>(
            ukr, U, sp.B, out->x, out->y, out->window);
        LNE_LAUNCH_CHECK();
        LNE_CUDA_TRY(cudaMemcpyAsync(out->cnt, cnt, sizeof(uint32_t) * U, cudaMemcpyDeviceToDevice, st));
    }
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    sort_release(ws);
    out->nnz = U;
    out->total_samples = total;
    return 0;
}

}  // namespace

int sparsifier_counts(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CountsResult *out,
                      cudaStream_t st) {
    if (sp.stratified) return strat_counts(ws, g, sp, out, st);
    if (sp.ds_C > 0.0 && !use_table(g, sp) && sp.aggregation == LNE_AGG_BUCKET)
        return fail(LNE_ERR_UNSUPPORTED, "edge downsampling needs the table or the sort aggregation");
    if (use_table(g, sp)) LNE_TRY(table_counts(ws, g, sp, out, st));
    else if (sp.aggregation == LNE_AGG_BUCKET) LNE_TRY(bucket_counts(ws, g, sp, out, st));
    else LNE_TRY(sort_counts(ws, g, sp, out, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int sparsifier_csr(Workspace &ws, const GraphView &g, const SamplerSpec &sp, CsrResult *out, cudaStream_t st) {
    if (sp.stratified) {
        Strata S;
        LNE_TRY(stratified_sample(ws, g, sp, &S, st));
        const int rc = stratified_csr(ws, g, sp, S, out, st);
        stratified_release(ws);
        return rc;
    }
    if (sp.ds_C > 0.0 && !use_table(g, sp) && sp.aggregation == LNE_AGG_BUCKET)
        return fail(LNE_ERR_UNSUPPORTED, "edge downsampling needs the table or the sort aggregation");
    if (use_table(g, sp)) return table_csr(ws, g, sp, out, st);
    if (sp.aggregation == LNE_AGG_BUCKET) return bucket_csr(ws, g, sp, out, st);
    return sort_csr(ws, g, sp, out, st);
}

}  // namespace lne
