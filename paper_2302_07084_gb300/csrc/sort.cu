// Sorting and run-length counting of 64-bit pair keys, for graphs whose pair
// space does not fit a dense count table (the hash aggregation of Sec. 5.2
// done as sort + run-length instead: exact counts, deterministic order).
//
// radix_sort_u64: stable LSD radix sort, 8 bits per pass over the low `bits`
// bits, optional 32-bit payload. One pass = three launches:
//   hist     per tile of 8192 keys, a 256-bin histogram -> offs[d][t];
//   scan     one CTA per digit turns its row into exclusive offsets (row total
//            last);
//   scatter  each tile ranks its keys stably (rounds of 256 in input order,
//            warp __match_any_sync groups per digit, a per-digit prefix over
//            warps), stages them grouped by digit in shared memory and writes
//            each digit's run contiguously to its global offset.
// run_length: unique keys of a sorted array and their multiplicities (tile
// flag counts, one scan over tiles, block scans inside tiles, each thread
// summing the run segments among its own items); run_length_weighted sums a
// per-arc 64-bit weight over each run instead (edge downsampling).
#include "common.cuh"
#include "runtime.h"

namespace lne {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 32;
constexpr int kSortTile = kSortThreads * kSortItems;   // 8192 keys per tile
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                                                  int shift, int64_t ntiles,
                                                                  int64_t *__restrict__ offs) {
    __shared__ uint32_t h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * kSortTile;
    const int nt = (int)imin64(kSortTile, n - i0);
    for (int i = tid; i < nt; i += kSortThreads) atomicAdd(&h[(uint32_t)(keys[i0 + i] >> shift) & 255u], 1u);
    __syncthreads();
    offs[(int64_t)tid * (ntiles + 1) + blockIdx.x] = h[tid];
}

// Exclusive scan of the 256 values v (one per thread) over the block.
__device__ __forceinline__ int64_t block_scan256(int64_t v, int64_t *s_warp) {
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

template <bool VALS>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, int64_t n, int shift, int64_t ntiles,
    const int64_t *__restrict__ offs, uint64_t *__restrict__ kout, uint32_t *__restrict__ vout) {
    extern __shared__ uint64_t sk[];                                   // kSortTile staged keys
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSortTile);      // kSortTile staged payloads
    __shared__ int64_t s_gbase[256];
    __shared__ uint32_t s_lbase[256], s_run[256];
    __shared__ uint32_t s_wc[kSortWarps][256];
    __shared__ int64_t s_warp[kSortWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t = blockIdx.x, i0 = t * kSortTile;
    const int nt = (int)imin64(kSortTile, n - i0);
    {
        const int64_t *row = offs + (int64_t)tid * (ntiles + 1);
        const int64_t tot = row[ntiles], mine = row[t], cnt = row[t + 1] - row[t];
        const int64_t dbase = block_scan256(tot, s_warp);    // start of digit tid in the output
        const int64_t lbase = block_scan256(cnt, s_warp);    // start of digit tid in this tile
        s_gbase[tid] = dbase + mine;
        s_lbase[tid] = (uint32_t)lbase;
        s_run[tid] = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s_wc[w][tid] = 0;
    }
    // every key (and payload) of the tile is requested up front: 32 independent
    // loads per thread in flight instead of one per round
    uint64_t kr[kSortItems];
    uint32_t vr[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int li = r * kSortThreads + tid;
        kr[r] = li < nt ? kin[i0 + li] : 0ull;
        vr[r] = (VALS && li < nt) ? vin[i0 + li] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int li = r * kSortThreads + tid;   // rounds in input order: stable
        const bool valid = li < nt;
        const uint64_t k = kr[r];
        const uint32_t v = vr[r];
        const uint32_t d = valid ? (uint32_t)(k >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lr = (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (valid && lr == 0) s_wc[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        {   // thread tid owns digit tid: warps' counts -> their starting ranks
            uint32_t p = s_run[tid];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = s_wc[w][tid];
                s_wc[w][tid] = p;
                p += c;
            }
            s_run[tid] = p;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_lbase[d] + s_wc[warp][d] + lr;
            sk[pos] = k;
            if (VALS) sv[pos] = v;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s_wc[w][tid] = 0;
        __syncthreads();
    }
    for (int li = tid; li < nt; li += kSortThreads) {
        const uint64_t k = sk[li];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const int64_t g = s_gbase[d] + (li - (int)s_lbase[d]);
        kout[g] = k;
        if (VALS) vout[g] = sv[li];
    }
}

// Run starts of a sorted array: count per tile.
__global__ void __launch_bounds__(kSortThreads) rle_count_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                                                 uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * kSortTile;
    const int nt = (int)imin64(kSortTile, n - i0);
    uint32_t c = 0;
    for (int i = threadIdx.x; i < nt; i += kSortThreads) {
        const int64_t g = i0 + i;
        c += (g == 0 || keys[g] != keys[g - 1]) ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = s;
}

// Unique keys and their run lengths (thread-blocked items, block scan). Each
// thread adds up the segments of runs among its own items: a run that starts
// and ends among them is stored, a piece of a run that crosses a thread
// boundary is added atomically (integer sums, so the result does not depend
// on the order), which keeps a run of any length parallel. The outputs are
// zeroed beforehand. WEIGHTED: instead of the length, the 64-bit sum of
// w[arc] over the run's payloads.
template <bool WEIGHTED>
__global__ void __launch_bounds__(kSortThreads) rle_write_kernel(const uint64_t *__restrict__ keys, int64_t n,
                                                                 const int64_t *__restrict__ tile_off,
                                                                 uint64_t *__restrict__ ukeys,
                                                                 uint32_t *__restrict__ counts,
                                                                 const uint32_t *__restrict__ arcs,
                                                                 const uint64_t *__restrict__ w,
                                                                 uint64_t *__restrict__ wsum) {
    __shared__ int64_t s_warp[kSortWarps];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * kSortTile + (int64_t)tid * kSortItems;
    uint32_t flags = 0;
    int c = 0;
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t g = i0 + j;
        if (g < n && (g == 0 || keys[g] != keys[g - 1])) {
            flags |= 1u << j;
            ++c;
        }
    }
    // index of the run holding the item before this thread's first one
    int64_t run = tile_off[blockIdx.x] + block_scan256(c, s_warp) - 1;
    if (i0 >= n) return;
    const int64_t iend = i0 + kSortItems < n ? i0 + kSortItems : n;
    auto flush = [&](uint64_t acc, bool complete) {
        if (WEIGHTED) {
            if (complete) wsum[run] = acc;
            else atomicAdd(reinterpret_cast<unsigned long long *>(wsum) + run, (unsigned long long)acc);
        } else {
            if (complete) counts[run] = (uint32_t)acc;
            else atomicAdd(counts + run, (uint32_t)acc);
        }
    };
    uint64_t acc = 0;
    bool started_here = false;
    for (int64_t g = i0; g < iend; ++g) {
        if (flags & (1u << (int)(g - i0))) {
            if (g > i0) flush(acc, started_here);   // the segment ends here
            ++run;
            ukeys[run] = keys[g];
            acc = 0;
            started_here = true;
        }
        acc += WEIGHTED ? __ldg(w + arcs[g]) : 1ull;
    }
    const bool ends = iend >= n || keys[iend] != keys[iend - 1];
    flush(acc, started_here && ends);
}

// Number of keys below `key` in a sorted array (one thread, binary search).
__global__ void lower_bound_kernel(const uint64_t *__restrict__ keys, int64_t n, uint64_t key,
                                   int64_t *__restrict__ out) {
    int64_t lo = 0, hi = n;   // keys[0, lo) < key <= keys[hi, n)
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    *out = lo;
}

}  // namespace

int count_below(Workspace &ws, const uint64_t *keys, int64_t n, uint64_t key, int64_t *count, cudaStream_t st) {
    int64_t *d = nullptr;
    LNE_TRY(ws.get("sort.bound", 1, &d));
    lower_bound_kernel<<<1, 1, 0, st>>>(keys, n, key, d);
    LNE_LAUNCH_CHECK();
    LNE_CUDA_TRY(cudaMemcpyAsync(count, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int radix_sort_u64(Workspace &ws, uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                   int64_t n, int bits, bool *in_alt, cudaStream_t st) {
    *in_alt = false;
    if (n <= 1) return 0;
    const int64_t ntiles = ceil_div(n, (int64_t)kSortTile);
    int64_t *offs = nullptr;
    LNE_TRY(ws.get("sort.offs", (size_t)256 * (ntiles + 1), &offs));
    const int smem = kSortTile * (8 + (vals ? 4 : 0));
    LNE_TRY(allow_dynamic_smem(radix_scatter_kernel<true>));
    LNE_TRY(allow_dynamic_smem(radix_scatter_kernel<false>));
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        LNE_TRACE("radix_pass", st);
        radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, st>>>(ka, n, shift, ntiles, offs);
        LNE_LAUNCH_CHECK();
        LNE_TRY(scan_exclusive_rows_i64(offs, 256, ntiles, st));
        if (vals)
            radix_scatter_kernel<true><<<(unsigned)ntiles, kSortThreads, smem, st>>>(ka, va, n, shift, ntiles, offs,
                                                                                     kb, vb);
        else
            radix_scatter_kernel<false><<<(unsigned)ntiles, kSortThreads, smem, st>>>(ka, nullptr, n, shift, ntiles,
                                                                                      offs, kb, nullptr);
        LNE_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
        *in_alt = !*in_alt;
    }
    return 0;
}

namespace {

int run_length_impl(Workspace &ws, const uint64_t *keys, int64_t n, uint64_t *ukeys, uint32_t *counts,
                    const uint32_t *arcs, const uint64_t *w, uint64_t *wsum, int64_t *nunique, cudaStream_t st) {
    *nunique = 0;
    if (n <= 0) return 0;
    const int64_t ntiles = ceil_div(n, (int64_t)kSortTile);
    uint32_t *tc = nullptr;
    int64_t *toff = nullptr;
    LNE_TRY(ws.get("rle.tile_cnt", (size_t)ntiles, &tc));
    LNE_TRY(ws.get("rle.tile_off", (size_t)ntiles + 1, &toff));
    LNE_TRACE("run_length", st);
    rle_count_kernel<<<(unsigned)ntiles, kSortThreads, 0, st>>>(keys, n, tc);
    LNE_LAUNCH_CHECK();
    LNE_TRY(scan_exclusive_u32_to_i64(tc, toff, ntiles, st));
    int64_t u = 0;
    LNE_CUDA_TRY(cudaMemcpyAsync(&u, toff + ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    if (wsum) LNE_CUDA_TRY(cudaMemsetAsync(wsum, 0, sizeof(uint64_t) * (size_t)u, st));
    else LNE_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)u, st));
    if (wsum)
        rle_write_kernel<true><<<(unsigned)ntiles, kSortThreads, 0, st>>>(keys, n, toff, ukeys, nullptr, arcs, w,
                                                                           wsum);
    else
        rle_write_kernel<false><<<(unsigned)ntiles, kSortThreads, 0, st>>>(keys, n, toff, ukeys, counts, nullptr,
                                                                            nullptr, nullptr);
    LNE_LAUNCH_CHECK();
    LNE_CUDA_TRY(cudaStreamSynchronize(st));
    *nunique = u;
    return 0;
}

}  // namespace

int run_length(Workspace &ws, const uint64_t *keys, int64_t n, uint64_t *ukeys, uint32_t *counts,
               int64_t *nunique, cudaStream_t st) {
    return run_length_impl(ws, keys, n, ukeys, counts, nullptr, nullptr, nullptr, nunique, st);
}

int run_length_weighted(Workspace &ws, const uint64_t *keys, const uint32_t *arcs, const uint64_t *w, int64_t n,
                        uint64_t *ukeys, uint64_t *wsum, int64_t *nunique, cudaStream_t st) {
    return run_length_impl(ws, keys, n, ukeys, nullptr, arcs, w, wsum, nunique, st);
}

}  // namespace lne
