/*
 * CPU oracle for the sampling stage of LightNE 2.0 -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load this library. The product path never calls it.
 *
 * A plain, slow restatement of the paper's sampling steps, written from:
 *   - Algorithm 1 (PathSampling): split s uniform in [0, r-1], walk u for s
 *     steps, walk v for r-1-s steps, return (u', v').
 *   - Algorithm 3 (per-edge PathSampling, Sec. 5.2): map over the edges; edge e
 *     gets n_e = floor(M/m) + Bernoulli({M/m}) samples; each sample draws the
 *     window length r from Multinomial(s_1..s_T).
 *   - Sec. 5.2, fetching a vertex's i-th edge: one walk step takes a uniform 32-bit value
 *     modulo the vertex degree.
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * implemented here from its published definition.
 *
 * Readings taken where the paper is silent:
 *   - the map runs over the 2m CSR arcs, each with S/(2m) expected samples;
 *   - Bernoulli({x}) is  word < floor(frac(x) * 2^32)  with the arc word below;
 *   - r = 1 + #{ i in 1..T-1 : thr_i <= word },
 *       thr_i = min(2^32, floor(2^32 * (s_1+..+s_i) / (s_1+..+s_T)));
 *   - split sigma = word mod r; walk step x <- nbr(x)[word mod deg(x)];
 *   - sample j of arc a uses Philox counter (j, a_lo, a_hi, blk), blk = 0,1,..,
 *     key (seed_lo, seed_hi); its words in order are: r, sigma, the
 *     downsampling coin, then the walk steps, u side first;
 *   - the arc's Bernoulli word is word 0 of counter
 *     (0xFFFFFFFF, a_lo, a_hi, 0xFFFFFFFF).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction:
 * every double operation here is a single IEEE-754 rounding).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* Philox4x32 with 10 rounds: each round multiplies counter words 0 and 2 by
 * the two round constants (full 64-bit products), swaps and xors the halves
 * with the other counter words and the key; the key is advanced by the two
 * Weyl constants before every round but the first. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Window-length thresholds thr[0..T-2] (thr_i for i = 1..T-1). */
void oracle_window_thresholds(int T, const double *s, uint64_t *thr)
{
    double total = 0.0;
    for (int t = 0; t < T; ++t) total += s[t];
    double cum = 0.0;
    for (int i = 0; i + 1 < T; ++i) {
        cum += s[i];
        double p = cum / total;
        double x = floor(p * 4294967296.0);
        if (x >= 4294967296.0) thr[i] = (uint64_t)1 << 32;
        else if (x <= 0.0) thr[i] = 0;
        else thr[i] = (uint64_t)x;
    }
}

/* Per-arc sample rate S/(2m): integer part and Bernoulli threshold of the
 * fractional part. */
void oracle_arc_rate(double S, int64_t n_arcs, uint64_t *base, uint64_t *thr_frac)
{
    double rate = S / (double)n_arcs;
    double b = floor(rate);
    double frac = rate - b;
    *base = (uint64_t)b;
    *thr_frac = (uint64_t)floor(frac * 4294967296.0);
}

static uint32_t seed_lo(uint64_t seed) { return (uint32_t)(seed & 0xFFFFFFFFu); }
static uint32_t seed_hi(uint64_t seed) { return (uint32_t)(seed >> 32); }

/* Number of samples drawn from arc a. */
uint64_t oracle_arc_samples(int64_t a, uint64_t base, uint64_t thr_frac, uint64_t seed)
{
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)((uint64_t)a & 0xFFFFFFFFu),
                       (uint32_t)((uint64_t)a >> 32), 0xFFFFFFFFu};
    uint32_t key[2] = {seed_lo(seed), seed_hi(seed)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    return base + ((uint64_t)w[0] < thr_frac ? 1u : 0u);
}

/* Stream of 32-bit words for sample j of arc a. */
typedef struct {
    uint32_t ctr[4];
    uint32_t key[2];
    uint32_t buf[4];
    int used;   /* words consumed from buf */
} word_stream;

static void ws_init(word_stream *st, uint64_t j, int64_t a, uint64_t seed)
{
    st->ctr[0] = (uint32_t)j;
    st->ctr[1] = (uint32_t)((uint64_t)a & 0xFFFFFFFFu);
    st->ctr[2] = (uint32_t)((uint64_t)a >> 32);
    st->ctr[3] = 0;   /* block index */
    st->key[0] = seed_lo(seed);
    st->key[1] = seed_hi(seed);
    st->used = 4;
}

static uint32_t ws_next(word_stream *st)
{
    if (st->used == 4) {
        oracle_philox4x32_10(st->ctr, st->key, st->buf);
        st->ctr[3] += 1;
        st->used = 0;
    }
    return st->buf[st->used++];
}

/* Source vertex of every arc (CSR row of the arc). */
static int64_t arc_source(int64_t n, const int64_t *indptr, int64_t a)
{
    int64_t lo = 0, hi = n;   /* indptr[lo] <= a < indptr[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (indptr[mid] <= a) lo = mid; else hi = mid;
    }
    return lo;
}

/* Weighted step (weighted graphs): with d = w_0 + .. + w_{deg-1} (< 2^32) and
 * prefixes P_j = w_0 + .. + w_j, the arc taken is the first j < deg - 1 with
 * word < floor(2^32 P_j / d), else the last: arc j with probability
 * w_j / d up to the 2^-32 rounding of the thresholds (inverse CDF). */
int64_t oracle_weighted_choice(const uint32_t *w, int64_t deg, uint32_t word)
{
    uint64_t d = 0;
    for (int64_t j = 0; j < deg; ++j) d += w[j];
    uint64_t prefix = 0;
    for (int64_t j = 0; j + 1 < deg; ++j) {
        prefix += w[j];
        if ((uint64_t)word < (prefix << 32) / d) return j;
    }
    return deg - 1;
}

static int64_t walk(const int64_t *indptr, const int32_t *indices, const uint32_t *weights, int64_t x,
                    int steps, word_stream *st)
{
    for (int t = 0; t < steps; ++t) {
        uint32_t w = ws_next(st);
        int64_t deg = indptr[x + 1] - indptr[x];
        int64_t j = weights ? oracle_weighted_choice(weights + indptr[x], deg, w)
                            : (int64_t)((uint64_t)w % (uint64_t)deg);
        x = indices[indptr[x] + j];
    }
    return x;
}

/* One sample: writes r, sigma and the ordered endpoints (u', v'). */
static void path_sample(const int64_t *indptr, const int32_t *indices, const uint32_t *weights, int T,
                        const uint64_t *thr, int64_t u, int64_t v, int64_t a, uint64_t j,
                        uint64_t seed, int *r_out, int *sigma_out, uint32_t *coin_out,
                        int64_t *u1, int64_t *v1)
{
    word_stream st;
    ws_init(&st, j, a, seed);
    uint32_t wr = ws_next(&st);
    int r = 1;
    for (int i = 0; i + 1 < T; ++i)
        if (thr[i] <= (uint64_t)wr) r += 1;
    uint32_t wsig = ws_next(&st);
    int sigma = (int)(wsig % (uint32_t)r);
    uint32_t coin = ws_next(&st);   /* the downsampling coin (Algorithm 3) */
    int64_t uu = walk(indptr, indices, weights, u, sigma, &st);
    int64_t vv = walk(indptr, indices, weights, v, r - 1 - sigma, &st);
    *r_out = r;
    *sigma_out = sigma;
    *coin_out = coin;
    *u1 = uu;
    *v1 = vv;
}

/* Weighted graphs: arc a of weight A_a draws S A_a / vol samples in
 * expectation (vol = sum of all arc weights), rate = fl(fl(S A_a) / vol). */
void oracle_arc_rate_w(double S, uint32_t weight, double vol, uint64_t *base, uint64_t *thr_frac)
{
    double rate = (S * (double)weight) / vol;
    double b = floor(rate);
    double frac = rate - b;
    *base = (uint64_t)b;
    *thr_frac = (uint64_t)floor(frac * 4294967296.0);
}

static double weight_volume(const uint32_t *weights, int64_t n_arcs)
{
    uint64_t vol = 0;
    for (int64_t a = 0; a < n_arcs; ++a) vol += weights[a];
    return (double)vol;
}

static uint64_t arc_samples_any(const uint32_t *weights, double vol, int64_t a, uint64_t base, uint64_t thr_frac,
                                double S, uint64_t seed)
{
    if (weights) oracle_arc_rate_w(S, weights[a], vol, &base, &thr_frac);
    return oracle_arc_samples(a, base, thr_frac, seed);
}

/* Total samples drawn by arcs [a0, a1) of a weighted graph. */
int64_t oracle_count_samples_w(const uint32_t *weights, int64_t n_arcs, int64_t a0, int64_t a1, double S,
                               uint64_t seed)
{
    double vol = weight_volume(weights, n_arcs);
    int64_t total = 0;
    for (int64_t a = a0; a < a1; ++a) total += (int64_t)arc_samples_any(weights, vol, a, 0, 0, S, seed);
    return total;
}

/* Total samples drawn by arcs [a0, a1). */
int64_t oracle_count_samples(int64_t n_arcs, int64_t a0, int64_t a1, double S, uint64_t seed)
{
    uint64_t base, thr_frac;
    oracle_arc_rate(S, n_arcs, &base, &thr_frac);
    int64_t total = 0;
    for (int64_t a = a0; a < a1; ++a) total += (int64_t)oracle_arc_samples(a, base, thr_frac, seed);
    return total;
}

/*
 * Every sample of arcs [a0, a1), in (arc, sample) order. Any output pointer may
 * be NULL. Returns the number of samples written.
 *   arc[k], r[k], sigma[k], u1[k], v1[k]: the sample's arc, window, split and
 *   ordered endpoints (u' from the arc's source side, v' from its target side);
 *   coin[k]: its downsampling coin word (the walk is drawn whatever the coin).
 */
int64_t oracle_sample_trace(int64_t n, const int64_t *indptr, const int32_t *indices, const uint32_t *weights,
                            int T, const double *s, double S, uint64_t seed,
                            int64_t a0, int64_t a1,
                            int64_t *arc, int32_t *r, int32_t *sigma, int64_t *u1, int64_t *v1,
                            uint32_t *coin)
{
    int64_t n_arcs = indptr[n];
    uint64_t thr[32];
    oracle_window_thresholds(T, s, thr);
    uint64_t base, thr_frac;
    oracle_arc_rate(S, n_arcs, &base, &thr_frac);
    double vol = weights ? weight_volume(weights, n_arcs) : 0.0;

    /* per-arc output offsets */
    int64_t count = a1 - a0;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(count + 1));
    off[0] = 0;
    for (int64_t i = 0; i < count; ++i)
        off[i + 1] = off[i] + (int64_t)arc_samples_any(weights, vol, a0 + i, base, thr_frac, S, seed);

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < count; ++i) {
        int64_t a = a0 + i;
        int64_t u = arc_source(n, indptr, a);
        int64_t v = indices[a];
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            uint64_t j = (uint64_t)(k - off[i]);
            int rr, ss;
            uint32_t cw;
            int64_t x, y;
            path_sample(indptr, indices, weights, T, thr, u, v, a, j, seed, &rr, &ss, &cw, &x, &y);
            if (coin) coin[k] = cw;
            if (arc) arc[k] = a;
            if (r) r[k] = rr;
            if (sigma) sigma[k] = ss;
            if (u1) u1[k] = x;
            if (v1) v1[k] = y;
        }
    }
    int64_t total = off[count];
    free(off);
    return total;
}

/* Raw Philox words of the Gaussian sketch: row i, column block cb uses
 * counter (i, cb, 0, 0) and key (seed_lo ^ 0x4f4d4547, seed_hi). Writes
 * words[(i * nblk + cb) * 4 + t]. */
void oracle_sketch_words(int64_t n, int64_t nblk, uint64_t seed, uint32_t *words)
{
    uint32_t key[2] = {seed_lo(seed) ^ 0x4f4d4547u, seed_hi(seed)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t cb = 0; cb < nblk; ++cb) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)cb, 0u, 0u};
            oracle_philox4x32_10(ctr, key, &words[(i * nblk + cb) * 4]);
        }
    }
}

/* Raw Philox words of the sparse sign sketch: row i, block b uses counter
 * (i, b, 0, 0x53505253) and the Gaussian sketch's key. Writes
 * words[(i * nblk + b) * 4 + t]. */
void oracle_sparse_sign_words(int64_t n, int64_t nblk, uint64_t seed, uint32_t *words)
{
    uint32_t key[2] = {seed_lo(seed) ^ 0x4f4d4547u, seed_hi(seed)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t b = 0; b < nblk; ++b) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)b, 0u, 0x53505253u};
            oracle_philox4x32_10(ctr, key, &words[(i * nblk + b) * 4]);
        }
    }
}

/* Raw Philox words of the very sparse projection: row i, block b uses counter
 * (i, b, 0, 0x56535250) and the Gaussian sketch's key. Writes
 * words[(i * nblk + b) * 4 + t]. */
void oracle_very_sparse_words(int64_t n, int64_t nblk, uint64_t seed, uint32_t *words)
{
    uint32_t key[2] = {seed_lo(seed) ^ 0x4f4d4547u, seed_hi(seed)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t b = 0; b < nblk; ++b) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)b, 0u, 0x56535250u};
            oracle_philox4x32_10(ctr, key, &words[(i * nblk + b) * 4]);
        }
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
