/*
 * Seeded synthetic input generators for the Mersenne-hashing Count Sketch
 * workloads.  This module holds no hashing, reduction or sketch arithmetic:
 * it only produces key, weight and value streams.  Both the CPU oracle and
 * the CUDA path consume its output, so it is kept separate from both.
 *
 * Every generator is counter based: element i of stream s under seed S is a
 * pure function of (S, s, i), so the output does not depend on the number of
 * threads used.  The word source is SplitMix64 (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the j-th
 * output of a generator whose state starts at x is mix(x + (j+1)*GAMMA).
 *
 * Recipes (stated again in the design notes):
 *   stream seed     sseed(S, s) = mix(S + (s+1)*GAMMA)        (output s of SplitMix64(S))
 *   word            w(S, s, i)  = mix(sseed(S, s) + (i+1)*GAMMA)
 *   u64 below B     floor(w * B / 2^64)                        (B = 0 means 2^64)
 *   u32 below B     floor((w >> 32) * B / 2^32)
 *   int32 in [lo,hi] lo + floor((w >> 32) * (hi-lo+1) / 2^32)
 *   bits-wide u128  lo = w(S,s,2i), hi = w(S,s,2i+1), masked to `bits` bits
 *   Zipf(alpha) over ranks [1, N]: rejection-inversion (Hoermann & Derflinger,
 *                   ACM TOMACS 6(3), 1996), attempt j of element i uses the
 *                   uniform double from w(S, s, 64*i + j); rank r is mapped to
 *                   the key (r * 0x9E3779B97F4A7C15) mod 2^61, a bijection on
 *                   [0, 2^61) because the multiplier is odd.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t dg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t dg_sseed(uint64_t seed, uint64_t stream) {
    return dg_mix(seed + (stream + 1) * DG_GAMMA);
}

static inline uint64_t dg_word_at(uint64_t sseed, uint64_t i) {
    return dg_mix(sseed + (i + 1) * DG_GAMMA);
}

/* Public: the i-th word of stream s (exported for tests of the generator). */
uint64_t dg_word(uint64_t seed, uint64_t stream, uint64_t i) {
    return dg_word_at(dg_sseed(seed, stream), i);
}

/* Public: first n outputs of sequential SplitMix64 started at state `seed`. */
void dg_splitmix64_seq(uint64_t seed, uint64_t n, uint64_t* out) {
    for (uint64_t j = 0; j < n; ++j) out[j] = dg_mix(seed + (j + 1) * DG_GAMMA);
}

static inline uint64_t dg_mulhi64(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

/* ---------------- threading helper ---------------- */

typedef void (*dg_range_fn)(void* ctx, uint64_t lo, uint64_t hi);

typedef struct {
    dg_range_fn fn;
    void* ctx;
    uint64_t lo, hi;
} dg_task;

static void* dg_thread_main(void* arg) {
    dg_task* t = (dg_task*)arg;
    t->fn(t->ctx, t->lo, t->hi);
    return NULL;
}

static void dg_parallel(uint64_t n, int nthreads, dg_range_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 65536 || nthreads == 1) {
        fn(ctx, 0, n);
        return;
    }
    pthread_t th[256];
    dg_task tasks[256];
    uint64_t chunk = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t lo = (uint64_t)t * chunk;
        uint64_t hi = lo + chunk < n ? lo + chunk : n;
        if (lo >= hi) break;
        tasks[t].fn = fn;
        tasks[t].ctx = ctx;
        tasks[t].lo = lo;
        tasks[t].hi = hi;
        if (pthread_create(&th[t], NULL, dg_thread_main, &tasks[t]) != 0) {
            fn(ctx, lo, hi); /* run inline if a thread cannot be created */
            tasks[t].fn = NULL;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (tasks[t].fn) pthread_join(th[t], NULL);
}

/* ---------------- uniform integers ---------------- */

typedef struct {
    uint64_t sseed, bound;
    void* out;
} dg_uni_ctx;

static void dg_u64_below_range(void* vctx, uint64_t lo, uint64_t hi) {
    dg_uni_ctx* c = (dg_uni_ctx*)vctx;
    uint64_t* out = (uint64_t*)c->out;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t w = dg_word_at(c->sseed, i);
        out[i] = c->bound ? dg_mulhi64(w, c->bound) : w;
    }
}

/* Keys uniform in [0, bound) (bound == 0: all of [0, 2^64)). */
void dg_u64_below(uint64_t seed, uint64_t stream, uint64_t bound, uint64_t n,
                  uint64_t* out, int nthreads) {
    dg_uni_ctx c = {dg_sseed(seed, stream), bound, out};
    dg_parallel(n, nthreads, dg_u64_below_range, &c);
}

static void dg_u32_below_range(void* vctx, uint64_t lo, uint64_t hi) {
    dg_uni_ctx* c = (dg_uni_ctx*)vctx;
    uint32_t* out = (uint32_t*)c->out;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t w = dg_word_at(c->sseed, i) >> 32;
        out[i] = c->bound ? (uint32_t)((w * c->bound) >> 32) : (uint32_t)w;
    }
}

/* Keys uniform in [0, bound) for bound <= 2^32 (bound == 0: [0, 2^32)). */
void dg_u32_below(uint64_t seed, uint64_t stream, uint64_t bound, uint64_t n,
                  uint32_t* out, int nthreads) {
    dg_uni_ctx c = {dg_sseed(seed, stream), bound, out};
    dg_parallel(n, nthreads, dg_u32_below_range, &c);
}

typedef struct {
    uint64_t sseed;
    int bits;
    uint64_t* out;
} dg_u128_ctx;

static void dg_u128_bits_range(void* vctx, uint64_t lo, uint64_t hi) {
    dg_u128_ctx* c = (dg_u128_ctx*)vctx;
    int bits = c->bits;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t l = dg_word_at(c->sseed, 2 * i);
        uint64_t h = dg_word_at(c->sseed, 2 * i + 1);
        if (bits <= 64) {
            h = 0;
            if (bits < 64) l &= (bits == 0) ? 0 : ((~0ULL) >> (64 - bits));
        } else if (bits < 128) {
            h &= (~0ULL) >> (128 - bits);
        }
        c->out[2 * i] = l;
        c->out[2 * i + 1] = h;
    }
}

/* Values uniform in [0, 2^bits), bits in [0, 128], as (lo, hi) u64 pairs. */
void dg_u128_bits(uint64_t seed, uint64_t stream, int bits, uint64_t n,
                  uint64_t* out_pairs, int nthreads) {
    dg_u128_ctx c = {dg_sseed(seed, stream), bits, out_pairs};
    dg_parallel(n, nthreads, dg_u128_bits_range, &c);
}

typedef struct {
    uint64_t sseed;
    int32_t lo;
    uint64_t span;
    int32_t* out;
} dg_w_ctx;

static void dg_i32_range_range(void* vctx, uint64_t lo, uint64_t hi) {
    dg_w_ctx* c = (dg_w_ctx*)vctx;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t w = dg_word_at(c->sseed, i) >> 32;
        c->out[i] = (int32_t)((int64_t)c->lo + (int64_t)((w * c->span) >> 32));
    }
}

/* Weights uniform in [lo, hi] (inclusive), hi - lo < 2^32. */
void dg_i32_range(uint64_t seed, uint64_t stream, int32_t lo, int32_t hi,
                  uint64_t n, int32_t* out, int nthreads) {
    dg_w_ctx c = {dg_sseed(seed, stream), lo,
                  (uint64_t)((int64_t)hi - (int64_t)lo + 1), out};
    dg_parallel(n, nthreads, dg_i32_range_range, &c);
}

/* ---------------- Zipf by rejection-inversion ---------------- */

/* log1p(x)/x and expm1(x)/x, continuous at 0 */
static double dg_log1p_over(double x) {
    return fabs(x) > 1e-8 ? log1p(x) / x : 1.0 - x * (0.5 - x / 3.0);
}
static double dg_expm1_over(double x) {
    return fabs(x) > 1e-8 ? expm1(x) / x : 1.0 + x * (0.5 + x / 6.0);
}

typedef struct {
    double alpha;       /* exponent */
    double n_ranks;     /* N */
    double area_lo;     /* H(1.5) - 1 */
    double area_hi;     /* H(N + 0.5) */
    double squeeze;     /* 2 - Hinv(H(2.5) - 2^-alpha) */
} dg_zipf_params;

/* H(x) = integral of t^-alpha from 1 to x, written stably. */
static double dg_zipf_H(const dg_zipf_params* z, double x) {
    double lx = log(x);
    return dg_expm1_over((1.0 - z->alpha) * lx) * lx;
}
static double dg_zipf_Hinv(const dg_zipf_params* z, double y) {
    double t = y * (1.0 - z->alpha);
    if (t < -1.0) t = -1.0; /* guard rounding at the boundary */
    return exp(dg_log1p_over(t) * y);
}
static double dg_zipf_h(const dg_zipf_params* z, double x) {
    return exp(-z->alpha * log(x));
}

static void dg_zipf_setup(dg_zipf_params* z, double alpha, double n_ranks) {
    z->alpha = alpha;
    z->n_ranks = n_ranks;
    z->area_lo = dg_zipf_H(z, 1.5) - 1.0;
    z->area_hi = dg_zipf_H(z, n_ranks + 0.5);
    z->squeeze = 2.0 - dg_zipf_Hinv(z, dg_zipf_H(z, 2.5) - dg_zipf_h(z, 2.0));
}

static uint64_t dg_zipf_rank(const dg_zipf_params* z, uint64_t sseed, uint64_t i) {
    for (uint64_t j = 0; j < 64; ++j) {
        uint64_t w = dg_word_at(sseed, 64 * i + j);
        double u01 = (double)(w >> 11) * (1.0 / 9007199254740992.0); /* [0,1) */
        double u = z->area_hi + u01 * (z->area_lo - z->area_hi);
        double x = dg_zipf_Hinv(z, u);
        double kf = floor(x + 0.5);
        if (kf < 1.0) kf = 1.0;
        if (kf > z->n_ranks) kf = z->n_ranks;
        if (kf - x <= z->squeeze || u >= dg_zipf_H(z, kf + 0.5) - dg_zipf_h(z, kf))
            return (uint64_t)kf;
    }
    return 1; /* 64 rejections in a row: probability far below 2^-100 */
}

typedef struct {
    dg_zipf_params z;
    uint64_t sseed;
    int map_to_keys;
    uint64_t* out;
} dg_zipf_ctx;

static void dg_zipf_range(void* vctx, uint64_t lo, uint64_t hi) {
    dg_zipf_ctx* c = (dg_zipf_ctx*)vctx;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t r = dg_zipf_rank(&c->z, c->sseed, i);
        c->out[i] = c->map_to_keys ? (r * DG_GAMMA) & ((1ULL << 61) - 1) : r;
    }
}

/* Zipf(alpha) ranks over [1, n_ranks]; map_to_keys != 0 maps each rank r to
 * the key (r * 0x9E3779B97F4A7C15) mod 2^61. */
void dg_zipf(uint64_t seed, uint64_t stream, double alpha, double n_ranks,
             int map_to_keys, uint64_t n, uint64_t* out, int nthreads) {
    dg_zipf_ctx c;
    dg_zipf_setup(&c.z, alpha, n_ranks);
    c.sseed = dg_sseed(seed, stream);
    c.map_to_keys = map_to_keys;
    c.out = out;
    dg_parallel(n, nthreads, dg_zipf_range, &c);
}

/* Uniform double in [0,1) from word i of stream s (53-bit mantissa). */
void dg_unit_doubles(uint64_t seed, uint64_t stream, uint64_t n, double* out) {
    uint64_t ss = dg_sseed(seed, stream);
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (double)(dg_word_at(ss, i) >> 11) * (1.0 / 9007199254740992.0);
}
