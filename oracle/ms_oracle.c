/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, definition-based CPU implementation of what the GPU library
 * computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never does.  It shares no code with the
 * CUDA library: no Mersenne folds, no branch-free division, no limb tricks.
 * Every reduction is the C `%` or `/` operator on unsigned __int128.
 *
 * Paper: Ahle, Knudsen, Thorup, "The Power of Hashing with Mersenne Primes".
 *
 *  - or_hash:      h_a(x) = sum_{i<k} a_i x^i mod p, the polynomial hash of
 *                  Sec. 1.2 (the k-universal family of the Definition there),
 *                  evaluated as that sum of powers.  Keys enter as x mod p.
 *  - or_draw_coeffs: coefficients a_i uniform in [0, p), drawn by rejection
 *                  from SplitMix64 (Steele, Lea & Flood 2014).  The paper only
 *                  requires them uniform (Sec. 1.2); the draw order is this
 *                  project's convention.
 *  - or_cs_update: Count Sketch "Process" (Algorithm count-sketch, Sec. 1.3):
 *                  C[i(x)] += s(x) * Delta, one row of m counters per hash
 *                  function, t rows.  The bucket i(x) = h(x) mod m and the
 *                  sign bit a(x) = floor(h(x) / 2^(b-1)), s = 1 - 2a, are the
 *                  two-for-one split of Algorithm h-and-s (Sec. 1.3, "Two-for-
 *                  one hash functions"), written with % and / rather than bit
 *                  masks.  In two-polynomial mode the sign bit comes from a
 *                  second, independent polynomial per row (Algorithm
 *                  count-sketch's two independent functions).
 *  - or_cs_row_sumsq / or_cs_f2: "Output" of Algorithm count-sketch,
 *                  X = sum_i C[i]^2 per row (mod 2^128), and the median over
 *                  the t rows (t odd) as the F2 estimate.
 *  - or_divmod:    floor(v / p) and v mod p for 128-bit v (what Algorithms
 *                  div-simple, division-generalized and mod-generalized of
 *                  Sec. 1.5 compute), by the C operators.
 *  - or_cs_point_query: the point-query estimate of f_x, median over rows of
 *                  s_r(x) C[r][i_r(x)] (Sec. 1.3, estimating a single value).
 *  - or_exact_f2:  F2 = sum_x f_x^2 of a weighted stream (Sec. 1.3 setup).
 *
 * Conventions shared with the library's contract (not its code): counters are
 * int64 and wrap modulo 2^64; row sums of squares wrap modulo 2^128.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

static inline u128 pack(const u64* pair) { return ((u128)pair[1] << 64) | pair[0]; }
static inline void unpack(u128 v, u64* pair) {
    pair[0] = (u64)v;
    pair[1] = (u64)(v >> 64);
}

/* p = 2^b - c.  The oracle accepts any 2 <= b <= 89 and 1 <= c < 2^b. */
static u128 or_prime(int b, u64 c) { return ((u128)1 << b) - c; }

int or_valid_prime_params(int b, u64 c) {
    if (b < 2 || b > 89) return 0;
    if (c < 1) return 0;
    if (b < 64 && c >= ((u64)1 << b) - 1) return 0;
    return 1;
}

/* (a * x) mod p for a, x < p.  For p <= 2^64 the product fits in 128 bits.
 * For larger p (up to 2^90) the multiplier x is taken 30 bits at a time, most
 * significant piece first: acc = (acc * 2^30 + a * piece) mod p, where every
 * intermediate stays below 2^121. */
static u128 or_mulmod(u128 a, u128 x, u128 p) {
    if (p <= ((u128)1 << 64)) return (a * x) % p;
    u128 acc = 0;
    for (int shift = 60; shift >= 0; shift -= 30) {
        u128 piece = (x >> shift) & (((u128)1 << 30) - 1);
        acc = ((acc << 30) % p + (a * piece) % p) % p;
    }
    return acc;
}

/* h_a(x) = sum_{i<k} a_i x^i mod p, by the sum of powers. */
static u128 or_hash_p(u128 p, int k, const u128* a, u128 x) {
    x %= p;
    u128 acc = 0;
    u128 xpow = 1 % p;
    for (int i = 0; i < k; ++i) {
        acc = (acc + or_mulmod(a[i] % p, xpow, p)) % p;
        xpow = or_mulmod(xpow, x, p);
    }
    return acc;
}

/* ---------------- SplitMix64 and the coefficient draw ---------------- */

typedef struct { u64 state; } or_sm64;

static u64 or_sm64_next(or_sm64* g) {
    g->state += 0x9E3779B97F4A7C15ULL;
    u64 z = g->state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void or_splitmix64(u64 seed, u64 n, u64* out) {
    or_sm64 g = {seed};
    for (u64 i = 0; i < n; ++i) out[i] = or_sm64_next(&g);
}

/* nfun * k coefficients, function-major, a_0 first; each one takes
 * ceil(b/64) words (low word first), keeps the low b bits, and is redrawn
 * while >= p. */
void or_draw_coeffs(int b, u64 c, int k, u64 nfun, u64 seed, u64* out_pairs) {
    u128 p = or_prime(b, c);
    u128 mask = (b >= 128) ? ~(u128)0 : (((u128)1 << b) - 1);
    or_sm64 g = {seed};
    for (u64 f = 0; f < nfun; ++f) {
        for (int i = 0; i < k; ++i) {
            u128 v;
            do {
                u128 lo = or_sm64_next(&g);
                u128 hi = (b > 64) ? (u128)or_sm64_next(&g) : 0;
                v = ((hi << 64) | lo) & mask;
            } while (v >= p);
            unpack(v, out_pairs + 2 * (f * (u64)k + (u64)i));
        }
    }
}

/* ---------------- hashing ---------------- */

/* key_kind: 32 -> uint32 keys, 64 -> uint64 keys, 128 -> (lo, hi) pairs */
static u128 or_key(const void* keys, int key_kind, u64 j) {
    if (key_kind == 32) return ((const uint32_t*)keys)[j];
    if (key_kind == 64) return ((const u64*)keys)[j];
    return pack((const u64*)keys + 2 * j);
}

static void or_load_coeffs(const u64* pairs, int k, u128* a) {
    for (int i = 0; i < k; ++i) a[i] = pack(pairs + 2 * i);
}

/* out[j] = h_a(keys[j]) for one function. */
void or_hash_eval(int b, u64 c, int k, const u64* coeff_pairs, const void* keys, int key_kind,
                  u64 n, u64* out_pairs) {
    u128 p = or_prime(b, c);
    u128 a[64];
    or_load_coeffs(coeff_pairs, k, a);
    for (u64 j = 0; j < n; ++j) unpack(or_hash_p(p, k, a, or_key(keys, key_kind, j)), out_pairs + 2 * j);
}

/* out[f * nkeys + j] = h_{a_f}(keys[j]) for nfun functions (enumeration pins). */
void or_hash_many(int b, u64 c, int k, const u64* coeff_pairs, u64 nfun, const u64* key_pairs,
                  u64 nkeys, u64* out_pairs) {
    u128 p = or_prime(b, c);
    u128 a[64];
    for (u64 f = 0; f < nfun; ++f) {
        or_load_coeffs(coeff_pairs + 2 * f * (u64)k, k, a);
        for (u64 j = 0; j < nkeys; ++j)
            unpack(or_hash_p(p, k, a, pack(key_pairs + 2 * j)), out_pairs + 2 * (f * nkeys + j));
    }
}

/* ---------------- Count Sketch ---------------- */

/* Bucket and sign of one key in one row.  mode bit 0 (two polynomials): the
 * sign comes from the row's second polynomial.  mode bit 1 (any m): the
 * bucket map for a number of buckets that need not be a power of two --
 *   c = 1 (Mersenne, Algorithm Mersenne-arb-r of Sec. 3.3): h' = h + 1 is
 *          nonzero in [2^b]; its low b-1 bits j give the bucket floor(j m /
 *          2^(b-1)) and, in two-for-one mode, its top bit a the sign s = 2a - 1
 *          (the sign convention of that section's text and proofs);
 *   c > 1 (pseudo-Mersenne, Sec. 1.5 "arbitrary number of buckets"): the most
 *          uniform map floor(h m / p); the sign then needs the second
 *          polynomial (the library accepts this case only in that mode).
 * Otherwise bucket = h mod m and the sign bit is floor(g / 2^(b-1)), s = 1 - 2a
 * (Algorithm h-and-s).  Plain % and / throughout. */
static void or_split(u128 p, int b, u64 c, int k, u64 m, int mode, const u128* a_bucket,
                     const u128* a_sign, u128 x, u64* bucket, int* sign) {
    u128 h = or_hash_p(p, k, a_bucket, x);
    u128 half = (u128)1 << (b - 1);
    if (mode & 2) {
        if (c == 1) {
            u128 hx = h + 1;
            u128 j = hx % half;
            *bucket = (u64)((j * (u128)m) / half);
            if (!(mode & 1)) {
                *sign = 2 * (int)(hx / half) - 1;
                return;
            }
        } else {
            *bucket = (u64)((h * (u128)m) / p);
        }
    } else {
        *bucket = (u64)(h % m);
    }
    u128 g = (mode & 1) ? or_hash_p(p, k, a_sign, x) : h;
    u128 bit = g / half;
    *sign = 1 - 2 * (int)bit;
}

/* C (t x m, row-major int64) += sketch of the stream (keys, w); w == NULL means
 * unit weights.  coeffs: t*k pairs (two-for-one) or 2*t*k pairs ordered row 0
 * bucket function, row 0 sign function, row 1 bucket function, ... */
void or_cs_update(int b, u64 c, int k, int t, u64 m, int mode, const u64* coeff_pairs,
                  const void* keys, int key_kind, const int32_t* w, u64 n, int64_t* C) {
    u128 p = or_prime(b, c);
    int nf = (mode & 1) ? 2 : 1;
    u128* a = (u128*)malloc(sizeof(u128) * (size_t)t * (size_t)nf * (size_t)k);
    for (int f = 0; f < t * nf; ++f) or_load_coeffs(coeff_pairs + 2 * (u64)f * (u64)k, k, a + f * k);
    for (u64 j = 0; j < n; ++j) {
        u128 x = or_key(keys, key_kind, j);
        int64_t wj = w ? (int64_t)w[j] : 1;
        for (int r = 0; r < t; ++r) {
            const u128* ab = a + (size_t)(r * nf) * k;
            const u128* as = (mode & 1) ? ab + k : ab;
            u64 bucket;
            int sign;
            or_split(p, b, c, k, m, mode, ab, as, x, &bucket, &sign);
            u64* cell = (u64*)&C[(u64)r * m + bucket];
            *cell += (u64)(sign * wj); /* two's-complement add, wraps mod 2^64 */
        }
    }
    free(a);
}

typedef struct {
    int b, k, t, mode, key_kind;
    u64 c, m, lo, hi;
    const u64* coeffs;
    const void* keys;
    const int32_t* w;
    int64_t* C;
} or_chunk;

static void* or_chunk_main(void* arg) {
    or_chunk* ch = (or_chunk*)arg;
    const char* kbase = (const char*)ch->keys;
    size_t kb = ch->key_kind == 32 ? 4 : ch->key_kind == 64 ? 8 : 16;
    or_cs_update(ch->b, ch->c, ch->k, ch->t, ch->m, ch->mode, ch->coeffs,
                 kbase + kb * ch->lo, ch->key_kind, ch->w ? ch->w + ch->lo : NULL,
                 ch->hi - ch->lo, ch->C);
    return NULL;
}

/* Same result as or_cs_update: the stream is cut into nthreads contiguous
 * pieces, each sketched into its own zeroed counters, and the counters are
 * summed (a Count Sketch is linear in the stream, Sec. 1.3). */
void or_cs_update_mt(int b, u64 c, int k, int t, u64 m, int mode, const u64* coeff_pairs,
                     const void* keys, int key_kind, const int32_t* w, u64 n, int64_t* C,
                     int nthreads) {
    if (nthreads < 2 || n < 1024) {
        or_cs_update(b, c, k, t, m, mode, coeff_pairs, keys, key_kind, w, n, C);
        return;
    }
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    or_chunk ch[256];
    int ran[256];
    u64 cells = (u64)t * m;
    u64 per = (n + (u64)nthreads - 1) / (u64)nthreads;
    for (int i = 0; i < nthreads; ++i) {
        ch[i] = (or_chunk){b, k, t, mode, key_kind, c, m, 0, 0, coeff_pairs, keys, w, NULL};
        ch[i].lo = (u64)i * per < n ? (u64)i * per : n;
        ch[i].hi = ch[i].lo + per < n ? ch[i].lo + per : n;
        ch[i].C = (int64_t*)calloc(cells, sizeof(int64_t));
        ran[i] = pthread_create(&th[i], NULL, or_chunk_main, &ch[i]) == 0;
        if (!ran[i]) or_chunk_main(&ch[i]);
    }
    for (int i = 0; i < nthreads; ++i) {
        if (ran[i]) pthread_join(th[i], NULL);
        for (u64 q = 0; q < cells; ++q) ((u64*)C)[q] += (u64)ch[i].C[q];
        free(ch[i].C);
    }
}

/* X_r = sum_i C[r][i]^2 modulo 2^128, for every row r. */
void or_cs_row_sumsq(int t, u64 m, const int64_t* C, u64* rows_pairs) {
    for (int r = 0; r < t; ++r) {
        u128 s = 0;
        for (u64 i = 0; i < m; ++i) {
            int64_t v = C[(u64)r * m + i];
            u64 mag = v < 0 ? (u64)0 - (u64)v : (u64)v;
            s += (u128)mag * mag;
        }
        unpack(s, rows_pairs + 2 * r);
    }
}

/* Median of the t row estimates (t odd: the middle one after sorting). */
void or_cs_f2(int t, u64 m, const int64_t* C, u64* out_pair) {
    u64* rows = (u64*)malloc(sizeof(u64) * 2 * (size_t)t);
    or_cs_row_sumsq(t, m, C, rows);
    u128* v = (u128*)malloc(sizeof(u128) * (size_t)t);
    for (int r = 0; r < t; ++r) v[r] = pack(rows + 2 * r);
    for (int i = 1; i < t; ++i) { /* insertion sort */
        u128 x = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
        v[j + 1] = x;
    }
    unpack(v[t / 2], out_pair);
    free(v);
    free(rows);
}

/* For each of nsets hash-function sets (1 function, or 2 in two-polynomial
 * mode), sketch the stream into ONE row of m counters and return that row's
 * X = sum C^2.  Used by the enumeration pins over all coefficient tuples. */
void or_cs_x_many(int b, u64 c, int k, u64 m, int mode, const u64* coeff_pairs, u64 nsets,
                  const void* keys, int key_kind, const int32_t* w, u64 n, u64* x_pairs) {
    int nf = (mode & 1) ? 2 : 1;
    int64_t* C = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    for (u64 s = 0; s < nsets; ++s) {
        memset(C, 0, sizeof(int64_t) * (size_t)m);
        or_cs_update(b, c, k, 1, m, mode, coeff_pairs + 2 * s * (u64)(nf * k), keys, key_kind,
                     w, n, C);
        or_cs_row_sumsq(1, m, C, x_pairs + 2 * s);
    }
    free(C);
}

/* Point query (Sec. 1.3): the estimate of f_x is the median over the t rows of
 * s_r(x) * C[r][i_r(x)] (t odd: the middle value after sorting). */
void or_cs_point_query(int b, u64 c, int k, int t, u64 m, int mode, const u64* coeff_pairs,
                       const int64_t* C, const void* keys, int key_kind, u64 n, int64_t* out) {
    u128 p = or_prime(b, c);
    int nf = (mode & 1) ? 2 : 1;
    u128* a = (u128*)malloc(sizeof(u128) * (size_t)t * (size_t)nf * (size_t)k);
    int64_t* est = (int64_t*)malloc(sizeof(int64_t) * (size_t)t);
    for (int f = 0; f < t * nf; ++f) or_load_coeffs(coeff_pairs + 2 * (u64)f * (u64)k, k, a + f * k);
    for (u64 j = 0; j < n; ++j) {
        u128 x = or_key(keys, key_kind, j);
        for (int r = 0; r < t; ++r) {
            const u128* ab = a + (size_t)(r * nf) * k;
            const u128* as = (mode & 1) ? ab + k : ab;
            u64 bucket;
            int sign;
            or_split(p, b, c, k, m, mode, ab, as, x, &bucket, &sign);
            u64 cv = (u64)C[(u64)r * m + bucket];
            est[r] = (int64_t)(sign > 0 ? cv : (u64)0 - cv);
        }
        for (int i = 1; i < t; ++i) {
            int64_t v = est[i];
            int q = i - 1;
            while (q >= 0 && est[q] > v) { est[q + 1] = est[q]; --q; }
            est[q + 1] = v;
        }
        out[j] = est[t / 2];
    }
    free(est);
    free(a);
}

/* ---------------- division and modulus ---------------- */

void or_divmod(int b, u64 c, const u64* v_pairs, u64 n, u64* q_pairs, u64* r_pairs) {
    u128 p = or_prime(b, c);
    for (u64 j = 0; j < n; ++j) {
        u128 v = pack(v_pairs + 2 * j);
        if (q_pairs) unpack(v / p, q_pairs + 2 * j);
        if (r_pairs) unpack(v % p, r_pairs + 2 * j);
    }
}

/* ---------------- exact F2 of a stream ---------------- */

typedef struct { u64 key; int64_t w; } or_kw;

static int or_kw_cmp(const void* x, const void* y) {
    u64 a = ((const or_kw*)x)->key, b = ((const or_kw*)y)->key;
    return a < b ? -1 : a > b ? 1 : 0;
}

/* F2 = sum over distinct keys of (sum of that key's weights)^2, mod 2^128. */
void or_exact_f2(const u64* keys, const int32_t* w, u64 n, u64* out_pair) {
    or_kw* v = (or_kw*)malloc(sizeof(or_kw) * (size_t)(n ? n : 1));
    for (u64 j = 0; j < n; ++j) {
        v[j].key = keys[j];
        v[j].w = w ? w[j] : 1;
    }
    qsort(v, (size_t)n, sizeof(or_kw), or_kw_cmp);
    u128 s = 0;
    u64 j = 0;
    while (j < n) {
        u64 key = v[j].key;
        int64_t f = 0;
        while (j < n && v[j].key == key) f += v[j++].w;
        u64 mag = f < 0 ? (u64)0 - (u64)f : (u64)f;
        s += (u128)mag * mag;
    }
    free(v);
    unpack(s, out_pair);
}
