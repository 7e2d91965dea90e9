// Device arithmetic modulo p = 2^b - c for the four supported primes.
//
// Each policy struct gives, for its prime:
//   key_t / val_t     key and hash-value types,
//   reduce_key(x)     x mod p, canonical,
//   Horner / power-sum building blocks with LAZY reduction: intermediate
//                     values stay below 2^b + 2^4 (not necessarily < p), and
//                     only the final value is made canonical,
//   bucket(h, mask)   the low bits of h (Algorithm h-and-s, Sec. 1.3),
//   sign_bit(h)       bit b-1 of h (the same algorithm).
//
// Mersenne reduction uses the fold y = (y mod 2^b) + floor(y / 2^b), which
// preserves y mod p because 2^b = 1 (mod p) (eq. Mersenne, Sec. 1.2).  The
// pseudo-Mersenne prime 2^64 - 59 uses Algorithm division-generalized and
// Algorithm mod-generalized (Sec. 1.5) with 3 steps.
//
// Every bound below is for the stated input ranges; the comments give the
// arithmetic so that each can be checked by hand.
#pragma once

#include <stdint.h>

namespace msf {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned __int128 u128;

struct u128x {  // a two-limb key/value as it sits in memory
    u64 lo, hi;
};

// 32x32 -> 64-bit multiply-add, a * b + c (one wide integer multiply-add).
__device__ __forceinline__ u64 madw(u32 a, u32 b, u64 c) {
    u64 d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// The signed form: a * b + c modulo 2^64, a and b signed 32-bit.
__device__ __forceinline__ u64 madws(int a, int b, u64 c) {
    u64 d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// ---------------------------------------------------------------- p = 2^61-1
//
// Elements are split into a 31-bit low part and a high part,
//     z = zh * 2^31 + zl,  zl < 2^31,
// so that every partial product fits 62 bits and sums of a few of them never
// carry out of 64 bits.  For z < 2^61 + 2^4 we have zh <= 2^30.
struct P61 {
    static constexpr int B = 61;
    static constexpr u64 P = (1ull << 61) - 1;
    typedef u64 key_t;
    typedef u64 val_t;

    struct Split {  // of a value < 2^61 + 2^4
        u32 lo;     // < 2^31
        u32 hi;     // <= 2^30
        u32 hi2;    // 2 * hi <= 2^31
    };

    __device__ static __forceinline__ Split split(u64 z) {
        Split s;
        s.lo = (u32)z & 0x7FFFFFFFu;
        s.hi = (u32)(z >> 31);
        s.hi2 = s.hi << 1;
        return s;
    }

    // x mod p for any 64-bit x: (x & p) + (x >> 61) < 2^61 + 8 < 2p.
    __device__ static __forceinline__ u64 reduce_key(u64 x) {
        return canon((x & P) + (x >> 61));
    }

    // y < 2p  ->  y mod p
    __device__ static __forceinline__ u64 canon(u64 y) { return y >= P ? y - P : y; }

    // Fold of a 64-bit value: (S & p) + (S >> 61) = S (mod p), result < 2^61 + 8.
    __device__ static __forceinline__ u64 fold(u64 S) { return (S & P) + (S >> 61); }

    // One Horner step (Algorithm Mersenne): returns y = z*x + a (mod p), lazily
    // reduced (< 2^61 + 8), for z, x < 2^61 + 8 (xs = split(x); lazy values
    // keep zh, xh <= 2^30 and zl, xl < 2^31, which is all the bounds use),
    // a < 2^61.
    //   z*x = zh*xh*2^62 + (zh*xl + zl*xh)*2^31 + zl*xl,   2^62 = 2 (mod p)
    //   A = zl*xl + a + zh*(2xh)   <= (2^31-1)^2 + 2^61 + 2^30*(2^31-2) < 2^63
    //   M = zh*xl + zl*xh          <  2^30*2^31 + 2^31*2^30 = 2^62
    //   M*2^31 = (M >> 30)*2^61 + (M mod 2^30)*2^31 = (M >> 30) + (M mod 2^30)*2^31
    //   S = A + (M >> 30) + (M mod 2^30)*2^31  < 2^63 + 2^32 + 2^61 < 2^64
    __device__ static __forceinline__ u64 mul_add(u64 z, const Split& xs, u64 a) {
        const u32 zl = (u32)z & 0x7FFFFFFFu;
        const u32 zh = (u32)(z >> 31);
        u64 A = (u64)zl * xs.lo + a;
        A += (u64)zh * xs.hi2;
        u64 M = (u64)zh * xs.lo;
        M += (u64)zl * xs.hi;
        const u64 S = A + (M >> 30) + ((M & 0x3FFFFFFFull) << 31);
        return fold(S);
    }

    __device__ static __forceinline__ u32 bucket(u64 h, u32 mask) { return (u32)h & mask; }
    __device__ static __forceinline__ u32 sign_bit(u64 h) { return (u32)(h >> 60) & 1u; }

    // Algorithm Mersenne-arb-r (Sec. 3.3) for a canonical h < p and r buckets:
    // h' = h + 1 is nonzero in [2^61]; the bucket is floor(r j / 2^60) for its
    // low 60 bits j (a most uniform map, Lemma most-uniform), a its top bit.
    __device__ static __forceinline__ void arb_split(u64 h, u32 r, u32& bucket, u32& a) {
        const u64 hx = h + 1;
        const u64 j = hx & ((1ull << 60) - 1);
        bucket = (u32)((__umul64hi(j, (u64)r) << 4) | ((j * (u64)r) >> 60));
        a = (u32)(hx >> 60);
    }

    // ---- power sum with signed digits (the update kernels' row hash) ----
    //
    // A row is y = a0 + a1 x + a2 x^2 + a3 x^3 (mod p) with the powers X_i of x
    // computed once per key, lazily reduced (X_i < 2^61 + 8).  Every operand
    // of the row's products is split into two SIGNED 31-bit digits:
    //   key side:  X - D = h 2^31 + l,  D = 2^60 + 2^30,
    //              l = (X mod 2^31) - 2^30 in [-2^30, 2^30),
    //              h = (X >> 31) - 2^29    in [-2^29, 2^29];
    //   row side:  c = a_i or a_i - p, whichever is in (-2^60, 2^60),
    //              c = ch 2^31 + cl,        cl in [-2^30, 2^30), ch in [-2^29, 2^29].
    // The key-side offset D is a constant: a_i X = c (X - D) + c D, and
    // sum_i c_i D joins a0 in the row constant K below.  With both digits that
    // small, c (X - D) = ch h 2^62 + (ch l + cl h) 2^31 + cl l, and 2^62 = 2
    // (mod p) gives, over the three terms,
    //   H = sum ch h    (|H| <= 3 2^58),
    //   A = sum cl l    (|A| <= 3 2^60),
    //   M = sum (ch l + cl h) = A + H + sum (cl - ch)(h - l)   (Karatsuba;
    //       |M| <= 3 2^60; |cl - ch|, |h - l| < 1.5 2^30 fit 32-bit operands),
    //   row = A + 2H + 2^31 M + K   (mod p).
    // Nine 32x32->64 multiply-adds in one chain give X1 = H, X2 = A + H and
    // X3 = M as exact two's-complement 64-bit values; A + 2H = X1 + X2.
    // With M = M1 2^30 + m0 (m0 = M mod 2^30, M1 = M >> 30 arithmetic,
    // |M1| <= 3 2^30) and 2^61 = 1 (mod p):
    //   2^31 M = M1 2^61 + m0 2^31 = M1 + m0 2^31                 (mod p)
    //   S = A + 2H + m0 2^31 + M1  in [-4.5 2^60 - 3 2^30, 6.5 2^60 + 3 2^30]
    // and K = (a0 + D (a1 + a2 + a3)) mod p + 3p lies in [6 2^60 - 3, 8 2^60),
    // so S + K is in [1.5 2^60 - 2^32, 14.5 2^60 + 2^32]: positive and far
    // below 2^64 - 8, and the 64-bit sum needs no carry word.
    // The row adds K + 1 (the "+1" of Algorithm div-simple, Sec. 1.5), so
    // S1 = S + K + 1 = v + 1 for v = S + K, and Algorithm div-simple gives
    //   z = floor(v / p) = ((S1 >> 61) + S1) >> 61,  v mod p = (v + z) & p,
    // the canonical residue, branch free; (S1 >> 61) + S1 < 2^64 again.
    struct Pow3 {
        int l[3], h[3], d[3];  // signed digits of X_i - D, and d = h - l
    };

    // Signed digits of a lazy X < 2^61 + 8 (above).  X >> 31 <= 2^30.
    __device__ static __forceinline__ void sdigits(u64 X, Pow3& xp, int i) {
        const u32 lo = (u32)X, hi = (u32)(X >> 32);
        const u32 lu = lo & 0x7FFFFFFFu;
        const u32 hu = __funnelshift_r(lo, hi, 31);
        xp.l[i] = (int)lu - (1 << 30);
        xp.h[i] = (int)hu - (1 << 29);
        xp.d[i] = (int)hu - (int)lu + ((1 << 30) - (1 << 29));  // h - l
    }

    // x^2 for x = xh 2^31 + xl (lazy, unsigned digits):
    //   x^2 = xh^2 2^62 + xh xl 2^32 + xl^2 = 2 xh^2 + xl^2 + Q 2^32 with Q = xh xl
    //   Q 2^32 = (Q >> 29) 2^61 + (Q mod 2^29) 2^32 = (Q >> 29) + (Q mod 2^29) 2^32
    //   sum < 2^62 + 2^61 + 2^32 + 2^61 < 2^64; one fold gives < 2^61 + 4.
    __device__ static __forceinline__ u64 square(u32 xl, u32 xh) {
        u64 A = madw(xl, xl, 0ull);
        A = madw(xh << 1, xh, A);
        const u64 Q = madw(xh, xl, 0ull);
        return fold(A + (Q >> 29) + ((Q & 0x1FFFFFFFull) << 32));
    }

    // x = key mod p (lazy: (key & p) + (key >> 61) < 2^61 + 8), x^2 and
    // x^3 = x^2 * x (lazy), each in signed digits.
    __device__ static __forceinline__ void powers3(u64 key, Pow3& xp) {
        const u64 x1 = fold(key);
        Split s1;
        s1.lo = (u32)x1 & 0x7FFFFFFFu;
        s1.hi = (u32)(x1 >> 31);
        s1.hi2 = s1.hi << 1;
        const u64 x2 = square(s1.lo, s1.hi);
        const u64 x3 = mul_add(x2, s1, 0ull);
        sdigits(x1, xp, 0);
        sdigits(x2, xp, 1);
        sdigits(x3, xp, 2);
    }

    // One row (above): cl/ch/nd = the signed digits of a1..a3 and cl - ch,
    // k1 = K + 1.  Returns the 64-bit word y64 = v + z with v mod p = y64 & p:
    // the canonical residue is (yhi mod 2^29 : ylo), its bit 60 is bit 28 of
    // yhi.  c2p31 = 2^31 arrives as a run-time operand so that m0 2^31 + X2
    // stays one wide multiply-add.
    __device__ static __forceinline__ void row_sd(const Pow3& xp, const int* cl, const int* ch,
                                                  const int* nd, u64 k1, u32 c2p31, u32& ylo,
                                                  u32& yhi) {
        long long X1 = (long long)ch[0] * xp.h[0];
        X1 += (long long)ch[1] * xp.h[1];
        X1 += (long long)ch[2] * xp.h[2];                // H
        long long X2 = X1 + (long long)cl[0] * xp.l[0];
        X2 += (long long)cl[1] * xp.l[1];
        X2 += (long long)cl[2] * xp.l[2];                // A + H
        long long X3 = X2 + (long long)nd[0] * xp.d[0];
        X3 += (long long)nd[1] * xp.d[1];
        X3 += (long long)nd[2] * xp.d[2];                // M
        const u32 m0 = (u32)X3 & 0x3FFFFFFFu;
        const long long M1 = X3 >> 30;
        const u64 T = (u64)m0 * c2p31 + (u64)X2;
        const u64 S1 = T + (u64)X1 + (u64)M1 + k1;      // S + K + 1 (no wrap)
        const u32 z = (u32)((S1 + (S1 >> 61)) >> 61);   // floor(v / p)
        const u64 y = S1 + z - 1;                        // v + z
        ylo = (u32)y;
        yhi = (u32)(y >> 32);
    }

    // Row-side constants of row_sd for canonical a0..a3 < p (host or device):
    // the signed digits of c_i = a_i or a_i - p (the one in (-2^60, 2^60)),
    // cl_i - ch_i, and k1 = K + 1 with K = (a0 + D (a1 + a2 + a3)) mod p + 3p,
    // D = 2^60 + 2^30.
    __host__ __device__ static inline void sd_coef(const u64* a, int* cl, int* ch, int* nd,
                                                   u64& k1) {
        u64 s = 0;  // (a1 + a2 + a3) mod p
        for (int i = 0; i < 3; ++i) {
            const u64 ai = a[i + 1];
            const long long c = ai <= (P >> 1) ? (long long)ai : (long long)ai - (long long)P;
            const int l = ((int)((u32)(u64)c << 1)) >> 1;  // low 31 bits, sign-extended
            cl[i] = l;
            ch[i] = (int)((c - l) >> 31);                 // exact: c - l = 0 mod 2^31
            nd[i] = cl[i] - ch[i];
            s += ai;
            if (s >= P) s -= P;
        }
        // 2^60 s = s / 2 (mod p), as 2^61 = 1: s / 2 for even s, (s + p) / 2 for odd s
        const u64 s60 = (s & 1ull) ? (s + P) >> 1 : s >> 1;
        // 2^30 s = (s mod 2^31) 2^30 + (s >> 31) 2^61 = (s mod 2^31) 2^30 + (s >> 31)
        u64 s30 = ((s & 0x7FFFFFFFull) << 30) + (s >> 31);
        if (s30 >= P) s30 -= P;
        u64 k = a[0] + s60;
        if (k >= P) k -= P;
        k += s30;
        if (k >= P) k -= P;
        k1 = k + 3 * P + 1;
    }

    // The canonical residue from row_sd's output.
    __device__ static __forceinline__ u64 canon_sd(u32 ylo, u32 yhi) {
        return ((u64)(yhi & 0x1FFFFFFFu) << 32) | ylo;
    }

    // Algorithm Mersenne-arb-r (Sec. 3.3) on row_sd's output: with h the
    // canonical residue and h + 1 = a 2^60 + j (j < 2^60), the bucket is
    // floor(r j / 2^60) -- taken from j's 28- and 32-bit halves as
    // floor((j_hi r + floor(j_lo r / 2^32)) / 2^28), the same integer -- and a
    // is returned (the update is subtracted when a = 0).
    __device__ static __forceinline__ void arb_split_sd(u32 ylo, u32 yhi, u32 r, u32& bucket,
                                                        u32& a) {
        const u32 hlo = ylo + 1u;  // h + 1 = (hhi : hlo), h < 2^61 - 1
        const u32 hhi = (yhi & 0x1FFFFFFFu) + (hlo == 0u ? 1u : 0u);
        bucket = (u32)(((u64)(hhi & 0x0FFFFFFFu) * r + __umulhi(hlo, r)) >> 28);
        a = hhi >> 28;
    }

    // Bucket (low bits) and sign bit (bit 60) of the canonical residue.
    __device__ static __forceinline__ void bucket_sign_sd(u32 ylo, u32 yhi, u32 mask, u32& bucket,
                                                          u32& sign) {
        bucket = ylo & mask;
        sign = (yhi >> 28) & 1u;
    }
};

// ---------------------------------------------------------------- p = 2^31-1
struct P31 {
    static constexpr int B = 31;
    static constexpr u32 P = 0x7FFFFFFFu;
    typedef u32 key_t;
    typedef u32 val_t;

    // x < 2^32: (x & p) + (x >> 31) <= 2^31 - 1 + 1 = 2^31 < 2p.
    __device__ static __forceinline__ u32 reduce_key(u32 x) { return canon((x & P) + (x >> 31)); }
    __device__ static __forceinline__ u32 canon(u32 y) { return y >= P ? y - P : y; }

    // y = z*x + a (mod p), lazily reduced (< 2^31 + 3), for z < 2^31 + 3,
    // x < p, a < p:
    //   v = z*x + a < (2^31+3)*2^31 + 2^31 < 2^63
    //   f = (v & p) + (v >> 31) < 2^31 + 2^32 + 4
    //   (f & p) + (f >> 31) < 2^31 + 3
    __device__ static __forceinline__ u32 mul_add(u32 z, u32 x, u32 a) {
        u64 v = (u64)z * x + a;
        v = (v & P) + (v >> 31);
        return (u32)((v & P) + (v >> 31));
    }

    __device__ static __forceinline__ u32 bucket(u32 h, u32 mask) { return h & mask; }
    __device__ static __forceinline__ u32 sign_bit(u32 h) { return (h >> 30) & 1u; }

    // ---- power sum (the update kernels' row hash for k = 4) ----
    //
    // x canonical, x^2 and x^3 lazy (< 2^31 + 3, from mul_add).
    struct Pow3 {
        u32 x[3];
    };

    __device__ static __forceinline__ void powers3(u32 key, Pow3& xp) {
        const u32 x = reduce_key(key);
        xp.x[0] = x;
        xp.x[1] = mul_add(x, x, 0u);
        xp.x[2] = mul_add(xp.x[1], x, 0u);
    }

    // Bucket and sign bit of y = a0 + a1 x + a2 x^2 + a3 x^3 (mod p), all a_i < p:
    //   S = a1 x + a2 x^2 + a3 x^3 + a0 < 3 2^31 (2^31 + 3) + 2^31 < 2^64
    //   2^32 = 2 (mod p):  v = 2 S.hi + S.lo < 3 2^32
    //   f = (v & p) + (v >> 31) < 2^31 + 6 < 2p
    // f >= p exactly when f + 1 >= 2^31; then the residue f - p = f + 1 - 2^31
    // is below 8 (bit 30 clear) and has the low bits of f + 1.
    __device__ static __forceinline__ void row_bs(const Pow3& xp, u32 a0, u32 a1, u32 a2, u32 a3,
                                                  u32 mask, u32& bucket, u32& sign) {
        u64 S = madw(a1, xp.x[0], (u64)a0);
        S = madw(a2, xp.x[1], S);
        S = madw(a3, xp.x[2], S);
        const u64 v = madw((u32)(S >> 32), 2u, S & 0xFFFFFFFFull);
        const u32 f = ((u32)v & P) + (u32)(v >> 31);
        const u32 over = (f + 1u) >> 31;
        bucket = (f + over) & mask;
        sign = over ? 0u : ((f >> 30) & 1u);
    }

    // Algorithm Mersenne-arb-r (Sec. 3.3): h' = h + 1, bucket floor(r j / 2^30)
    // for its low 30 bits j, a = its top bit.
    __device__ static __forceinline__ void arb_split(u32 h, u32 r, u32& bucket, u32& a) {
        const u32 hx = h + 1u;
        bucket = (u32)(((u64)(hx & 0x3FFFFFFFu) * r) >> 30);
        a = hx >> 30;
    }
};

// ---------------------------------------------------------------- p = 2^89-1
//
// Values are unsigned __int128 below 2^89 + 2^4 (lazy).
struct P89 {
    static constexpr int B = 89;
    typedef u128x key_t;
    typedef u128x val_t;

    // The 32x32->64 multiply-adds of this prime's limb arithmetic as plain C++
    // (they shadow the inline-PTX madw / madws inside this struct): on the
    // 2^30-key sweep the compiler's own scheduling of these rows was 6% faster
    // (22.6 vs 24.1 ms), while the other primes' rows are faster with the PTX
    // form.
    __device__ static __forceinline__ u64 madw(u32 a, u32 b, u64 c) {
        return (u64)a * (u64)b + c;
    }
    __device__ static __forceinline__ u64 madws(int a, int b, u64 c) {
        return (u64)((long long)a * (long long)b) + c;
    }

    __device__ static __forceinline__ u128 Pv() { return (((u128)1) << 89) - 1; }

    __device__ static __forceinline__ u128 load(const u128x& v) {
        return ((u128)v.hi << 64) | v.lo;
    }
    __device__ static __forceinline__ u128x store(u128 v) {
        u128x r;
        r.lo = (u64)v;
        r.hi = (u64)(v >> 64);
        return r;
    }

    // x < 2^128: (x & p) + (x >> 89) < 2^89 + 2^39 < 2p.
    __device__ static __forceinline__ u128 reduce_key(u128 x) {
        return canon((x & Pv()) + (x >> 89));
    }
    __device__ static __forceinline__ u128 canon(u128 y) { return y >= Pv() ? y - Pv() : y; }

    // y = z*x + a (mod p), lazily reduced (< 2^89 + 4), for z < 2^89 + 4,
    // x < p, a < p.  With z = z1*2^64 + z0, x = x1*2^64 + x0 (z1 <= 2^25,
    // x1 < 2^25):
    //   z*x = z1 x1 2^128 + (z1 x0 + z0 x1) 2^64 + z0 x0
    //   2^128 = 2^39 (mod p), so z1 x1 2^128 = z1 x1 2^39, and z1 x1 2^39 < 2^89+2^64
    //   T = z1 x0 + z0 x1 < 2^90;  T 2^64 = (T >> 25) + (T mod 2^25) 2^64  (mod p)
    //   z0 x0 < 2^128;  z0 x0 = (z0 x0 >> 89) + (z0 x0 mod 2^89)  (mod p)
    //   S = sum of those six terms + a < 2^91
    __device__ static __forceinline__ u128 mul_add(u128 z, u128 x, u128 a) {
        const u64 z0 = (u64)z, z1 = (u64)(z >> 64);
        const u64 x0 = (u64)x, x1 = (u64)(x >> 64);
        const u128 p00 = (u128)z0 * x0;
        const u128 T = (u128)z1 * x0 + (u128)z0 * x1;
        const u128 p11 = (u128)(z1 * x1);  // < 2^51, fits 64 bits
        u128 S = (p11 << 39) + (T >> 25) + ((T & ((((u128)1) << 25) - 1)) << 64) + (p00 >> 89) +
                 (p00 & Pv()) + a;
        return (S & Pv()) + (S >> 89);
    }

    __device__ static __forceinline__ u32 bucket(u128 h, u32 mask) { return (u32)h & mask; }
    __device__ static __forceinline__ u32 sign_bit(u128 h) { return (u32)(h >> 88) & 1u; }

    // ---- power sum with 30-bit limbs (the update kernels' row hash, k = 4) ----
    //
    // A value is z = z0 + z1 2^30 + z2 2^60 with z0, z1 < 2^30 and z2 <= 2^29
    // (so z < 2^90; lazy, not necessarily below p).  Since 2^89 = 1 (mod p),
    //   2^90 = 2  and  2^120 = 2^31 = 2 * 2^30  (mod p),
    // so the columns 3 and 4 of a 3-limb product wrap onto columns 0 and 1
    // with a factor 2, and every product of two values is
    //   L0 + L1 2^30 + L2 2^60  with
    //   L0 = y0 z0 + y1 (2 z2) + y2 (2 z1),  L1 = y0 z1 + y1 z0 + y2 (2 z2),
    //   L2 = y0 z2 + y1 z1 + y2 z0,
    // nine 32x32->64 products (2 z1 < 2^31, 2 z2 <= 2^30).
    static constexpr u32 M30 = (1u << 30) - 1u;
    static constexpr u32 M29 = (1u << 29) - 1u;

    struct Pow3 {
        u32 l[3][3];  // x, x^2, x^3, three limbs each
        int d[3][3];  // per power: l1 - l0, l2 - l0, l2 - l1
    };

    // Limbs of (L0 + L1 2^30 + L2 2^60) mod p for L0 < 2^64 - 2^34,
    // L1, L2 < 2^64 - 2^35 (every caller's sums are below 12 2^60 + 2^30):
    //   r0 = L0 mod 2^30, L1' = L1 + (L0 >> 30), r1 = L1' mod 2^30,
    //   L2' = L2 + (L1' >> 30) < 2^64;  L2' 2^60 = (L2' mod 2^29) 2^60 + (L2' >> 29) (mod p)
    //   s0 = r0 + (L2' >> 29) < 2^30 + 2^35; carries: s1 = r1 + (s0 >> 30) < 2^30 + 33,
    //   r2 = (L2' mod 2^29) + (s1 >> 30) <= 2^29.
    __device__ static __forceinline__ void norm3(u64 L0, u64 L1, u64 L2, u32 (&r)[3]) {
        L1 += L0 >> 30;
        L2 += L1 >> 30;
        const u64 s0 = (u64)((u32)L0 & M30) + (L2 >> 29);
        const u32 s1 = ((u32)L1 & M30) + (u32)(s0 >> 30);
        r[0] = (u32)s0 & M30;
        r[1] = s1 & M30;
        r[2] = ((u32)L2 & M29) + (s1 >> 30);
    }

    // y * z (mod p), lazy, for lazy y, z (bounds above: L0 < 3 2^60).
    __device__ static __forceinline__ void mul3(const u32 (&y)[3], const u32 (&z)[3], u32 (&r)[3]) {
        const u32 z1d = z[1] << 1, z2d = z[2] << 1;
        u64 L0 = madw(y[0], z[0], 0ull);
        L0 = madw(y[1], z2d, L0);
        L0 = madw(y[2], z1d, L0);
        u64 L1 = madw(y[0], z[1], 0ull);
        L1 = madw(y[1], z[0], L1);
        L1 = madw(y[2], z2d, L1);
        u64 L2 = madw(y[0], z[2], 0ull);
        L2 = madw(y[1], z[1], L2);
        L2 = madw(y[2], z[0], L2);
        norm3(L0, L1, L2, r);
    }

    // One Horner step (Algorithm Mersenne) on limbs: r = y x + a (mod p), lazy,
    // for lazy y, x and a canonical a: a's limbs join the columns before the
    // carry pass (L0 < 3 2^60 + 2^30, within norm3's bounds).
    __device__ static __forceinline__ void mul_add3(const u32 (&y)[3], const u32 (&x)[3],
                                                    const u32 (&a)[3], u32 (&r)[3]) {
        const u32 x1d = x[1] << 1, x2d = x[2] << 1;
        u64 L0 = madw(y[0], x[0], (u64)a[0]);
        L0 = madw(y[1], x2d, L0);
        L0 = madw(y[2], x1d, L0);
        u64 L1 = madw(y[0], x[1], (u64)a[1]);
        L1 = madw(y[1], x[0], L1);
        L1 = madw(y[2], x2d, L1);
        u64 L2 = madw(y[0], x[2], (u64)a[2]);
        L2 = madw(y[1], x[1], L2);
        L2 = madw(y[2], x[0], L2);
        norm3(L0, L1, L2, r);
    }

    // The three limbs of a value below 2^90.
    __device__ static __forceinline__ void limbs(u128 v, u32 (&l)[3]) {
        l[0] = (u32)v & M30;
        l[1] = (u32)(v >> 30) & M30;
        l[2] = (u32)(v >> 60);
    }

    // The canonical residue of lazy limbs (value < 2^89 + 2^60 < 2p).
    __device__ static __forceinline__ u128 canon3(const u32 (&l)[3]) {
        return canon((u128)l[0] | ((u128)l[1] << 30) | ((u128)l[2] << 60));
    }

    // x = (key & p) + (key >> 89) < 2^89 + 2^39 (limb 2 <= 2^29), then x^2, x^3.
    __device__ static __forceinline__ void powers3(const u128x& key, Pow3& xp) {
        const u128 v = load(key);
        const u128 x = (v & Pv()) + (v >> 89);
        xp.l[0][0] = (u32)x & M30;
        xp.l[0][1] = (u32)(x >> 30) & M30;
        xp.l[0][2] = (u32)(x >> 60);
        mul3(xp.l[0], xp.l[0], xp.l[1]);
        mul3(xp.l[1], xp.l[0], xp.l[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            xp.d[i][0] = (int)xp.l[i][1] - (int)xp.l[i][0];
            xp.d[i][1] = (int)xp.l[i][2] - (int)xp.l[i][0];
            xp.d[i][2] = (int)xp.l[i][2] - (int)xp.l[i][1];
        }
    }

    // Bucket and sign bit of y = a0 + a1 x + a2 x^2 + a3 x^3 (mod p).
    // c: 21 words precomputed on the host from canonical coefficients: c[0..2]
    // the limbs of a0; for i = 1..3, c[6i-3 .. 6i+2] = (l0, l1, l2, l0 - l1,
    // l0 - l2, l1 - l2) of a_i (l0, l1 < 2^30, l2 < 2^29; differences signed).
    // Each product a_i x^i is taken by Karatsuba, six 32x32->64 products
    // instead of nine: with P_jj = l_j x_j and D_jk = (l_j - l_k)(x_k - x_j),
    //   l0 x1 + l1 x0 = P00 + P11 + D01,  l0 x2 + l2 x0 = P00 + P22 + D02,
    //   l1 x2 + l2 x1 = P11 + P22 + D12,
    // and the wrapped columns of mul3 become
    //   L0 = P00 + 2 (P11 + P22 + D12),  L1 = P00 + P11 + 2 P22 + D01,
    //   L2 = P00 + P11 + P22 + D02.
    // Summed over the three terms (S_jj, T_jk) with U = S00 + S11 + S22:
    //   L0 = 2 (U + T12) - S00 + a0.l0,  L1 = U + S22 + T01 + a0.l1,
    //   L2 = U + T02 + a0.l2,
    // computed modulo 2^64 (the T's are signed); each column's true value is
    // below 12 2^60 + 2^30 (as in the nine-product form), so the results are
    // exact.  Then the columns are normalised as below.
    __device__ static __forceinline__ void row_bs(const Pow3& xp, const u32 (&c)[21], u32 mask,
                                                  u32& bucket, u32& sign) {
        u64 S00 = 0, S11 = 0, S22 = 0;
        u64 T01 = c[1], T02 = c[2], T12 = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const u32* a = c + 3 + 6 * i;
            S00 = madw(a[0], xp.l[i][0], S00);
            S11 = madw(a[1], xp.l[i][1], S11);
            S22 = madw(a[2], xp.l[i][2], S22);
            T01 = madws((int)a[3], xp.d[i][0], T01);
            T02 = madws((int)a[4], xp.d[i][1], T02);
            T12 = madws((int)a[5], xp.d[i][2], T12);
        }
        const u64 U = S00 + S11 + S22;
        u64 L2 = U + T02;
        u64 L1 = U + S22 + T01;
        u64 L0 = 2ull * (U + T12) - S00 + c[0];
        // With y = s0 + r1 2^30 + r2 2^60 after norm3's first pass (s0 < 2^36
        // unreduced), the carries of y are u1 = r1 + (s0 >> 30) and
        // u2 = r2 + (u1 >> 30) <= 2^29, y < 2^89 + 2^36 < 2p, and
        //   y >= p  <=>  y + 1 >= 2^89  <=>  u2 + [s0, u1 both end in 30 one bits] >= 2^29.
        // Then the residue y - p = y + 1 - 2^89 < 2^37 has bit 88 clear and the
        // low 30 bits of s0 + 1; otherwise bit 88 of y is bit 28 of u2.
        L1 += L0 >> 30;
        L2 += L1 >> 30;
        const u64 s0 = (u64)((u32)L0 & M30) + (L2 >> 29);
        const u32 u1 = ((u32)L1 & M30) + (u32)(s0 >> 30);
        const u32 u2 = ((u32)L2 & M29) + (u1 >> 30);
        const u32 ones = (((u32)s0 & u1 & M30) == M30) ? 1u : 0u;
        const u32 over = (u2 + ones) >> 29;
        bucket = ((u32)s0 + over) & mask;
        sign = over ? 0u : ((u2 >> 28) & 1u);
    }

    // Algorithm Mersenne-arb-r (Sec. 3.3): h' = h + 1, bucket floor(r j / 2^88)
    // for its low 88 bits j (r j < 2^120), a = its top bit.
    __device__ static __forceinline__ void arb_split(u128 h, u32 r, u32& bucket, u32& a) {
        const u128 hx = h + 1;
        const u128 j = hx & ((((u128)1) << 88) - 1);
        bucket = (u32)((j * (u128)r) >> 88);
        a = (u32)(hx >> 88);
    }
};

// ------------------------------------------------------------ p = 2^64-59
//
// Pseudo-Mersenne: reduction by Algorithm division-generalized (3 steps, which
// covers every v < (2^64/59)^2 (2^64 - 59), i.e. all v < 2^128 by the theorem
// of Sec. 4) and Algorithm mod-generalized.  Values are canonical (< p).
struct P64 {
    static constexpr int B = 64;
    static constexpr u64 C = 59;
    static constexpr u64 P = 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59
    typedef u64 key_t;
    typedef u64 val_t;

    // x < 2^64 < 2p
    __device__ static __forceinline__ u64 reduce_key(u64 x) { return x >= P ? x - P : x; }

    // v mod p for v <= (p-1)^2 + (p-1) (a product of residues plus a residue):
    //   v' = v + c < 2^128 (no carry out: (p-1)p + c < 2^128 - 2^70)
    //   z  = v' >> 64;  z = (z c + v') >> 64  (twice)   -> floor(v / p) < 2^64
    //   y  = (v + z c) mod 2^64                          -> v mod p
    __device__ static __forceinline__ u64 mod_p(u128 v) { return (u64)v + div_p(v) * C; }

    // floor(v / p) for the same v (the three division steps above).
    __device__ static __forceinline__ u64 div_p(u128 v) {
        const u128 vp = v + C;
        u64 z = (u64)(vp >> 64);
        z = (u64)(((u128)z * C + vp) >> 64);
        z = (u64)(((u128)z * C + vp) >> 64);
        return z;
    }

    // Any number r of buckets for a pseudo-Mersenne prime: the most uniform map
    // floor(h r / p) (Sec. 1.5, "Applications to an arbitrary number of
    // buckets"), by Algorithm division-generalized.  h r < 2^96 is in range.
    // There is no sign bit to pair with it; sketches take the sign from a
    // second polynomial.
    __device__ static __forceinline__ void arb_split(u64 h, u32 r, u32& bucket, u32& a) {
        bucket = (u32)div_p((u128)h * r);
        a = 0;
    }

    __device__ static __forceinline__ u64 mul_add(u64 z, u64 x, u64 a) {
        return mod_p((u128)z * x + a);
    }

    __device__ static __forceinline__ u32 bucket(u64 h, u32 mask) { return (u32)h & mask; }
    __device__ static __forceinline__ u32 sign_bit(u64 h) { return (u32)(h >> 63); }

    // ---- power sum (the update kernels' row hash for k = 4) ----
    //
    // x, x^2, x^3 (canonical) as limbs of 29, 29 and 6 bits:
    //   x^i = l0 + l1 2^29 + l2 2^58.
    static constexpr u32 M29 = (1u << 29) - 1u;
    struct Pow3 {
        u32 l[3][3];
    };

    __device__ static __forceinline__ void split29(u64 z, u32 (&l)[3]) {
        l[0] = (u32)z & M29;
        l[1] = (u32)(z >> 29) & M29;
        l[2] = (u32)(z >> 58);
    }

    __device__ static __forceinline__ void powers3(u64 key, Pow3& xp) {
        const u64 x = reduce_key(key);
        const u64 x2 = mod_p((u128)x * x);
        split29(x, xp.l[0]);
        split29(x2, xp.l[1]);
        split29(mod_p((u128)x2 * x), xp.l[2]);
    }

    // Bucket and sign bit of y = a0 + a1 x + a2 x^2 + a3 x^3 (mod p).
    // c: 18 words precomputed on the host, for i = 1..3 and v = 0..2 the low and
    // high 32-bit halves of b_iv = a_i 2^(29 v) mod p, at c[6(i-1) + 2v + {0,1}];
    // then a_i x^i = sum_v l_iv b_iv (mod p).  Columns of weight 1 and 2^32:
    //   L0 = a0.lo + sum l_iv b_iv.lo,  L1 = a0.hi + sum l_iv b_iv.hi,
    // each below 2^32 + 6 2^61 + 3 2^38 < 2^64 (l_i0, l_i1 < 2^29, l_i2 < 2^6).
    // V = L0 + L1 2^32 = vh 2^64 + vl with vh < 2^32 (L1 < 0.76 2^64).
    // V < 2^96 < (2^64/59)^2, so two steps of Algorithm division-generalized
    // give z = floor(V / p) (Thm simple-div, Sec. 4), and Algorithm
    // mod-generalized the canonical y = (V + 59 z) mod 2^64:
    //   v' = V + 59;  z = v' >> 64;  z = (59 z + v') >> 64
    //     = v'.hi + carry(v'.lo + 59 v'.hi).
    __device__ static __forceinline__ void row_bs(const Pow3& xp, u64 a0, const u32 (&c)[18],
                                                  u32 mask, u32& bucket, u32& sign) {
        u64 L0 = a0 & 0xFFFFFFFFull, L1 = a0 >> 32;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                L0 = madw(xp.l[i][v], c[6 * i + 2 * v], L0);
                L1 = madw(xp.l[i][v], c[6 * i + 2 * v + 1], L1);
            }
        }
        const u64 t = (L0 >> 32) + (L1 & 0xFFFFFFFFull);  // < 2^33
        const u64 vl = (L0 & 0xFFFFFFFFull) | (t << 32);
        const u32 vh = (u32)(L1 >> 32) + (u32)(t >> 32);
        const u64 vpl = vl + C;
        const u32 vph = vh + (vpl < vl ? 1u : 0u);
        const u64 q = (u64)vph * C;
        const u32 z = vph + ((vpl + q) < vpl ? 1u : 0u);
        const u64 y = vl + (u64)z * C;
        bucket = (u32)y & mask;
        sign = (u32)(y >> 63);
    }
};

}  // namespace msf
