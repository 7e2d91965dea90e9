// Count Sketch update kernel (Algorithm count-sketch "Process", Sec. 1.3) and
// the per-prime hashing glue it needs.  Included by one translation unit per
// prime, which instantiates the launch dispatcher for that prime.
//
// Per block:
//   1. zero its counter tile (PLACE_SMEM: all t x m counters as int32 in shared
//      memory; PLACE_DSMEM: a 1/cluster slice of every row, the slices of the
//      cluster's blocks together covering the sketch; PLACE_GLOBAL: none);
//   2. grid-stride over groups of 4 consecutive keys (16-byte vector loads when
//      aligned), reduce each key mod p, hash it with every row's polynomial,
//      split each hash value into (bucket, sign) (Algorithm h-and-s), and add
//      sign * weight to the counter with a shared-memory (or distributed
//      shared-memory) atomic;
//   3. add its tile into the int64 counters in global memory (a sketch is
//      linear in the stream, so per-block partial sketches add up exactly).
// Weights whose magnitude could overflow an int32 tile counter (|w| > w_safe,
// computed on the host from the keys one tile can see) go straight to the
// int64 counters instead, so the result is exact for every int32 weight.
#pragma once

#include <stdint.h>

#include <type_traits>

#include "ms_field.cuh"
#include "ms_kernels.h"

namespace msk {

using msf::u128;
using msf::u128x;

// ------------------------------------------------------------ field glue
//
// FieldOps<F> gives a uniform interface over the four primes:
//   val_t         hash value type used in registers
//   Prep          a key prepared for multiplication (reduced, maybe split)
//   prep(key)     key -> Prep
//   mul_add(z, P, a)  lazy  z*x + a
//   canon(y)      final canonical residue
//   from_words(w) coefficient from its 64-bit limbs
template <class F>
struct FieldOps;

template <>
struct FieldOps<msf::P61> {
    typedef msf::P61 F;
    typedef u64 val_t;
    typedef F::Split Prep;
    typedef u64 key_t;
    static constexpr int WORDS = 1;
    __device__ static __forceinline__ Prep prep(u64 key) { return F::split(F::reduce_key(key)); }
    __device__ static __forceinline__ val_t mul_add(val_t z, const Prep& x, val_t a) {
        return F::mul_add(z, x, a);
    }
    __device__ static __forceinline__ val_t canon(val_t y) { return F::canon(y); }
    __device__ static __forceinline__ val_t from_words(const u64* w) { return w[0]; }
    __device__ static __forceinline__ u32 bucket(val_t h, u32 mask) { return F::bucket(h, mask); }
    __device__ static __forceinline__ u32 sign_bit(val_t h) { return F::sign_bit(h); }
    __device__ static __forceinline__ void arb_split(val_t h, u32 r, u32& bucket, u32& a) {
        F::arb_split(h, r, bucket, a);
    }
};

template <>
struct FieldOps<msf::P31> {
    typedef msf::P31 F;
    typedef u32 val_t;
    typedef u32 Prep;
    typedef u32 key_t;
    static constexpr int WORDS = 1;
    __device__ static __forceinline__ Prep prep(u32 key) { return F::reduce_key(key); }
    __device__ static __forceinline__ val_t mul_add(val_t z, const Prep& x, val_t a) {
        return F::mul_add(z, x, a);
    }
    __device__ static __forceinline__ val_t canon(val_t y) { return F::canon(y); }
    __device__ static __forceinline__ val_t from_words(const u64* w) { return (u32)w[0]; }
    __device__ static __forceinline__ u32 bucket(val_t h, u32 mask) { return F::bucket(h, mask); }
    __device__ static __forceinline__ u32 sign_bit(val_t h) { return F::sign_bit(h); }
    __device__ static __forceinline__ void arb_split(val_t h, u32 r, u32& bucket, u32& a) {
        F::arb_split(h, r, bucket, a);
    }
};

template <>
struct FieldOps<msf::P64> {
    typedef msf::P64 F;
    typedef u64 val_t;
    typedef u64 Prep;
    typedef u64 key_t;
    static constexpr int WORDS = 1;
    __device__ static __forceinline__ Prep prep(u64 key) { return F::reduce_key(key); }
    __device__ static __forceinline__ val_t mul_add(val_t z, const Prep& x, val_t a) {
        return F::mul_add(z, x, a);
    }
    __device__ static __forceinline__ val_t canon(val_t y) { return y; }  // already canonical
    __device__ static __forceinline__ val_t from_words(const u64* w) { return w[0]; }
    __device__ static __forceinline__ u32 bucket(val_t h, u32 mask) { return F::bucket(h, mask); }
    __device__ static __forceinline__ u32 sign_bit(val_t h) { return F::sign_bit(h); }
    __device__ static __forceinline__ void arb_split(val_t h, u32 r, u32& bucket, u32& a) {
        F::arb_split(h, r, bucket, a);
    }
};

template <>
struct FieldOps<msf::P89> {
    typedef msf::P89 F;
    typedef u128 val_t;
    typedef u128 Prep;
    typedef u128x key_t;
    static constexpr int WORDS = 2;
    __device__ static __forceinline__ Prep prep(const u128x& key) {
        return F::reduce_key(F::load(key));
    }
    __device__ static __forceinline__ val_t mul_add(val_t z, const Prep& x, val_t a) {
        return F::mul_add(z, x, a);
    }
    __device__ static __forceinline__ val_t canon(val_t y) { return F::canon(y); }
    __device__ static __forceinline__ val_t from_words(const u64* w) {
        return ((u128)w[1] << 64) | w[0];
    }
    __device__ static __forceinline__ u32 bucket(val_t h, u32 mask) { return F::bucket(h, mask); }
    __device__ static __forceinline__ u32 sign_bit(val_t h) { return F::sign_bit(h); }
    __device__ static __forceinline__ void arb_split(val_t h, u32 r, u32& bucket, u32& a) {
        F::arb_split(h, r, bucket, a);
    }
};

// Bucket and sign flag (1: the update is subtracted) of one row from its hash
// value(s).  arb_r == 0: Algorithm h-and-s (the low bits of h and its bit
// b-1).  arb_r > 0, any number of buckets: Algorithm Mersenne-arb-r for c = 1,
// whose two-for-one sign is s = 2a - 1 from the same h + 1 (Sec. 3.3), or
// floor(h r / p) for 2^64 - 59; with two polynomials the sign is always bit
// b-1 of the second one.
template <class F, int NF>
__device__ __forceinline__ void split_row(const typename FieldOps<F>::val_t& h,
                                          const typename FieldOps<F>::val_t& g, u32 mask,
                                          u32 arb_r, u32& bucket, u32& sign) {
    typedef FieldOps<F> Ops;
    if (arb_r) {
        u32 a;
        Ops::arb_split(h, arb_r, bucket, a);
        sign = (NF == 2) ? Ops::sign_bit(g) : (a ^ 1u);
    } else {
        bucket = Ops::bucket(h, mask);
        sign = Ops::sign_bit(g);
    }
}

// ------------------------------------------------------------ coefficients
//
// Compile-time (t, k): the coefficients travel in the kernel's parameter
// space.  With the row and coefficient loops unrolled, every access has a
// constant offset, so the multiply instructions read them straight from the
// constant bank.  For p = 2^61-1 the 31-bit splits used by the power-sum
// evaluation are precomputed on the host.
// For 2^89-1 and 2^64-59 the power sum also takes 21 and 18 precomputed words
// per function (k = 4), built by fill_param_coef.
template <class F>
struct PsLimbs {
    static constexpr int N = std::is_same<F, msf::P89>::value   ? 21
                             : std::is_same<F, msf::P64>::value ? 18
                                                                : 0;
};

template <class F, int NFUN, int K>
struct ParamCoef {
    static constexpr int SD = (NFUN > 0 && K == 4 && std::is_same<F, msf::P61>::value) ? NFUN : 0;
    u64 w[NFUN > 0 ? NFUN * K * FieldOps<F>::WORDS : 1];
    // P61, k = 4 (row_sd): signed digits of a1..a3 of function f at [3f + i - 1],
    // cl - ch, and the row constant K + 1
    int cl[SD > 0 ? 3 * SD : 1];
    int ch[SD > 0 ? 3 * SD : 1];
    int nd[SD > 0 ? 3 * SD : 1];
    u64 k1[SD > 0 ? SD : 1];
    u32 ps[(NFUN > 0 && K == 4 && PsLimbs<F>::N > 0) ? NFUN * PsLimbs<F>::N : 1];  // P89, P64
    u32 c2p31, c4;                    // 2^31 and 4, as run-time operands
};

// Coefficient a_i of function f.  Generic kernels read the shared-memory copy
// (k runtime); specialized kernels index the parameter struct directly, so
// after unrolling each access is a constant-bank operand.
template <class F, int NFUN, int K>
__device__ __forceinline__ typename FieldOps<F>::val_t coef_at(const ParamCoef<F, NFUN, K>& pc,
                                                               const u64* scoef, bool generic,
                                                               int k, int f, int i) {
    typedef typename FieldOps<F>::val_t val_t;
    constexpr int W = FieldOps<F>::WORDS;
    if (generic) {
        const u64* w = scoef + ((size_t)f * k + i) * W;
        if (W == 1) return (val_t)w[0];
        return (val_t)(((u128)w[1] << 64) | w[0]);
    }
    const int idx = f * K + i;
    if (W == 1) return (val_t)pc.w[idx];
    return (val_t)(((u128)pc.w[2 * idx + 1] << 64) | pc.w[2 * idx]);
}

// ------------------------------------------------------------ key loading
//
// load4: 4 consecutive keys and weights starting at index j (j % 4 == 0).
// Returns how many are in range; out-of-range keys read as 0 with weight 0.
template <class F>
struct KeyIO;

template <>
struct KeyIO<msf::P61> {
    __device__ static __forceinline__ void load(const void* keys, u64 j, u64 n, bool vec,
                                                u64 (&x)[4]) {
        const u64* k = (const u64*)keys + j;
        if (vec && j + 3 < n) {
            const ulonglong2 a = __ldcs((const ulonglong2*)k);
            const ulonglong2 b = __ldcs((const ulonglong2*)k + 1);
            x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = (j + q < n) ? __ldcs(k + q) : 0ull;
        }
    }
};
template <>
struct KeyIO<msf::P64> : KeyIO<msf::P61> {};

template <>
struct KeyIO<msf::P31> {
    __device__ static __forceinline__ void load(const void* keys, u64 j, u64 n, bool vec,
                                                u32 (&x)[4]) {
        const u32* k = (const u32*)keys + j;
        if (vec && j + 3 < n) {
            const uint4 a = __ldcs((const uint4*)k);
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = (j + q < n) ? __ldcs(k + q) : 0u;
        }
    }
};

template <>
struct KeyIO<msf::P89> {
    __device__ static __forceinline__ void load(const void* keys, u64 j, u64 n, bool vec,
                                                u128x (&x)[4]) {
        const ulonglong2* k = (const ulonglong2*)keys + j;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ulonglong2 v = make_ulonglong2(0ull, 0ull);
            if (j + q < n) v = __ldcs(k + q);  // 16-byte keys: always one vector load
            x[q].lo = v.x;
            x[q].hi = v.y;
        }
        (void)vec;
    }
};

__device__ __forceinline__ void load_weights4(const int32_t* w, u64 j, u64 n, bool vec,
                                              int (&wt)[4]) {
    if (w == nullptr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) wt[q] = (j + q < n) ? 1 : 0;
        return;
    }
    if (vec && j + 3 < n) {
        const int4 a = __ldcs((const int4*)(w + j));
        wt[0] = a.x; wt[1] = a.y; wt[2] = a.z; wt[3] = a.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) wt[q] = (j + q < n) ? __ldcs(w + q + j) : 0;
    }
}

// ------------------------------------------------------------ warp matching

// Mask of the lanes of this (converged) warp that hold the same key.
__device__ __forceinline__ u32 match_key(u64 k) { return __match_any_sync(0xffffffffu, k); }
__device__ __forceinline__ u32 match_key(u32 k) { return __match_any_sync(0xffffffffu, k); }
__device__ __forceinline__ u32 match_key(const u128x& k) {
    // equal keys have equal limbs: intersect the two limb matches
    return __match_any_sync(0xffffffffu, k.lo) & __match_any_sync(0xffffffffu, k.hi);
}

// ------------------------------------------------------------ de-duplication
//
// Unit weights, global placement, one-word keys.  A Count Sketch is linear in
// the stream (Sec. 1.3), so c occurrences of key x add exactly what one update
// of x with weight c adds.  Each block keeps a direct-mapped table in shared
// memory, slot i holding a key (or DEDUP_EMPTY) and how often the block has
// seen it: a key that owns its slot, or claims an empty one, is only counted,
// and is hashed once, with its count, when the block has finished its share of
// the stream.  The other keys go to their warp's queue in shared memory and
// are hashed 128 at a time (four per lane), so the lanes of a warp hash only
// keys the table did not absorb.
constexpr u64 DEDUP_EMPTY = ~0ull;

template <class K>
struct DedupKey {
    static constexpr bool OK = false;
};
template <>
struct DedupKey<u64> {
    static constexpr bool OK = true;
};
template <>
struct DedupKey<u32> {
    static constexpr bool OK = true;
};

// Counts c occurrences of `key` in the table; false when the key's slot holds
// another key (or the key is DEDUP_EMPTY itself, which never enters the table).
__device__ __forceinline__ bool dedup_count(u64* tk, int* tc, int log2slots, u64 key, int c) {
    if (key == DEDUP_EMPTY) return false;
    const u32 slot = (u32)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2slots));
    u64 cur = tk[slot];
    if (cur == DEDUP_EMPTY) {
        cur = atomicCAS((unsigned long long*)&tk[slot], DEDUP_EMPTY, key);
        if (cur == DEDUP_EMPTY) cur = key;  // claimed by this thread
    }
    if (cur != key) return false;
    atomicAdd(&tc[slot], c);
    return true;
}

// Second-level table in global memory (L2-resident), two-way: a key's place is
// the aligned pair of slots at `base` (the slot hash with its low bit
// cleared).  gtable_count2 counts c occurrences of `key` when either slot holds
// it or one was free (claimed here, the pair's first slot first); false
// otherwise.  cur0, cur1 are the pair's keys as loaded before by one 16-byte
// load (so that a warp's loads overlap).  Should a key ever hold both slots,
// each count is still hashed with its key, so the result stays exact.
__device__ __forceinline__ u32 gtable_slot(u64 key, int glog2) {
    return (u32)((key * 0xD6E8FEB86659FD93ull) >> (64 - glog2));
}

__device__ __forceinline__ bool gtable_count2(unsigned long long* gk, int* gc, u32 base, u64 key,
                                              u64 cur0, u64 cur1, int c) {
    if (key == DEDUP_EMPTY) return false;
    if (cur0 == key) {
        atomicAdd(gc + base, c);
        return true;
    }
    if (cur1 == key) {
        atomicAdd(gc + base + 1, c);
        return true;
    }
    if (cur0 == DEDUP_EMPTY) {
        cur0 = atomicCAS(gk + base, DEDUP_EMPTY, (unsigned long long)key);
        if (cur0 == DEDUP_EMPTY || cur0 == key) {
            atomicAdd(gc + base, c);
            return true;
        }
    }
    if (cur1 == DEDUP_EMPTY) {
        cur1 = atomicCAS(gk + base + 1, DEDUP_EMPTY, (unsigned long long)key);
        if (cur1 == DEDUP_EMPTY || cur1 == key) {
            atomicAdd(gc + base + 1, c);
            return true;
        }
    }
    return false;
}

// ------------------------------------------------------------ cluster helpers

__device__ __forceinline__ u32 cluster_rank() {
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Adds v to the 32-bit counter at shared address `laddr` of block `rank` of
// this cluster.
__device__ __forceinline__ void dsmem_add(u32 laddr, u32 rank, int v) {
    u32 raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
    asm volatile("red.relaxed.cluster.shared::cluster.add.u32 [%0], %1;" ::"r"(raddr), "r"(v)
                 : "memory");
}

__device__ __forceinline__ void global_add64(long long* p, long long v) {
    atomicAdd((unsigned long long*)p, (unsigned long long)v);
}

// ------------------------------------------------------------ the kernel

// One counter update: C[row][bucket] += (sign ? -w : w).  For PLACE_GLOBAL,
// `tile` is this block's int32 replica of the counters in global memory (or
// NULL: int64 atomics on the counters themselves).
template <int PLACE>
__device__ __forceinline__ void apply_update(int* tile, u32 tile_saddr, long long* counters,
                                             int row, u32 bucket, u32 sign, int w, bool big,
                                             u32 m, int log2m, int lcs) {
    if (big || (PLACE == PLACE_GLOBAL && tile == nullptr)) {
        const long long d = sign ? -(long long)w : (long long)w;
        global_add64(counters + (((u64)row) << log2m) + bucket, d);
        return;
    }
    const int d = sign ? -w : w;
    if (PLACE == PLACE_GLOBAL) {
        atomicAdd(tile + (row << log2m) + bucket, d);  // red.global.add.s32 on the replica
    } else if (PLACE == PLACE_SMEM) {
        atomicAdd(tile + (row << log2m) + bucket, d);
    } else {  // PLACE_DSMEM: owner block = high bits of the bucket
        const int lshift = log2m - lcs;
        const u32 owner = bucket >> lshift;
        const u32 local = ((u32)row << lshift) + (bucket & ((1u << lshift) - 1u));
        dsmem_add(tile_saddr + local * 4u, owner, d);
    }
}

// Counter update on the unchecked path: |w| is within the tile's safe range.
// A zero delta is still added to shared memory (cheaper than a test); the
// global placements skip it.
template <int PLACE>
__device__ __forceinline__ void apply_fast(int* tile, u32 tile_saddr, long long* counters, int row,
                                           u32 bucket, int d, int log2m, int lcs) {
    if (PLACE == PLACE_SMEM) {
        asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(tile_saddr + ((((u32)row << log2m) + bucket) << 2)),
                     "r"(d)
                     : "memory");
    } else if (PLACE == PLACE_DSMEM) {
        const int lshift = log2m - lcs;
        const u32 owner = bucket >> lshift;
        const u32 local = ((u32)row << lshift) + (bucket & ((1u << lshift) - 1u));
        dsmem_add(tile_saddr + local * 4u, owner, d);
    } else if (d != 0) {
        if (tile)
            atomicAdd(tile + (row << log2m) + bucket, d);
        else
            global_add64(counters + (((u64)row) << log2m) + bucket, (long long)d);
    }
}

// Bucket and sign bit of row r for p = 2^61-1, k = 4 (signed-digit power sum,
// row_sd): two-for-one (both from one polynomial) or two polynomials (the sign
// from the second one's bit 60).
template <int NF, bool ANY = false, class PC>
__device__ __forceinline__ void p61_row_bs(const msf::P61::Pow3& xp, const PC& pc, int r, u32 mask,
                                           u32 arb_r, u32& bucket, u32& sign) {
    typedef msf::P61 F;
    const int fb = r * NF;
    u32 ylo, yhi;
    F::row_sd(xp, pc.cl + 3 * fb, pc.ch + 3 * fb, pc.nd + 3 * fb, pc.k1[fb], pc.c2p31, ylo, yhi);
    if (ANY) {  // Algorithm Mersenne-arb-r on the canonical value
        u32 a;
        F::arb_split(F::canon_sd(ylo, yhi), arb_r, bucket, a);
        sign = a ^ 1u;  // s = 2a - 1: subtract when a = 0
    } else {
        F::bucket_sign_sd(ylo, yhi, mask, bucket, sign);
    }
    if (NF == 2) {
        const int fs = fb + 1;
        u32 unused;
        F::row_sd(xp, pc.cl + 3 * fs, pc.ch + 3 * fs, pc.nd + 3 * fs, pc.k1[fs], pc.c2p31, ylo,
                  yhi);
        F::bucket_sign_sd(ylo, yhi, mask, unused, sign);
    }
}

// Bucket and sign bit of row r for p = 2^31-1, 2^89-1, 2^64-59 and k = 4 (power
// sum of the prime's field policy), two-for-one or two polynomials.
template <class F, int NF, class PC>
__device__ __forceinline__ void ps_row_bs(const typename F::Pow3& xp, const PC& pc, int r, u32 mask,
                                          u32& bucket, u32& sign) {
    const int fb = r * NF;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const int f = fb + j;
        u32 b, s;
        if constexpr (std::is_same<F, msf::P31>::value) {
            F::row_bs(xp, (u32)pc.w[f * 4], (u32)pc.w[f * 4 + 1], (u32)pc.w[f * 4 + 2],
                      (u32)pc.w[f * 4 + 3], mask, b, s);
        } else {
            constexpr int N = PsLimbs<F>::N;
            u32 c[N];
#pragma unroll
            for (int i = 0; i < N; ++i) c[i] = pc.ps[f * N + i];
            if constexpr (std::is_same<F, msf::P64>::value)
                F::row_bs(xp, pc.w[f * 4], c, mask, b, s);
            else
                F::row_bs(xp, c, mask, b, s);
        }
        if (j == 0) bucket = b;
        sign = s;  // two polynomials: the second one's bit b-1
    }
}

// One key whose weight could overflow an int32 tile counter (|w| > w_safe):
// every row is hashed by Horner from the device copy of the coefficients and
// added to the int64 counters.  Rolled loops keep this rare path small.
template <class F, int NF>
__device__ __forceinline__ void update_big_key(const typename FieldOps<F>::Prep& xq, int w,
                                               const u64* coef, int t, int k, int log2m,
                                               u32 arb_r, long long* counters) {
    typedef FieldOps<F> Ops;
    typedef typename Ops::val_t val_t;
    constexpr int W = Ops::WORDS;
    const u32 mask = (1u << log2m) - 1u;
#pragma unroll 1
    for (int r = 0; r < t; ++r) {
        const u64* cb = coef + (size_t)r * NF * k * W;
        val_t y = Ops::from_words(cb + (size_t)(k - 1) * W);
#pragma unroll 1
        for (int i = k - 2; i >= 0; --i) y = Ops::mul_add(y, xq, Ops::from_words(cb + (size_t)i * W));
        const val_t h = Ops::canon(y);
        val_t g = h;
        if (NF == 2) {
            const u64* cs = cb + (size_t)k * W;
            val_t z = Ops::from_words(cs + (size_t)(k - 1) * W);
#pragma unroll 1
            for (int i = k - 2; i >= 0; --i) z = Ops::mul_add(z, xq, Ops::from_words(cs + (size_t)i * W));
            g = Ops::canon(z);
        }
        u32 bucket, sb;
        split_row<F, NF>(h, g, mask, arb_r, bucket, sb);
        global_add64(counters + ((u64)r << log2m) + bucket, sb ? -(long long)w : (long long)w);
    }
}

// T, K > 0: compile-time rows and degree with ParamCoef; T = K = 0: runtime t
// and k with coefficients staged from coef_dev into shared memory.
// Two-for-one kernels are capped at 64 registers (two 512-thread blocks per SM);
// two-polynomial kernels keep twice the key state live and get 128, except for
// 2^61-1 in global placement, where the kernel waits on memory and two blocks
// per SM at 64 registers were 15% faster on the 2^28-key Zipf sketch (2.90 vs
// 3.41 ms); the wider primes' rows would spill at 64.
template <class F, int T, int K, int MODE, int PLACE, int STRAT>
__global__ void __launch_bounds__(512, (MODE == CS_TWO_POLY &&
                                        !(PLACE == PLACE_GLOBAL && std::is_same<F, msf::P61>::value))
                                           ? 1
                                           : 2)
k_cs_update(const UpdateArgs a, const ParamCoef<F, (MODE == CS_TWO_POLY ? 2 : 1) * T, K> pc) {
    typedef FieldOps<F> Ops;
    typedef typename Ops::val_t val_t;
    typedef typename Ops::Prep Prep;
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    constexpr bool GENERIC = (T == 0);
    constexpr int W = Ops::WORDS;

    extern __shared__ __align__(16) unsigned char smem[];
    const int t = GENERIC ? a.t : T;
    const int k = GENERIC ? a.k : K;
    const int log2m = a.log2m;
    const u32 m = 1u << log2m;
    const u32 mask = m - 1u;
    const int lcs = (PLACE == PLACE_DSMEM) ? a.cluster_log2 : 0;
    const u32 mloc = m >> lcs;

    // PLACE_GLOBAL: `tile` is this block's replica in global memory (or NULL)
    int* tile = (PLACE == PLACE_GLOBAL)
                    ? (a.replicas ? a.replicas + (size_t)(blockIdx.x & a.replica_mask) * ((u32)t << log2m)
                                  : nullptr)
                    : reinterpret_cast<int*>(smem);
    const u32 tile_cells = (PLACE == PLACE_GLOBAL) ? 0u : (u32)t * mloc;
    u64* scoef = reinterpret_cast<u64*>(smem + (size_t)tile_cells * 4u);
    // PLACE_GLOBAL with unit weights: the de-duplication table (12 bytes a slot)
    // and the warps' queues (12 bytes an entry) after the coefficients
    constexpr bool DEDUP_OK = PLACE == PLACE_GLOBAL && DedupKey<typename Ops::key_t>::OK;
    const int dd_log2 = (DEDUP_OK && a.weights == nullptr) ? a.dedup_log2 : 0;
    const u32 dd_slots = dd_log2 ? (1u << dd_log2) : 0u;
    u64* tk = reinterpret_cast<u64*>(
        smem + (((size_t)tile_cells * 4u + (GENERIC ? (size_t)t * NF * k * W * 8 : 0) + 15) & ~(size_t)15));
    int* tc = reinterpret_cast<int*>(tk + dd_slots);
    u64* qk = reinterpret_cast<u64*>(tc + dd_slots) + (size_t)(threadIdx.x >> 5) * DEDUP_QCAP;
    int* qc = reinterpret_cast<int*>(reinterpret_cast<u64*>(tc + dd_slots) +
                                     (size_t)(blockDim.x >> 5) * DEDUP_QCAP) +
              (threadIdx.x >> 5) * DEDUP_QCAP;
    for (u32 i = threadIdx.x; i < dd_slots; i += blockDim.x) {
        tk[i] = DEDUP_EMPTY;
        tc[i] = 0;
    }
    const u32 tile_saddr = (PLACE == PLACE_GLOBAL) ? 0u : (u32)__cvta_generic_to_shared(tile);

    if (PLACE != PLACE_GLOBAL)
        for (u32 i = threadIdx.x; i < tile_cells; i += blockDim.x) tile[i] = 0;
    if (GENERIC) {
        const int nw = t * NF * k * W;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) scoef[i] = a.coef_dev[i];
    }
    __syncthreads();
    if (PLACE == PLACE_DSMEM) cluster_sync_all();

    // coefficient a_i of function f (row r: bucket f = r*NF, sign f = r*NF+1)
#define MSK_COEF(f, i) coef_at<F, NF * T, K>(pc, scoef, GENERIC, k, (f), (i))

    const u64 n = a.n;
    const bool vec = a.vec_ok != 0;
    const u32 w_safe = a.w_safe;
    const bool unit_safe = a.weights == nullptr && w_safe >= 1u;  // every weight is 0 or 1
    const u32 row_bytes = m << 2;  // PLACE_SMEM: one row of the int32 tile
    const u64 stride = (u64)gridDim.x * blockDim.x * 4ull;
    const u32 lane = threadIdx.x & 31u;
    const u32 lanes_below = (1u << lane) - 1u;
    int drain = -1;  // de-duplication: -1 while streaming, then the batch being drained
    // De-duplication state of this warp (warp-uniform), packed in one word:
    // bits 0..8 the queue length, 9..14 chunks seen (up to 32), 15..26 keys the
    // table missed in chunks 16..31 (counting from 0), bit 31 set while the
    // table is in use.  It stays in use if it absorbed at least 1/8 of those
    // chunks' keys (a stream without repeats turns it off once it has filled).
    u32 dd = dd_log2 != 0 ? 0x80000000u : 0u;
    // The loop runs on the block's first key index, so every warp of a block
    // takes the same number of iterations (warps and lanes past the end load
    // weight-0 keys): warp-wide matching relies on it, and so does the drain of
    // the de-duplication table, which starts with a block barrier.
    for (u64 jb = (u64)blockIdx.x * blockDim.x * 4ull;;) {
        typename Ops::key_t key[4];
        int wt[4];
        if (drain < 0) {
            if (jb >= n) {
                if (!DEDUP_OK || dd_log2 == 0) break;
                drain = 0;
                __syncthreads();  // every warp is done with the table
                continue;
            }
            const u64 j = jb + (u64)threadIdx.x * 4ull;
            jb += stride;
            KeyIO<F>::load(a.keys, j, n, vec, key);
            load_weights4(a.weights, j, n, vec, wt);
            if (PLACE == PLACE_GLOBAL && a.aggregate == 1 && a.weights == nullptr) {
                // Unit weights: lanes of this warp holding the same key would add
                // to the same t counters.  The lowest such lane takes the group's
                // count; the others keep weight 0.
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u32 valid = __ballot_sync(0xffffffffu, wt[q] != 0);
                    u32 grp = match_key(key[q]) & valid;
                    if (wt[q] != 0) wt[q] = ((grp & lanes_below) == 0u) ? __popc(grp) : 0;
                }
            }
            if constexpr (DEDUP_OK) {
                if (dd >> 31) {
                    // the table counts what it can; the rest waits in the queue
                    // until 128 keys (four a lane) are there to hash
                    const u32 qn = dd & 0x1FFu;
                    u32 missed = 0;
                    bool miss[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        miss[q] = wt[q] != 0 && !dedup_count(tk, tc, dd_log2, (u64)key[q], wt[q]);
                    if (a.glog2) {
                        // the block's misses try the second-level table (the four
                        // slot-pair loads of a lane are in flight together)
                        u32 gs[4];
                        ulonglong2 gcur[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            gs[q] = gtable_slot((u64)key[q], a.glog2) & ~1u;
                            gcur[q] = miss[q] ? __ldcg(reinterpret_cast<const ulonglong2*>(a.gkeys + gs[q]))
                                              : make_ulonglong2(DEDUP_EMPTY, DEDUP_EMPTY);
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (miss[q] && gtable_count2(a.gkeys, a.gcounts, gs[q], (u64)key[q], gcur[q].x,
                                                         gcur[q].y, wt[q]))
                                miss[q] = false;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const u32 mb = __ballot_sync(0xffffffffu, miss[q]);
                        if (miss[q]) {
                            const u32 pos = qn + missed + __popc(mb & lanes_below);
                            qk[pos] = (u64)key[q];
                            qc[pos] = wt[q];
                        }
                        missed += __popc(mb);
                    }
                    dd += missed;  // queue length
                    const u32 chunk = (dd >> 9) & 0x3Fu;
                    if (chunk < 32u) {
                        dd += 1u << 9;
                        if (chunk >= 16u) dd += missed << 15;
                        if (chunk == 31u && ((dd >> 15) & 0xFFFu) > 16u * 128u * 7u / 8u) dd &= 0x7FFFFFFFu;
                    }
                    if ((dd & 0x1FFu) < 128u) continue;
                    __syncwarp();
                    dd -= 128u;
                    const u32 top = dd & 0x1FFu;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        key[q] = (typename Ops::key_t)qk[top + lane + 32u * q];
                        wt[q] = qc[top + lane + 32u * q];
                    }
                    __syncwarp();
                }
            }
        } else if constexpr (DEDUP_OK) {
            // batch 0: what is left in this warp's queue; then the table, four
            // slots a thread per batch
            if (drain == 0) {
                const u32 qn = dd & 0x1FFu;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u32 e = lane + 32u * q;
                    key[q] = (typename Ops::key_t)(e < qn ? qk[e] : 0ull);
                    wt[q] = e < qn ? qc[e] : 0;
                }
            } else {
                const u32 base = (u32)(drain - 1) * blockDim.x * 4u;
                if (base >= dd_slots) break;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u32 sl = base + threadIdx.x + blockDim.x * (u32)q;
                    const u64 kw = sl < dd_slots ? tk[sl] : DEDUP_EMPTY;
                    key[q] = (typename Ops::key_t)(kw == DEDUP_EMPTY ? 0ull : kw);
                    wt[q] = kw == DEDUP_EMPTY ? 0 : tc[sl];
                }
            }
            ++drain;
        } else {
            break;
        }
        if (a.hashed) {  // measurement: entries about to be hashed with a non-zero count
            u32 c = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) c += __popc(__ballot_sync(0xffffffffu, wt[q] != 0));
            if (lane == 0 && c) atomicAdd(a.hashed, (unsigned long long)c);
        }
        bool big[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const u32 aw = wt[q] < 0 ? 0u - (u32)wt[q] : (u32)wt[q];
            big[q] = !unit_safe && aw > w_safe;
        }

        if constexpr (!GENERIC && STRAT >= STRAT_POWER_SUM && std::is_same<F, msf::P61>::value &&
                      K == 4) {
            // Keys whose weight could overflow an int32 tile counter (rare)
            // go straight to the int64 counters; the hot loops below see
            // them with weight 0.
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (big[q]) {
                    update_big_key<F, NF>(Ops::prep(key[q]), wt[q], a.coef_dev, t, k, log2m,
                                          a.arb_r, a.counters);
                    wt[q] = 0;
                }
            }
            if constexpr (PLACE == PLACE_GLOBAL && NF == 2) {
                // two polynomials: one key's powers live at a time (a rolled
                // loop over the four keys, whose registers rotate), so the
                // kernel fits 64 registers without spilling (6% faster on the
                // 2^28-key Zipf sketch than two keys at a time)
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {
                    msf::P61::Pow3 xs;
                    msf::P61::powers3(key[0], xs);
                    const int ws = wt[0];
                    key[0] = key[1];
                    key[1] = key[2];
                    key[2] = key[3];
                    wt[0] = wt[1];
                    wt[1] = wt[2];
                    wt[2] = wt[3];
#pragma unroll
                    for (int r = 0; r < T; ++r) {
                        u32 bucket, sb;
                        p61_row_bs<NF, STRAT == STRAT_POWER_SUM_ANY_R>(xs, pc, r, mask, a.arb_r,
                                                                       bucket, sb);
                        apply_fast<PLACE>(tile, tile_saddr, a.counters, r, bucket, sb ? -ws : ws,
                                          log2m, lcs);
                    }
                }
            } else if constexpr (PLACE == PLACE_GLOBAL) {
                // two keys' powers live at a time (a rolled loop over the two
                // pairs, whose registers rotate; rows outer within a pair): with
                // all four keys' powers live the de-duplicating path spilled
                // under the 64-register cap
#pragma unroll 1
                for (int qq = 0; qq < 2; ++qq) {
                    msf::P61::Pow3 xp[2];
                    msf::P61::powers3(key[0], xp[0]);
                    msf::P61::powers3(key[1], xp[1]);
                    const int w0 = wt[0], w1 = wt[1];
                    key[0] = key[2];
                    key[1] = key[3];
                    wt[0] = wt[2];
                    wt[1] = wt[3];
#pragma unroll
                    for (int r = 0; r < T; ++r) {
                        u32 bucket, sb;
                        p61_row_bs<NF, STRAT == STRAT_POWER_SUM_ANY_R>(xp[0], pc, r, mask, a.arb_r,
                                                                       bucket, sb);
                        apply_fast<PLACE>(tile, tile_saddr, a.counters, r, bucket, sb ? -w0 : w0,
                                          log2m, lcs);
                        p61_row_bs<NF, STRAT == STRAT_POWER_SUM_ANY_R>(xp[1], pc, r, mask, a.arb_r,
                                                                       bucket, sb);
                        apply_fast<PLACE>(tile, tile_saddr, a.counters, r, bucket, sb ? -w1 : w1,
                                          log2m, lcs);
                    }
                }
            } else {
                // keys outer: one key's powers live at a time
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    msf::P61::Pow3 xp;
                    msf::P61::powers3(key[q], xp);
                    const int w = wt[q], w2 = -2 * w;
                    u32 rbase = tile_saddr;  // shared address of row r's counters
#pragma unroll
                    for (int r = 0; r < T; ++r) {
                        u32 bucket, sb;
                        p61_row_bs<NF, STRAT == STRAT_POWER_SUM_ANY_R>(xp, pc, r, mask, a.arb_r,
                                                                       bucket, sb);
                        const int d = (int)sb * w2 + w;
                        if (PLACE == PLACE_SMEM) {
                            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(rbase + (bucket << 2)), "r"(d)
                                         : "memory");
                            rbase += row_bytes;
                        } else {
                            apply_fast<PLACE>(tile, tile_saddr, a.counters, r, bucket, d, log2m, lcs);
                        }
                    }
                }
            }
        } else if constexpr (!GENERIC && STRAT >= STRAT_POWER_SUM && K == 4 &&
                             !std::is_same<F, msf::P61>::value) {
            // the other primes' power sum: keys outer, one key's powers live
            // at a time, in every placement
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (big[q]) {
                    update_big_key<F, NF>(Ops::prep(key[q]), wt[q], a.coef_dev, t, k, log2m,
                                          a.arb_r, a.counters);
                    wt[q] = 0;
                }
            }
            // A rolled loop over the four keys (the key registers rotate, so no
            // array is indexed at run time): unrolled, the compiler interleaves
            // the keys and runs out of registers.
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                typename F::Pow3 xp;
                F::powers3(key[0], xp);
                const int w = wt[0], w2 = -2 * w;
                key[0] = key[1];
                key[1] = key[2];
                key[2] = key[3];
                wt[0] = wt[1];
                wt[1] = wt[2];
                wt[2] = wt[3];
                u32 rbase = tile_saddr;  // shared address of row r's counters
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    u32 bucket, sb;
                    ps_row_bs<F, NF>(xp, pc, r, mask, bucket, sb);
                    const int d = (int)sb * w2 + w;
                    if (PLACE == PLACE_SMEM) {
                        asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(rbase + (bucket << 2)), "r"(d)
                                     : "memory");
                        rbase += row_bytes;
                    } else {
                        apply_fast<PLACE>(tile, tile_saddr, a.counters, r, bucket, d, log2m, lcs);
                    }
                }
            }
        } else {
            Prep xp[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) xp[q] = Ops::prep(key[q]);
#pragma unroll(GENERIC ? 1 : (T > 0 ? T : 1))
            for (int r = 0; r < t; ++r) {
                const int fb = r * NF;
                val_t h[4], g[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    val_t y = MSK_COEF(fb, k - 1);
#pragma unroll(GENERIC ? 1 : (K > 1 ? K - 1 : 1))
                    for (int i = k - 2; i >= 0; --i) y = Ops::mul_add(y, xp[q], MSK_COEF(fb, i));
                    h[q] = Ops::canon(y);
                    if (MODE == CS_TWO_POLY) {
                        val_t z = MSK_COEF(fb + 1, k - 1);
#pragma unroll(GENERIC ? 1 : (K > 1 ? K - 1 : 1))
                        for (int i = k - 2; i >= 0; --i) z = Ops::mul_add(z, xp[q], MSK_COEF(fb + 1, i));
                        g[q] = Ops::canon(z);
                    } else {
                        g[q] = h[q];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (wt[q] != 0) {
                        u32 bucket, sb;
                        split_row<F, NF>(h[q], g[q], mask, a.arb_r, bucket, sb);
                        apply_update<PLACE>(tile, tile_saddr, a.counters, r, bucket, sb, wt[q],
                                            big[q], m, log2m, lcs);
                    }
                }
            }
        }
    }

    if (PLACE == PLACE_GLOBAL) return;
#undef MSK_COEF
    if (PLACE == PLACE_DSMEM)
        cluster_sync_all();  // every remote add into this block's slice has landed
    else
        __syncthreads();
    const u32 rank = (PLACE == PLACE_DSMEM) ? cluster_rank() : 0u;
    const int lshift = log2m - lcs;
    for (u32 i = threadIdx.x; i < tile_cells; i += blockDim.x) {
        const int v = tile[i];
        if (v != 0) {
            const u32 row = i >> lshift;
            const u32 b = (rank << lshift) + (i & (mloc - 1u));
            global_add64(a.counters + (((u64)row) << log2m) + b, (long long)v);
        }
    }
}

// ------------------------------------------------------------ second-level table drain
//
// After an update that used the second-level key table: every key the table
// holds is hashed once, with its count (Horner from the device copy of the
// coefficients, the sketch's split), into the int64 counters -- exact by the
// linearity of the Count Sketch (Sec. 1.3) -- and its slot is emptied for the
// next update.  With the statistics hook on, each drained key counts as one
// hashed entry.
template <class F, int NF>
__global__ void __launch_bounds__(256) k_gtable_drain(const UpdateArgs a) {
    typedef FieldOps<F> Ops;
    const u32 slots = 1u << a.glog2;
    const u32 lane = threadIdx.x & 31u;
    for (u32 i0 = blockIdx.x * blockDim.x; i0 < slots; i0 += gridDim.x * blockDim.x) {
        const u32 i = i0 + threadIdx.x;
        const u64 k = i < slots ? a.gkeys[i] : DEDUP_EMPTY;
        const bool held = k != DEDUP_EMPTY;
        if (a.hashed) {
            const u32 b = __ballot_sync(0xffffffffu, held);
            if (lane == 0 && b) atomicAdd(a.hashed, (unsigned long long)__popc(b));
        }
        if (!held) continue;
        const int c = a.gcounts[i];
        a.gkeys[i] = DEDUP_EMPTY;
        a.gcounts[i] = 0;
        const typename Ops::key_t key = (typename Ops::key_t)k;
        update_big_key<F, NF>(Ops::prep(key), c, a.coef_dev, a.t, a.k, a.log2m, a.arb_r,
                              a.counters);
    }
}

// The same drain for p = 2^61-1, k = 4 and compile-time t: each held key's
// rows by the signed-digit power sum (row_sd, x^2 and x^3 once per key) with
// the coefficients in the parameter space, as in the update kernels, so the
// drain waits on its slot loads and counter atomics only.
template <int T, int NF, bool ANY>
__global__ void __launch_bounds__(256) k_gtable_drain_sd(const UpdateArgs a,
                                                         const ParamCoef<msf::P61, NF * T, 4> pc) {
    const u32 slots = 1u << a.glog2;
    const u32 lane = threadIdx.x & 31u;
    const int log2m = a.log2m;
    const u32 mask = (1u << log2m) - 1u;
    for (u32 i0 = blockIdx.x * blockDim.x; i0 < slots; i0 += gridDim.x * blockDim.x) {
        const u32 i = i0 + threadIdx.x;
        const u64 k = i < slots ? a.gkeys[i] : DEDUP_EMPTY;
        const bool held = k != DEDUP_EMPTY;
        if (a.hashed) {
            const u32 b = __ballot_sync(0xffffffffu, held);
            if (lane == 0 && b) atomicAdd(a.hashed, (unsigned long long)__popc(b));
        }
        if (!held) continue;
        const int c = a.gcounts[i];
        a.gkeys[i] = DEDUP_EMPTY;
        a.gcounts[i] = 0;
        msf::P61::Pow3 xp;
        msf::P61::powers3(k, xp);
#pragma unroll
        for (int r = 0; r < T; ++r) {
            u32 bucket, sb;
            p61_row_bs<NF, ANY>(xp, pc, r, mask, a.arb_r, bucket, sb);
            global_add64(a.counters + ((u64)r << log2m) + bucket, sb ? -(long long)c : (long long)c);
        }
    }
}

// ------------------------------------------------------------ point queries
//
// The median of t = 5 or 7 estimates by a comparator network: Batcher's
// odd-even merge sort on 8 wires, the wires past t fixed at +infinity (their
// comparators drop out), pruned to the comparators the middle wire depends on,
// and where only one output of a comparator is used, only that min (lo, on
// the first wire) or max (hi, on the second).  A min/max network selects the
// middle value of every input iff it does so on every 0/1 input;
// tests/test_median_networks.py checks that on the networks as written here.
__device__ __forceinline__ void med_ce(long long& x, long long& y) {
    const long long a = x < y ? x : y;
    y = x < y ? y : x;
    x = a;
}
__device__ __forceinline__ void med_lo(long long& x, long long y) { x = x < y ? x : y; }
__device__ __forceinline__ void med_hi(long long x, long long& y) { y = x < y ? y : x; }

__device__ __forceinline__ long long median_of(long long (&e)[5]) {
    // median network, t = 5
    med_ce(e[0], e[1]); med_ce(e[2], e[3]); med_ce(e[0], e[2]); med_lo(e[1], e[3]);
    med_ce(e[1], e[2]); med_hi(e[0], e[4]); med_lo(e[2], e[4]); med_hi(e[1], e[2]);
    return e[2];
}

__device__ __forceinline__ long long median_of(long long (&e)[7]) {
    // median network, t = 7
    med_ce(e[0], e[1]); med_ce(e[2], e[3]); med_ce(e[4], e[5]); med_ce(e[0], e[2]);
    med_ce(e[1], e[3]); med_ce(e[4], e[6]); med_ce(e[1], e[2]); med_ce(e[5], e[6]);
    med_hi(e[0], e[4]); med_hi(e[1], e[5]); med_lo(e[2], e[6]); med_hi(e[2], e[4]);
    med_lo(e[3], e[5]); med_lo(e[3], e[4]);
    return e[3];
}
//
// Point queries for p = 2^61-1, k = 4 and compile-time t: the estimate of f_x
// is the median over the rows of s_r(x) C[r][i_r(x)] (Sec. 1.3).  Each key's
// rows by the update kernels' signed-digit power sum (x^2, x^3 once per key,
// the coefficients in the parameter space), the split of the sketch's mode
// (ANY: Algorithm Mersenne-arb-r, P61::arb_split_sd), the t estimates in
// registers, and their median by the network above.
template <int T, int NF, bool ANY>
__global__ void __launch_bounds__(256) k_cs_point_query_sd(const QueryArgs a,
                                                            const ParamCoef<msf::P61, NF * T, 4> pc) {
    typedef msf::P61 F;
    const int log2m = a.log2m;
    const u32 mask = (1u << log2m) - 1u;
    const u64* keys = reinterpret_cast<const u64*>(a.keys);
    for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < a.n;
         j += (u64)gridDim.x * blockDim.x) {
        F::Pow3 xp;
        F::powers3(__ldcs(keys + j), xp);
        long long est[T];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            u32 ylo, yhi;
            F::row_sd(xp, pc.cl + 3 * NF * r, pc.ch + 3 * NF * r, pc.nd + 3 * NF * r,
                      pc.k1[NF * r], pc.c2p31, ylo, yhi);
            u32 bucket, neg;
            if constexpr (ANY) {
                u32 keep;
                F::arb_split_sd(ylo, yhi, a.arb_r, bucket, keep);
                neg = keep ^ 1u;  // subtract when a = 0
            } else {
                bucket = ylo & mask;
                neg = (yhi >> 28) & 1u;  // bit 60 of the residue
            }
            if (NF == 2) {  // the sign from the second polynomial's bit 60
                F::row_sd(xp, pc.cl + 3 * (2 * r + 1), pc.ch + 3 * (2 * r + 1),
                          pc.nd + 3 * (2 * r + 1), pc.k1[2 * r + 1], pc.c2p31, ylo, yhi);
                neg = (yhi >> 28) & 1u;
            }
            const long long c = __ldg(a.counters + ((u64)r << log2m) + bucket);
            est[r] = neg ? -c : c;
        }
        a.out[j] = median_of(est);
    }
}

// ------------------------------------------------------------ lean tile kernel
//
// The hot configuration on its own: p = 2^61-1, k = 4 (signed-digit power
// sum, row_sd), compile-time t, one int32 counter tile per block in shared
// memory (t * 2^log2m cells), two-for-one or two polynomials, int32 weights or
// unit weights, log2m fixed at compile time (LOG2M > 0) or read at run time.
// A thread takes four consecutive keys (and weights) per grid-stride step --
// 16-byte loads when the stream is aligned and the group is whole, else
// element loads with weight 0 past the end -- and hashes them one after the
// other, each row ending in one shared atomic at tile + r * 4m + 4 * bucket.
// A key whose weight could overflow an int32 tile counter (|w| > w_safe) goes
// to the int64 counters through the cold Horner path.  The tile is added into
// the int64 counters at the end (tile cell r * 2^log2m + b is counter
// r * 2^log2m + b).  The t = 5 two-for-one kernels are capped at 42 registers
// (three 512-thread blocks per SM), the others at 64.  With unit weights the
// four keys go through a rolled loop (their registers rotate): unrolled, the
// compiler interleaves them and spills.  ANY: any number of buckets r
// (Algorithm Mersenne-arb-r, Sec. 3.3, P61::arb_split_sd) in rows 2^log2m >= r
// wide, the update subtracted when a = 0 (two polynomials: the sign is still
// bit 60 of the second one).
template <int T, int MODE, bool WEIGHTED, int LOG2M, bool ANY = false>
__global__ void __launch_bounds__(512, (MODE != CS_TWO_POLY && T == 5) ? 3 : 2)
k_cs_update_tile(const UpdateArgs a,
                 const ParamCoef<msf::P61, (MODE == CS_TWO_POLY ? 2 : 1) * T, 4> pc) {
    typedef msf::P61 F;
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    int* tile = reinterpret_cast<int*>(smem);
    const int log2m = LOG2M > 0 ? LOG2M : a.log2m;
    const u32 mask = (1u << log2m) - 1u;
    const u32 row_bytes = 4u << log2m;
    const u32 cells = (u32)T << log2m;
    for (u32 i = threadIdx.x; i < cells; i += blockDim.x) tile[i] = 0;
    __syncthreads();
    const u32 base = (u32)__cvta_generic_to_shared(tile);
    const u64 n = a.n;
    const u32 w_safe = a.w_safe;
    const bool vec = a.vec_ok != 0;
    const u64* keys = reinterpret_cast<const u64*>(a.keys);
    const u64 groups = (n + 3) / 4;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const u64 j = 4 * g;
        u64 key[4];
        int wt[4];
        if (vec && j + 3 < n) {
            const ulonglong2 k0 = __ldcs(reinterpret_cast<const ulonglong2*>(keys + j));
            const ulonglong2 k1 = __ldcs(reinterpret_cast<const ulonglong2*>(keys + j) + 1);
            key[0] = k0.x; key[1] = k0.y; key[2] = k1.x; key[3] = k1.y;
            if (WEIGHTED) {
                const int4 w4 = __ldcs(reinterpret_cast<const int4*>(a.weights + j));
                wt[0] = w4.x; wt[1] = w4.y; wt[2] = w4.z; wt[3] = w4.w;
            } else {
                wt[0] = wt[1] = wt[2] = wt[3] = 1;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // past the end: key 0 with weight 0 (adds nothing)
                const bool in = j + q < n;
                key[q] = in ? __ldcs(keys + j + q) : 0ull;
                wt[q] = in ? (WEIGHTED ? __ldcs(a.weights + j + q) : 1) : 0;
            }
        }
#pragma unroll(WEIGHTED ? 4 : 1)
        for (int q = 0; q < 4; ++q) {
            const u64 kq = key[0];
            const int w = wt[0];
            key[0] = key[1];
            key[1] = key[2];
            key[2] = key[3];
            wt[0] = wt[1];
            wt[1] = wt[2];
            wt[2] = wt[3];
            if (WEIGHTED && (u32)w + w_safe > 2u * w_safe) {  // |w| > w_safe (w_safe < 2^31)
                update_big_key<F, NF>(FieldOps<F>::prep(kq), w, a.coef_dev, T, 4, log2m,
                                      ANY ? a.arb_r : 0u, a.counters);
                continue;
            }
            F::Pow3 xp;
            F::powers3(kq, xp);
#pragma unroll
            for (int r = 0; r < T; ++r) {
                u32 ylo, yhi;
                F::row_sd(xp, pc.cl + 3 * NF * r, pc.ch + 3 * NF * r, pc.nd + 3 * NF * r,
                          pc.k1[NF * r], pc.c2p31, ylo, yhi);
                u32 bucket, keep = 0;
                if constexpr (ANY) {
                    F::arb_split_sd(ylo, yhi, a.arb_r, bucket, keep);  // add when a = 1
                } else {
                    bucket = ylo & mask;
                }
                if (NF == 2)  // the sign from the second polynomial's bit 60
                    F::row_sd(xp, pc.cl + 3 * (2 * r + 1), pc.ch + 3 * (2 * r + 1),
                              pc.nd + 3 * (2 * r + 1), pc.k1[2 * r + 1], pc.c2p31, ylo, yhi);
                int d;
                if (ANY && NF == 1)
                    d = keep ? w : -w;
                else
                    d = (yhi & 0x10000000u) ? -w : w;  // bit 60 of the residue
                asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(base + (u32)r * row_bytes + (bucket << 2)),
                             "r"(d)
                             : "memory");
            }
        }
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < cells; i += blockDim.x) {
        const int v = tile[i];
        if (v != 0) global_add64(a.counters + i, (long long)v);
    }
}

// The same lean kernel for p = 2^31-1, k = 4 (32-bit keys, four a thread by
// one 16-byte load; the prime's power-sum rows, row_bs, with the coefficients
// in the parameter space), power-of-two buckets.
template <int T, int MODE, bool WEIGHTED, int LOG2M>
__global__ void __launch_bounds__(512, (MODE != CS_TWO_POLY && T == 5) ? 3 : 2)
k_cs_update_tile31(const UpdateArgs a,
                   const ParamCoef<msf::P31, (MODE == CS_TWO_POLY ? 2 : 1) * T, 4> pc) {
    typedef msf::P31 F;
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    int* tile = reinterpret_cast<int*>(smem);
    const int log2m = LOG2M > 0 ? LOG2M : a.log2m;
    const u32 mask = (1u << log2m) - 1u;
    const u32 row_bytes = 4u << log2m;
    const u32 cells = (u32)T << log2m;
    for (u32 i = threadIdx.x; i < cells; i += blockDim.x) tile[i] = 0;
    __syncthreads();
    const u32 base = (u32)__cvta_generic_to_shared(tile);
    const u64 n = a.n;
    const u32 w_safe = a.w_safe;
    const bool vec = a.vec_ok != 0;
    const u32* keys = reinterpret_cast<const u32*>(a.keys);
    const u64 groups = (n + 3) / 4;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const u64 j = 4 * g;
        u32 key[4];
        int wt[4];
        if (vec && j + 3 < n) {
            const uint4 k4 = __ldcs(reinterpret_cast<const uint4*>(keys + j));
            key[0] = k4.x; key[1] = k4.y; key[2] = k4.z; key[3] = k4.w;
            if (WEIGHTED) {
                const int4 w4 = __ldcs(reinterpret_cast<const int4*>(a.weights + j));
                wt[0] = w4.x; wt[1] = w4.y; wt[2] = w4.z; wt[3] = w4.w;
            } else {
                wt[0] = wt[1] = wt[2] = wt[3] = 1;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // past the end: key 0 with weight 0 (adds nothing)
                const bool in = j + q < n;
                key[q] = in ? __ldcs(keys + j + q) : 0u;
                wt[q] = in ? (WEIGHTED ? __ldcs(a.weights + j + q) : 1) : 0;
            }
        }
#pragma unroll(WEIGHTED ? 4 : 1)
        for (int q = 0; q < 4; ++q) {
            const u32 kq = key[0];
            const int w = wt[0];
            key[0] = key[1];
            key[1] = key[2];
            key[2] = key[3];
            wt[0] = wt[1];
            wt[1] = wt[2];
            wt[2] = wt[3];
            if (WEIGHTED && (u32)w + w_safe > 2u * w_safe) {  // |w| > w_safe (w_safe < 2^31)
                update_big_key<F, NF>(FieldOps<F>::prep(kq), w, a.coef_dev, T, 4, log2m, 0u,
                                      a.counters);
                continue;
            }
            F::Pow3 xp;
            F::powers3(kq, xp);
#pragma unroll
            for (int r = 0; r < T; ++r) {
                u32 bucket, sb;
                ps_row_bs<F, NF>(xp, pc, r, mask, bucket, sb);
                const int d = sb ? -w : w;
                asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(base + (u32)r * row_bytes + (bucket << 2)),
                             "r"(d)
                             : "memory");
            }
        }
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < cells; i += blockDim.x) {
        const int v = tile[i];
        if (v != 0) global_add64(a.counters + i, (long long)v);
    }
}

// The lean kernel for the wider primes' power sum (p = 2^89-1 and 2^64-59,
// k = 4, power-of-two buckets): the keys of a four-key group through the
// prime's key loader, then one key at a time (a rolled loop, the registers
// rotating) through x^2, x^3 and the rows (ps_row_bs), the coefficients in the
// parameter space.
template <class F, int T, int MODE, bool WEIGHTED, int LOG2M>
__global__ void __launch_bounds__(512, 2)
k_cs_update_tile_ps(const UpdateArgs a, const ParamCoef<F, (MODE == CS_TWO_POLY ? 2 : 1) * T, 4> pc) {
    typedef FieldOps<F> Ops;
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    int* tile = reinterpret_cast<int*>(smem);
    const int log2m = LOG2M > 0 ? LOG2M : a.log2m;
    const u32 mask = (1u << log2m) - 1u;
    const u32 row_bytes = 4u << log2m;
    const u32 cells = (u32)T << log2m;
    for (u32 i = threadIdx.x; i < cells; i += blockDim.x) tile[i] = 0;
    __syncthreads();
    const u32 base = (u32)__cvta_generic_to_shared(tile);
    const u64 n = a.n;
    const u32 w_safe = a.w_safe;
    const bool vec = a.vec_ok != 0;
    const u64 groups = (n + 3) / 4;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const u64 j = 4 * g;
        typename Ops::key_t key[4];
        int wt[4];
        KeyIO<F>::load(a.keys, j, n, vec, key);
        load_weights4(WEIGHTED ? a.weights : nullptr, j, n, vec, wt);
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const typename Ops::key_t kq = key[0];
            const int w = wt[0];
            key[0] = key[1];
            key[1] = key[2];
            key[2] = key[3];
            wt[0] = wt[1];
            wt[1] = wt[2];
            wt[2] = wt[3];
            if (WEIGHTED && (u32)w + w_safe > 2u * w_safe) {  // |w| > w_safe (w_safe < 2^31)
                update_big_key<F, NF>(Ops::prep(kq), w, a.coef_dev, T, 4, log2m, 0u, a.counters);
                continue;
            }
            typename F::Pow3 xp;
            F::powers3(kq, xp);
#pragma unroll
            for (int r = 0; r < T; ++r) {
                u32 bucket, sb;
                ps_row_bs<F, NF>(xp, pc, r, mask, bucket, sb);
                const int d = sb ? -w : w;
                asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(base + (u32)r * row_bytes + (bucket << 2)),
                             "r"(d)
                             : "memory");
            }
        }
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < cells; i += blockDim.x) {
        const int v = tile[i];
        if (v != 0) global_add64(a.counters + i, (long long)v);
    }
}

}  // namespace msk
