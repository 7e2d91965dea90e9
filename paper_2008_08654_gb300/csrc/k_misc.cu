// F2 estimate, point query, hash evaluation, division/modulus, counter
// utilities and the integer-multiply throughput probe.
#include <cuda_runtime.h>
#include <stdint.h>

#include "k_update.cuh"
#include "ms_kernels.h"

namespace msk {

// ================================================================ F2 estimate
//
// Output of Algorithm count-sketch per row, X_r = sum_i C[r][i]^2, as an exact
// 128-bit sum (two 64-bit limbs with carry), then the median of the t rows.
// Small sketches (t * m <= F2_ONE_BLOCK_CELLS): one block, its warps split
// evenly over the rows.  Larger ones: t * splits blocks, block (row, split)
// sums one slice of one row and writes a partial; the last block to finish
// (atomic ticket) adds the partials, takes the median, writes the result and
// re-arms the ticket.

struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ void add128(U128& acc, u64 lo, u64 hi) {
    const u64 s = acc.lo + lo;
    acc.hi += hi + (s < lo ? 1ull : 0ull);
    acc.lo = s;
}

__device__ __forceinline__ bool less128(const U128& a, const U128& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

constexpr u32 F2_ONE_BLOCK_CELLS = 1u << 15;

// acc += sum of C[i]^2 over the counters this lane visits (i = begin, begin +
// step, ... < end), eight loads in flight before any of them is used
__device__ __forceinline__ void sumsq(U128& acc, const long long* c, u32 begin, u32 end, u32 step) {
    for (u32 i = begin; i < end; i += 8u * step) {
        long long v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const u32 j = i + (u32)u * step;
            v[u] = j < end ? __ldcg(c + j) : 0ll;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const u64 mag = v[u] < 0 ? 0ull - (u64)v[u] : (u64)v[u];
            add128(acc, mag * mag, __umul64hi(mag, mag));
        }
    }
}

__device__ __forceinline__ void warp_sum128(U128& acc) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const u64 lo = __shfl_down_sync(0xffffffffu, acc.lo, off);
        const u64 hi = __shfl_down_sync(0xffffffffu, acc.hi, off);
        add128(acc, lo, hi);
    }
}

// The median of the t row values in shared memory (t odd): thread r < t finds
// the rank of row r, ties broken by index, and the one of rank t/2 writes it.
// Also writes the row values when asked.  Called by every thread of a block.
__device__ __forceinline__ void median_rows(const U128* rows, int t, ms_u128* out, ms_u128* rows_out) {
    const int r = threadIdx.x;
    if (r < t) {
        const U128 x = rows[r];
        int rank = 0;
        for (int j = 0; j < t; ++j) {
            const U128 y = rows[j];
            rank += (less128(y, x) || (j < r && y.lo == x.lo && y.hi == x.hi)) ? 1 : 0;
        }
        if (rank == t / 2) {
            out->lo = x.lo;
            out->hi = x.hi;
        }
        if (rows_out) {
            rows_out[r].lo = x.lo;
            rows_out[r].hi = x.hi;
        }
    }
}

__global__ void __launch_bounds__(1024) k_cs_f2_one(const F2Args a) {
    __shared__ U128 warp_sums[32];
    __shared__ U128 rows[MAX_T];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpr = (int)(blockDim.x >> 5) / a.t;  // warps per row (>= 2: t <= 15)
    const int row = warp / wpr, sub = warp % wpr;
    U128 acc = {0ull, 0ull};
    if (row < a.t)
        sumsq(acc, a.counters + (u64)row * a.m, (u32)(sub * 32 + lane), a.m, (u32)wpr * 32u);
    warp_sum128(acc);
    if (lane == 0) warp_sums[warp] = acc;
    __syncthreads();
    if ((int)threadIdx.x < a.t) {
        U128 s = {0ull, 0ull};
        for (int q = 0; q < wpr; ++q) add128(s, warp_sums[threadIdx.x * wpr + q].lo,
                                             warp_sums[threadIdx.x * wpr + q].hi);
        rows[threadIdx.x] = s;
    }
    __syncthreads();
    median_rows(rows, a.t, a.out, a.rows);
}

__global__ void __launch_bounds__(1024) k_cs_f2(const F2Args a) {
    __shared__ U128 warp_sums[32];
    __shared__ U128 rows[MAX_T];
    __shared__ bool is_last;
    const int row = blockIdx.x / a.splits;
    const int split = blockIdx.x % a.splits;
    const u32 slice = a.m / (u32)a.splits;

    U128 acc = {0ull, 0ull};
    sumsq(acc, a.counters + (u64)row * a.m + (u64)split * slice, threadIdx.x, slice, blockDim.x);
    warp_sum128(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_sums[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        U128 s = {0ull, 0ull};
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) add128(s, warp_sums[w].lo, warp_sums[w].hi);
        a.partial[blockIdx.x].lo = s.lo;
        a.partial[blockIdx.x].hi = s.hi;
        __threadfence();
        const u32 prev = atomicAdd(a.ticket, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;

    // the last block: thread r adds row r's partials (loads from L2, where the
    // other blocks' fenced writes are)
    __threadfence();
    if ((int)threadIdx.x < a.t) {
        U128 s = {0ull, 0ull};
        const ms_u128* pr = a.partial + threadIdx.x * a.splits;
        for (int q = 0; q < a.splits; ++q) add128(s, __ldcg(&pr[q].lo), __ldcg(&pr[q].hi));
        rows[threadIdx.x] = s;
    }
    __syncthreads();
    median_rows(rows, a.t, a.out, a.rows);
    if (threadIdx.x == 0) *a.ticket = 0u;  // re-arm for the next launch on this scratch
}

cudaError_t launch_cs_f2(const F2Args& a, int threads, cudaStream_t stream) {
    if ((u64)a.t * a.m <= F2_ONE_BLOCK_CELLS)
        k_cs_f2_one<<<1, 1024, 0, stream>>>(a);
    else
        k_cs_f2<<<a.t * a.splits, threads, 0, stream>>>(a);
    return cudaGetLastError();
}

// ================================================================ update dispatch

cudaError_t launch_cs_update(int prime, const UpdateArgs& a, const u64* coef_host,
                             const LaunchCfg& cfg, cudaStream_t stream, int* specialized) {
    switch (prime) {
        case PRIME_31: return launch_update_p31(a, coef_host, cfg, stream, specialized, nullptr);
        case PRIME_61: return launch_update_p61(a, coef_host, cfg, stream, specialized, nullptr);
        case PRIME_89: return launch_update_p89(a, coef_host, cfg, stream, specialized, nullptr);
        default: return launch_update_p64(a, coef_host, cfg, stream, specialized, nullptr);
    }
}

cudaError_t launch_gtable_drain(int prime, const UpdateArgs& a, const u64* coef_host,
                                cudaStream_t stream) {
    switch (prime) {
        case PRIME_31: return launch_gtable_drain_p31(a, coef_host, stream);
        case PRIME_61: return launch_gtable_drain_p61(a, coef_host, stream);
        case PRIME_89: return launch_gtable_drain_p89(a, coef_host, stream);
        default: return launch_gtable_drain_p64(a, coef_host, stream);
    }
}

cudaError_t query_cs_update_occupancy(int prime, const UpdateArgs& a, const u64* coef_host,
                                      const LaunchCfg& cfg, int* result) {
    *result = 0;
    switch (prime) {
        case PRIME_31: return launch_update_p31(a, coef_host, cfg, nullptr, nullptr, result);
        case PRIME_61: return launch_update_p61(a, coef_host, cfg, nullptr, nullptr, result);
        case PRIME_89: return launch_update_p89(a, coef_host, cfg, nullptr, nullptr, result);
        default: return launch_update_p64(a, coef_host, cfg, nullptr, nullptr, result);
    }
}

// ================================================================ point query
//
// X_x = s(x) C[i(x)] per row, and the median over rows (Sec. 1.3, the
// point-query use of the Count Sketch).  Runtime t and k; coefficients are
// staged in shared memory.
template <class F, int MODE>
__global__ void __launch_bounds__(256) k_cs_point_query(const QueryArgs a) {
    typedef FieldOps<F> Ops;
    typedef typename Ops::val_t val_t;
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    constexpr int W = Ops::WORDS;
    __shared__ u64 scoef[MAX_COEF_WORDS];
    const int nw = a.t * NF * a.k * W;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) scoef[i] = a.coef_dev[i];
    __syncthreads();
    const ParamCoef<F, 0, 0> dummy = {};
    const u32 mask = (1u << a.log2m) - 1u;
    for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < a.n;
         j += (u64)gridDim.x * blockDim.x) {
        typename Ops::key_t key[4];
        KeyIO<F>::load(a.keys, j, j + 1, false, key);  // scalar load of key j
        const typename Ops::Prep x = Ops::prep(key[0]);
        long long est[MAX_T];
        for (int r = 0; r < a.t; ++r) {
            const int fb = r * NF;
            val_t y = coef_at<F, 0, 0>(dummy, scoef, true, a.k, fb, a.k - 1);
            for (int i = a.k - 2; i >= 0; --i)
                y = Ops::mul_add(y, x, coef_at<F, 0, 0>(dummy, scoef, true, a.k, fb, i));
            const val_t h = Ops::canon(y);
            val_t g = h;
            if (MODE == CS_TWO_POLY) {
                val_t z = coef_at<F, 0, 0>(dummy, scoef, true, a.k, fb + 1, a.k - 1);
                for (int i = a.k - 2; i >= 0; --i)
                    z = Ops::mul_add(z, x, coef_at<F, 0, 0>(dummy, scoef, true, a.k, fb + 1, i));
                g = Ops::canon(z);
            }
            u32 bucket, sb;
            split_row<F, NF>(h, g, mask, a.arb_r, bucket, sb);
            const long long cval = a.counters[((u64)r << a.log2m) + bucket];
            est[r] = sb ? -cval : cval;
        }
        for (int i = 1; i < a.t; ++i) {
            const long long v = est[i];
            int q = i - 1;
            while (q >= 0 && est[q] > v) {
                est[q + 1] = est[q];
                --q;
            }
            est[q + 1] = v;
        }
        a.out[j] = est[a.t / 2];
    }
}

template <class F>
static cudaError_t launch_pq(const QueryArgs& a, cudaStream_t stream) {
    const int threads = 256;
    u64 blocks = (a.n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (a.mode == CS_TWO_POLY)
        k_cs_point_query<F, CS_TWO_POLY><<<(unsigned)blocks, threads, 0, stream>>>(a);
    else
        k_cs_point_query<F, CS_TWO_FOR_ONE><<<(unsigned)blocks, threads, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cs_point_query(int prime, const QueryArgs& a, const u64* coef_host,
                                  cudaStream_t stream) {
    switch (prime) {
        case PRIME_31: return launch_pq<msf::P31>(a, stream);
        case PRIME_61:
            if (a.k == 4 && (a.t == 5 || a.t == 7))
                return launch_point_query_p61_sd(a, coef_host, stream);
            return launch_pq<msf::P61>(a, stream);
        case PRIME_89: return launch_pq<msf::P89>(a, stream);
        default: return launch_pq<msf::P64>(a, stream);
    }
}

// ================================================================ utilities

__global__ void k_add_counters(long long* __restrict__ dst, const long long* __restrict__ src,
                               u64 n) {
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (u64)gridDim.x * blockDim.x)
        dst[i] = (long long)((u64)dst[i] + (u64)src[i]);
}

cudaError_t launch_add_counters(long long* dst, const long long* src, u64 n, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    u64 blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_add_counters<<<(unsigned)blocks, 256, 0, stream>>>(dst, src, n);
    return cudaGetLastError();
}

// counters += the sum of the nrep int32 replicas, and the replicas back to zero
// for the next update.  Four cells a thread with 16-byte loads when the replica
// size allows (every replica 16-byte aligned); all of a thread's replica loads
// are issued before its stores.
__global__ void k_reduce_replicas(long long* __restrict__ counters, int* __restrict__ rep, int nrep,
                                  u64 cells) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 first = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if ((cells & 3u) == 0) {
        const u64 n4 = cells >> 2;
        int4* r4 = reinterpret_cast<int4*>(rep);
        longlong2* c2 = reinterpret_cast<longlong2*>(counters);
        for (u64 i = first; i < n4; i += stride) {
            long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll 8
            for (int r = 0; r < nrep; ++r) {
                const int4 v = r4[(u64)r * n4 + i];
                s0 += v.x;
                s1 += v.y;
                s2 += v.z;
                s3 += v.w;
            }
#pragma unroll 8
            for (int r = 0; r < nrep; ++r) r4[(u64)r * n4 + i] = make_int4(0, 0, 0, 0);
            if ((s0 | s1 | s2 | s3) != 0) {
                longlong2 a = c2[2 * i], b = c2[2 * i + 1];
                a.x = (long long)((u64)a.x + (u64)s0);
                a.y = (long long)((u64)a.y + (u64)s1);
                b.x = (long long)((u64)b.x + (u64)s2);
                b.y = (long long)((u64)b.y + (u64)s3);
                c2[2 * i] = a;
                c2[2 * i + 1] = b;
            }
        }
        return;
    }
    for (u64 i = first; i < cells; i += stride) {
        long long s = 0;
        for (int r = 0; r < nrep; ++r) {
            int* p = rep + (u64)r * cells + i;
            s += (long long)*p;
            *p = 0;
        }
        if (s != 0) counters[i] = (long long)((u64)counters[i] + (u64)s);
    }
}

cudaError_t launch_reduce_replicas(long long* counters, int* replicas, int nrep, u64 cells,
                                   cudaStream_t stream) {
    if (cells == 0 || nrep < 1) return cudaSuccess;
    const u64 work = (cells & 3u) == 0 ? cells >> 2 : cells;
    u64 blocks = (work + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    k_reduce_replicas<<<(unsigned)blocks, 256, 0, stream>>>(counters, replicas, nrep, cells);
    return cudaGetLastError();
}

__global__ void k_zero(uint4* dst, u64 n16, unsigned char* tail, u64 ntail) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
        dst[i] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0 && threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

// dst must be 16-byte aligned (device allocations are).
cudaError_t launch_zero(void* dst, u64 bytes, cudaStream_t stream) {
    if (bytes == 0) return cudaSuccess;
    const u64 n16 = bytes / 16;
    u64 blocks = (n16 + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 8192) blocks = 8192;
    k_zero<<<(unsigned)blocks, 256, 0, stream>>>((uint4*)dst, n16,
                                                 (unsigned char*)dst + n16 * 16, bytes % 16);
    return cudaGetLastError();
}

// ================================================================ hash eval
//
// out[j] = h(keys[j]): Algorithm Mersenne (Horner with lazy reduction) and one
// final canonicalization.  K > 0: compile-time degree; K = 0: runtime k.
template <class F>
struct ValIO;
template <>
struct ValIO<msf::P61> {
    __device__ static __forceinline__ void store(void* out, u64 j, u64 v) { ((u64*)out)[j] = v; }
};
template <>
struct ValIO<msf::P64> : ValIO<msf::P61> {};
template <>
struct ValIO<msf::P31> {
    __device__ static __forceinline__ void store(void* out, u64 j, u32 v) { ((u32*)out)[j] = v; }
};
template <>
struct ValIO<msf::P89> {
    __device__ static __forceinline__ void store(void* out, u64 j, u128 v) {
        ((ulonglong2*)out)[j] = make_ulonglong2((u64)v, (u64)(v >> 64));
    }
};

template <class F, int K>
__global__ void __launch_bounds__(256) k_hash_eval(const void* keys, void* out, u64 n, int k_rt,
                                                   int vec, const HashCoef coef) {
    typedef FieldOps<F> Ops;
    typedef typename Ops::val_t val_t;
    constexpr int W = Ops::WORDS;
    const int k = K ? K : k_rt;
    const u64 stride = (u64)gridDim.x * blockDim.x * 4ull;
    for (u64 j = ((u64)blockIdx.x * blockDim.x + threadIdx.x) * 4ull; j < n; j += stride) {
        typename Ops::key_t key[4];
        KeyIO<F>::load(keys, j, n, vec != 0, key);
        val_t h[4];
        // Horner's rule (Algorithm Mersenne) with the prime's lazy multiply-add
        auto horner = [&]() {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const typename Ops::Prep x = Ops::prep(key[q]);
                val_t y;
                if (W == 1)
                    y = (val_t)coef.w[k - 1];
                else
                    y = (val_t)(((u128)coef.w[2 * (k - 1) + 1] << 64) | coef.w[2 * (k - 1)]);
#pragma unroll(K > 1 ? K - 1 : 1)
                for (int i = k - 2; i >= 0; --i) {
                    val_t ai;
                    if (W == 1)
                        ai = (val_t)coef.w[i];
                    else
                        ai = (val_t)(((u128)coef.w[2 * i + 1] << 64) | coef.w[2 * i]);
                    y = Ops::mul_add(y, x, ai);
                }
                h[q] = Ops::canon(y);
            }
        };
        if constexpr (std::is_same<F, msf::P89>::value) {
            if (k >= 3) {
                // 2^89-1, k >= 3: Horner on three 30-bit limbs (nine 32x32->64
                // products a step; at k = 2 the single step does not repay the limb
                // conversions: 0.092 vs 0.081 ms per 10^7 keys, while k = 4 and 8
                // run 21% and 25% faster than on 128-bit values)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u128 v = F::load(key[q]);
                    u32 x[3], y[3], ai[3];
                    F::limbs((v & F::Pv()) + (v >> 89), x);
                    F::limbs(((u128)coef.w[2 * (k - 1) + 1] << 64) | coef.w[2 * (k - 1)], y);
#pragma unroll(K > 1 ? K - 1 : 1)
                    for (int i = k - 2; i >= 0; --i) {
                        F::limbs(((u128)coef.w[2 * i + 1] << 64) | coef.w[2 * i], ai);
                        F::mul_add3(y, x, ai, y);
                    }
                    h[q] = F::canon3(y);
                }
            } else {
                horner();
            }
        } else {
            horner();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (j + q < n) ValIO<F>::store(out, j + q, h[q]);
    }
}

template <class F>
static cudaError_t launch_he(const void* keys, void* out, u64 n, int k, const HashCoef& coef,
                             int vec, cudaStream_t stream) {
    const int threads = 256;
    u64 blocks = (n + 4ull * threads - 1) / (4ull * threads);
    if (blocks > 152ull * 32) blocks = 152ull * 32;
    if (blocks < 1) blocks = 1;
    switch (k) {
        case 2: k_hash_eval<F, 2><<<(unsigned)blocks, threads, 0, stream>>>(keys, out, n, k, vec, coef); break;
        case 4: k_hash_eval<F, 4><<<(unsigned)blocks, threads, 0, stream>>>(keys, out, n, k, vec, coef); break;
        case 8: k_hash_eval<F, 8><<<(unsigned)blocks, threads, 0, stream>>>(keys, out, n, k, vec, coef); break;
        default: k_hash_eval<F, 0><<<(unsigned)blocks, threads, 0, stream>>>(keys, out, n, k, vec, coef);
    }
    return cudaGetLastError();
}

cudaError_t launch_hash_eval(int prime, const void* keys, void* out, u64 n, int k,
                             const HashCoef& coef, bool vec, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int v = vec ? 1 : 0;
    switch (prime) {
        case PRIME_31: return launch_he<msf::P31>(keys, out, n, k, coef, v, stream);
        case PRIME_61: return launch_he<msf::P61>(keys, out, n, k, coef, v, stream);
        case PRIME_89: return launch_he<msf::P89>(keys, out, n, k, coef, v, stream);
        default: return launch_he<msf::P64>(keys, out, n, k, coef, v, stream);
    }
}

// ================================================================ division
//
// Algorithm division-generalized (Sec. 1.5) on a 129-bit running value: the
// input v < 2^128 plus c can carry into bit 128, so (value, carry) pairs are
// kept and shifted together.  STEPS covers all of [0, 2^128) by the theorem
// of Sec. 4.  Algorithm mod-generalized then gives the remainder from the low
// b bits of v + z*c.
template <int B, unsigned C, int STEPS>
__global__ void __launch_bounds__(256) k_divmod(const ulonglong2* __restrict__ v,
                                                ulonglong2* __restrict__ q, void* __restrict__ r,
                                                u64 n) {
    const u128 MASK = (B == 128) ? ~(u128)0 : ((((u128)1) << B) - 1);
    for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (u64)gridDim.x * blockDim.x) {
        const ulonglong2 in = __ldcs(v + j);
        const u128 x = ((u128)in.y << 64) | in.x;
        const u128 xp = x + C;                 // v' = v + c (mod 2^128) ...
        const u64 xcarry = xp < x ? 1ull : 0ull;  // ... and its bit 128
        // z = v' >> b
        u128 z = (xp >> B) | ((u128)xcarry << (128 - B));
#pragma unroll
        for (int s = 1; s < STEPS; ++s) {
            const u128 zc = z * C;             // z < 2^98, so no overflow
            const u128 sum = zc + xp;
            const u64 carry = xcarry + (sum < xp ? 1ull : 0ull);
            z = (sum >> B) | ((u128)carry << (128 - B));
        }
        if (q) __stcs(q + j, make_ulonglong2((u64)z, (u64)(z >> 64)));
        if (r) {
            const u128 y = (x + z * C) & MASK;  // Algorithm mod-generalized
            if (B <= 64)
                __stcs((u64*)r + j, (u64)y);
            else
                __stcs((ulonglong2*)r + j, make_ulonglong2((u64)y, (u64)(y >> 64)));
        }
    }
}

cudaError_t launch_divmod(int prime, const ms_u128* v, ms_u128* q, void* r, u64 n,
                          cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    u64 blocks = (n + threads - 1) / threads;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    const ulonglong2* vi = (const ulonglong2*)v;
    ulonglong2* qo = (ulonglong2*)q;
    switch (prime) {
        case PRIME_31: k_divmod<31, 1u, 5><<<(unsigned)blocks, threads, 0, stream>>>(vi, qo, r, n); break;
        case PRIME_61: k_divmod<61, 1u, 3><<<(unsigned)blocks, threads, 0, stream>>>(vi, qo, r, n); break;
        case PRIME_89: k_divmod<89, 1u, 2><<<(unsigned)blocks, threads, 0, stream>>>(vi, qo, r, n); break;
        default: k_divmod<64, 59u, 3><<<(unsigned)blocks, threads, 0, stream>>>(vi, qo, r, n);
    }
    return cudaGetLastError();
}

// ================================================================ probe
//
// Throughput of independent integer multiplies on every SM.  Each thread runs
// 8 independent chains so that latency is hidden; the chains' final values are
// folded into one checksum so nothing can be removed.
//  variant 0: a <- lo64(a*b) ^ hi64(a*b): one full 64x64->128 product (low half
//             by multiplication, high half by __umul64hi) per step
//  variant 1: w <- lo32(w)*b + w (mad.wide.u32): one 32x32->64 multiply-add per
//             step whose multiplicand is the previous result, so the compiler
//             cannot hoist the product out of the loop
//  variant 2: x <- x*b + y (mad.lo.u32): one dependent 32-bit multiply-add
//  variant 3: x <- x + y; y <- y + x (add.u32): two dependent 32-bit adds
//  variant 4: a <- lo32(c)*b + a, c <- lo32(a)*b + c (mad.wide.u32) on eight
//             pairs of accumulators per thread: each multiplicand is the other
//             accumulator's latest value, so no product can be hoisted, and the
//             sixteen chains per thread measure the multiplier's throughput
//             rather than its latency
__global__ void __launch_bounds__(256) k_probe(int variant, int iters, u64 seed, u64* sink) {
    u64 a[8], wv[8];
    u32 x[8], y[8];
    const u64 b = seed | 1ull;
    const u32 b32 = (u32)(seed >> 7) | 1u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        a[c] = seed * (threadIdx.x + 1 + c) + blockIdx.x;
        x[c] = (u32)a[c];
        y[c] = (u32)(a[c] >> 29) ^ (u32)c;
        wv[c] = a[c] ^ 0x5555ull;
    }
    if (variant == 0) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < 8; ++c) a[c] = (a[c] * b) ^ __umul64hi(a[c], b);
        }
    } else if (variant == 1) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(wv[c]) : "r"((u32)wv[c]), "r"(b32));
        }
    } else if (variant == 2) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(b32), "r"(y[c]));
        }
    } else if (variant == 3) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                asm volatile("add.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(y[c]));
                asm volatile("add.u32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[c]));
            }
        }
    } else {
        u64 acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = wv[c] ^ 0xAAAAull;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(wv[c]) : "r"((u32)acc[c]), "r"(b32));
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[c]) : "r"((u32)wv[c]), "r"(b32));
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) wv[c] ^= acc[c];
    }
    u64 s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s ^= a[c] ^ wv[c] ^ x[c] ^ ((u64)y[c] << 32);
    if (s == 0x1234567ull) *sink = s;  // practically never taken; keeps the work live
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicXor(sink, s);
}

cudaError_t run_probe_mul128(int variant, int iters, u64* sink, double* rate, double* ms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe, 256, 0);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe<<<blocks, 256>>>(variant, iters / 8 + 1, 0x9E3779B97F4A7C15ull, sink);  // warm-up
    cudaEventRecord(e0);
    k_probe<<<blocks, 256>>>(variant, iters, 0x9E3779B97F4A7C15ull, sink);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double ops = (double)blocks * 256.0 * 8.0 * (double)iters *
                       ((variant == 3 || variant == 4) ? 2.0 : 1.0);
    *ms = t;
    *rate = ops / (t * 1e-3);
    return cudaSuccess;
}

// L2 atomic throughput: every thread adds 1 to `iters` pseudo-random words of
// buf (words a power of two), four independent additions in flight per step.
// Sized like the update's int32 replicas, the buffer stays in L2, so the rate
// is that of the L2's atomic units for scattered 32-bit reductions.
__global__ void __launch_bounds__(256) k_probe_red(int* buf, u32 mask, int iters, u32 seed) {
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    u32 base = (tid * 0x9E3779B1u) ^ seed;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            u32 h = (base + (u32)c) * 0x85EBCA6Bu;
            h ^= h >> 13;
            atomicAdd(buf + (h & mask), 1);
        }
        base += 0x632BE5ABu;
    }
}

cudaError_t run_probe_red(int* buf, u64 words, int iters, double* rate, double* ms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_red, 256, 0);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const u32 mask = (u32)(words - 1);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe_red<<<blocks, 256>>>(buf, mask, iters / 8 + 1, 0x1234567u);  // warm-up
    cudaEventRecord(e0);
    k_probe_red<<<blocks, 256>>>(buf, mask, iters, 0x7654321u);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *ms = t;
    *rate = (double)blocks * 256.0 * 4.0 * (double)iters / (t * 1e-3);
    return cudaSuccess;
}

}  // namespace msk
