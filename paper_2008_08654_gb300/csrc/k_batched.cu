// Batched Count Sketch updates: many independent sketches (each with its own
// coefficients, width m, row count t and stream) in ONE persistent launch.
//
// The host cuts every job (one stream applied to one sketch) into work items
// of at most `chunk` keys and `rows_per_item` rows.  Persistent blocks pull
// item numbers from a device counter.  For an item, a block stages the rows'
// coefficients in shared memory, then either
//   - zeroes an int32 tile of (rows x m) counters in shared memory, adds the
//     chunk's updates there, and adds the tile into the sketch's int64
//     counters (when the chunk has at least smem_min_ratio * m keys), or
//   - adds every update straight into the int64 counters (small chunks, where
//     zeroing and flushing a tile would cost more than the updates).
// The arithmetic is the same as the single-sketch kernel (k_update.cuh).
#include <cuda_runtime.h>
#include <stdint.h>

#include "k_update.cuh"
#include "ms_batch_internal.h"

namespace msk {

struct PsCoef {  // one polynomial, signed-digit power-sum form (p = 2^61-1, k = 4; row_sd)
    u64 k1;
    int cl[3], ch[3];
    int nd[3];  // cl - ch
    u32 pad;
};

// C[r][bucket] += sign ? -w : w, into the item's tile (rows r0..) or, for
// `direct`, straight into the sketch's int64 counters.
__device__ __forceinline__ void batched_add(int* tile, long long* counters, int r, int r0,
                                            int log2m, u32 bucket, u32 sign, int w, bool direct) {
    if (direct) {
        global_add64(counters + (((u64)r) << log2m) + bucket, sign ? -(long long)w : (long long)w);
    } else {
        atomicAdd(tile + ((r - r0) << log2m) + bucket, sign ? -w : w);
    }
}

template <class F, int MODE, bool PS>
__global__ void __launch_bounds__(1024) k_cs_update_batched(const BatchArgs a) {
    typedef FieldOps<F> Ops;
    typedef typename Ops::val_t val_t;
    typedef typename Ops::Prep Prep;
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    constexpr int W = Ops::WORDS;

    extern __shared__ __align__(16) unsigned char smem[];
    // layout: [coefficients: MAX_T*NF*MAX_K*W u64 | PsCoef MAX_T*NF] [tile int32]
    u64* scoef = reinterpret_cast<u64*>(smem);
    PsCoef* sps = reinterpret_cast<PsCoef*>(smem + MAX_COEF_WORDS * 8);
    int* tile = reinterpret_cast<int*>(smem + MAX_COEF_WORDS * 8 + MAX_T * 2 * sizeof(PsCoef));
    __shared__ u32 s_item;
    const int k = a.k;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const u32 item = s_item;
        if (item >= a.total_items) break;
        // job = last j with first_item[j] <= item
        int lo = 0, hi = a.njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&a.jobs[mid].first_item) <= item) lo = mid; else hi = mid - 1;
        }
        const BatchJobDev job = a.jobs[lo];
        const u32 local = item - job.first_item;
        const u32 ngroups = (job.t + a.rows_per_item - 1) / a.rows_per_item;
        const u32 chunk_idx = local / ngroups;
        const int r0 = (int)(local % ngroups) * a.rows_per_item;
        const int r1 = min((int)job.t, r0 + a.rows_per_item);
        const u64 j0 = (u64)chunk_idx * a.chunk;
        const u64 j1 = min(job.n, j0 + a.chunk);
        const int log2m = (int)job.log2m;
        const u32 m = 1u << log2m;
        const u32 mask = m - 1u;
        const bool use_tile = (j1 - j0) >= (u64)a.smem_min_ratio * m;
        const u32 tile_cells = use_tile ? (u32)(r1 - r0) * m : 0u;

        // stage this item's coefficients (rows r0..r1)
        const int nw = (r1 - r0) * NF * k * W;
        const u64* src = job.coef + (size_t)r0 * NF * k * W;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) scoef[i] = src[i];
        if (PS) {
            for (int f = threadIdx.x; f < (r1 - r0) * NF; f += blockDim.x) {
                PsCoef pc;
                msf::P61::sd_coef(src + (size_t)f * 4, pc.cl, pc.ch, pc.nd, pc.k1);
                pc.pad = 0;
                sps[f] = pc;
            }
        }
        for (u32 i = threadIdx.x; i < tile_cells; i += blockDim.x) tile[i] = 0;
        __syncthreads();

        const bool vec = job.vec_ok != 0;
        const u32 w_safe = a.w_safe;
        for (u64 j = j0 + (u64)threadIdx.x * 4ull; j < j1; j += (u64)blockDim.x * 4ull) {
            typename Ops::key_t key[4];
            int wt[4];
            KeyIO<F>::load(job.keys, j, j1, vec, key);
            load_weights4(job.w, j, j1, vec, wt);
            bool big[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const u32 aw = wt[q] < 0 ? 0u - (u32)wt[q] : (u32)wt[q];
                big[q] = !use_tile || aw > w_safe;
            }
            if constexpr (PS) {
                const u32 row_bytes = 4u << log2m;
                const int nr = r1 - r0;
                // A key that goes to the int64 counters (every key of a direct
                // item; in a tile item the rare key whose weight could overflow
                // an int32 cell): its rows one at a time.  Rolled over the four
                // keys (their registers rotate), so the cold path stays small.
                if (big[0] | big[1] | big[2] | big[3]) {
#pragma unroll 1
                    for (int q = 0; q < 4; ++q) {
                        // key 0 is taken here (its weight then 0 for the tile
                        // path) and moves to the back: after four turns the
                        // keys are in their places again
                        const u64 kq = (u64)key[0];
                        const int wq = big[0] ? wt[0] : 0;
                        const int wk = big[0] ? 0 : wt[0];
                        key[0] = key[1];
                        key[1] = key[2];
                        key[2] = key[3];
                        key[3] = (typename Ops::key_t)kq;
                        wt[0] = wt[1];
                        wt[1] = wt[2];
                        wt[2] = wt[3];
                        wt[3] = wk;
                        big[0] = big[1];
                        big[1] = big[2];
                        big[2] = big[3];
                        big[3] = false;
                        if (wq == 0) continue;
                        msf::P61::Pow3 xp;
                        msf::P61::powers3(kq, xp);
#pragma unroll 1
                        for (int rr = 0; rr < nr; ++rr) {
                            const PsCoef cb = sps[rr * NF];
                            u32 ylo, yhi;
                            msf::P61::row_sd(xp, cb.cl, cb.ch, cb.nd, cb.k1, a.c2p31, ylo, yhi);
                            const u32 bucket = ylo & mask;
                            if (MODE == CS_TWO_POLY) {
                                const PsCoef cs = sps[rr * NF + 1];
                                msf::P61::row_sd(xp, cs.cl, cs.ch, cs.nd, cs.k1, a.c2p31, ylo, yhi);
                            }
                            global_add64(job.counters + (((u64)(r0 + rr)) << log2m) + bucket,
                                         (yhi & 0x10000000u) ? -(long long)wq : (long long)wq);
                        }
                    }
                }
                if (use_tile) {
                    // Two keys at a time, so each row's coefficients are read from
                    // shared memory once for both; a zero weight adds 0.
                    const u32 tbase = (u32)__cvta_generic_to_shared(tile);
#pragma unroll 1
                    for (int qq = 0; qq < 2; ++qq) {
                        msf::P61::Pow3 xa, xb;
                        msf::P61::powers3(key[0], xa);
                        msf::P61::powers3(key[1], xb);
                        const int wa = wt[0], wb = wt[1];
                        key[0] = key[2];
                        key[1] = key[3];
                        wt[0] = wt[2];
                        wt[1] = wt[3];
                        auto row = [&](int rr, u32 rbase) {
                            const PsCoef cb = sps[rr * NF];
                            u32 alo, ahi, blo, bhi;
                            msf::P61::row_sd(xa, cb.cl, cb.ch, cb.nd, cb.k1, a.c2p31, alo, ahi);
                            msf::P61::row_sd(xb, cb.cl, cb.ch, cb.nd, cb.k1, a.c2p31, blo, bhi);
                            const u32 ba = alo & mask, bb = blo & mask;
                            if (MODE == CS_TWO_POLY) {
                                const PsCoef cs = sps[rr * NF + 1];
                                msf::P61::row_sd(xa, cs.cl, cs.ch, cs.nd, cs.k1, a.c2p31, alo, ahi);
                                msf::P61::row_sd(xb, cs.cl, cs.ch, cs.nd, cs.k1, a.c2p31, blo, bhi);
                            }
                            const int da = (ahi & 0x10000000u) ? -wa : wa;  // bit 60 of the residue
                            const int db = (bhi & 0x10000000u) ? -wb : wb;
                            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(rbase + (ba << 2)), "r"(da)
                                         : "memory");
                            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(rbase + (bb << 2)), "r"(db)
                                         : "memory");
                        };
                        u32 rbase = tbase;  // shared address of the item's row rr
                        if (MODE != CS_TWO_POLY && nr == 5) {
                            // five rows (every item of a t = 5 sketch): unrolled, so
                            // the rows' multiply chains interleave (with two
                            // polynomials a row has four chains already, and the
                            // unrolled rows spilled)
#pragma unroll
                            for (int rr = 0; rr < 5; ++rr) {
                                row(rr, rbase);
                                rbase += row_bytes;
                            }
                        } else {
                            for (int rr = 0; rr < nr; ++rr) {
                                row(rr, rbase);
                                rbase += row_bytes;
                            }
                        }
                    }
                }
            } else {
                Prep xp[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) xp[q] = Ops::prep(key[q]);
                for (int r = r0; r < r1; ++r) {
                    const u64* cb = scoef + (size_t)(r - r0) * NF * k * W;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        val_t y = Ops::from_words(cb + (size_t)(k - 1) * W);
                        for (int i = k - 2; i >= 0; --i)
                            y = Ops::mul_add(y, xp[q], Ops::from_words(cb + (size_t)i * W));
                        const val_t h = Ops::canon(y);
                        val_t g = h;
                        if (MODE == CS_TWO_POLY) {
                            const u64* cs = cb + (size_t)k * W;
                            val_t z = Ops::from_words(cs + (size_t)(k - 1) * W);
                            for (int i = k - 2; i >= 0; --i)
                                z = Ops::mul_add(z, xp[q], Ops::from_words(cs + (size_t)i * W));
                            g = Ops::canon(z);
                        }
                        if (wt[q] != 0)
                            batched_add(tile, job.counters, r, r0, log2m, Ops::bucket(h, mask),
                                        Ops::sign_bit(g), wt[q], big[q]);
                    }
                }
            }
        }
        __syncthreads();
        for (u32 i = threadIdx.x; i < tile_cells; i += blockDim.x) {
            const int v = tile[i];
            if (v != 0) {
                const u32 row = (u32)r0 + (i >> log2m);
                global_add64(job.counters + (((u64)row) << log2m) + (i & mask), (long long)v);
            }
        }
        __syncthreads();  // tile and coefficients are reused by the next item
    }
}

__global__ void k_batch_reset(u32* work_counter) { *work_counter = 0u; }

size_t batched_smem_bytes(int rows_per_item, int max_log2m) {
    return (size_t)MAX_COEF_WORDS * 8 + MAX_T * 2 * sizeof(PsCoef) +
           (size_t)rows_per_item * ((size_t)1 << max_log2m) * 4;
}

template <class F, int MODE, bool PS>
static cudaError_t launch_b(const BatchArgs& a, const BatchLaunch& l, cudaStream_t s,
                            int* occupancy) {
    auto kern = k_cs_update_batched<F, MODE, PS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)l.smem);
    if (e != cudaSuccess) return e;
    if (occupancy) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, kern, l.threads, l.smem);
    k_batch_reset<<<1, 1, 0, s>>>(a.work_counter);
    kern<<<l.blocks, l.threads, l.smem, s>>>(a);
    return cudaGetLastError();
}

template <class F, int MODE>
static cudaError_t launch_bm(const BatchArgs& a, const BatchLaunch& l, cudaStream_t s, int* occ) {
    constexpr bool PS_OK = std::is_same<F, msf::P61>::value;
    if (PS_OK && a.k == 4 && l.strategy == STRAT_POWER_SUM)
        return launch_b<F, MODE, PS_OK>(a, l, s, occ);
    return launch_b<F, MODE, false>(a, l, s, occ);
}

template <class F>
static cudaError_t launch_bf(const BatchArgs& a, const BatchLaunch& l, cudaStream_t s, int* occ) {
    if (a.mode == CS_TWO_POLY) return launch_bm<F, CS_TWO_POLY>(a, l, s, occ);
    return launch_bm<F, CS_TWO_FOR_ONE>(a, l, s, occ);
}

// Enqueues the work-counter reset and the persistent kernel on `s`, or (with
// occupancy != NULL) only reports resident blocks per SM.
cudaError_t launch_cs_update_batched(int prime, const BatchArgs& a, const BatchLaunch& l,
                                     cudaStream_t s, int* occupancy) {
    switch (prime) {
        case PRIME_31: return launch_bf<msf::P31>(a, l, s, occupancy);
        case PRIME_61: return launch_bf<msf::P61>(a, l, s, occupancy);
        case PRIME_89: return launch_bf<msf::P89>(a, l, s, occupancy);
        default: return launch_bf<msf::P64>(a, l, s, occupancy);
    }
}

}  // namespace msk
