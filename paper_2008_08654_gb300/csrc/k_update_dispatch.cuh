// Runtime -> compile-time dispatch of the Count Sketch update kernel for one
// prime.  Each k_update_p*.cu includes this file and instantiates
// launch_update_for<F>() for its prime, so the four primes compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

#include "k_update.cuh"

namespace msk {

// Fill the parameter-space coefficient pack from the host copy of the
// coefficient words (function-major, a_0 first, W limbs each).
template <class F, int NFUN, int K>
static void fill_param_coef(ParamCoef<F, NFUN, K>& pc, const u64* words) {
    constexpr int W = FieldOps<F>::WORDS;
    pc.c2p31 = 0x80000000u;
    pc.c4 = 4u;
    pc.cl[0] = pc.ch[0] = pc.nd[0] = 0;
    pc.k1[0] = 0;
    if (NFUN == 0) {
        pc.w[0] = 0;
        return;
    }
    for (int i = 0; i < NFUN * K * W; ++i) pc.w[i] = words[i];
    if constexpr (ParamCoef<F, NFUN, K>::SD > 0) {
        for (int f = 0; f < NFUN; ++f)
            msf::P61::sd_coef(words + (size_t)f * K, pc.cl + 3 * f, pc.ch + 3 * f, pc.nd + 3 * f,
                              pc.k1[f]);
    }
    if constexpr (K == 4 && PsLimbs<F>::N > 0) {
        for (int f = 0; f < NFUN; ++f) {
            u32* c = pc.ps + f * PsLimbs<F>::N;
            const u64* a = words + (size_t)f * K * W;
            if constexpr (std::is_same<F, msf::P89>::value) {
                // a0's 30-bit limbs, then (l0, l1, l2, l0 - l1, l0 - l2, l1 - l2)
                // of a1, a2, a3 (the differences as two's-complement words)
                for (int i = 0; i < 4; ++i) {
                    const unsigned __int128 v = ((unsigned __int128)a[2 * i + 1] << 64) | a[2 * i];
                    const u32 l0 = (u32)(v & 0x3FFFFFFFu), l1 = (u32)((v >> 30) & 0x3FFFFFFFu);
                    const u32 l2 = (u32)(v >> 60);
                    if (i == 0) {
                        c[0] = l0; c[1] = l1; c[2] = l2;
                    } else {
                        u32* d = c + 3 + 6 * (i - 1);
                        d[0] = l0; d[1] = l1; d[2] = l2;
                        d[3] = (u32)((int)l0 - (int)l1);
                        d[4] = (u32)((int)l0 - (int)l2);
                        d[5] = (u32)((int)l1 - (int)l2);
                    }
                }
            } else {
                // b_iv = a_i 2^(29 v) mod (2^64 - 59), low and high halves
                const unsigned __int128 p = (((unsigned __int128)1) << 64) - 59;
                for (int i = 1; i < 4; ++i)
                    for (int v = 0; v < 3; ++v) {
                        const u64 b = (u64)((((unsigned __int128)a[i]) << (29 * v)) % p);
                        c[6 * (i - 1) + 2 * v] = (u32)b;
                        c[6 * (i - 1) + 2 * v + 1] = (u32)(b >> 32);
                    }
            }
        }
    }
}

template <class F, int T, int K, int MODE, int PLACE, int STRAT>
static cudaError_t launch_exact(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                                cudaStream_t stream, int* occupancy) {
    constexpr int NF = (MODE == CS_TWO_POLY) ? 2 : 1;
    auto kern = k_cs_update<F, T, K, MODE, PLACE, STRAT>;
    // 2^61-1, k = 4, shared-memory tile: the lean kernel (the statistics hook
    // counts entries only in the general one)
    if constexpr (std::is_same<F, msf::P61>::value && T > 0 && K == 4 && PLACE == PLACE_SMEM &&
                  STRAT == STRAT_POWER_SUM_ANY_R) {
        // any number of buckets: the lean kernel with the any-m map, run-time row stride
        if (update_uses_lean_tile(PRIME_61, a, cfg.place, cfg.strategy))
            kern = a.weights ? k_cs_update_tile<T, MODE, true, 0, true>
                             : k_cs_update_tile<T, MODE, false, 0, true>;
    }
    if constexpr (std::is_same<F, msf::P31>::value && T > 0 && K == 4 && PLACE == PLACE_SMEM &&
                  STRAT == STRAT_POWER_SUM) {
        if (update_uses_lean_tile(PRIME_31, a, cfg.place, cfg.strategy)) {
            if (a.weights)
                kern = a.log2m == 10   ? k_cs_update_tile31<T, MODE, true, 10>
                       : a.log2m == 12 ? k_cs_update_tile31<T, MODE, true, 12>
                                       : k_cs_update_tile31<T, MODE, true, 0>;
            else
                kern = a.log2m == 10   ? k_cs_update_tile31<T, MODE, false, 10>
                       : a.log2m == 12 ? k_cs_update_tile31<T, MODE, false, 12>
                                       : k_cs_update_tile31<T, MODE, false, 0>;
        }
    }
    if constexpr ((std::is_same<F, msf::P89>::value || std::is_same<F, msf::P64>::value) && T > 0 &&
                  K == 4 && PLACE == PLACE_SMEM && STRAT == STRAT_POWER_SUM) {
        constexpr int PR = std::is_same<F, msf::P89>::value ? PRIME_89 : PRIME_64_59;
        if (update_uses_lean_tile(PR, a, cfg.place, cfg.strategy)) {
            if (a.weights)
                kern = a.log2m == 10   ? k_cs_update_tile_ps<F, T, MODE, true, 10>
                       : a.log2m == 12 ? k_cs_update_tile_ps<F, T, MODE, true, 12>
                                       : k_cs_update_tile_ps<F, T, MODE, true, 0>;
            else
                kern = a.log2m == 10   ? k_cs_update_tile_ps<F, T, MODE, false, 10>
                       : a.log2m == 12 ? k_cs_update_tile_ps<F, T, MODE, false, 12>
                                       : k_cs_update_tile_ps<F, T, MODE, false, 0>;
        }
    }
    if constexpr (std::is_same<F, msf::P61>::value && T > 0 && K == 4 && PLACE == PLACE_SMEM &&
                  STRAT == STRAT_POWER_SUM) {
        if (update_uses_lean_tile(PRIME_61, a, cfg.place, cfg.strategy)) {
            // m = 2^10 and 2^12 (the workloads' widths) with compile-time row strides
            if (a.weights)
                kern = a.log2m == 10   ? k_cs_update_tile<T, MODE, true, 10>
                       : a.log2m == 12 ? k_cs_update_tile<T, MODE, true, 12>
                                       : k_cs_update_tile<T, MODE, true, 0>;
            else
                kern = a.log2m == 10   ? k_cs_update_tile<T, MODE, false, 10>
                       : a.log2m == 12 ? k_cs_update_tile<T, MODE, false, 12>
                                       : k_cs_update_tile<T, MODE, false, 0>;
        }
    }
    cudaError_t e;
    if (T == 0) {  // the generic kernel stages the coefficients after the tile
        const size_t tile = PLACE == PLACE_GLOBAL ? 0
                            : ((size_t)a.t << a.log2m) * 4 / (size_t)(cfg.cluster > 0 ? cfg.cluster : 1);
        const size_t coef = (size_t)a.t * NF * a.k * FieldOps<F>::WORDS * 8;
        if (cfg.smem < tile + coef) return cudaErrorInvalidValue;
    }
    if (cfg.smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        if (e != cudaSuccess) return e;
    }
    if (PLACE == PLACE_DSMEM && cfg.cluster > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)cfg.blocks);
    lc.blockDim = dim3((unsigned)cfg.threads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    if (PLACE == PLACE_DSMEM) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cfg.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
    }
    if (occupancy) {
        if (PLACE == PLACE_DSMEM)
            return cudaOccupancyMaxActiveClusters(occupancy, kern, &lc);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, kern, cfg.threads,
                                                             cfg.smem);
    }
    ParamCoef<F, NF * T, K> pc;
    fill_param_coef<F, NF * T, K>(pc, coef_host);
    return cudaLaunchKernelEx(&lc, kern, a, pc);
}

template <class F, int T, int K, int MODE, int PLACE>
static cudaError_t launch_strat(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                                cudaStream_t stream, int* occupancy) {
    // the power sum: every prime at k = 4; the any-m map only for 2^61-1 (the
    // other primes' any-m sketches take the generic kernel)
    constexpr bool PS_OK = K == 4;
    constexpr bool ANY_OK = std::is_same<F, msf::P61>::value && K == 4;
    if (PS_OK && cfg.strategy == STRAT_POWER_SUM) {
        if (a.arb_r)
            return launch_exact<F, T, K, MODE, PLACE, ANY_OK ? STRAT_POWER_SUM_ANY_R : STRAT_HORNER>(
                a, coef_host, cfg, stream, occupancy);
        return launch_exact<F, T, K, MODE, PLACE, PS_OK ? STRAT_POWER_SUM : STRAT_HORNER>(
            a, coef_host, cfg, stream, occupancy);
    }
    return launch_exact<F, T, K, MODE, PLACE, STRAT_HORNER>(a, coef_host, cfg, stream, occupancy);
}

template <class F, int T, int K, int MODE>
static cudaError_t launch_place(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                                cudaStream_t stream, int* occupancy) {
    switch (cfg.place) {
        case PLACE_SMEM:
            return launch_strat<F, T, K, MODE, PLACE_SMEM>(a, coef_host, cfg, stream, occupancy);
        case PLACE_DSMEM:
            return launch_strat<F, T, K, MODE, PLACE_DSMEM>(a, coef_host, cfg, stream, occupancy);
        default:
            return launch_strat<F, T, K, MODE, PLACE_GLOBAL>(a, coef_host, cfg, stream, occupancy);
    }
}

template <class F, int T, int K>
static cudaError_t launch_mode(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                               cudaStream_t stream, int* occupancy) {
    if (a.mode == CS_TWO_POLY)
        return launch_place<F, T, K, CS_TWO_POLY>(a, coef_host, cfg, stream, occupancy);
    return launch_place<F, T, K, CS_TWO_FOR_ONE>(a, coef_host, cfg, stream, occupancy);
}

// The specializations: (t, k) = (5, 4) and (7, 4), the workloads' shapes;
// everything else takes the generic kernel (runtime t and k).
template <class F>
cudaError_t launch_update_for(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                              cudaStream_t stream, int* specialized, int* occupancy) {
    constexpr int PRIME = std::is_same<F, msf::P31>::value   ? PRIME_31
                          : std::is_same<F, msf::P61>::value ? PRIME_61
                          : std::is_same<F, msf::P89>::value ? PRIME_89
                                                             : PRIME_64_59;
    if (update_is_specialized(PRIME, a.t, a.k, a.arb_r)) {
        if (specialized) *specialized = update_uses_lean_tile(PRIME, a, cfg.place, cfg.strategy) ? 2 : 1;
        return a.t == 5 ? launch_mode<F, 5, 4>(a, coef_host, cfg, stream, occupancy)
                        : launch_mode<F, 7, 4>(a, coef_host, cfg, stream, occupancy);
    }
    if (specialized) *specialized = 0;
    return launch_mode<F, 0, 0>(a, coef_host, cfg, stream, occupancy);
}

// The second-level table's drain (one-word keys only: 2^89-1 never uses it).
// The 2^61-1, k = 4, t = 5 or 7 drain (signed-digit rows, coefficients in
// the parameter space).
template <int T, int NF, bool ANY>
static cudaError_t drain_sd(const UpdateArgs& a, const u64* coef_host, unsigned blocks,
                            cudaStream_t stream) {
    ParamCoef<msf::P61, NF * T, 4> pc;
    fill_param_coef<msf::P61, NF * T, 4>(pc, coef_host);
    k_gtable_drain_sd<T, NF, ANY><<<blocks, 256, 0, stream>>>(a, pc);
    return cudaGetLastError();
}

// Point queries, 2^61-1 with k = 4 and t = 5 or 7 (the signed-digit rows).
template <int T, int NF, bool ANY>
static cudaError_t point_query_sd(const QueryArgs& a, const u64* coef_host, cudaStream_t stream) {
    ParamCoef<msf::P61, NF * T, 4> pc;
    fill_param_coef<msf::P61, NF * T, 4>(pc, coef_host);
    const int threads = 256;
    u64 blocks = (a.n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    k_cs_point_query_sd<T, NF, ANY><<<(unsigned)blocks, threads, 0, stream>>>(a, pc);
    return cudaGetLastError();
}

template <class F>
cudaError_t launch_gtable_drain_for(const UpdateArgs& a, const u64* coef_host, cudaStream_t stream) {
    if constexpr (!DedupKey<typename FieldOps<F>::key_t>::OK) {
        return cudaErrorInvalidValue;
    } else {
        const u32 slots = 1u << a.glog2;
        const unsigned blocks = (unsigned)((slots + 255u) / 256u < 4096u ? (slots + 255u) / 256u : 4096u);
        if constexpr (std::is_same<F, msf::P61>::value) {
            if (a.k == 4 && (a.t == 5 || a.t == 7)) {
                const bool two = a.mode == CS_TWO_POLY, any = a.arb_r != 0;
                if (a.t == 5) {
                    if (two) return any ? drain_sd<5, 2, true>(a, coef_host, blocks, stream)
                                        : drain_sd<5, 2, false>(a, coef_host, blocks, stream);
                    return any ? drain_sd<5, 1, true>(a, coef_host, blocks, stream)
                               : drain_sd<5, 1, false>(a, coef_host, blocks, stream);
                }
                if (two) return any ? drain_sd<7, 2, true>(a, coef_host, blocks, stream)
                                    : drain_sd<7, 2, false>(a, coef_host, blocks, stream);
                return any ? drain_sd<7, 1, true>(a, coef_host, blocks, stream)
                           : drain_sd<7, 1, false>(a, coef_host, blocks, stream);
            }
        }
        if (a.mode == CS_TWO_POLY)
            k_gtable_drain<F, 2><<<blocks, 256, 0, stream>>>(a);
        else
            k_gtable_drain<F, 1><<<blocks, 256, 0, stream>>>(a);
        return cudaGetLastError();
    }
}

}  // namespace msk
