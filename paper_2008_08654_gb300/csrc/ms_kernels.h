// Internal interface between the host ABI code (ms_host.cu) and the kernel
// translation units.  Not installed; the public interface is include/ms.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ms.h"

namespace msk {

typedef unsigned long long u64;
typedef unsigned int u32;

// Prime identifiers (p = 2^b - c).
enum PrimeId { PRIME_31 = 0, PRIME_61 = 1, PRIME_89 = 2, PRIME_64_59 = 3 };

// Counter placement of the update kernel.
enum Place {
    PLACE_SMEM = 0,   // whole t x m int32 tile in each block's shared memory
    PLACE_DSMEM = 1,  // tile split over a thread-block cluster (distributed smem)
    PLACE_GLOBAL = 2  // int64 atomics straight into the counters in HBM/L2
};

// Row-hash evaluation strategy (both give the same canonical value).
enum Strategy {
    STRAT_HORNER = 0,    // Algorithm Mersenne, k-1 lazy multiply-add steps per row
    STRAT_POWER_SUM = 1, // x^2..x^(k-1) once per key, then sum a_i x^i per row
    STRAT_POWER_SUM_ANY_R = 2  // internal: the power sum with the any-m bucket map
};

constexpr int MAX_T = 15;
// De-duplication (PLACE_GLOBAL, unit weights): entries of each warp's queue of
// keys waiting to be hashed (fewer than 128 wait, one chunk adds at most 128).
constexpr u32 DEDUP_QCAP = 256;
constexpr int MAX_K = 8;
constexpr int MAX_COEF_WORDS = MAX_T * 2 * MAX_K * 2;  // t * functions * k * limbs

struct UpdateArgs {
    const void* keys;
    const int32_t* weights;  // NULL: unit weights
    u64 n;
    long long* counters;     // t * m int64, row-major
    const u64* coef_dev;     // device copy of the coefficients (generic kernels)
    int t, k, log2m, mode;
    int cluster_log2;        // DSMEM: log2(cluster size)
    int vec_ok;              // keys and weights are 16-byte aligned
    u32 w_safe;              // |w| <= w_safe may use int32 tile/replica counters
    int* replicas;           // PLACE_GLOBAL: R int32 copies of the t x m counters,
                             // or NULL for direct int64 atomics
    u32 replica_mask;        // R - 1 (R a power of two)
    int aggregate;           // PLACE_GLOBAL, unit weights: merge equal keys of a warp
    int dedup_log2;          // PLACE_GLOBAL, unit weights, one-word keys: log2 slots of
                             // the per-block de-duplication table (0 = none)
    u32 arb_r;               // any number of buckets: r (rows are 2^log2m >= r wide);
                             // 0: power-of-two buckets (generic kernels only)
    unsigned long long* hashed;  // optional: += entries hashed with a non-zero count
    int keys_per_thread_hint;    // 0: any kernel; 4: the general kernel (4 keys a thread)
    // With the de-duplication table: the second-level key table in global
    // memory (L2-resident), 2^glog2 slots of keys (DEDUP_EMPTY = free) and
    // int32 counts; glog2 = 0: none.  Keys the block's table misses are
    // counted there when they own (or claim) their slot.
    unsigned long long* gkeys;
    int* gcounts;
    int glog2;
};

// Whether cs_update runs a compile-time (t, k) kernel (coefficients in the
// parameter space) or the generic one (coefficients staged in shared memory
// after the counter tile, which the launch's shared memory must cover).  The
// host's launch choice and the dispatcher both ask this one function.
inline bool update_is_specialized(int prime, int t, int k, u32 arb_r) {
    return k == 4 && (t == 5 || t == 7) && (arb_r == 0 || prime == PRIME_61);
}

// Whether a specialized update with a shared-memory tile runs a lean
// one-key-a-thread kernel rather than the general one: 2^61-1 (k_cs_update_tile,
// power-of-two or any number of buckets), 2^31-1 (k_cs_update_tile31) and the
// wider primes (k_cs_update_tile_ps) with power-of-two buckets; no statistics
// hook, no request for the general kernel.
inline bool update_uses_lean_tile(int prime, const UpdateArgs& a, int place, int strategy) {
    return (prime == PRIME_61 || a.arb_r == 0) && a.k == 4 &&
           (a.t == 5 || a.t == 7) && place == PLACE_SMEM && strategy == STRAT_POWER_SUM &&
           a.hashed == nullptr && a.keys_per_thread_hint == 0;
}

// Second-level key table: hashes every key it holds with its count into the
// int64 counters (t rows, the split of the sketch's mode) and empties the
// table for the next update.  2^61-1 with k = 4 and t = 5 or 7: signed-digit
// rows with the coefficients from coef_host in the parameter space; else
// Horner from coef_dev.
cudaError_t launch_gtable_drain(int prime, const UpdateArgs& a, const u64* coef_host,
                                cudaStream_t stream);

// Launch configuration chosen on the host.
struct LaunchCfg {
    int place;
    int strategy;
    int threads;
    int blocks;       // total blocks (a multiple of the cluster size)
    int cluster;      // 1 unless PLACE_DSMEM
    int replicas;     // PLACE_GLOBAL: int32 replica count (0 = direct int64 atomics)
    size_t smem;      // dynamic shared memory bytes
};

// Returns cudaSuccess or the launch error.  `specialized` is set to whether a
// compile-time (t, k) specialization served the call.
// coef_host: the sketch's coefficient limbs (function-major, a_0 first).
cudaError_t launch_cs_update(int prime, const UpdateArgs& a, const u64* coef_host,
                             const LaunchCfg& cfg, cudaStream_t stream, int* specialized);

// Occupancy query for a configuration: resident blocks per SM (SMEM/GLOBAL)
// or co-resident clusters on the device (DSMEM).
cudaError_t query_cs_update_occupancy(int prime, const UpdateArgs& a, const u64* coef_host,
                                      const LaunchCfg& cfg, int* result);

// Per-prime entry points (one translation unit each).
cudaError_t launch_update_p31(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                              cudaStream_t stream, int* specialized, int* occupancy);
cudaError_t launch_update_p61(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                              cudaStream_t stream, int* specialized, int* occupancy);
cudaError_t launch_update_p89(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                              cudaStream_t stream, int* specialized, int* occupancy);
cudaError_t launch_update_p64(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                              cudaStream_t stream, int* specialized, int* occupancy);
cudaError_t launch_gtable_drain_p31(const UpdateArgs& a, const u64* coef_host,
                                    cudaStream_t stream);
cudaError_t launch_gtable_drain_p61(const UpdateArgs& a, const u64* coef_host,
                                    cudaStream_t stream);
cudaError_t launch_gtable_drain_p64(const UpdateArgs& a, const u64* coef_host,
                                    cudaStream_t stream);
cudaError_t launch_gtable_drain_p89(const UpdateArgs& a, const u64* coef_host,
                                    cudaStream_t stream);

struct F2Args {
    const long long* counters;
    int t;
    u32 m;
    int splits;          // blocks per row (power of two, divides m)
    ms_u128* partial;    // t * splits scratch
    u32* ticket;         // scratch counter, zero between launches
    ms_u128* out;        // median
    ms_u128* rows;       // optional t row values
};
cudaError_t launch_cs_f2(const F2Args& a, int threads, cudaStream_t stream);

struct QueryArgs {
    const void* keys;
    u64 n;
    const long long* counters;
    const u64* coef_dev;
    int t, k, log2m, mode;
    u32 arb_r;  // as in UpdateArgs
    long long* out;
};
// coef_host: the sketch's coefficient limbs (2^61-1 with k = 4 and t = 5 or 7
// run the signed-digit rows with them in the parameter space; the others
// Horner from coef_dev).
cudaError_t launch_cs_point_query(int prime, const QueryArgs& a, const u64* coef_host,
                                  cudaStream_t stream);
cudaError_t launch_point_query_p61_sd(const QueryArgs& a, const u64* coef_host,
                                      cudaStream_t stream);

cudaError_t launch_add_counters(long long* dst, const long long* src, u64 n, cudaStream_t stream);

// counters[i] += sum_r replicas[r * cells + i] (sign-extended), then every
// replica cell is zeroed for the next update.
cudaError_t launch_reduce_replicas(long long* counters, int* replicas, int nrep, u64 cells,
                                   cudaStream_t stream);
cudaError_t launch_zero(void* dst, u64 bytes, cudaStream_t stream);

struct HashCoef {
    u64 w[MAX_K * 2];  // k coefficients, 1 or 2 limbs each
};
cudaError_t launch_hash_eval(int prime, const void* keys, void* out, u64 n, int k,
                             const HashCoef& coef, bool vec, cudaStream_t stream);

cudaError_t launch_divmod(int prime, const ms_u128* v, ms_u128* q, void* r, u64 n,
                          cudaStream_t stream);

cudaError_t run_probe_mul128(int variant, int iters, u64* sink, double* rate, double* ms);
cudaError_t run_probe_red(int* buf, u64 words, int iters, double* rate, double* ms);

}  // namespace msk
