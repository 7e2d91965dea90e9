// Internal interface of the batched update kernel (k_batched.cu) and its
// host plan (ms_batch.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ms_kernels.h"

namespace msk {

// One job as the kernel sees it (device table, 64-byte entries).
struct BatchJobDev {
    const void* keys;
    const int32_t* w;
    u64 n;
    long long* counters;
    const u64* coef;     // the sketch's device coefficient words
    u32 log2m;
    u32 t;
    u32 first_item;      // first work item of this job
    u32 vec_ok;          // keys/weights 16-byte aligned
};

struct BatchArgs {
    const BatchJobDev* jobs;
    int njobs;
    u32 total_items;
    u32* work_counter;   // device scratch, reset before each launch
    int k, mode;
    int rows_per_item;
    u32 chunk;           // keys per work item
    u32 smem_min_ratio;  // shared-memory tile when chunk keys >= ratio * m
    u32 w_safe;          // |w| <= w_safe may use int32 tile counters
    u32 c2p31 = 0x80000000u, c4 = 4u;  // run-time operands of the p = 2^61-1 row hash
};

struct BatchLaunch {
    int threads;
    int blocks;
    int strategy;
    size_t smem;
};

size_t batched_smem_bytes(int rows_per_item, int max_log2m);
cudaError_t launch_cs_update_batched(int prime, const BatchArgs& a, const BatchLaunch& l,
                                     cudaStream_t s, int* occupancy);

}  // namespace msk
