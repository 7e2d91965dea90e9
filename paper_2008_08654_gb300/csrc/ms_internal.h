// Internal host-side state of the library's handles.  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ms.h"
#include "ms_kernels.h"

// A forced launch configuration (fields < 0 or == 0 mean "choose").
struct LaunchOverride {
    int place = -1;
    int strategy = -1;
    int threads = 0;
    int blocks = 0;
    int blocks_per_sm = 0;
    int cluster = 0;
    int replicas = 0;    // PLACE_GLOBAL: use this many of the sketch's replicas
    int aggregate = -1;  // warp aggregation of equal keys (unit weights, global placement)
};

struct cs_sketch {
    int t, k, b, mode, prime, log2m;
    uint32_t m;                   // counters per row in memory (a power of two)
    uint32_t r = 0;               // CS_ANY_R: the number of buckets (<= m); 0 otherwise
    uint64_t c;
    std::vector<msk::u64> words;  // host copy of the coefficients (limbs)
    void* block = nullptr;        // single device allocation holding everything below
    long long* counters = nullptr;    // t * m int64
    msk::u64* coef_dev = nullptr;     // device copy of `words`
    ms_u128* f2_partial = nullptr;    // F2 scratch: t * f2_splits partial sums
    msk::u32* f2_ticket = nullptr;    // F2 scratch: completion ticket
    int f2_splits = 1;
    int* replicas = nullptr;          // update scratch: nrep int32 copies of the counters
    int nrep = 0;                     // (large sketches only; zero between calls)
    // cs_update_host: two staging chunks, a copy stream and its events (lazy)
    void* hstage = nullptr;
    // second-level key table of the de-duplicating update (lazy; empty
    // between calls): 2^glog2 keys, then 2^glog2 int32 counts
    void* gtable = nullptr;
    int glog2 = 0;
    cudaStream_t hcopy = nullptr;
    cudaEvent_t hcopied[2] = {nullptr, nullptr};
    cudaEvent_t hfree[2] = {nullptr, nullptr};
    LaunchOverride launch;
    unsigned long long* hashed = nullptr;  // cs_set_stats: device counter of hashed entries
    msk::LaunchCfg last_cfg = {};
    int last_specialized = 0;
};

namespace msi {
// NVTX tracing (ms_set_tracing / MS_NVTX=1): off by default.  A range is
// pushed only while tracing is on; the NVTX v3 calls are header-only and go
// to a profiler's injection library when one is attached, else nowhere, so
// the library links nothing extra.
bool tracing();
void trace_push(const char* name);
void trace_pop();
struct TraceRange {
    bool on;
    explicit TraceRange(const char* name) : on(tracing()) {
        if (on) trace_push(name);
    }
    ~TraceRange() {
        if (on) trace_pop();
    }
};

ms_status cuda_fail(cudaError_t e, const char* where);
int prime_id(int b, uint64_t c);
int words_per_value(int prime);
size_t key_bytes(int prime);
bool less_than_p(msk::u64 lo, msk::u64 hi, int b, uint64_t c);
void draw_uniform_below_p(int b, uint64_t c, uint64_t seed, int nvals, msk::u64* out);
ms_status dev_alloc(void** p, size_t bytes);
ms_status choose_update_config(const cs_sketch* sk, uint64_t n, bool unit_weights,
                               msk::UpdateArgs& a, msk::LaunchCfg& cfg);
}  // namespace msi
