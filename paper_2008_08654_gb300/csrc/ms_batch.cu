// Host side of the batched plan (include/ms_batch.h): job table, work-item
// numbering, launch shape, CUDA-graph capture, and the autotuner.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <set>
#include <vector>

#include "ms_batch.h"
#include "ms_batch_internal.h"
#include "ms_internal.h"

using msk::u32;
using msk::u64;

struct cs_batch {
    int prime = 0, k = 0, mode = 0;
    uint64_t total_keys = 0;
    void* block = nullptr;
    msk::BatchArgs args = {};
    msk::BatchLaunch launch = {};
    cudaGraphExec_t exec = nullptr;
};

namespace {

ms_status fail(cudaError_t e, const char* where) { return msi::cuda_fail(e, where); }

bool is_pow2(u64 v) { return v && !(v & (v - 1)); }

void destroy_plan(cs_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->block) cudaFree(b->block);
    delete b;
}

}  // namespace

extern "C" ms_status cs_batch_default_tuning(cs_batch_tuning* out) {
    if (!out) return MS_ERR_INVALID_ARG;
    out->threads = 1024;
    out->blocks_per_sm = 0;
    out->chunk_keys = 1u << 19;
    out->smem_min_ratio = 2;
    out->rows_per_item = 0;
    out->strategy = msk::STRAT_POWER_SUM;
    return MS_OK;
}

extern "C" ms_status cs_batch_create(cs_batch** out, const cs_batch_job* jobs_host, int count,
                                     const cs_batch_tuning* tuning, void* stream) {
    if (!out) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!jobs_host || count < 1) return MS_ERR_INVALID_ARG;
    cs_batch_tuning tu;
    if (tuning)
        tu = *tuning;
    else
        cs_batch_default_tuning(&tu);
    if (tu.threads < 32 || tu.threads > 1024 || tu.threads % 32 != 0) return MS_ERR_INVALID_ARG;
    if (!is_pow2(tu.chunk_keys) || tu.chunk_keys < 1024u || tu.chunk_keys > (1u << 24))
        return MS_ERR_INVALID_ARG;
    if (tu.rows_per_item < 0 || tu.rows_per_item > msk::MAX_T || tu.blocks_per_sm < 0)
        return MS_ERR_INVALID_ARG;
    if (tu.strategy != msk::STRAT_HORNER && tu.strategy != msk::STRAT_POWER_SUM)
        return MS_ERR_INVALID_ARG;

    const cs_sketch* s0 = jobs_host[0].sketch;
    if (!s0) return MS_ERR_INVALID_ARG;
    const int rpi_req = tu.rows_per_item == 0 ? msk::MAX_T : tu.rows_per_item;
    std::vector<msk::BatchJobDev> table((size_t)count);
    u64 items = 0, total_keys = 0;
    int max_log2m = 1, max_t = 1;
    for (int j = 0; j < count; ++j) {
        const cs_batch_job& jb = jobs_host[j];
        const cs_sketch* sk = jb.sketch;
        if (!sk || sk->prime != s0->prime || sk->k != s0->k || sk->mode != s0->mode ||
            sk->r != 0)  // power-of-two bucket counts only
            return MS_ERR_INVALID_ARG;
        if (jb.n > 0 && !jb.keys_dev) return MS_ERR_INVALID_ARG;
        const size_t kb = msi::key_bytes(sk->prime);
        if ((uintptr_t)jb.keys_dev % kb || (uintptr_t)jb.weights_dev % 4) return MS_ERR_MISALIGNED;
        msk::BatchJobDev& d = table[(size_t)j];
        d.keys = jb.keys_dev;
        d.w = jb.weights_dev;
        d.n = jb.n;
        d.counters = sk->counters;
        d.coef = sk->coef_dev;
        d.log2m = (u32)sk->log2m;
        d.t = (u32)sk->t;
        d.first_item = (u32)items;
        d.vec_ok = ((uintptr_t)jb.keys_dev % 16 == 0) &&
                   (!jb.weights_dev || (uintptr_t)jb.weights_dev % 16 == 0);
        const u64 chunks = (jb.n + tu.chunk_keys - 1) / tu.chunk_keys;
        const u64 groups = (u64)((sk->t + rpi_req - 1) / rpi_req);
        items += chunks * groups;
        if (items >= 0xFFFFFFFFull) return MS_ERR_INVALID_ARG;
        total_keys += jb.n;
        if (jb.n > 0) {
            max_log2m = std::max(max_log2m, sk->log2m);
            max_t = std::max(max_t, sk->t);
        }
    }
    // Longest streams first: the persistent blocks take work items in table
    // order, so the items handed out last are the short ones and no block is
    // left with a whole chunk after the others have run out of work.
    std::stable_sort(table.begin(), table.end(),
                     [](const msk::BatchJobDev& x, const msk::BatchJobDev& y) { return x.n > y.n; });
    u64 first = 0;
    for (msk::BatchJobDev& d : table) {
        d.first_item = (u32)first;
        first += ((d.n + tu.chunk_keys - 1) / tu.chunk_keys) * (u64)((d.t + rpi_req - 1) / rpi_req);
    }
    const int rpi = std::min(rpi_req, max_t);

    cs_batch* b = new (std::nothrow) cs_batch;
    if (!b) return MS_ERR_OOM;
    b->prime = s0->prime;
    b->k = s0->k;
    b->mode = s0->mode;
    b->total_keys = total_keys;

    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    b->launch.threads = tu.threads;
    b->launch.strategy = tu.strategy;
    b->launch.smem = msk::batched_smem_bytes(rpi, max_log2m);
    if (b->launch.smem > (size_t)optin) {
        destroy_plan(b);
        return MS_ERR_INVALID_ARG;  // the widest sketch's tile does not fit
    }

    const size_t table_bytes = table.size() * sizeof(msk::BatchJobDev);
    const size_t counter_off = (table_bytes + 255) / 256 * 256;
    ms_status st = msi::dev_alloc(&b->block, counter_off + 256);
    if (st != MS_OK) {
        destroy_plan(b);
        return st;
    }
    cudaError_t e = cudaMemcpy(b->block, table.data(), table_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        destroy_plan(b);
        return fail(e, "cs_batch_create");
    }

    msk::BatchArgs& a = b->args;
    a.jobs = (const msk::BatchJobDev*)b->block;
    a.njobs = count;
    a.total_items = (u32)items;
    a.work_counter = (u32*)((char*)b->block + counter_off);
    a.k = s0->k;
    a.mode = s0->mode;
    a.rows_per_item = rpi;
    a.chunk = tu.chunk_keys;
    a.smem_min_ratio = tu.smem_min_ratio;
    a.w_safe = (u32)(0x7FFFFFFFull / tu.chunk_keys);

    int occ = 0;
    e = msk::launch_cs_update_batched(b->prime, a, b->launch, nullptr, &occ);
    if (e != cudaSuccess || occ < 1) {
        destroy_plan(b);
        return e != cudaSuccess ? fail(e, "batched occupancy") : MS_ERR_INVALID_ARG;
    }
    if (tu.blocks_per_sm > 0) occ = std::min(occ, tu.blocks_per_sm);
    u64 blocks = (u64)occ * (u64)sms;
    if (blocks > items) blocks = std::max<u64>(items, 1);
    b->launch.blocks = (int)blocks;

    // capture [reset, kernel] into a graph on a private stream
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = msk::launch_cs_update_batched(b->prime, a, b->launch, cs, nullptr);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        destroy_plan(b);
        return fail(e, "cs_batch_create graph");
    }
    (void)stream;
    *out = b;
    return MS_OK;
}

extern "C" ms_status cs_batch_launch(cs_batch* b, void* stream) {
    msi::TraceRange trace_("cs_batch_launch");
    if (!b || !b->exec) return MS_ERR_INVALID_ARG;
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? MS_OK : fail(e, "cs_batch_launch");
}

extern "C" ms_status cs_batch_launch_direct(cs_batch* b, void* stream) {
    msi::TraceRange trace_("cs_batch_launch_direct");
    if (!b) return MS_ERR_INVALID_ARG;
    cudaError_t e = msk::launch_cs_update_batched(b->prime, b->args, b->launch, (cudaStream_t)stream,
                                                  nullptr);
    return e == cudaSuccess ? MS_OK : fail(e, "cs_batch_launch_direct");
}

extern "C" ms_status cs_batch_destroy(cs_batch* b) {
    destroy_plan(b);
    return MS_OK;
}

extern "C" ms_status cs_batch_info(const cs_batch* b, uint64_t* total_keys, uint32_t* total_items,
                                   int* blocks, int* threads, size_t* smem_bytes) {
    if (!b) return MS_ERR_INVALID_ARG;
    if (total_keys) *total_keys = b->total_keys;
    if (total_items) *total_items = b->args.total_items;
    if (blocks) *blocks = b->launch.blocks;
    if (threads) *threads = b->launch.threads;
    if (smem_bytes) *smem_bytes = b->launch.smem;
    return MS_OK;
}

extern "C" ms_status cs_batch_tune(const cs_batch_job* jobs_host, int count,
                                   const cs_batch_tuning* candidates, int ncand, int reps,
                                   cs_batch_tuning* best, double* times_ms, void* stream) {
    msi::TraceRange trace_("cs_batch_tune");
    if (!jobs_host || count < 1 || !candidates || ncand < 1 || reps < 1 || !best)
        return MS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // save the counters of every sketch involved
    std::vector<cs_sketch*> sketches;
    {
        std::set<cs_sketch*> seen;
        for (int j = 0; j < count; ++j)
            if (jobs_host[j].sketch && seen.insert(jobs_host[j].sketch).second)
                sketches.push_back(jobs_host[j].sketch);
    }
    std::vector<void*> saved(sketches.size(), nullptr);
    ms_status st = MS_OK;
    for (size_t i = 0; i < sketches.size() && st == MS_OK; ++i) {
        const size_t bytes = (size_t)sketches[i]->t * sketches[i]->m * 8;
        st = msi::dev_alloc(&saved[i], bytes);
        if (st == MS_OK) {
            cudaError_t e = cudaMemcpyAsync(saved[i], sketches[i]->counters, bytes,
                                            cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = fail(e, "cs_batch_tune save");
        }
    }
    double best_ms = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c = 0; c < ncand && st == MS_OK; ++c) {
        if (times_ms) times_ms[c] = -1.0;
        cs_batch* plan = nullptr;
        if (cs_batch_create(&plan, jobs_host, count, &candidates[c], stream) != MS_OK) continue;
        std::vector<double> t;
        bool ok = cs_batch_launch(plan, stream) == MS_OK;  // warm-up
        for (int r = 0; r < reps && ok; ++r) {
            cudaEventRecord(e0, s);
            ok = cs_batch_launch(plan, stream) == MS_OK;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms);
        }
        cs_batch_destroy(plan);
        if (!ok || t.empty()) {
            cudaGetLastError();
            continue;
        }
        std::sort(t.begin(), t.end());
        const double med = t[t.size() / 2];
        if (times_ms) times_ms[c] = med;
        if (best_ms < 0 || med < best_ms) {
            best_ms = med;
            *best = candidates[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t i = 0; i < sketches.size(); ++i) {
        if (saved[i]) {
            if (st == MS_OK) {
                cudaError_t e = cudaMemcpyAsync(sketches[i]->counters, saved[i],
                                                (size_t)sketches[i]->t * sketches[i]->m * 8,
                                                cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) st = fail(e, "cs_batch_tune restore");
            }
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    for (void* p : saved)
        if (p) cudaFree(p);
    if (st == MS_OK && e != cudaSuccess) st = fail(e, "cs_batch_tune");
    if (st == MS_OK && best_ms < 0) st = MS_ERR_INVALID_ARG;  // no candidate could run
    return st;
}
