// Continuous-batching server (include/ms_server.h).
//
// One worker thread owns the GPU work.  Requests are queued in submission
// order.  Whenever fewer than kMaxInflight batches are on the GPU and requests
// are waiting, the worker forms a batch from the head of the queue:
//   - an update is admitted if its payload fits the device staging ring;
//   - a query is evaluated after the batch's updates;
//   - the batch closes before an update to a sketch that already has a query
//     in the batch (so a query sees exactly the updates submitted before it),
//     or at max_batch_requests / max_batch_keys, or when the ring is full.
// Page-locked payloads are read in place by the update kernel (through their
// device alias; no staging copy, no ring space: per-request copies of about a
// megabyte ran at 116 GB/s against the link's 211, whatever the number of copy
// streams).  Pageable payloads are copied host->device on the copy stream; the
// compute stream waits for them, runs the batched update kernel over the batch's jobs
// (one persistent launch), then one F2 kernel per query, and copies the
// answers back.  While one batch computes, the next one's copies proceed.
// Completed batches are retired in order by polling their events; that frees
// their part of the ring and their slots.  Every blocking host wait is bounded
// by timeout_s; no kernel waits on anything.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "ms_batch.h"
#include "ms_batch_internal.h"
#include "ms_internal.h"
#include "ms_server.h"

using msk::u32;
using msk::u64;

namespace {

constexpr int kMaxInflight = 2;      // batches on the GPU at once
constexpr u64 kAlign = 256;          // staging allocations are 256-byte aligned

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

enum { MS_REQ_UPDATE = 0, MS_REQ_QUERY = 1 };

struct Req {
    int kind = MS_REQ_UPDATE;
    int sketch = 0;
    const void* keys = nullptr;
    const int32_t* w = nullptr;
    const void* dkeys = nullptr;  // device alias of page-locked keys (read in place), or NULL
    const int32_t* dw = nullptr;  // ... of page-locked weights
    u64 n = 0;
    bool done = false;
    ms_status status = MS_OK;
    ms_u128 f2 = {0, 0};
    double submit_s = 0, done_s = 0;
};

struct Batch {
    std::vector<u64> tickets;
    std::vector<u64> query_tickets;
    u64 ring_end = 0;       // ring position to release to when done
    u64 keys = 0;
    cudaEvent_t done_ev = nullptr;
    int slot = 0;
};

}  // namespace

struct ms_server {
    ms_server_config cfg;
    std::vector<uint32_t> widths;
    std::vector<cs_sketch*> sketches;
    int prime = 0;
    size_t key_bytes = 8;

    // staging ring (device) in "virtual" positions: [tail, head) is in use
    unsigned char* ring = nullptr;
    u64 ring_cap = 0, head = 0, tail = 0;

    // per in-flight slot: device job table, work counter, F2 answers; pinned mirrors
    msk::BatchJobDev* jobs_dev = nullptr;
    msk::BatchJobDev* jobs_host = nullptr;
    u32* work_counters = nullptr;
    ms_u128* answers_dev = nullptr;
    ms_u128* answers_host = nullptr;
    void* dev_block = nullptr;

    cudaStream_t copy_stream = nullptr, compute_stream = nullptr;
    cudaEvent_t copy_ev[kMaxInflight] = {nullptr, nullptr};
    msk::BatchLaunch launch = {};
    msk::BatchArgs args_proto = {};
    int device = 0;

    std::mutex mu;
    std::condition_variable cv_work;   // worker waits for requests
    std::condition_variable cv_slots;  // submitters wait for a slot; drain waits for done
    std::deque<Req> reqs;              // reqs[ticket - base]
    u64 base = 1;
    std::deque<u64> queue;             // tickets not yet in a batch
    std::deque<Batch> inflight;
    int outstanding = 0;
    bool free_slot[kMaxInflight] = {true, true};
    bool stop = false;
    std::thread worker;

    u64 stat_done = 0, stat_keys = 0, stat_batches = 0;

    Req& at(u64 ticket) { return reqs[ticket - base]; }
};

namespace {

// Reserve `bytes` of the ring (aligned); returns false when it does not fit.
bool ring_alloc(ms_server* s, u64 bytes, u64* off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    if (s->head == s->tail) {  // empty: restart at the ring's physical start
        const u64 r = (s->head + s->ring_cap - 1) / s->ring_cap * s->ring_cap;
        s->head = s->tail = r;
    }
    if (bytes == 0) {
        *off = s->head % s->ring_cap;
        return true;
    }
    u64 phys = s->head % s->ring_cap;
    u64 waste = 0;
    if (phys + bytes > s->ring_cap) waste = s->ring_cap - phys;  // wrap to the start
    if (s->head - s->tail + waste + bytes > s->ring_cap) return false;
    s->head += waste;
    *off = s->head % s->ring_cap;
    s->head += bytes;
    return true;
}

void finish_batch(ms_server* s, Batch& b, ms_status st) {
    const double t = now_s();
    size_t qi = 0;
    for (u64 tk : b.tickets) {
        Req& r = s->at(tk);
        r.done = true;
        r.status = st;
        r.done_s = t;
        if (r.kind == MS_REQ_QUERY && st == MS_OK) {
            r.f2 = s->answers_host[(size_t)b.slot * s->cfg.max_batch_requests + qi];
            ++qi;
        } else if (r.kind == MS_REQ_QUERY) {
            ++qi;
        }
        --s->outstanding;
        ++s->stat_done;
    }
    s->stat_keys += b.keys;
    s->tail = b.ring_end;
    s->free_slot[b.slot] = true;
}

// An update whose keys (and weights, if any) are page-locked is read in place.
bool in_place(const Req& r) { return r.dkeys != nullptr && (r.w == nullptr || r.dw != nullptr); }

// The device alias of a page-locked host buffer (allocated or registered with
// CUDA), or NULL for pageable memory, on device `dev`; the calling thread's
// current device is left as it was.
const void* device_alias(const void* p, int dev) {
    if (!p) return nullptr;
    int old = 0;
    if (cudaGetDevice(&old) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (old != dev && cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaPointerAttributes at;
    const void* d = nullptr;
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess) {
        if (at.type == cudaMemoryTypeHost) d = at.devicePointer;
    } else {
        cudaGetLastError();  // not a pointer CUDA knows: pageable
    }
    if (old != dev) cudaSetDevice(old);
    return d;
}

// Forms and launches one batch from the head of the queue (lock held on entry;
// released around the CUDA calls).  Returns true if a batch was launched.
bool launch_batch(ms_server* s, std::unique_lock<std::mutex>& lk) {
    int slot = -1;
    for (int i = 0; i < kMaxInflight; ++i)
        if (s->free_slot[i]) { slot = i; break; }
    if (slot < 0 || s->queue.empty()) return false;

    Batch b;
    b.slot = slot;
    std::set<int> queried;
    struct Up { u64 ticket, koff, woff; };
    std::vector<Up> ups;
    const size_t kb = s->key_bytes;
    while (!s->queue.empty() && (int)b.tickets.size() < s->cfg.max_batch_requests &&
           b.keys < s->cfg.max_batch_keys) {
        const u64 tk = s->queue.front();
        Req& r = s->at(tk);
        if (r.kind == MS_REQ_UPDATE) {
            if (queried.count(r.sketch)) break;  // it must follow the query: next batch
            u64 koff = 0, woff = 0;
            const u64 h0 = s->head;
            if (!in_place(r)) {
                if (!ring_alloc(s, r.n * kb, &koff)) break;
                if (r.w && !ring_alloc(s, r.n * 4, &woff)) {
                    s->head = h0;  // undo the key reservation
                    break;
                }
            }
            ups.push_back({tk, koff, woff});
            b.keys += r.n;
        } else {
            queried.insert(r.sketch);
            b.query_tickets.push_back(tk);
        }
        b.tickets.push_back(tk);
        s->queue.pop_front();
    }
    if (b.tickets.empty()) return false;
    b.ring_end = s->head;
    s->free_slot[slot] = false;

    // Everything below only reads requests that no one else writes now.
    std::vector<const Req*> up_reqs;
    for (auto& u : ups) up_reqs.push_back(&s->at(u.ticket));
    std::vector<int> q_sketch;
    for (u64 tk : b.query_tickets) q_sketch.push_back(s->at(tk).sketch);
    lk.unlock();

    ms_status st = MS_OK;
    cudaError_t e = cudaSuccess;
    cudaSetDevice(s->device);
    msk::BatchJobDev* jh = s->jobs_host + (size_t)slot * s->cfg.max_batch_requests;
    u64 items = 0;
    const int rpi = s->args_proto.rows_per_item;
    for (size_t i = 0; i < ups.size() && e == cudaSuccess; ++i) {
        const Req& r = *up_reqs[i];
        cs_sketch* sk = s->sketches[(size_t)r.sketch];
        msk::BatchJobDev& j = jh[i];
        if (in_place(r)) {
            j.keys = r.dkeys;
            j.w = r.dw;
            j.vec_ok = ((uintptr_t)r.dkeys % 16 == 0 && (uintptr_t)r.dw % 16 == 0) ? 1u : 0u;
        } else {
            unsigned char* kd = s->ring + ups[i].koff;
            unsigned char* wd = r.w ? s->ring + ups[i].woff : nullptr;
            if (r.n) e = cudaMemcpyAsync(kd, r.keys, r.n * kb, cudaMemcpyHostToDevice, s->copy_stream);
            if (e == cudaSuccess && r.w && r.n)
                e = cudaMemcpyAsync(wd, r.w, r.n * 4, cudaMemcpyHostToDevice, s->copy_stream);
            j.keys = kd;
            j.w = (const int32_t*)wd;
            j.vec_ok = 1;  // ring offsets are 256-byte aligned
        }
        j.n = r.n;
        j.counters = sk->counters;
        j.coef = sk->coef_dev;
        j.log2m = (u32)sk->log2m;
        j.t = (u32)sk->t;
        j.first_item = (u32)items;
        items += ((r.n + s->args_proto.chunk - 1) / s->args_proto.chunk) *
                 (u64)((sk->t + rpi - 1) / rpi);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->copy_ev[slot], s->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->compute_stream, s->copy_ev[slot], 0);
    if (e == cudaSuccess && !ups.empty()) {
        msk::BatchJobDev* jd = s->jobs_dev + (size_t)slot * s->cfg.max_batch_requests;
        e = cudaMemcpyAsync(jd, jh, ups.size() * sizeof(msk::BatchJobDev), cudaMemcpyHostToDevice,
                            s->compute_stream);
        if (e == cudaSuccess && items > 0) {
            msk::BatchArgs a = s->args_proto;
            a.jobs = jd;
            a.njobs = (int)ups.size();
            a.total_items = (u32)items;
            a.work_counter = s->work_counters + slot * 64;
            e = msk::launch_cs_update_batched(s->prime, a, s->launch, s->compute_stream, nullptr);
        }
    }
    ms_u128* ad = s->answers_dev + (size_t)slot * s->cfg.max_batch_requests;
    for (size_t qi = 0; qi < q_sketch.size() && e == cudaSuccess && st == MS_OK; ++qi)
        st = cs_estimate_f2(s->sketches[(size_t)q_sketch[qi]], ad + qi, nullptr, s->compute_stream);
    if (e == cudaSuccess && st == MS_OK && !q_sketch.empty())
        e = cudaMemcpyAsync(s->answers_host + (size_t)slot * s->cfg.max_batch_requests, ad,
                            q_sketch.size() * sizeof(ms_u128), cudaMemcpyDeviceToHost,
                            s->compute_stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b.done_ev, s->compute_stream);
    if (e != cudaSuccess) st = msi::cuda_fail(e, "ms_server batch");

    lk.lock();
    ++s->stat_batches;
    if (st != MS_OK) {
        if (b.done_ev) cudaEventDestroy(b.done_ev);
        b.done_ev = nullptr;
        finish_batch(s, b, st);
        s->cv_slots.notify_all();
        return true;
    }
    s->inflight.push_back(b);
    return true;
}

// Retires finished batches in order (lock held).  Returns true if any finished.
bool retire(ms_server* s) {
    bool any = false;
    while (!s->inflight.empty()) {
        Batch& b = s->inflight.front();
        cudaError_t q = cudaEventQuery(b.done_ev);
        if (q == cudaErrorNotReady) break;
        ms_status st = (q == cudaSuccess) ? MS_OK : msi::cuda_fail(q, "ms_server batch");
        cudaEventDestroy(b.done_ev);
        finish_batch(s, b, st);
        s->inflight.pop_front();
        any = true;
    }
    if (any) s->cv_slots.notify_all();
    return any;
}

void worker_main(ms_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        retire(s);
        bool launched = false;
        if ((int)s->inflight.size() < kMaxInflight && !s->queue.empty()) launched = launch_batch(s, lk);
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        if (!launched) {
            if (s->inflight.empty() && s->queue.empty())
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else {  // GPU busy: poll its events again shortly
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
    }
}

ms_status submit(ms_server* s, Req r, int try_only, uint64_t* ticket) {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) return MS_ERR_INVALID_ARG;
    if (s->outstanding >= s->cfg.max_inflight) {
        if (try_only) return MS_ERR_BUSY;
        const auto limit = std::chrono::duration<double>(s->cfg.timeout_s);
        if (!s->cv_slots.wait_for(lk, limit, [&] { return s->outstanding < s->cfg.max_inflight; }))
            return MS_ERR_TIMEOUT;
    }
    r.submit_s = now_s();
    s->reqs.push_back(r);
    const u64 tk = s->base + s->reqs.size() - 1;
    s->queue.push_back(tk);
    ++s->outstanding;
    if (ticket) *ticket = tk;
    s->cv_work.notify_one();
    return MS_OK;
}

}  // namespace

extern "C" ms_status ms_server_create(ms_server** out, const ms_server_config* cfg) {
    if (!out || !cfg) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    if ((cfg->mode & ~CS_TWO_POLY) != 0) return MS_ERR_INVALID_ARG;  // no CS_ANY_R here
    if (cfg->num_sketches < 1 || !cfg->m_per_sketch || cfg->staging_bytes < 4096 ||
        cfg->max_inflight < 1 || cfg->max_batch_requests < 1 || cfg->max_batch_keys < 1 ||
        cfg->timeout_s <= 0)
        return MS_ERR_INVALID_ARG;
    const int prime = msi::prime_id(cfg->b, cfg->c);
    if (prime < 0) return MS_ERR_UNSUPPORTED_PRIME;
    ms_server* s = new (std::nothrow) ms_server;
    if (!s) return MS_ERR_OOM;
    s->cfg = *cfg;
    s->widths.assign(cfg->m_per_sketch, cfg->m_per_sketch + cfg->num_sketches);
    s->cfg.m_per_sketch = s->widths.data();
    s->prime = prime;
    s->key_bytes = msi::key_bytes(prime);
    cudaGetDevice(&s->device);

    ms_status st = MS_OK;
    int max_log2m = 1, max_t = cfg->t;
    for (int i = 0; i < cfg->num_sketches && st == MS_OK; ++i) {
        cs_sketch* sk = nullptr;
        st = cs_create(&sk, cfg->t, s->widths[(size_t)i], cfg->k, cfg->b, cfg->c,
                       cfg->seed_base + (uint64_t)i, cfg->mode);
        if (st == MS_OK) {
            s->sketches.push_back(sk);
            max_log2m = std::max(max_log2m, sk->log2m);
        }
    }
    const int R = cfg->max_batch_requests;
    s->ring_cap = cfg->staging_bytes / kAlign * kAlign;
    const size_t jobs_bytes = (size_t)kMaxInflight * R * sizeof(msk::BatchJobDev);
    const size_t ans_bytes = (size_t)kMaxInflight * R * sizeof(ms_u128);
    const size_t wc_bytes = (size_t)kMaxInflight * 64 * sizeof(u32);
    if (st == MS_OK) st = msi::dev_alloc((void**)&s->ring, s->ring_cap);
    if (st == MS_OK) st = msi::dev_alloc(&s->dev_block, jobs_bytes + ans_bytes + wc_bytes);
    cudaError_t e = cudaSuccess;
    if (st == MS_OK) {
        s->jobs_dev = (msk::BatchJobDev*)s->dev_block;
        s->answers_dev = (ms_u128*)((char*)s->dev_block + jobs_bytes);
        s->work_counters = (u32*)((char*)s->dev_block + jobs_bytes + ans_bytes);
        e = cudaMallocHost((void**)&s->jobs_host, jobs_bytes);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&s->answers_host, ans_bytes);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute_stream, cudaStreamNonBlocking);
        for (int i = 0; i < kMaxInflight && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&s->copy_ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) st = msi::cuda_fail(e, "ms_server_create");
    }
    if (st == MS_OK) {
        // Serving batches are small and latency matters: shorter chunks than the
        // throughput default, so a batch of a few updates still spreads over
        // every SM.
        cs_batch_tuning tu;
        cs_batch_default_tuning(&tu);
        tu.chunk_keys = 1u << 16;
        tu.smem_min_ratio = 8;
        const int rpi = std::min(tu.rows_per_item == 0 ? msk::MAX_T : tu.rows_per_item, max_t);
        msk::BatchArgs& a = s->args_proto;
        a.k = cfg->k;
        a.mode = cfg->mode;
        a.rows_per_item = rpi;
        a.chunk = tu.chunk_keys;
        a.smem_min_ratio = tu.smem_min_ratio;
        a.w_safe = (u32)(0x7FFFFFFFull / tu.chunk_keys);
        s->launch.threads = tu.threads;
        s->launch.strategy = tu.strategy;
        s->launch.smem = msk::batched_smem_bytes(rpi, max_log2m);
        int occ = 0, sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        e = msk::launch_cs_update_batched(prime, a, s->launch, nullptr, &occ);
        if (e != cudaSuccess || occ < 1)
            st = e != cudaSuccess ? msi::cuda_fail(e, "ms_server occupancy") : MS_ERR_INVALID_ARG;
        s->launch.blocks = std::max(1, occ) * sms;
    }
    if (st != MS_OK) {
        ms_server_destroy(s);
        return st;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return MS_OK;
}

extern "C" ms_status ms_server_submit_update(ms_server* s, int sketch_id, const void* keys_host,
                                             const int32_t* weights_host, uint64_t n, int try_only,
                                             uint64_t* ticket) {
    msi::TraceRange trace_("ms_server_submit_update");
    if (!s || sketch_id < 0 || sketch_id >= (int)s->sketches.size() || (n && !keys_host))
        return MS_ERR_INVALID_ARG;
    Req r;
    r.kind = MS_REQ_UPDATE;
    r.sketch = sketch_id;
    r.keys = keys_host;
    r.w = weights_host;
    r.n = n;
    if (n) {
        r.dkeys = device_alias(keys_host, s->device);
        r.dw = (const int32_t*)device_alias(weights_host, s->device);
    }
    const u64 need = (n * s->key_bytes + kAlign - 1) / kAlign * kAlign +
                     (weights_host ? (n * 4 + kAlign - 1) / kAlign * kAlign : 0);
    if (!in_place(r) && need > s->ring_cap) return MS_ERR_OUT_OF_RANGE;
    return submit(s, r, try_only, ticket);
}

extern "C" ms_status ms_server_submit_query(ms_server* s, int sketch_id, int try_only,
                                            uint64_t* ticket) {
    msi::TraceRange trace_("ms_server_submit_query");
    if (!s || sketch_id < 0 || sketch_id >= (int)s->sketches.size()) return MS_ERR_INVALID_ARG;
    Req r;
    r.kind = MS_REQ_QUERY;
    r.sketch = sketch_id;
    return submit(s, r, try_only, ticket);
}

extern "C" ms_status ms_server_poll(ms_server* s, uint64_t ticket, ms_request_result* res) {
    if (!s || !res) return MS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket < s->base || ticket >= s->base + s->reqs.size()) return MS_ERR_INVALID_ARG;
    const Req& r = s->at(ticket);
    res->done = r.done ? 1 : 0;
    res->status = r.status;
    res->f2 = r.f2;
    res->submit_s = r.submit_s;
    res->done_s = r.done_s;
    return MS_OK;
}

extern "C" ms_status ms_server_drain(ms_server* s) {
    msi::TraceRange trace_("ms_server_drain");
    if (!s) return MS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto limit = std::chrono::duration<double>(s->cfg.timeout_s);
    s->cv_work.notify_one();
    if (!s->cv_slots.wait_for(lk, limit, [&] { return s->outstanding == 0; })) return MS_ERR_TIMEOUT;
    return MS_OK;
}

extern "C" ms_status ms_server_sketch_counters(ms_server* s, int sketch_id, int64_t* counters_host) {
    if (!s || !counters_host || sketch_id < 0 || sketch_id >= (int)s->sketches.size())
        return MS_ERR_INVALID_ARG;
    ms_status st = ms_server_drain(s);
    if (st != MS_OK) return st;
    const cs_sketch* sk = s->sketches[(size_t)sketch_id];
    cudaError_t e = cudaMemcpy(counters_host, sk->counters, (size_t)sk->t * sk->m * 8,
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MS_OK : msi::cuda_fail(e, "ms_server_sketch_counters");
}

extern "C" ms_status ms_server_stats(ms_server* s, uint64_t* requests_done, uint64_t* keys_done,
                                     uint64_t* batches) {
    if (!s) return MS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (requests_done) *requests_done = s->stat_done;
    if (keys_done) *keys_done = s->stat_keys;
    if (batches) *batches = s->stat_batches;
    return MS_OK;
}

extern "C" ms_status ms_server_destroy(ms_server* s) {
    if (!s) return MS_OK;
    ms_status st = MS_OK;
    if (s->worker.joinable()) {
        st = ms_server_drain(s);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    if (s->compute_stream) cudaStreamSynchronize(s->compute_stream);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    for (auto* sk : s->sketches) cs_destroy(sk);
    for (int i = 0; i < kMaxInflight; ++i)
        if (s->copy_ev[i]) cudaEventDestroy(s->copy_ev[i]);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->compute_stream) cudaStreamDestroy(s->compute_stream);
    if (s->jobs_host) cudaFreeHost(s->jobs_host);
    if (s->answers_host) cudaFreeHost(s->answers_host);
    if (s->dev_block) cudaFree(s->dev_block);
    if (s->ring) cudaFree(s->ring);
    delete s;
    return st;
}

// ------------------------------------------------------------------ load generator

namespace {
struct Sm64 {
    u64 s;
    u64 next() {
        s += 0x9E3779B97F4A7C15ull;
        u64 z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

double percentile(std::vector<double>& v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    size_t i = (size_t)std::min<double>((double)v.size() - 1, std::floor(q * (double)v.size()));
    return v[i];
}
}  // namespace

extern "C" ms_status ms_server_run_load(ms_server* s, const ms_load_spec* sp, ms_load_result* out) {
    msi::TraceRange trace_("ms_server_run_load");
    if (!s || !sp || !out || sp->count < 1 || sp->rate_per_s <= 0 || sp->min_keys < 1 ||
        sp->max_keys < sp->min_keys || !sp->key_pool_host || sp->pool_keys < sp->max_keys ||
        sp->query_fraction < 0 || sp->query_fraction > 1)
        return MS_ERR_INVALID_ARG;
    Sm64 g{sp->seed};
    struct Plan { double at; int kind, sketch; uint64_t off, n; };
    std::vector<Plan> plan((size_t)sp->count);
    double t = 0;
    const double lr = std::log((double)sp->max_keys / (double)sp->min_keys);
    const int S = (int)s->sketches.size();
    for (auto& p : plan) {
        t += -std::log(1.0 - g.unit()) / sp->rate_per_s;
        p.at = t;
        p.kind = g.unit() < sp->query_fraction ? MS_REQ_QUERY : MS_REQ_UPDATE;
        p.sketch = (int)(g.next() % (u64)S);
        p.n = (uint64_t)std::floor(std::exp(g.unit() * lr) * (double)sp->min_keys);
        p.n = std::min<uint64_t>(std::max<uint64_t>(p.n, sp->min_keys), sp->max_keys);
        p.off = (uint64_t)(g.next() % (u64)(sp->pool_keys - p.n + 1));
    }
    std::vector<uint64_t> tickets(plan.size());
    uint64_t b0 = 0;
    ms_server_stats(s, nullptr, nullptr, &b0);
    const double t0 = now_s();
    const unsigned char* pool = (const unsigned char*)sp->key_pool_host;
    for (size_t i = 0; i < plan.size(); ++i) {
        const double target = t0 + plan[i].at;
        while (now_s() < target) {
        }
        ms_status st = plan[i].kind == MS_REQ_QUERY
                           ? ms_server_submit_query(s, plan[i].sketch, 0, &tickets[i])
                           : ms_server_submit_update(s, plan[i].sketch,
                                                     pool + plan[i].off * s->key_bytes, nullptr,
                                                     plan[i].n, 0, &tickets[i]);
        if (st != MS_OK) return st;
    }
    ms_status st = ms_server_drain(s);
    if (st != MS_OK) return st;
    std::vector<double> lu, lq;
    double last = t0;
    uint64_t keys = 0;
    for (size_t i = 0; i < plan.size(); ++i) {
        ms_request_result r;
        ms_server_poll(s, tickets[i], &r);
        if (r.status != MS_OK) return r.status;
        const double lat = (r.done_s - (t0 + plan[i].at)) * 1e3;
        last = std::max(last, r.done_s);
        if (plan[i].kind == MS_REQ_QUERY) {
            lq.push_back(lat);
        } else {
            lu.push_back(lat);
            keys += plan[i].n;
        }
    }
    uint64_t b1 = 0;
    ms_server_stats(s, nullptr, nullptr, &b1);
    out->wall_s = last - t0;
    out->keys = keys;
    out->keys_per_s = out->wall_s > 0 ? (double)keys / out->wall_s : 0.0;
    out->updates = lu.size();
    out->queries = lq.size();
    out->batches = b1 - b0;
    out->update_p50_ms = percentile(lu, 0.50);
    out->update_p99_ms = percentile(lu, 0.99);
    out->query_p50_ms = percentile(lq, 0.50);
    out->query_p99_ms = percentile(lq, 0.99);
    const double mean_n = (double)(sp->max_keys - sp->min_keys) / std::max(lr, 1e-12);
    out->offered_keys_per_s = sp->rate_per_s * (1.0 - sp->query_fraction) * mean_n;
    return MS_OK;
}
