// Host side of the C ABI declared in include/ms.h: argument validation,
// handle ownership, the coefficient draw, launch-configuration choice, and
// error reporting.  Every computation is delegated to the kernels.
#include <atomic>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "ms.h"
#include "ms_internal.h"
#include "ms_kernels.h"

using msk::u32;
using msk::u64;

namespace {
thread_local char g_cuda_err[256] = "";
}  // namespace

// Records the failing call for ms_last_cuda_error() and clears the sticky
// runtime error state where that is possible.
ms_status msi::cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    cudaGetLastError();
    return MS_ERR_CUDA;
}

using msi::cuda_fail;

// Largest int32 counter tile kept in one block's shared memory by default
// (two such blocks fit an SM).
static const size_t kSmemTileBudget = 112 * 1024;
static const int kMaxReplicas = 32;   // replicas a large sketch owns (<= 64 MiB)
static const int kDefaultReplicas = 16;  // replicas a default launch uses
static const int kDedupReplicas = 8;     // ... when the de-duplication table is on
static const int kDedupLog2 = 12;        // de-duplication table: 4096 slots (48 KiB) per block
// Second-level key table: 2^21 slots (24 MiB: keys and int32 counts, resident
// in the L2 beside the replicas), used by de-duplicating updates of at least
// 2^22 keys (aggregate 3 forces it, aggregate 2 turns it off).
static const int kGTableLog2 = 21;
static const uint64_t kGTableMinKeys = 1ull << 22;

namespace {

#define MS_CUDA(call, where)                              \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

namespace msi {

// ------------------------------------------------------------ primes

int prime_id(int b, uint64_t c) {
    if (b == 31 && c == 1) return msk::PRIME_31;
    if (b == 61 && c == 1) return msk::PRIME_61;
    if (b == 89 && c == 1) return msk::PRIME_89;
    if (b == 64 && c == 59) return msk::PRIME_64_59;
    return -1;
}

int words_per_value(int prime) { return prime == msk::PRIME_89 ? 2 : 1; }

size_t key_bytes(int prime) {
    return prime == msk::PRIME_31 ? 4 : prime == msk::PRIME_89 ? 16 : 8;
}

// p as (lo, hi)
void prime_words(int b, uint64_t c, u64* lo, u64* hi) {
    if (b < 64) {
        *lo = (1ull << b) - c;
        *hi = 0;
    } else if (b == 64) {
        *lo = 0ull - c;  // 2^64 - c
        *hi = 0;
    } else {
        // 2^b - c with 64 < b < 128: hi = 2^(b-64) - (c > 0 ? 1 : 0) when c <= 2^64
        *lo = 0ull - c;
        *hi = (1ull << (b - 64)) - 1ull;
    }
}

bool less_than_p(u64 lo, u64 hi, int b, uint64_t c) {
    u64 plo, phi;
    prime_words(b, c, &plo, &phi);
    return hi < phi || (hi == phi && lo < plo);
}

// ------------------------------------------------------------ SplitMix64
//
// Steele, Lea & Flood (OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the
// output is the state passed through the mixing function below.
struct SplitMix64 {
    u64 state;
    u64 next() {
        state += 0x9E3779B97F4A7C15ull;
        u64 z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// nvals values uniform in [0, p) as W limbs each: ceil(b/64) words (low first),
// the low b bits kept, redrawn while >= p.
void draw_uniform_below_p(int b, uint64_t c, uint64_t seed, int nvals, u64* out) {
    SplitMix64 g{seed};
    const int W = b > 64 ? 2 : 1;
    for (int v = 0; v < nvals; ++v) {
        u64 lo, hi;
        do {
            lo = g.next();
            hi = (b > 64) ? g.next() : 0ull;
            if (b < 64) lo &= (1ull << b) - 1ull;
            if (b > 64) hi &= (1ull << (b - 64)) - 1ull;
        } while (!less_than_p(lo, hi, b, c));
        out[v * W] = lo;
        if (W == 2) out[v * W + 1] = hi;
    }
}

// ------------------------------------------------------------ allocation
//
// Host-side fault injection: with MS_FAULT_ALLOC=n in the environment, the
// n-th device allocation made by the library (counting from 1) reports
// MS_ERR_OOM without calling cudaMalloc.
std::mutex g_alloc_mu;
long g_alloc_count = 0;

ms_status dev_alloc(void** p, size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        ++g_alloc_count;
        const char* f = getenv("MS_FAULT_ALLOC");
        if (f && atol(f) == g_alloc_count) {
            *p = nullptr;
            return MS_ERR_OOM;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return MS_ERR_OOM;
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    return MS_OK;
}

// ------------------------------------------------------------ device info

struct DevInfo {
    int sms = 0;
    int smem_optin = 0;
    bool ok = false;
};

DevInfo device_info() {
    static std::mutex mu;
    static DevInfo cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DevInfo{};
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev].ok) {
        DevInfo d;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ==
                cudaSuccess)
            d.ok = true;
        cache[dev] = d;
    }
    return cache[dev];
}

}  // namespace msi

using namespace msi;

// ====================================================================== misc

extern "C" const char* ms_status_str(ms_status s) {
    switch (s) {
        case MS_OK: return "ok";
        case MS_ERR_INVALID_ARG: return "invalid argument";
        case MS_ERR_UNSUPPORTED_PRIME: return "unsupported prime";
        case MS_ERR_OUT_OF_RANGE: return "value out of range";
        case MS_ERR_OOM: return "out of memory";
        case MS_ERR_CUDA: return "CUDA error";
        case MS_ERR_TIMEOUT: return "timeout";
        case MS_ERR_BUSY: return "busy";
        case MS_ERR_MISALIGNED: return "misaligned pointer";
    }
    return "unknown status";
}

extern "C" const char* ms_last_cuda_error(void) { return g_cuda_err; }

extern "C" const char* ms_version(void) { return "1.0.0"; }

// ---------------------------------------------------------------- tracing

static std::atomic<int> g_tracing{-1};  // -1: not yet read from the environment

bool msi::tracing() {
    int v = g_tracing.load(std::memory_order_relaxed);
    if (v < 0) {
        const char* e = getenv("MS_NVTX");
        v = (e && e[0] == '1') ? 1 : 0;
        int expected = -1;
        g_tracing.compare_exchange_strong(expected, v);
        v = g_tracing.load(std::memory_order_relaxed);
    }
    return v == 1;
}

void msi::trace_push(const char* name) { nvtxRangePushA(name); }
void msi::trace_pop() { nvtxRangePop(); }

extern "C" int ms_set_tracing(int on) {
    const int before = msi::tracing() ? 1 : 0;
    g_tracing.store(on ? 1 : 0, std::memory_order_relaxed);
    return before;
}

// ====================================================================== hashing

struct ms_hash {
    int k, b, prime;
    uint64_t c;
    std::vector<u64> words;  // k * W limbs
};

static ms_status hash_make(ms_hash** out, int k, int b, uint64_t c, const u64* words) {
    ms_hash* h = new (std::nothrow) ms_hash;
    if (!h) return MS_ERR_OOM;
    h->k = k;
    h->b = b;
    h->c = c;
    h->prime = prime_id(b, c);
    h->words.assign(words, words + (size_t)k * words_per_value(h->prime));
    *out = h;
    return MS_OK;
}

extern "C" ms_status ms_hash_init(ms_hash** out, int k, int b, uint64_t c, uint64_t seed) {
    if (!out) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    if (k < 1 || k > msk::MAX_K) return MS_ERR_INVALID_ARG;
    const int prime = prime_id(b, c);
    if (prime < 0) return MS_ERR_UNSUPPORTED_PRIME;
    u64 w[msk::MAX_K * 2];
    draw_uniform_below_p(b, c, seed, k, w);
    return hash_make(out, k, b, c, w);
}

extern "C" ms_status ms_hash_init_coeffs(ms_hash** out, int k, int b, uint64_t c,
                                         const ms_u128* coeffs_host) {
    if (!out) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    if (k < 1 || k > msk::MAX_K || !coeffs_host) return MS_ERR_INVALID_ARG;
    const int prime = prime_id(b, c);
    if (prime < 0) return MS_ERR_UNSUPPORTED_PRIME;
    const int W = words_per_value(prime);
    u64 w[msk::MAX_K * 2];
    for (int i = 0; i < k; ++i) {
        if (!less_than_p(coeffs_host[i].lo, coeffs_host[i].hi, b, c)) return MS_ERR_OUT_OF_RANGE;
        w[i * W] = coeffs_host[i].lo;
        if (W == 2) w[i * W + 1] = coeffs_host[i].hi;
    }
    return hash_make(out, k, b, c, w);
}

extern "C" ms_status ms_hash_coeffs(const ms_hash* h, ms_u128* coeffs_host) {
    if (!h || !coeffs_host) return MS_ERR_INVALID_ARG;
    const int W = words_per_value(h->prime);
    for (int i = 0; i < h->k; ++i) {
        coeffs_host[i].lo = h->words[(size_t)i * W];
        coeffs_host[i].hi = W == 2 ? h->words[(size_t)i * W + 1] : 0ull;
    }
    return MS_OK;
}

extern "C" ms_status ms_hash_params(const ms_hash* h, int* k, int* b, uint64_t* c) {
    if (!h) return MS_ERR_INVALID_ARG;
    if (k) *k = h->k;
    if (b) *b = h->b;
    if (c) *c = h->c;
    return MS_OK;
}

extern "C" ms_status ms_hash_eval(const ms_hash* h, const void* keys_dev, void* out_dev, size_t n,
                                  void* stream) {
    msi::TraceRange trace_("ms_hash_eval");
    if (!h) return MS_ERR_INVALID_ARG;
    if (n == 0) return MS_OK;
    if (!keys_dev || !out_dev) return MS_ERR_INVALID_ARG;
    const size_t kb = key_bytes(h->prime);
    if (!aligned(keys_dev, kb) || !aligned(out_dev, h->prime == msk::PRIME_31 ? 4 : kb))
        return MS_ERR_MISALIGNED;
    msk::HashCoef coef;
    memset(&coef, 0, sizeof(coef));
    for (size_t i = 0; i < h->words.size(); ++i) coef.w[i] = h->words[i];
    const bool vec = aligned(keys_dev, 16);
    MS_CUDA(msk::launch_hash_eval(h->prime, keys_dev, out_dev, n, h->k, coef, vec,
                                  (cudaStream_t)stream),
            "ms_hash_eval");
    return MS_OK;
}

extern "C" ms_status ms_hash_destroy(ms_hash* h) {
    delete h;
    return MS_OK;
}

// ====================================================================== division

static ms_status divmod_common(int b, uint64_t c, const ms_u128* v, ms_u128* q, void* r, size_t n,
                               void* stream) {
    const int prime = prime_id(b, c);
    if (prime < 0) return MS_ERR_UNSUPPORTED_PRIME;
    if (n == 0) return MS_OK;
    if (!v || (!q && !r)) return MS_ERR_INVALID_ARG;
    if (!aligned(v, 16) || (q && !aligned(q, 16)) || (r && !aligned(r, b > 64 ? 16 : 8)))
        return MS_ERR_MISALIGNED;
    MS_CUDA(msk::launch_divmod(prime, v, q, r, n, (cudaStream_t)stream), "ms_div");
    return MS_OK;
}

extern "C" ms_status ms_div(int b, uint64_t c, const ms_u128* v_dev, ms_u128* q_dev, void* r_dev,
                            size_t n, void* stream) {
    msi::TraceRange trace_("ms_div");
    return divmod_common(b, c, v_dev, q_dev, r_dev, n, stream);
}

extern "C" ms_status ms_mod(int b, uint64_t c, const ms_u128* v_dev, void* r_dev, size_t n,
                            void* stream) {
    msi::TraceRange trace_("ms_mod");
    if (n > 0 && !r_dev) return MS_ERR_INVALID_ARG;
    return divmod_common(b, c, v_dev, nullptr, r_dev, n, stream);
}

// ====================================================================== sketch

static int ilog2_exact(uint32_t m) {
    if (m == 0 || (m & (m - 1)) != 0) return -1;
    int l = 0;
    while ((1u << l) < m) ++l;
    return l;
}

static void sketch_free_device(cs_sketch* sk) {
    if (sk->block) cudaFree(sk->block);
    sk->block = nullptr;
    if (sk->hcopy) cudaStreamSynchronize(sk->hcopy);
    for (int i = 0; i < 2; ++i) {
        if (sk->hcopied[i]) cudaEventDestroy(sk->hcopied[i]);
        if (sk->hfree[i]) cudaEventDestroy(sk->hfree[i]);
        sk->hcopied[i] = sk->hfree[i] = nullptr;
    }
    if (sk->hcopy) cudaStreamDestroy(sk->hcopy);
    sk->hcopy = nullptr;
    if (sk->hstage) cudaFree(sk->hstage);
    sk->hstage = nullptr;
    if (sk->gtable) cudaFree(sk->gtable);
    sk->gtable = nullptr;
    sk->glog2 = 0;
}

// The second-level key table (allocated on first use, then kept): every key
// slot free (all ones), every count zero.  The drain after each update leaves
// it that way again.
static ms_status ensure_gtable(cs_sketch* sk, int glog2) {
    if (sk->gtable && sk->glog2 == glog2) return MS_OK;
    if (sk->gtable) cudaFree(sk->gtable);
    sk->gtable = nullptr;
    sk->glog2 = 0;
    const size_t slots = (size_t)1 << glog2;
    ms_status st = msi::dev_alloc(&sk->gtable, slots * 12);
    if (st != MS_OK) return st;
    cudaError_t e = cudaMemset(sk->gtable, 0xFF, slots * 8);
    if (e == cudaSuccess) e = cudaMemset((char*)sk->gtable + slots * 8, 0, slots * 4);
    if (e != cudaSuccess) {
        cudaFree(sk->gtable);
        sk->gtable = nullptr;
        return msi::cuda_fail(e, "second-level key table");
    }
    sk->glog2 = glog2;
    return MS_OK;
}

static uint32_t next_pow2(uint32_t m) {
    uint32_t s = 1;
    while (s < m) s <<= 1;
    return s;
}

// m_req: the number of buckets as created (any value for CS_ANY_R); the rows
// are stored m = m_req wide, or 2^ceil(log2 m_req) wide for CS_ANY_R.
static ms_status sketch_make(cs_sketch** out, int t, uint32_t m_req, int k, int b, uint64_t c,
                             int mode, const u64* words) {
    const int prime = prime_id(b, c);
    cs_sketch* sk = new (std::nothrow) cs_sketch;
    if (!sk) return MS_ERR_OOM;
    sk->t = t;
    sk->r = (mode & CS_ANY_R) ? m_req : 0u;
    sk->m = (mode & CS_ANY_R) ? next_pow2(m_req) : m_req;
    sk->log2m = ilog2_exact(sk->m);
    const uint32_t m = sk->m;  // every size below is in rows of the storage width
    sk->k = k;
    sk->b = b;
    sk->c = c;
    sk->mode = mode;
    sk->prime = prime;
    const int nf = (mode & CS_TWO_POLY) ? 2 : 1;
    const size_t nwords = (size_t)t * nf * k * words_per_value(prime);
    sk->words.assign(words, words + nwords);
    sk->f2_splits = 1;
    while (sk->f2_splits < 64 && (m / (uint32_t)(sk->f2_splits * 2)) >= 4096) sk->f2_splits *= 2;

    // Sketches whose int32 tile does not fit the shared-memory budget update
    // through R int32 replicas in global memory (R a power of two <= 32, at
    // most 64 MiB of replicas): block b adds into replica b mod R, which splits
    // the atomic traffic on a hot counter R ways.
    const size_t tile_bytes = (size_t)t * m * 4;
    int nrep = 0;
    if (tile_bytes > kSmemTileBudget) {
        nrep = kMaxReplicas;
        while (nrep > 1 && (size_t)nrep * tile_bytes > (64ull << 20)) nrep /= 2;
        if ((size_t)nrep * tile_bytes > (64ull << 20)) nrep = 0;
    }
    sk->nrep = nrep;

    // one device block: counters | coefficients | F2 partials | F2 ticket | replicas
    const size_t counters_bytes = (size_t)t * m * 8;
    const size_t coef_off = (counters_bytes + 255) / 256 * 256;
    const size_t part_off = coef_off + (nwords * 8 + 255) / 256 * 256;
    const size_t ticket_off = part_off + ((size_t)t * sk->f2_splits * 16 + 255) / 256 * 256;
    const size_t rep_off = ticket_off + 256;
    const size_t total = rep_off + (size_t)nrep * tile_bytes;
    void* blk = nullptr;
    ms_status st = dev_alloc(&blk, total);
    if (st != MS_OK) {
        delete sk;
        return st;
    }
    sk->block = blk;
    sk->counters = (long long*)blk;
    sk->coef_dev = (u64*)((char*)blk + coef_off);
    sk->f2_partial = (ms_u128*)((char*)blk + part_off);
    sk->f2_ticket = (u32*)((char*)blk + ticket_off);
    sk->replicas = nrep ? (int*)((char*)blk + rep_off) : nullptr;
    cudaError_t e = cudaMemcpy(sk->coef_dev, sk->words.data(), nwords * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(sk->counters, 0, counters_bytes);
    if (e == cudaSuccess) e = cudaMemset(sk->f2_ticket, 0, 256);
    if (e == cudaSuccess && nrep) e = cudaMemset(sk->replicas, 0, (size_t)nrep * tile_bytes);
    if (e != cudaSuccess) {
        sketch_free_device(sk);
        delete sk;
        return cuda_fail(e, "cs_create");
    }
    *out = sk;
    return MS_OK;
}

static ms_status validate_sketch_params(int t, uint32_t m, int k, int b, uint64_t c, int mode) {
    if (prime_id(b, c) < 0) return MS_ERR_UNSUPPORTED_PRIME;
    if (t < 1 || t > msk::MAX_T || (t % 2) == 0) return MS_ERR_INVALID_ARG;
    if (k < 1 || k > msk::MAX_K) return MS_ERR_INVALID_ARG;
    if ((mode & ~(CS_TWO_POLY | CS_ANY_R)) != 0) return MS_ERR_INVALID_ARG;
    if (mode & CS_ANY_R) {
        if (m < 2 || m > (1u << 24) || (uint64_t)m > (1ull << (b - 2))) return MS_ERR_INVALID_ARG;
        // floor(h m / p) has no sign bit to pair with (pseudo-Mersenne)
        if (c != 1 && !(mode & CS_TWO_POLY)) return MS_ERR_INVALID_ARG;
        return MS_OK;
    }
    const int l = ilog2_exact(m);
    if (l < 1 || l > 24 || l >= b - 1) return MS_ERR_INVALID_ARG;
    return MS_OK;
}

extern "C" ms_status cs_create(cs_sketch** out, int t, uint32_t m, int k, int b, uint64_t c,
                               uint64_t seed, int mode) {
    if (!out) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    ms_status st = validate_sketch_params(t, m, k, b, c, mode);
    if (st != MS_OK) return st;
    const int nf = (mode & CS_TWO_POLY) ? 2 : 1;
    const int W = words_per_value(prime_id(b, c));
    std::vector<u64> w((size_t)t * nf * k * W);
    draw_uniform_below_p(b, c, seed, t * nf * k, w.data());
    return sketch_make(out, t, m, k, b, c, mode, w.data());
}

extern "C" ms_status cs_create_coeffs(cs_sketch** out, int t, uint32_t m, int k, int b, uint64_t c,
                                      int mode, const ms_u128* coeffs_host) {
    if (!out) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!coeffs_host) return MS_ERR_INVALID_ARG;
    ms_status st = validate_sketch_params(t, m, k, b, c, mode);
    if (st != MS_OK) return st;
    const int nf = (mode & CS_TWO_POLY) ? 2 : 1;
    const int W = words_per_value(prime_id(b, c));
    const int nv = t * nf * k;
    std::vector<u64> w((size_t)nv * W);
    for (int i = 0; i < nv; ++i) {
        if (!less_than_p(coeffs_host[i].lo, coeffs_host[i].hi, b, c)) return MS_ERR_OUT_OF_RANGE;
        w[(size_t)i * W] = coeffs_host[i].lo;
        if (W == 2) w[(size_t)i * W + 1] = coeffs_host[i].hi;
    }
    return sketch_make(out, t, m, k, b, c, mode, w.data());
}

extern "C" ms_status cs_destroy(cs_sketch* sk) {
    if (!sk) return MS_OK;
    sketch_free_device(sk);
    delete sk;
    return MS_OK;
}

extern "C" ms_status cs_params(const cs_sketch* sk, int* t, uint32_t* m, int* k, int* b,
                               uint64_t* c, int* mode) {
    if (!sk) return MS_ERR_INVALID_ARG;
    if (t) *t = sk->t;
    if (m) *m = sk->r ? sk->r : sk->m;
    if (k) *k = sk->k;
    if (b) *b = sk->b;
    if (c) *c = sk->c;
    if (mode) *mode = sk->mode;
    return MS_OK;
}

extern "C" ms_status cs_row_stride(const cs_sketch* sk, uint32_t* stride) {
    if (!sk || !stride) return MS_ERR_INVALID_ARG;
    *stride = sk->m;
    return MS_OK;
}

extern "C" ms_status cs_coeffs(const cs_sketch* sk, ms_u128* coeffs_host) {
    if (!sk || !coeffs_host) return MS_ERR_INVALID_ARG;
    const int W = words_per_value(sk->prime);
    const size_t nv = sk->words.size() / W;
    for (size_t i = 0; i < nv; ++i) {
        coeffs_host[i].lo = sk->words[i * W];
        coeffs_host[i].hi = W == 2 ? sk->words[i * W + 1] : 0ull;
    }
    return MS_OK;
}

// Launch configuration for one cs_update call (see ms_internal.h).
ms_status msi::choose_update_config(const cs_sketch* sk, uint64_t n, bool unit_weights,
                                    msk::UpdateArgs& a, msk::LaunchCfg& cfg) {
    const DevInfo d = device_info();
    if (!d.ok) return cuda_fail(cudaGetLastError(), "device query");
    const LaunchOverride& ov = sk->launch;
    const int nf = (sk->mode & CS_TWO_POLY) ? 2 : 1;
    const size_t coef_bytes = (size_t)sk->t * nf * sk->k * words_per_value(sk->prime) * 8;
    const bool generic = !msk::update_is_specialized(sk->prime, sk->t, sk->k, sk->r);
    const size_t extra = generic ? (coef_bytes + 15) / 16 * 16 : 0;
    const size_t tile_bytes = (size_t)sk->t * sk->m * 4;
    const size_t optin = (size_t)d.smem_optin;

    cfg.threads = ov.threads > 0 ? ov.threads : 256;
    cfg.strategy = ov.strategy >= 0 ? ov.strategy : msk::STRAT_POWER_SUM;
    // strategy 2 (cs_set_launch): the power sum in the general kernel (four
    // keys a thread) rather than the lean shared-memory-tile kernel
    a.keys_per_thread_hint = 0;
    if (cfg.strategy == 2) {
        cfg.strategy = msk::STRAT_POWER_SUM;
        a.keys_per_thread_hint = 4;
    }
    cfg.cluster = 1;
    int place = ov.place;
    bool direct = false;  // PLACE_GLOBAL without replicas
    if (place == 3) {
        place = msk::PLACE_GLOBAL;
        direct = true;
    }
    if (place < 0) place = (tile_bytes + extra <= kSmemTileBudget) ? msk::PLACE_SMEM : msk::PLACE_GLOBAL;
    if (place == msk::PLACE_SMEM && tile_bytes + extra > optin) place = msk::PLACE_GLOBAL;
    if (place == msk::PLACE_DSMEM) {
        int cl = ov.cluster > 0 ? ov.cluster : 0;
        if (cl == 0) {  // smallest cluster whose slice allows 2 blocks per SM, else one that fits
            for (int c = 2; c <= 16; c *= 2)
                if (tile_bytes / c + extra <= 112 * 1024) { cl = c; break; }
            if (cl == 0)
                for (int c = 2; c <= 16; c *= 2)
                    if (tile_bytes / c + extra <= optin) { cl = c; break; }
        }
        if (cl < 2 || (cl & (cl - 1)) != 0 || (uint32_t)cl > sk->m || tile_bytes / cl + extra > optin)
            place = msk::PLACE_GLOBAL;
        else
            cfg.cluster = cl;
    }
    cfg.place = place;
    // 512-thread blocks for the shared-memory tile and global placements (the
    // global one measured 3% faster than 256 on the 2^28-key Zipf sketch; with
    // t = 5, m = 4096 tiles, where shared memory admits two blocks per SM,
    // 512 threads were 6-8% faster than 256 for every prime)
    if (ov.threads <= 0 && place != msk::PLACE_DSMEM) cfg.threads = 512;
    cfg.replicas = 0;
    // With the de-duplication table (unit weights, one-word keys) the hottest
    // keys reach the counters once per block, so fewer replicas suffice (8 vs
    // 16 measured 2% faster on the 2^28-key Zipf sketch, with half the reduce).
    const int aggregate = ov.aggregate >= 0 ? ov.aggregate : 3;
    const bool dedup_wanted = unit_weights && aggregate >= 2 && sk->prime != msk::PRIME_89;
    if (place == msk::PLACE_GLOBAL && !direct && sk->nrep > 0) {
        int r = ov.replicas > 0 ? ov.replicas : (dedup_wanted ? kDedupReplicas : kDefaultReplicas);
        if (r > sk->nrep) r = sk->nrep;
        cfg.replicas = r;
    }
    int lcs = 0;
    while ((1 << lcs) < cfg.cluster) ++lcs;
    cfg.smem = (place == msk::PLACE_GLOBAL ? 0 : tile_bytes / cfg.cluster) + extra;

    a.t = sk->t;
    a.k = sk->k;
    a.log2m = sk->log2m;
    a.mode = sk->mode & CS_TWO_POLY;
    a.arb_r = sk->r;
    a.hashed = sk->hashed;
    a.cluster_log2 = lcs;
    a.coef_dev = sk->coef_dev;
    a.counters = sk->counters;
    a.n = n;
    a.replicas = cfg.replicas ? sk->replicas : nullptr;
    a.replica_mask = cfg.replicas ? (u32)(cfg.replicas - 1) : 0u;
    a.aggregate = aggregate;
    // De-duplication (unit weights, one-word keys, global placement): a table of
    // 12-byte slots and a 12-byte-entry queue per warp follow the coefficients in
    // shared memory.  Re-derived after every change of placement below, so
    // cfg.smem always covers what the kernel will touch.
    auto set_dedup = [&](bool allow) {
        const bool on = allow && dedup_wanted && cfg.place == msk::PLACE_GLOBAL;
        a.dedup_log2 = on ? kDedupLog2 : 0;
        cfg.smem = (cfg.place == msk::PLACE_GLOBAL ? 0 : tile_bytes / cfg.cluster) + extra;
        if (on)
            cfg.smem = (cfg.smem + 15) / 16 * 16 + ((size_t)12 << kDedupLog2) +
                       (size_t)(cfg.threads / 32) * msk::DEDUP_QCAP * 12;
    };
    set_dedup(true);

    // resident capacity (the cluster query needs a grid that is a whole cluster)
    cfg.blocks = cfg.cluster;
    int occ = 0;
    cudaError_t e = msk::query_cs_update_occupancy(sk->prime, a, sk->words.data(), cfg, &occ);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (occ < 1) {
        if (place == msk::PLACE_GLOBAL) return cuda_fail(cudaErrorInvalidConfiguration, "occupancy");
        // fall back to direct global atomics
        cfg.place = msk::PLACE_GLOBAL;
        cfg.cluster = 1;
        cfg.blocks = 1;
        cfg.replicas = sk->nrep < kDefaultReplicas ? sk->nrep : kDefaultReplicas;
        a.cluster_log2 = 0;
        a.replicas = cfg.replicas ? sk->replicas : nullptr;
        a.replica_mask = cfg.replicas ? (u32)(cfg.replicas - 1) : 0u;
        set_dedup(true);
        e = msk::query_cs_update_occupancy(sk->prime, a, sk->words.data(), cfg, &occ);
        if (e != cudaSuccess || occ < 1) return cuda_fail(e, "occupancy");
    }
    // Two waves of resident blocks: the second wave fills the gaps the first
    // leaves as its blocks finish at different times.  With the
    // de-duplication table, one wave: each block's table then sees twice the
    // keys and half as many tables are drained (2^28 Zipf keys: 2.49-2.53 vs
    // 2.52-2.57 ms best of 10 against two waves).
    long long capacity;
    if (cfg.place == msk::PLACE_DSMEM)
        capacity = (long long)occ * cfg.cluster;  // occ = co-resident clusters
    else if (cfg.place == msk::PLACE_GLOBAL && a.dedup_log2)
        capacity = (long long)occ * d.sms;
    else
        capacity = 2ll * occ * d.sms;
    if (ov.blocks_per_sm > 0 && cfg.place != msk::PLACE_DSMEM) {
        long long want = (long long)ov.blocks_per_sm * d.sms;
        if (want < capacity) capacity = want;
    }
    // The lean tile kernel over two or three rounds of four keys a thread:
    // with 512-thread blocks the last round would run on a few of them while
    // the rest of the GPU idles, so one wave of blocks is launched with the
    // threads sized for every thread to take the same number of rounds (2^20
    // keys at t = 5, m = 2^10: 288 threads x 456 blocks, 21.7 against 23.7 us
    // per update; 2^21 keys: 384 x 456, 31.8 against 33.9 us; one round or
    // four and more measured no gain).
    long long balanced_blocks = 0;
    if (ov.threads <= 0 && ov.blocks <= 0 && ov.blocks_per_sm <= 0 && cfg.place == msk::PLACE_SMEM &&
        msk::update_uses_lean_tile(sk->prime, a, cfg.place, cfg.strategy)) {
        const u64 wave = (u64)occ * (u64)d.sms;
        const u64 groups = (n + 3) / 4;
        const u64 rounds = (groups + wave * 512 - 1) / (wave * 512);
        const u64 useful = (n * (u64)sk->t) / ((u64)sk->t * sk->m * 2ull + 1);
        if (rounds >= 2 && rounds <= 3 && useful >= wave) {
            const u64 per_block = (groups + rounds * wave - 1) / (rounds * wave);
            cfg.threads = (int)((per_block + 31) / 32 * 32);
            balanced_blocks = (long long)((groups + rounds * cfg.threads - 1) / (rounds * cfg.threads));
        }
    }
    const u64 per_iter = 4ull * cfg.threads;
    long long need = (long long)((n + per_iter - 1) / per_iter);
    if (balanced_blocks) need = balanced_blocks;
    if (cfg.place != msk::PLACE_GLOBAL) {
        // each tile should see >= 2 updates per counter on average (the tile's
        // zeroing and flush are cheap next to the keys: 2^20 keys at t = 5,
        // m = 2^10 measured 20.3 us per update with 456 blocks, 22.8 us with
        // the 255 that >= 4 updates per counter gave)
        const u64 cells = (u64)sk->t * sk->m;
        long long useful = (long long)((n * (u64)sk->t) / (cells * 2ull / cfg.cluster + 1));
        if (useful < d.sms) useful = d.sms;
        if (useful < need) need = useful;
    }
    long long blocks = need < capacity ? need : capacity;
    if (ov.blocks > 0) blocks = ov.blocks;
    if (blocks < 1) blocks = 1;
    if (cfg.place == msk::PLACE_DSMEM) blocks = (blocks + cfg.cluster - 1) / cfg.cluster * cfg.cluster;
    cfg.blocks = (int)blocks;

    // int32 tile/replica counters: the most keys any one of them can see, times |w|
    const u64 iters = (n + (u64)blocks * per_iter - 1) / ((u64)blocks * per_iter);
    u64 per_tile = iters * per_iter * (u64)cfg.cluster;
    if (cfg.place == msk::PLACE_GLOBAL && cfg.replicas)
        per_tile = iters * per_iter * (((u64)blocks + cfg.replicas - 1) / cfg.replicas);
    a.w_safe = per_tile >= 0x7FFFFFFFull ? 0u : (u32)(0x7FFFFFFFull / (per_tile ? per_tile : 1));
    if (per_tile >= 0x7FFFFFFFull && (cfg.place != msk::PLACE_GLOBAL || cfg.replicas)) {
        // even unit weights could overflow an int32 counter: int64 atomics only
        cfg.place = msk::PLACE_GLOBAL;
        cfg.cluster = 1;
        cfg.replicas = 0;
        a.cluster_log2 = 0;
        a.replicas = nullptr;
        a.replica_mask = 0;
        set_dedup(false);  // per-block counts could overflow int32 too
    }
    // the table's int32 counts hold at most the keys one block sees
    if (a.dedup_log2 && iters * per_iter >= 0x7FFFFFFFull) set_dedup(false);
    // the second-level key table (its int32 counts hold at most n); the
    // caller points gkeys/gcounts at the sketch's table
    a.glog2 = 0;
    a.gkeys = nullptr;
    a.gcounts = nullptr;
    if (a.dedup_log2 && aggregate >= 3 && n < 0x7FFFFFFFull &&
        (ov.aggregate == 3 || n >= kGTableMinKeys))
        a.glog2 = kGTableLog2;
    return MS_OK;
}

// Points an update's arguments at the sketch's second-level table (allocated
// on first use) when the configuration asked for it.
static ms_status attach_gtable(cs_sketch* sk, msk::UpdateArgs& a) {
    if (!a.glog2) return MS_OK;
    ms_status st = ensure_gtable(sk, a.glog2);
    if (st != MS_OK) return st;
    const size_t slots = (size_t)1 << a.glog2;
    a.gkeys = (unsigned long long*)sk->gtable;
    a.gcounts = (int*)((char*)sk->gtable + slots * 8);
    return MS_OK;
}

extern "C" ms_status cs_update(cs_sketch* sk, const void* keys_dev, const int32_t* weights_dev,
                               size_t n, void* stream) {
    msi::TraceRange trace_("cs_update");
    if (!sk) return MS_ERR_INVALID_ARG;
    if (n == 0) return MS_OK;
    if (!keys_dev) return MS_ERR_INVALID_ARG;
    const size_t kb = key_bytes(sk->prime);
    if (!aligned(keys_dev, kb) || (weights_dev && !aligned(weights_dev, 4))) return MS_ERR_MISALIGNED;
    msk::UpdateArgs a;
    memset(&a, 0, sizeof(a));
    msk::LaunchCfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    ms_status st = choose_update_config(sk, n, weights_dev == nullptr, a, cfg);
    if (st != MS_OK) return st;
    a.keys = keys_dev;
    a.weights = weights_dev;
    a.vec_ok = aligned(keys_dev, 16) && (!weights_dev || aligned(weights_dev, 16));
    st = attach_gtable(sk, a);
    if (st != MS_OK) return st;
    int spec = 0;
    MS_CUDA(msk::launch_cs_update(sk->prime, a, sk->words.data(), cfg, (cudaStream_t)stream, &spec),
            "cs_update");
    if (a.glog2)
        MS_CUDA(msk::launch_gtable_drain(sk->prime, a, sk->words.data(), (cudaStream_t)stream),
                "cs_update drain");
    if (a.replicas)
        MS_CUDA(msk::launch_reduce_replicas(sk->counters, sk->replicas, cfg.replicas,
                                            (u64)sk->t * sk->m, (cudaStream_t)stream),
                "cs_update replicas");
    sk->last_cfg = cfg;
    sk->last_specialized = spec;
    return MS_OK;
}

static const uint64_t kHostChunk = 1ull << 24;  // keys per staging chunk of cs_update_host

extern "C" ms_status cs_update_host(cs_sketch* sk, const void* keys_host, const int32_t* weights_host,
                                    size_t n, void* stream) {
    msi::TraceRange trace_("cs_update_host");
    if (!sk) return MS_ERR_INVALID_ARG;
    if (n == 0) return MS_OK;
    if (!keys_host) return MS_ERR_INVALID_ARG;
    const size_t kb = key_bytes(sk->prime);
    const size_t chunk_bytes = (size_t)kHostChunk * (kb + 4);  // keys, then weights
    cudaStream_t st = (cudaStream_t)stream;
    if (!sk->hstage) {
        ms_status a = dev_alloc(&sk->hstage, 2 * chunk_bytes);
        if (a != MS_OK) return a;
        cudaError_t e = cudaStreamCreateWithFlags(&sk->hcopy, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&sk->hcopied[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sk->hfree[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            cudaFree(sk->hstage);
            sk->hstage = nullptr;
            return cuda_fail(e, "cs_update_host setup");
        }
    }
    // one configuration for the whole stream: replica counters are sized for
    // all n keys and reduced once at the end
    msk::UpdateArgs a;
    memset(&a, 0, sizeof(a));
    msk::LaunchCfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    ms_status stt = choose_update_config(sk, n, weights_host == nullptr, a, cfg);
    if (stt != MS_OK) return stt;
    stt = attach_gtable(sk, a);
    if (stt != MS_OK) return stt;
    // the copies start after the work already on `stream` (which may still read
    // the staging chunks of an earlier call)
    MS_CUDA(cudaEventRecord(sk->hfree[0], st), "cs_update_host");
    MS_CUDA(cudaEventRecord(sk->hfree[1], st), "cs_update_host");
    const char* kh = (const char*)keys_host;
    int spec = 0;
    for (uint64_t off = 0, c = 0; off < n; off += kHostChunk, ++c) {
        const int buf = (int)(c & 1);
        const uint64_t len = (n - off) < kHostChunk ? (n - off) : kHostChunk;
        char* kd = (char*)sk->hstage + (size_t)buf * chunk_bytes;
        int32_t* wd = (int32_t*)(kd + (size_t)kHostChunk * kb);
        MS_CUDA(cudaStreamWaitEvent(sk->hcopy, sk->hfree[buf], 0), "cs_update_host");
        MS_CUDA(cudaMemcpyAsync(kd, kh + off * kb, len * kb, cudaMemcpyHostToDevice, sk->hcopy),
                "cs_update_host copy");
        if (weights_host)
            MS_CUDA(cudaMemcpyAsync(wd, weights_host + off, len * 4, cudaMemcpyHostToDevice,
                                    sk->hcopy),
                    "cs_update_host copy");
        MS_CUDA(cudaEventRecord(sk->hcopied[buf], sk->hcopy), "cs_update_host");
        MS_CUDA(cudaStreamWaitEvent(st, sk->hcopied[buf], 0), "cs_update_host");
        a.keys = kd;
        a.weights = weights_host ? wd : nullptr;
        a.n = len;
        a.vec_ok = 1;  // staging chunks are 256-byte aligned
        MS_CUDA(msk::launch_cs_update(sk->prime, a, sk->words.data(), cfg, st, &spec), "cs_update_host");
        MS_CUDA(cudaEventRecord(sk->hfree[buf], st), "cs_update_host");
    }
    if (a.glog2) MS_CUDA(msk::launch_gtable_drain(sk->prime, a, sk->words.data(), st), "cs_update_host drain");
    if (a.replicas)
        MS_CUDA(msk::launch_reduce_replicas(sk->counters, sk->replicas, cfg.replicas,
                                            (u64)sk->t * sk->m, st),
                "cs_update_host replicas");
    sk->last_cfg = cfg;
    sk->last_specialized = spec;
    return MS_OK;
}

extern "C" ms_status cs_estimate_f2(const cs_sketch* sk, ms_u128* out_dev, ms_u128* rows_dev,
                                    void* stream) {
    msi::TraceRange trace_("cs_estimate_f2");
    if (!sk || !out_dev) return MS_ERR_INVALID_ARG;
    if (!aligned(out_dev, 16) || (rows_dev && !aligned(rows_dev, 16))) return MS_ERR_MISALIGNED;
    msk::F2Args a;
    a.counters = sk->counters;
    a.t = sk->t;
    a.m = sk->m;
    a.splits = sk->f2_splits;
    a.partial = sk->f2_partial;
    a.ticket = sk->f2_ticket;
    a.out = out_dev;
    a.rows = rows_dev;
    MS_CUDA(msk::launch_cs_f2(a, 512, (cudaStream_t)stream), "cs_estimate_f2");
    return MS_OK;
}

extern "C" ms_status cs_point_query(const cs_sketch* sk, const void* keys_dev, int64_t* out_dev,
                                    size_t n, void* stream) {
    msi::TraceRange trace_("cs_point_query");
    if (!sk) return MS_ERR_INVALID_ARG;
    if (n == 0) return MS_OK;
    if (!keys_dev || !out_dev) return MS_ERR_INVALID_ARG;
    if (!aligned(keys_dev, key_bytes(sk->prime)) || !aligned(out_dev, 8)) return MS_ERR_MISALIGNED;
    msk::QueryArgs a;
    a.keys = keys_dev;
    a.n = n;
    a.counters = sk->counters;
    a.coef_dev = sk->coef_dev;
    a.t = sk->t;
    a.k = sk->k;
    a.log2m = sk->log2m;
    a.mode = sk->mode & CS_TWO_POLY;
    a.arb_r = sk->r;
    a.out = (long long*)out_dev;
    MS_CUDA(msk::launch_cs_point_query(sk->prime, a, sk->words.data(), (cudaStream_t)stream),
            "cs_point_query");
    return MS_OK;
}

extern "C" ms_status cs_counters(const cs_sketch* sk, int64_t** counters_dev) {
    if (!sk || !counters_dev) return MS_ERR_INVALID_ARG;
    *counters_dev = (int64_t*)sk->counters;
    return MS_OK;
}

extern "C" ms_status cs_reset(cs_sketch* sk, void* stream) {
    msi::TraceRange trace_("cs_reset");
    if (!sk) return MS_ERR_INVALID_ARG;
    MS_CUDA(msk::launch_zero(sk->counters, (u64)sk->t * sk->m * 8, (cudaStream_t)stream), "cs_reset");
    return MS_OK;
}

extern "C" ms_status cs_merge(cs_sketch* dst, const cs_sketch* src, void* stream) {
    msi::TraceRange trace_("cs_merge");
    if (!dst || !src) return MS_ERR_INVALID_ARG;
    if (dst->t != src->t || dst->m != src->m || dst->r != src->r || dst->k != src->k ||
        dst->prime != src->prime || dst->mode != src->mode || dst->words != src->words)
        return MS_ERR_INVALID_ARG;
    if (dst == src) return MS_ERR_INVALID_ARG;
    MS_CUDA(msk::launch_add_counters(dst->counters, src->counters, (u64)dst->t * dst->m,
                                     (cudaStream_t)stream),
            "cs_merge");
    return MS_OK;
}

// checkpoint layout: magic, version, t, m, k, b, c, mode, nwords | words | counters
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t t;
    uint32_t m;
    int32_t k;
    int32_t b;
    int32_t mode;
    uint64_t c;
    uint64_t nwords;
};
const char kMagic[8] = {'M', 'S', 'C', 'S', 'K', 'E', 'T', '1'};
}  // namespace

extern "C" ms_status cs_export(const cs_sketch* sk, void* buf_host, size_t* size, void* stream) {
    msi::TraceRange trace_("cs_export");
    if (!sk || !size) return MS_ERR_INVALID_ARG;
    const size_t need = sizeof(CkptHeader) + sk->words.size() * 8 + (size_t)sk->t * sk->m * 8;
    if (!buf_host) {
        *size = need;
        return MS_OK;
    }
    if (*size < need) {
        *size = need;
        return MS_ERR_INVALID_ARG;
    }
    CkptHeader h;
    memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.t = sk->t;
    h.m = sk->r ? sk->r : sk->m;  // as created; the counters follow in rows of sk->m
    h.k = sk->k;
    h.b = sk->b;
    h.mode = sk->mode;
    h.c = sk->c;
    h.nwords = sk->words.size();
    char* p = (char*)buf_host;
    memcpy(p, &h, sizeof(h));
    memcpy(p + sizeof(h), sk->words.data(), sk->words.size() * 8);
    MS_CUDA(cudaMemcpyAsync(p + sizeof(h) + sk->words.size() * 8, sk->counters,
                            (size_t)sk->t * sk->m * 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream),
            "cs_export");
    MS_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "cs_export");
    *size = need;
    return MS_OK;
}

extern "C" ms_status cs_import(cs_sketch** out, const void* buf_host, size_t size) {
    msi::TraceRange trace_("cs_import");
    if (!out || !buf_host || size < sizeof(CkptHeader)) return MS_ERR_INVALID_ARG;
    *out = nullptr;
    CkptHeader h;
    memcpy(&h, buf_host, sizeof(h));
    if (memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) return MS_ERR_INVALID_ARG;
    ms_status st = validate_sketch_params(h.t, h.m, h.k, h.b, h.c, h.mode);
    if (st != MS_OK) return st;
    const int nf = (h.mode & CS_TWO_POLY) ? 2 : 1;
    const int W = words_per_value(prime_id(h.b, h.c));
    if (h.nwords != (uint64_t)h.t * nf * h.k * W) return MS_ERR_INVALID_ARG;
    const uint32_t stride = (h.mode & CS_ANY_R) ? next_pow2(h.m) : h.m;
    const size_t need = sizeof(h) + h.nwords * 8 + (size_t)h.t * stride * 8;
    if (size < need) return MS_ERR_INVALID_ARG;
    const u64* words = (const u64*)((const char*)buf_host + sizeof(h));
    for (uint64_t i = 0; i < h.nwords / W; ++i)
        if (!less_than_p(words[i * W], W == 2 ? words[i * W + 1] : 0ull, h.b, h.c))
            return MS_ERR_OUT_OF_RANGE;
    cs_sketch* sk = nullptr;
    st = sketch_make(&sk, h.t, h.m, h.k, h.b, h.c, h.mode, words);
    if (st != MS_OK) return st;
    cudaError_t e = cudaMemcpy(sk->counters, (const char*)buf_host + sizeof(h) + h.nwords * 8,
                               (size_t)h.t * stride * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cs_destroy(sk);
        return cuda_fail(e, "cs_import");
    }
    *out = sk;
    return MS_OK;
}

// Tuning hook: force a launch configuration for later cs_update calls on this
// sketch (any field < 0 or 0 keeps the automatic choice).
extern "C" ms_status cs_set_launch(cs_sketch* sk, int place, int strategy, int threads, int blocks,
                                   int blocks_per_sm, int cluster, int replicas, int aggregate) {
    if (!sk) return MS_ERR_INVALID_ARG;
    if (place > 3 || strategy > 2) return MS_ERR_INVALID_ARG;  // 2: power sum, general kernel
    if (threads != 0 && threads != -1 &&
        (threads < 32 || threads > 512 || threads % 32 != 0))
        return MS_ERR_INVALID_ARG;
    if (cluster > 16 || (cluster > 0 && (cluster & (cluster - 1)) != 0)) return MS_ERR_INVALID_ARG;
    if (replicas > 32 || (replicas > 0 && (replicas & (replicas - 1)) != 0) || aggregate > 3)
        return MS_ERR_INVALID_ARG;
    sk->launch.place = place;
    sk->launch.strategy = strategy;
    sk->launch.threads = threads;
    sk->launch.blocks = blocks;
    sk->launch.blocks_per_sm = blocks_per_sm;
    sk->launch.cluster = cluster;
    sk->launch.replicas = replicas;
    sk->launch.aggregate = aggregate;
    return MS_OK;
}

// Measurement hook: later cs_update calls add the entries they hash into
// *hashed_dev (NULL turns it off).
extern "C" ms_status cs_set_stats(cs_sketch* sk, uint64_t* hashed_dev) {
    if (!sk) return MS_ERR_INVALID_ARG;
    if (hashed_dev && !aligned(hashed_dev, 8)) return MS_ERR_MISALIGNED;
    sk->hashed = (unsigned long long*)hashed_dev;
    return MS_OK;
}

// The configuration the last cs_update on this sketch launched with.
extern "C" ms_status cs_last_launch(const cs_sketch* sk, int* place, int* strategy, int* threads,
                                    int* blocks, int* cluster, int* smem, int* specialized,
                                    int* replicas) {
    if (!sk) return MS_ERR_INVALID_ARG;
    if (place)
        *place = (sk->last_cfg.place == msk::PLACE_GLOBAL && sk->last_cfg.replicas == 0)
                     ? 3 : sk->last_cfg.place;
    if (strategy) *strategy = sk->last_cfg.strategy;
    if (threads) *threads = sk->last_cfg.threads;
    if (blocks) *blocks = sk->last_cfg.blocks;
    if (cluster) *cluster = sk->last_cfg.cluster;
    if (smem) *smem = (int)sk->last_cfg.smem;
    if (specialized) *specialized = sk->last_specialized;
    if (replicas) *replicas = sk->last_cfg.replicas;
    return MS_OK;
}

// ====================================================================== probe

extern "C" ms_status ms_probe_mul128(int variant, int iters, uint64_t* sink_dev, double* rate,
                                     double* ms) {
    if (!sink_dev || !rate || !ms || iters < 1 || variant < 0 || variant > 4)
        return MS_ERR_INVALID_ARG;
    MS_CUDA(msk::run_probe_mul128(variant, iters, (u64*)sink_dev, rate, ms), "ms_probe_mul128");
    return MS_OK;
}

extern "C" ms_status ms_probe_red(int32_t* buf_dev, size_t words, int iters, double* rate,
                                  double* ms) {
    if (!buf_dev || !rate || !ms || iters < 1 || words < 32 || words > (1ull << 31) ||
        (words & (words - 1)) != 0)
        return MS_ERR_INVALID_ARG;
    if (!aligned(buf_dev, 4)) return MS_ERR_MISALIGNED;
    MS_CUDA(msk::run_probe_red((int*)buf_dev, (u64)words, iters, rate, ms), "ms_probe_red");
    return MS_OK;
}
