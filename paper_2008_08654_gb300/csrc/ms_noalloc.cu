// cs_estimate_f2_noalloc: the F2 estimate of a caller's counter array without
// any allocation.  The scratch that cs_estimate_f2 keeps inside a sketch handle
// (one 128-bit partial sum per block and a completion ticket) lives here in a
// file-scope device array instead.  Every GPU that loads the library holds this
// array until the process exits, and every call shares it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ms.h"
#include "ms_internal.h"
#include "ms_kernels.h"

namespace {

// At most MAX_T rows x 64 blocks per row partial sums (16 bytes each), then the
// ticket in its own 256-byte line.
constexpr int kMaxSplits = 64;
constexpr size_t kPartialBytes = (size_t)msk::MAX_T * kMaxSplits * 16;  // 15,360 bytes
constexpr size_t kScratchBytes = kPartialBytes + 256;                   // 15,616 bytes

}  // namespace

// The static scratch.  In host code this name is only a handle for
// cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_f2_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void* g_scratch_dev[256];  // per device: device address of g_f2_scratch

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
ms_status scratch_on_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return msi::cuda_fail(e, "cs_estimate_f2_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 256) return MS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_f2_scratch);
        if (e != cudaSuccess || !p)
            return msi::cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                  "cs_estimate_f2_noalloc: cudaGetSymbolAddress");
        g_scratch_dev[dev] = p;
    }
    *out = (unsigned char*)g_scratch_dev[dev];
    return MS_OK;
}

}  // namespace

extern "C" ms_status cs_estimate_f2_noalloc(const int64_t* counters_dev, int t, uint32_t m,
                                            ms_u128* out_dev, ms_u128* rows_dev, void* stream) {
    if (!counters_dev || !out_dev) return MS_ERR_INVALID_ARG;
    if (t < 1 || (t % 2) == 0 || m < 2 || (m & (m - 1)) != 0) return MS_ERR_INVALID_ARG;
    if (t > msk::MAX_T || m > (1u << 24)) return MS_ERR_OUT_OF_RANGE;  // beyond the scratch's size
    if ((uintptr_t)counters_dev % 8 || (uintptr_t)out_dev % 16 || (uintptr_t)rows_dev % 16)
        return MS_ERR_MISALIGNED;
    int splits = 1;  // one block per 4096 counters of a row, at most 64
    while (splits < kMaxSplits && (m / (uint32_t)(splits * 2)) >= 4096) splits *= 2;
    if ((size_t)t * splits * 16 > kPartialBytes) return MS_ERR_OUT_OF_RANGE;

    unsigned char* scratch = nullptr;
    ms_status st = scratch_on_current_device(&scratch);
    if (st != MS_OK) return st;
    msk::u32* ticket = (msk::u32*)(scratch + kPartialBytes);
    cudaStream_t s = (cudaStream_t)stream;
    // The ticket must start at zero; the array keeps whatever the last call left.
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(msk::u32), s);
    if (e != cudaSuccess) return msi::cuda_fail(e, "cs_estimate_f2_noalloc: clear");
    msk::F2Args a;
    a.counters = (const long long*)counters_dev;
    a.t = t;
    a.m = m;
    a.splits = splits;
    a.partial = (ms_u128*)scratch;
    a.ticket = ticket;
    a.out = out_dev;
    a.rows = rows_dev;
    e = msk::launch_cs_f2(a, 512, s);
    if (e != cudaSuccess) return msi::cuda_fail(e, "cs_estimate_f2_noalloc");
    return MS_OK;
}
