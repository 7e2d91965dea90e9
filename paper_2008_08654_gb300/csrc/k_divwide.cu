// Quotient and remainder of wide values by p = 2^b - c (b up to 1024):
// Algorithm division-generalized (Sec. 1.5; step count from the theorem of
// Sec. 4), then Algorithm mod-generalized.
//
// Layout on the GPU: a warp is cut into segments of S lanes (S a power of two,
// S >= the limbs of v); segment s of the warp holds one value, lane l of the
// segment its 64-bit limb l (little-endian), so loads and stores of
// consecutive limbs are coalesced.  Multi-limb additions resolve their carries
// across the segment with two ballots: with per-lane generate g (the 64-bit add
// wrapped) and propagate p (the sum is all ones), the carries into the lanes
// are ((G | P) + G) ^ P, where G and P are the warp's g and p masks with the
// segments' top lanes cleared, so no carry crosses from one value to the next.
// Shifts by b bits are shuffles of whole limbs plus a funnel shift.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ms_internal.h"

namespace {

typedef unsigned long long u64;
typedef unsigned int u32;

// s = a + b across the segment; returns the carry out of the segment's top
// limb (valid in every lane of the segment).
__device__ __forceinline__ u64 seg_add(u64 a, u64 b, u32 top, int S, int seg_base, u32& carry_out) {
    u64 s = a + b;
    const bool g = s < a;
    const bool p = s == ~0ull;
    const u32 G = __ballot_sync(0xffffffffu, g) & ~top;
    const u32 P = __ballot_sync(0xffffffffu, p) & ~top;
    const u32 CI = ((G | P) + G) ^ P;
    const u32 lane = threadIdx.x & 31u;
    const u32 cin = (CI >> lane) & 1u;
    s += cin;
    const u32 co = (u32)(g | (p & (cin != 0)));
    carry_out = __shfl_sync(0xffffffffu, co, seg_base + S - 1);
    return s;
}

// (x + cbit * 2^(64 S)) >> b for a segment value x (cbit: the carry out of the
// top limb, 0 or 1).
__device__ __forceinline__ u64 seg_shr(u64 x, u32 cbit, int b, int S, int l) {
    const int qb = b >> 6, rb = b & 63;
    const u64 lo_s = __shfl_down_sync(0xffffffffu, x, qb, S);
    const u64 hi_s = __shfl_down_sync(0xffffffffu, x, qb + 1, S);
    const u64 lo = (l + qb < S) ? lo_s : (l + qb == S ? (u64)cbit : 0ull);
    const u64 hi = (l + qb + 1 < S) ? hi_s : (l + qb + 1 == S ? (u64)cbit : 0ull);
    return rb ? ((lo >> rb) | (hi << (64 - rb))) : lo;
}

// z * c across the segment (z < 2^(64 S - 64), so no carry leaves it).
__device__ __forceinline__ u64 seg_mul_small(u64 z, u64 c, u32 top, int S, int seg_base, int l) {
    const u64 lo = z * c;
    const u64 hi = __umul64hi(z, c);
    u64 hp = __shfl_up_sync(0xffffffffu, hi, 1, S);
    if (l == 0) hp = 0;
    u32 unused;
    return seg_add(lo, hp, top, S, seg_base, unused);
}

// Each warp handles V groups of 32/S values; the V groups are independent, so
// their shuffle and ballot chains overlap.
template <int V>
__global__ void __launch_bounds__(256) k_divwide(const u64* __restrict__ v, int lv, u64* q, int lq,
                                                 u64* r, int lr, u64 n, int b, u64 c, int steps,
                                                 int S) {
    const int lane = (int)(threadIdx.x & 31u);
    const int l = lane & (S - 1);
    const int seg_base = lane & ~(S - 1);
    const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const u64 per_group = (u64)(32 / S);
    u32 top = 0;
    for (int s = S - 1; s < 32; s += S) top |= 1u << s;
    const int tb = 2 * b;

    u64 x[V], z[V], y[V];
    bool valid[V];
    u64 idx[V];
#pragma unroll
    for (int g = 0; g < V; ++g) {
        idx[g] = (warp * V + g) * per_group + (u64)(lane / S);
        valid[g] = idx[g] < n;
        // v mod 2^(2b): limbs at or above bit 2b are cleared
        u64 xv = (valid[g] && l < lv) ? __ldcs(v + idx[g] * (u64)lv + l) : 0ull;
        if (64 * l >= tb)
            xv = 0;
        else if (64 * (l + 1) > tb)
            xv &= (1ull << (tb - 64 * l)) - 1ull;
        x[g] = xv;
    }
    // v' = v + c;  z = v' >> b
    u64 vp[V];
    u32 co_vp[V];
#pragma unroll
    for (int g = 0; g < V; ++g) {
        vp[g] = seg_add(x[g], l == 0 ? c : 0ull, top, S, seg_base, co_vp[g]);
        z[g] = seg_shr(vp[g], co_vp[g], b, S, l);
    }
    // z = (z c + v') >> b, steps - 1 times (z c = z when c = 1)
    for (int it = 1; it < steps; ++it) {
#pragma unroll
        for (int g = 0; g < V; ++g) {
            const u64 zc = c == 1 ? z[g] : seg_mul_small(z[g], c, top, S, seg_base, l);
            u32 co;
            const u64 t = seg_add(zc, vp[g], top, S, seg_base, co);
            z[g] = seg_shr(t, co | co_vp[g], b, S, l);
        }
    }
    // y = (v + z c) mod 2^b
#pragma unroll
    for (int g = 0; g < V; ++g) {
        const u64 zc = c == 1 ? z[g] : seg_mul_small(z[g], c, top, S, seg_base, l);
        u32 unused;
        u64 yv = seg_add(x[g], zc, top, S, seg_base, unused);
        if (64 * l >= b)
            yv = 0;
        else if (64 * (l + 1) > b)
            yv &= (1ull << (b - 64 * l)) - 1ull;
        y[g] = yv;
    }
#pragma unroll
    for (int g = 0; g < V; ++g) {
        if (valid[g]) {
            if (q && l < lq) q[idx[g] * (u64)lq + l] = z[g];
            if (r && l < lr) r[idx[g] * (u64)lr + l] = y[g];
        }
    }
}

constexpr int kDivWideV = 4;

// ---------------------------------------------------------------------------
// Limb-aligned b (b = 64 NB: the Table 2 sizes from 64 to 1024): one value per
// thread, limbs in registers, so a shift by b is a renaming of limbs and the
// carries ride the integer adds.  A block's values are contiguous in memory;
// they are staged through shared memory with coalesced 8-byte accesses (one
// padding limb per value keeps the per-thread reads free of bank conflicts),
// and the quotients and remainders leave the same way.
constexpr int kAlignedThreads = 128;

template <int NB>
__global__ void __launch_bounds__(kAlignedThreads) k_divwide_aligned(const u64* __restrict__ v,
                                                                     u64* q, u64* r, u64 n, u64 c,
                                                                     int steps) {
    constexpr int L = 2 * NB;       // limbs of v
    constexpr int LQ = NB + 1;      // limbs of the quotient (< 2^(b+1))
    constexpr int LDS = L + 1;      // padded stride in shared memory
    extern __shared__ u64 stage[];  // kAlignedThreads * LDS limbs
    const u64 base = (u64)blockIdx.x * kAlignedThreads;
    const int nv = (int)(n - base < (u64)kAlignedThreads ? n - base : (u64)kAlignedThreads);

    for (int e = threadIdx.x; e < nv * L; e += kAlignedThreads)
        stage[(e / L) * LDS + (e % L)] = __ldcs(v + base * L + e);
    __syncthreads();

    const int i = threadIdx.x;
    u64 x[L];
#pragma unroll
    for (int j = 0; j < L; ++j) x[j] = i < nv ? stage[i * LDS + j] : 0ull;

    // v' = v + c, with its carry out of the top limb
    u64 vp[L];
    u64 carry = c;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const unsigned __int128 s = (unsigned __int128)x[j] + carry;
        vp[j] = (u64)s;
        carry = (u64)(s >> 64);
    }
    const u64 cv = carry;
    // z = v' >> b
    u64 z[LQ];
#pragma unroll
    for (int j = 0; j < NB; ++j) z[j] = vp[NB + j];
    z[NB] = cv;
    // z = (z c + v') >> b, steps - 1 times
    for (int it = 1; it < steps; ++it) {
        u64 t[L];
        u64 cy = 0;
        if (c == 1) {
#pragma unroll
            for (int j = 0; j < L; ++j) {
                const unsigned __int128 s = (unsigned __int128)vp[j] + (j < LQ ? z[j] : 0ull) + cy;
                t[j] = (u64)s;
                cy = (u64)(s >> 64);
            }
        } else {
            u64 mcarry = 0;  // z c, limb by limb (c < 2^32), added into v'
#pragma unroll
            for (int j = 0; j < L; ++j) {
                u64 zc = 0;
                if (j <= LQ) {
                    const unsigned __int128 pr =
                        (unsigned __int128)(j < LQ ? z[j] : 0ull) * c + mcarry;
                    zc = (u64)pr;
                    mcarry = (u64)(pr >> 64);
                }
                const unsigned __int128 s = (unsigned __int128)vp[j] + zc + cy;
                t[j] = (u64)s;
                cy = (u64)(s >> 64);
            }
        }
        cy += cv;  // the carry of v' itself (the sum stays below 2^(2b+1))
#pragma unroll
        for (int j = 0; j < NB; ++j) z[j] = t[NB + j];
        z[NB] = cy;
    }
    // y = (v + z c) mod 2^b
    u64 y[NB];
    {
        u64 cy = 0, mcarry = 0;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            u64 zc;
            if (c == 1) {
                zc = z[j];
            } else {
                const unsigned __int128 pr = (unsigned __int128)z[j] * c + mcarry;
                zc = (u64)pr;
                mcarry = (u64)(pr >> 64);
            }
            const unsigned __int128 s = (unsigned __int128)x[j] + zc + cy;
            y[j] = (u64)s;
            cy = (u64)(s >> 64);
        }
    }

    // quotients (LQ limbs) then remainders (NB limbs), staged and stored coalesced
    __syncthreads();
    if (q) {
#pragma unroll
        for (int j = 0; j < LQ; ++j) stage[i * LDS + j] = z[j];
        __syncthreads();
        for (int e = threadIdx.x; e < nv * LQ; e += kAlignedThreads)
            q[base * LQ + e] = stage[(e / LQ) * LDS + (e % LQ)];
        __syncthreads();
    }
    if (r) {
#pragma unroll
        for (int j = 0; j < NB; ++j) stage[i * LDS + j] = y[j];
        __syncthreads();
        for (int e = threadIdx.x; e < nv * NB; e += kAlignedThreads)
            r[base * NB + e] = stage[(e / NB) * LDS + (e % NB)];
    }
}

template <int NB>
cudaError_t launch_aligned(const u64* v, u64* q, u64* r, u64 n, u64 c, int steps,
                           cudaStream_t stream) {
    const size_t smem = (size_t)kAlignedThreads * (2 * NB + 1) * 8;
    auto kern = k_divwide_aligned<NB>;
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const u64 blocks = (n + kAlignedThreads - 1) / kAlignedThreads;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, kAlignedThreads, smem, stream>>>(v, q, r, n, c, steps);
    return cudaGetLastError();
}

// 32 <= b < 64: v < 2^(2b) fits 128 bits, so one thread does the whole
// division in unsigned __int128 (v + c cannot overflow), reading one or two
// limbs and writing one limb of quotient (< 2^(b+1) <= 2^64) and remainder.
__global__ void __launch_bounds__(256) k_divwide_narrow(const u64* __restrict__ v, int lv, u64* q,
                                                        u64* r, u64 n, int b, u64 c, int steps) {
    typedef unsigned __int128 u128;
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u128 x = (u128)__ldcs(v + i * (u64)lv);
    if (lv == 2) x |= (u128)__ldcs(v + i * (u64)lv + 1) << 64;
    x &= (((u128)1) << (2 * b)) - 1;  // v mod 2^(2b)
    const u128 vp = x + c;
    u128 z = vp >> b;
    for (int it = 1; it < steps; ++it) z = (z * c + vp) >> b;
    if (q) q[i] = (u64)z;
    if (r) r[i] = (u64)((x + z * c) & ((((u128)1) << b) - 1));
}

int limbs(int bits) { return (bits + 63) / 64; }

}  // namespace

// Steps of Algorithm division-generalized that cover every v < 2^(2b) (the
// theorem of Sec. 4): c = 1 divides q = 2^b, so 2 steps reach x <= 2^(2b) - 1;
// otherwise x < (2^b / c)^n suffices, i.e. n (b - log2 c) >= 2b, and one step
// is added as a margin against rounding in log2 (extra steps leave the result
// unchanged).
extern "C" int ms_div_wide_steps(int b, uint64_t c) {
    if (b < 2 || c < 1) return -1;
    if (c == 1) return 2;
    const long double lc = log2l((long double)c);
    if (lc >= (long double)b - 1) return -1;
    return (int)floorl(2.0L * b / ((long double)b - lc)) + 1;
}

extern "C" ms_status ms_div_wide(int b, uint64_t c, const uint64_t* v_dev, uint64_t* q_dev,
                                 uint64_t* r_dev, size_t n, void* stream) {
    msi::TraceRange trace_("ms_div_wide");
    if (b < 32 || b > 1024 || c < 1 || c >= (1ull << 32) || (c > 1 && (uint64_t)b <= 64 &&
                                                              c >= (1ull << (b / 2))))
        return MS_ERR_INVALID_ARG;
    if (n == 0) return MS_OK;
    if (!v_dev || (!q_dev && !r_dev)) return MS_ERR_INVALID_ARG;
    if (((uintptr_t)v_dev | (uintptr_t)q_dev | (uintptr_t)r_dev) & 7u) return MS_ERR_MISALIGNED;
    const int steps = ms_div_wide_steps(b, c);
    if (steps < 1 || steps > 64) return MS_ERR_INVALID_ARG;
    if (b < 64) {  // the whole value fits 128 bits: one value per thread
        const u64 blocks = (n + 255) / 256;
        if (blocks > 0x7FFFFFFFull) return MS_ERR_INVALID_ARG;
        k_divwide_narrow<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
            (const u64*)v_dev, limbs(2 * b), (u64*)q_dev, (u64*)r_dev, (u64)n, b, (u64)c, steps);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? MS_OK : msi::cuda_fail(e, "ms_div_wide");
    }
    const int nb = b / 64;
    if (b % 64 == 0 && (nb & (nb - 1)) == 0) {  // 64..1024, a power of two limbs: one value per thread
        const u64* vv = (const u64*)v_dev;
        u64 *qq = (u64*)q_dev, *rr = (u64*)r_dev;
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaSuccess;
        switch (nb) {
            case 1: e = launch_aligned<1>(vv, qq, rr, (u64)n, (u64)c, steps, st); break;
            case 2: e = launch_aligned<2>(vv, qq, rr, (u64)n, (u64)c, steps, st); break;
            case 4: e = launch_aligned<4>(vv, qq, rr, (u64)n, (u64)c, steps, st); break;
            case 8: e = launch_aligned<8>(vv, qq, rr, (u64)n, (u64)c, steps, st); break;
            default: e = launch_aligned<16>(vv, qq, rr, (u64)n, (u64)c, steps, st); break;
        }
        return e == cudaSuccess ? MS_OK : msi::cuda_fail(e, "ms_div_wide");
    }
    // any other b: the warp-segment kernel
    const int lv = limbs(2 * b), lq = limbs(b + 1), lr = limbs(b);
    // segment: the limbs of v, and of z*c (b + 1 + 32 bits), as a power of two
    int need = lv > limbs(b + 33) ? lv : limbs(b + 33);
    int S = 1;
    while (S < need) S <<= 1;
    if (S < 2) S = 2;
    if (S > 32) return MS_ERR_INVALID_ARG;
    const u64 per_block = (u64)(256 / 32) * kDivWideV * (u64)(32 / S);  // values per block
    const u64 blocks = (n + per_block - 1) / per_block;
    if (blocks > 0x7FFFFFFFull) return MS_ERR_INVALID_ARG;
    k_divwide<kDivWideV><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        (const u64*)v_dev, lv, (u64*)q_dev, lq, (u64*)r_dev, lr, (u64)n, b, (u64)c, steps, S);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MS_OK : msi::cuda_fail(e, "ms_div_wide");
}
