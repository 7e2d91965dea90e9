/*
 * ms.h -- C ABI of the GB300 Mersenne-prime hashing and Count Sketch library.
 *
 * Paper: T. D. Ahle, J. T. B. Knudsen, M. Thorup, "The Power of Hashing with
 * Mersenne Primes" (arXiv 2008.08654).
 *
 * Conventions for every call
 *  - Primes are p = 2^b - c.  Supported (b, c): (31, 1), (61, 1), (89, 1) and
 *    the pseudo-Mersenne (64, 59).  Anything else: MS_ERR_UNSUPPORTED_PRIME.
 *  - Key element type by prime:
 *        (31, 1)            uint32_t
 *        (61, 1), (64, 59)  uint64_t
 *        (89, 1)            ms_u128 (two little-endian 64-bit limbs)
 *    Keys may be any value of their type; a key x is hashed as x mod p, since
 *    the polynomial only depends on x mod p (Sec. 1.2).
 *  - Hash values are canonical residues in [0, p): uint32_t for (31, 1),
 *    uint64_t for (61, 1) and (64, 59), ms_u128 for (89, 1).
 *  - Pointers named *_dev are device pointers (e.g. a torch tensor's
 *    data_ptr); *_host are host pointers.  The caller owns every buffer it
 *    passes; the library owns its opaque handles (ms_hash, cs_sketch,
 *    cs_batch, ms_server) and the device memory inside them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream only enqueue work and return; results
 *    are ready when the stream reaches that point.
 *  - No call throws; each returns an ms_status.  Argument errors are detected
 *    on the host before anything is enqueued, and leave all state unchanged.
 *  - There is no floating point anywhere on these paths: every result is an
 *    exact integer, identical from run to run.
 *  - The library holds no CPU fallback: every computation below runs in its
 *    own CUDA kernels for sm_103a.
 */
#ifndef MS_H_
#define MS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    uint64_t lo, hi;
} ms_u128;

typedef enum {
    MS_OK = 0,
    MS_ERR_INVALID_ARG = 1,       /* null handle/pointer, bad k, t, m, mode, size */
    MS_ERR_UNSUPPORTED_PRIME = 2, /* (b, c) not in the supported list */
    MS_ERR_OUT_OF_RANGE = 3,      /* a value outside a documented domain */
    MS_ERR_OOM = 4,               /* device or host allocation failed */
    MS_ERR_CUDA = 5,              /* a CUDA runtime call failed */
    MS_ERR_TIMEOUT = 6,           /* a bounded wait ran out */
    MS_ERR_BUSY = 7,              /* serving admission is full */
    MS_ERR_MISALIGNED = 8         /* a pointer lacks its element alignment */
} ms_status;

/* Static text for a status code. */
const char* ms_status_str(ms_status s);

/* Text of the last CUDA error seen by this thread inside the library. */
const char* ms_last_cuda_error(void);

/* Library version, e.g. "1.0.0". */
const char* ms_version(void);

/*
 * ms_set_tracing -- NVTX ranges (a tracing aid, not in the paper) around the
 * library's compute and transfer entry points (hashing, division, sketch
 * update / F2 / point query / merge / reset / export / import, batched
 * launches and tuning, server submissions, drain and load runs), named after
 * the call.  Off by default; MS_NVTX=1 in the environment turns it on when the
 * library first checks.  The ranges go to a profiler that injects NVTX (Nsight
 * Systems, Nsight Compute) and cost nothing otherwise; the library needs no
 * NVTX library at run time.  on: 0 or 1.  Returns the previous setting.
 */
int ms_set_tracing(int on);

/* ------------------------------------------------------------------ hashing */

typedef struct ms_hash ms_hash;

/*
 * ms_hash_init -- a random degree-(k-1) polynomial h_a(x) = sum_{i<k} a_i x^i
 * mod p over Z_p (Sec. 1.2, the k-universal family of Carter and Wegman).
 *  k in [1, 8].  The k coefficients are uniform in [0, p), drawn on the host
 *  from SplitMix64 started at `seed` (Steele, Lea & Flood 2014): each takes
 *  ceil(b/64) words (low word first), keeps the low b bits and is redrawn
 *  while >= p.  Coefficients are copied to the device; the handle owns them.
 *  Errors: INVALID_ARG (out null, k out of range), UNSUPPORTED_PRIME, OOM.
 */
ms_status ms_hash_init(ms_hash** out, int k, int b, uint64_t c, uint64_t seed);

/* As ms_hash_init with explicit coefficients a_0..a_{k-1} (host array of k
 * ms_u128).  Each must be < p, else MS_ERR_OUT_OF_RANGE. */
ms_status ms_hash_init_coeffs(ms_hash** out, int k, int b, uint64_t c, const ms_u128* coeffs_host);

/* Copies the k coefficients (a_0 first) to coeffs_host. */
ms_status ms_hash_coeffs(const ms_hash* h, ms_u128* coeffs_host);

/* Parameters of a hash handle; any output pointer may be NULL. */
ms_status ms_hash_params(const ms_hash* h, int* k, int* b, uint64_t* c);

/*
 * ms_hash_eval -- out_dev[j] = h(keys_dev[j]) for j < n (Algorithm Mersenne,
 * Sec. 1.2, with every intermediate kept below 2^b + 2^4 so that keys up to
 * the full key type are allowed, then one final conditional subtraction).
 *  keys_dev: n keys of the prime's key type; out_dev: n hash values of the
 *  prime's hash type.  Both need the natural alignment of their element type.
 *  n == 0 is a no-op.  Errors: INVALID_ARG (null with n > 0), CUDA.
 */
ms_status ms_hash_eval(const ms_hash* h, const void* keys_dev, void* out_dev, size_t n,
                       void* stream);

ms_status ms_hash_destroy(ms_hash* h);

/* ------------------------------------------------------- division and modulus */

/*
 * ms_div -- quotient and remainder of 128-bit values by p = 2^b - c, branch
 * free: Algorithm division-generalized (Sec. 1.5; its correctness range is the
 * theorem of Sec. 4) computes z = floor(v / p) with enough steps to cover all
 * of [0, 2^128): (31,1): 5 steps, (61,1): 3, (89,1): 2, (64,59): 3.  For
 * c = 1 and v < 2^(2b) the first two steps are Algorithm div-simple.
 * Algorithm mod-generalized then gives y = (v + z*c) mod 2^b = v mod p.
 *  v_dev: n ms_u128 inputs (16-byte aligned).
 *  q_dev: n ms_u128 quotients (the quotient of a 128-bit value by 2^64-59 can
 *         exceed 64 bits), or NULL.
 *  r_dev: n remainders, uint64_t for b <= 64 and ms_u128 for (89, 1), or NULL.
 *  Every input value is in range; there is no OUT_OF_RANGE case.
 *  Errors: INVALID_ARG (v null with n > 0, or both outputs null), UNSUPPORTED_PRIME,
 *  MISALIGNED, CUDA.
 */
ms_status ms_div(int b, uint64_t c, const ms_u128* v_dev, ms_u128* q_dev, void* r_dev, size_t n,
                 void* stream);

/* ms_mod -- remainders only: r_dev[j] = v_dev[j] mod p (same types as ms_div). */
ms_status ms_mod(int b, uint64_t c, const ms_u128* v_dev, void* r_dev, size_t n, void* stream);

/*
 * ms_div_wide -- quotient and remainder of wide values by p = 2^b - c, the
 * setting of Table 2 (Sec. 5: 2b-bit values, b up to 1024): Algorithm
 * division-generalized (Sec. 1.5) with ms_div_wide_steps(b, c) steps, which
 * the theorem of Sec. 4 shows cover every v < 2^(2b), then Algorithm
 * mod-generalized.  p need not be prime.
 *  b: 32..1024; c: 1 <= c < 2^32, and c < 2^(b/2) when b <= 64.
 *  v_dev: n values of ceil(2b/64) uint64 limbs each, little-endian, value-major;
 *         the value used is v mod 2^(2b) (bits at and above 2b are ignored).
 *  q_dev: n quotients of ceil((b+1)/64) limbs (floor(v/p) < 2^(b+1)), or NULL.
 *  r_dev: n remainders of ceil(b/64) limbs, or NULL (not both NULL).
 *  All three 8-byte aligned.  n == 0 is a no-op.
 *  Errors: INVALID_ARG (b or c out of range, null buffers), MISALIGNED, CUDA.
 */
ms_status ms_div_wide(int b, uint64_t c, const uint64_t* v_dev, uint64_t* q_dev, uint64_t* r_dev,
                      size_t n, void* stream);

/* Steps ms_div_wide runs for (b, c): 2 for c = 1, else floor(2b / (b - log2 c)) + 1;
 * -1 when c >= 2^(b-1).  Host only. */
int ms_div_wide_steps(int b, uint64_t c);

/* ------------------------------------------------------------- Count Sketch */

typedef struct cs_sketch cs_sketch;

enum {
    CS_TWO_FOR_ONE = 0, /* bucket and sign from ONE hash value (Algorithm h-and-s) */
    CS_TWO_POLY = 1,    /* bucket from one polynomial, sign from a second one */
    CS_ANY_R = 2        /* flag: m need not be a power of two (Sec. 3.3 / Sec. 1.5) */
};

/*
 * cs_create -- a t-row Count Sketch (Algorithm count-sketch, Sec. 1.3) with
 * m counters per row, each row with its own hash function(s) of degree k-1
 * over p = 2^b - c.
 *  t: odd, 1..15 (the F2 estimate is the median of the t row estimates).
 *  m: power of two, 2 <= m <= 2^24, and m < 2^(b-1) so that the bucket bits
 *     and the sign bit are disjoint (Sec. 1.3).
 *  k: 1..8.  mode: CS_TWO_FOR_ONE or CS_TWO_POLY, optionally | CS_ANY_R.
 *  Two-for-one (Algorithm h-and-s): for hash value h of row r,
 *      bucket = h & (m - 1)   (the log2(m) least significant bits)
 *      a      = h >> (b - 1)  (the most significant of the b bits)
 *      sign   = 1 - 2a.
 *  Two-poly: bucket from polynomial P_r as above, a = bit b-1 of Q_r(x).
 *  CS_ANY_R: m is any number of buckets, 2 <= m <= 2^24 (and m <= 2^(b-2)).
 *    c = 1 (Algorithm Mersenne-arb-r, Sec. 3.3): h' = h + 1, j = h' mod
 *      2^(b-1), bucket = floor(m j / 2^(b-1)); in two-for-one mode
 *      a = floor(h' / 2^(b-1)) and sign = 2a - 1 (the sign convention of that
 *      section's text and proofs).
 *    c > 1 (2^64 - 59): bucket = floor(h m / p), the most uniform map of
 *      Sec. 1.5; there is no sign bit to pair with it, so this needs
 *      CS_TWO_POLY (else INVALID_ARG).
 *    With CS_TWO_POLY the sign is always bit b-1 of Q_r(x), as above.
 *    Storage: rows are cs_row_stride = 2^ceil(log2 m) counters wide; the
 *    columns from m on stay zero.  Batched plans and the server take only
 *    power-of-two sketches.
 *  Coefficients: drawn as in ms_hash_init from one SplitMix64 sequence started
 *  at `seed`, in the order row 0 bucket polynomial, row 0 sign polynomial
 *  (two-poly only), row 1 bucket polynomial, ..., each a_0 first.
 *  The t*m int64 counters (row-major) are allocated on the device and zeroed.
 *  Errors: INVALID_ARG, UNSUPPORTED_PRIME, OOM, CUDA.
 */
ms_status cs_create(cs_sketch** out, int t, uint32_t m, int k, int b, uint64_t c, uint64_t seed,
                    int mode);

/* As cs_create with explicit coefficients: t*k (two-for-one) or 2*t*k
 * (two-poly) ms_u128 on the host, in the order described above. */
ms_status cs_create_coeffs(cs_sketch** out, int t, uint32_t m, int k, int b, uint64_t c, int mode,
                           const ms_u128* coeffs_host);

ms_status cs_destroy(cs_sketch* sk);

/* Parameters of a sketch (m as created); any output pointer may be NULL. */
ms_status cs_params(const cs_sketch* sk, int* t, uint32_t* m, int* k, int* b, uint64_t* c,
                    int* mode);

/* Counters per row in memory: m, or 2^ceil(log2 m) for CS_ANY_R sketches.
 * cs_counters, cs_export and cs_import use rows of this width. */
ms_status cs_row_stride(const cs_sketch* sk, uint32_t* stride);

/* Copies the sketch's coefficients (t*k or 2*t*k ms_u128) to the host. */
ms_status cs_coeffs(const cs_sketch* sk, ms_u128* coeffs_host);

/*
 * cs_update -- Process(x, Delta) of Algorithm count-sketch for every (key,
 * weight) of a stream: C[r][bucket_r(x)] += sign_r(x) * Delta for r < t.
 *  keys_dev: n keys of the prime's key type.
 *  weights_dev: n int32 weights, or NULL for unit weights (Delta = 1).
 *  Counters are int64 and add modulo 2^64 (two's complement); integer
 *  addition commutes, so the result does not depend on the order in which
 *  the GPU applies updates.  n == 0 is a no-op.
 *  Errors: INVALID_ARG, CUDA.
 */
ms_status cs_update(cs_sketch* sk, const void* keys_dev, const int32_t* weights_dev, size_t n,
                    void* stream);

/*
 * cs_update_host -- cs_update for a stream held in HOST memory.  The library
 * copies it to the GPU in chunks of 2^24 keys on a copy stream of its own,
 * double-buffered, so the copy of one chunk overlaps the update of the one
 * before; all chunks add into the same counters (the sketch is linear in its
 * stream), so the result equals cs_update on the whole stream.
 *  keys_host: n keys of the prime's key type; weights_host: n int32 weights or
 *  NULL.  Page-locked (pinned) host memory lets the copies run asynchronously;
 *  pageable memory works but each copy then blocks the calling thread.
 *  The work is enqueued on `stream` (the copies wait for the work already on it,
 *  and `stream` waits for the copies): the host buffers must stay valid until
 *  `stream` has been synchronized.
 *  On first use the sketch allocates two staging chunks in device memory
 *  (2 * 2^24 * (key bytes + 4) bytes), a copy stream and four events, kept
 *  until cs_destroy.  Calls on one sketch must not overlap.
 *  Errors: INVALID_ARG, OOM, CUDA.
 */
ms_status cs_update_host(cs_sketch* sk, const void* keys_host, const int32_t* weights_host,
                         size_t n, void* stream);

/*
 * cs_estimate_f2 -- Output of Algorithm count-sketch per row, X_r = sum_i
 * C[r][i]^2 (computed modulo 2^128), and the F2 estimate = the median of the t
 * row values (t odd, so the middle one).  Writes one ms_u128 to out_dev
 * (device pointer, 16-byte aligned).  rows_dev, if not NULL, receives the t
 * row values.
 *  Errors: INVALID_ARG, MISALIGNED, CUDA.
 */
ms_status cs_estimate_f2(const cs_sketch* sk, ms_u128* out_dev, ms_u128* rows_dev, void* stream);

/*
 * cs_estimate_f2_noalloc -- the same F2 estimate (and optional row values) as
 * cs_estimate_f2, computed from a caller's counter array, and allocating
 * nothing.  The paper has no counterpart: this is for callers that cannot
 * call cudaMalloc, such as a serving loop that must not allocate once it is
 * running (a device allocation can block and synchronize the whole device) or
 * code that works inside a memory budget that is already spent.
 *  counters_dev: t*m int64 counters, row-major (for a sketch: cs_counters).
 *  out_dev, rows_dev: as in cs_estimate_f2 (rows_dev may be NULL).
 *  t odd, m a power of two >= 2; t > 15 or m > 2^24 is beyond the scratch
 *  array and returns MS_ERR_OUT_OF_RANGE.
 *  Scratch: one file-scope device array of 15,616 bytes (up to 960 partial
 *  sums and a ticket), which every GPU that loads the library holds until the
 *  process exits.  The first call on a device looks up that array's device
 *  address (once per device, with that device current); make that first call
 *  before any stream capture begins.  The address stays cached for the life of
 *  the process: after a cudaDeviceReset of that device it is stale, as is
 *  every sketch handle made before it, so do not call into the library on a
 *  device after resetting it.  Each call first clears the ticket on
 *  `stream`.  All calls share the one array, so calls that overlap on the GPU
 *  (for example on two streams) race and give wrong results: keep them ordered
 *  on one stream.
 *  Errors: INVALID_ARG, OUT_OF_RANGE, MISALIGNED, CUDA.
 */
ms_status cs_estimate_f2_noalloc(const int64_t* counters_dev, int t, uint32_t m, ms_u128* out_dev,
                                 ms_u128* rows_dev, void* stream);

/*
 * cs_point_query -- the estimate of f_x for each key: median over rows r of
 * sign_r(x) * C[r][bucket_r(x)] (the point-query use of the Count Sketch,
 * Sec. 1.3).  out_dev: n int64.  Errors: INVALID_ARG, CUDA.
 */
ms_status cs_point_query(const cs_sketch* sk, const void* keys_dev, int64_t* out_dev, size_t n,
                         void* stream);

/* Device pointer to the t*m int64 counters (row-major).  Owned by the sketch. */
ms_status cs_counters(const cs_sketch* sk, int64_t** counters_dev);

/* Sets every counter to zero (enqueued on `stream`). */
ms_status cs_reset(cs_sketch* sk, void* stream);

/*
 * cs_merge -- dst += src counter by counter.  A Count Sketch is linear in the
 * stream (Sec. 1.3), so the result is the sketch of the concatenated streams.
 * Both sketches must have identical t, m, k, prime, mode and coefficients,
 * else INVALID_ARG.
 */
ms_status cs_merge(cs_sketch* dst, const cs_sketch* src, void* stream);

/*
 * cs_export / cs_import -- checkpoint a sketch (parameters, coefficients and
 * counters) into a host byte buffer and back.  cs_export with buf == NULL
 * writes the needed size to *size.  Synchronises `stream`.
 */
ms_status cs_export(const cs_sketch* sk, void* buf_host, size_t* size, void* stream);
ms_status cs_import(cs_sketch** out, const void* buf_host, size_t size);

/*
 * cs_set_launch -- pin the launch configuration of later cs_update calls on
 * this sketch (tuning and benchmarking; not in the paper).  Any argument < 0
 * (place, strategy) or == 0 (the others) keeps the library's own choice.
 *  place:    0 = int32 tile in each block's shared memory, 1 = tile split
 *            over a thread-block cluster's distributed shared memory,
 *            2 = global memory: int32 replicas of the counters (block b adds
 *            into replica b mod R, then one kernel adds the replicas into the
 *            int64 counters; a sketch whose tile exceeds 112 KiB owns up to
 *            32 replicas, at most 64 MiB of them), 3 = int64 atomics straight
 *            into the counters.
 *  Default: 0 when the t*m int32 tile fits 112 KiB, else 2.
 *  strategy: 0 = Horner per row (Algorithm Mersenne), 1 = powers of x once per
 *            key, then sum a_i x^i per row (k = 4 with t = 5 or 7, every prime;
 *            for the other primes only with a power-of-two m; other sketches
 *            use Horner); 2 = the power sum as 1, but with a shared-memory
 *            tile in the general kernel (four keys a thread) instead of the
 *            lean one (one key a thread; the default there for every prime
 *            with a power-of-two m, and for 2^61-1 with any m).
 *            All give identical hash values.
 *  threads (multiple of 32, <= 512; default 512, 256 for place 1; the lean
 *  kernel on a stream of two or three rounds of four keys a thread takes one
 *  wave of blocks with the threads sized for equal rounds), blocks
 *  (total), blocks_per_sm (cap), cluster (power of two <= 16, place 1 only),
 *  replicas (power of two <= 32, place 2 only; capped at the replicas the
 *  sketch owns; default 16),
 *  aggregate (0 to 3, default 3; unit weights and place 2 or 3 only):
 *  1 = lanes of a warp holding the same key send one update carrying their
 *  count; 2 = a per-block table of 4096 keys in shared memory (one-word keys:
 *  every prime but 2^89-1): a key the table holds is only counted, and is
 *  hashed once, with its count, when the block ends; the other keys are hashed
 *  128 at a time from a per-warp queue.  A warp whose table takes under 1/8 of
 *  the keys of its 17th to 32nd chunks of 128 stops using it.  3 = as 2, and a
 *  key the block's table misses is counted in a second-level table of 2^21
 *  keys in global memory (24 MiB, allocated by the sketch on first use and
 *  kept, L2-resident) when it owns or can claim one of its two slots there
 *  (the aligned pair its hash picks); after the
 *  update one kernel hashes each key that table holds once, with its count,
 *  and empties it.  The default uses the second level for streams of at least
 *  2^22 keys (3 forces it for any length).  The counters are identical for
 *  every setting (a sketch is linear in the stream).
 * Errors: INVALID_ARG.
 */
ms_status cs_set_launch(cs_sketch* sk, int place, int strategy, int threads, int blocks,
                        int blocks_per_sm, int cluster, int replicas, int aggregate);

/*
 * cs_set_stats -- measurement hook (not in the paper): while `hashed_dev` (a
 * device uint64, 8-byte aligned) is set, every cs_update / cs_update_host on
 * this sketch atomically adds to it the number of entries it hashed with a
 * non-zero count: the keys with a non-zero weight, or with the
 * de-duplication table the distinct (block, key) entries it counted.  Each
 * hashed entry costs t polynomial evaluations and t counter additions.  It adds
 * one atomic per warp per 128 entries.  NULL turns it off.
 * Errors: INVALID_ARG, MISALIGNED.
 */
ms_status cs_set_stats(cs_sketch* sk, uint64_t* hashed_dev);

/* The configuration the most recent cs_update on this sketch launched with;
 * `specialized` is 1 when a compile-time (t, k) kernel served it, 2 when that
 * was the lean one-key-a-thread shared-memory-tile kernel.  Any output
 * pointer may be NULL. */
ms_status cs_last_launch(const cs_sketch* sk, int* place, int* strategy, int* threads, int* blocks,
                         int* cluster, int* smem, int* specialized, int* replicas);

/* ---------------------------------------------------- peak probes */

/*
 * ms_probe_mul128 -- measures this GPU's throughput of independent integer
 * multiplies with a kernel that runs 8 independent chains of `iters` steps per
 * thread on every SM.  Writes operations/s to *rate and the kernel time in ms
 * to *ms.  `sink_dev` (8 bytes) receives a checksum so the work cannot be
 * elided.  Synchronous.
 *  variant 0: one full 64x64->128 product per step (low 64 bits by
 *             multiplication, high 64 bits by __umul64hi) -- the unit the
 *             hashing roofline is counted in.
 *  variant 1: one 32x32->64 multiply-add (mad.wide.u32), the partial product
 *             the limb arithmetic is built of; its multiplicand is the previous
 *             result, so the product cannot be hoisted out of the loop.
 *  variant 2: one dependent 32-bit multiply-add (low word only).
 *  variant 3: one 32-bit integer add (two dependent adds per step, both counted).
 *  variant 4: one 32x32->64 multiply-add (mad.wide.u32) whose multiplicand is
 *             another accumulator's latest value, sixteen accumulators per thread
 *             in cross-coupled pairs (throughput, not latency).
 */
ms_status ms_probe_mul128(int variant, int iters, uint64_t* sink_dev, double* rate, double* ms);

/*
 * ms_probe_red -- measures the throughput of scattered 32-bit atomic additions
 * (red.global.add.s32) into `buf_dev` (`words` int32, a power of two from 32 to
 * 2^31): every thread of a full-occupancy grid adds 1 to 4 * `iters`
 * pseudo-random words.  A buffer the size of the update's replica counters
 * stays in L2, so the rate is the L2's atomic throughput, the unit the global
 * placement's counter updates are bounded by.  Writes additions/s to *rate and
 * the kernel time to *ms; the buffer's words are incremented.  Synchronous.
 * Errors: INVALID_ARG, MISALIGNED, CUDA.
 */
ms_status ms_probe_red(int32_t* buf_dev, size_t words, int iters, double* rate, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* MS_H_ */
