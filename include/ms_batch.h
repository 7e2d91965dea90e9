/*
 * ms_batch.h -- many independent Count Sketches updated in ONE persistent,
 * CUDA-graph-captured kernel launch, with a launch-shape autotuner.
 *
 * Not in the paper: this applies Process(x, Delta) of Algorithm count-sketch
 * (Sec. 1.3) to thousands of sketches at once.  Each sketch keeps its own
 * coefficients, t and m; the arithmetic and the result are exactly those of
 * cs_update (include/ms.h) applied job by job, since integer addition commutes.
 *
 * Conventions are those of include/ms.h.
 */
#ifndef MS_BATCH_H_
#define MS_BATCH_H_

#include "ms.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One update job: a stream (keys, weights, n) applied to one sketch.  Several
 * jobs may name the same sketch; their updates add. */
typedef struct {
    cs_sketch* sketch;
    const void* keys_dev;       /* n keys of the sketch's key type */
    const int32_t* weights_dev; /* n int32 weights, or NULL for unit weights */
    uint64_t n;
} cs_batch_job;

/* Launch shape of a batched plan (one point of the autotuner's search space). */
typedef struct {
    int threads;             /* threads per block: a multiple of 32, 32..1024 */
    int blocks_per_sm;       /* persistent blocks per SM (0 = as many as fit) */
    uint32_t chunk_keys;     /* keys per work item (power of two, 2^10..2^24) */
    uint32_t smem_min_ratio; /* an item uses a shared-memory counter tile when it
                                has >= smem_min_ratio * m keys; smaller items add
                                straight into the int64 counters */
    int rows_per_item;       /* rows of one sketch handled by one work item
                                (0 = all rows) */
    int strategy;            /* 0 = Horner, 1 = power sum (2^61-1, k = 4 only) */
} cs_batch_tuning;

typedef struct cs_batch cs_batch;

/* Built-in launch shape used when `tuning` is NULL: 1024 threads, blocks
 * from occupancy, 2^19-key chunks, shared-memory tiles when a chunk has at
 * least 2 m keys, all rows per item, power sum (the tuner's pick for the
 * 4096-sketch workload on GB300). */
ms_status cs_batch_default_tuning(cs_batch_tuning* out);

/*
 * cs_batch_create -- a reusable plan that applies `count` jobs (host array) in
 * one persistent kernel launch.  All sketches must share the prime, k and mode
 * and have a power-of-two number of buckets (no CS_ANY_R; else INVALID_ARG).
 * The job table is copied to the device; the plan owns a
 * small device allocation (job table and work counter) and a CUDA graph of
 * [work-counter reset, persistent kernel].  The keys, weights and sketches must
 * stay alive while the plan is used.  Errors: INVALID_ARG, MISALIGNED, OOM, CUDA.
 */
ms_status cs_batch_create(cs_batch** out, const cs_batch_job* jobs_host, int count,
                          const cs_batch_tuning* tuning, void* stream);

/* Enqueue the plan on `stream` as a CUDA-graph replay.  Counters are not reset
 * first: every launch adds the jobs' updates once more.  Launches of one plan
 * must not overlap (they share the plan's work counter). */
ms_status cs_batch_launch(cs_batch* batch, void* stream);

/* The same work as two ordinary kernel launches (no graph). */
ms_status cs_batch_launch_direct(cs_batch* batch, void* stream);

ms_status cs_batch_destroy(cs_batch* batch);

/* Plan facts: total keys, work items, persistent blocks and shared memory. */
ms_status cs_batch_info(const cs_batch* batch, uint64_t* total_keys, uint32_t* total_items,
                        int* blocks, int* threads, size_t* smem_bytes);

/*
 * cs_batch_tune -- times every candidate launch shape on the real jobs (`reps`
 * graph replays each, CUDA events on `stream`) and returns the fastest in
 * *best; times_ms (ncand entries, may be NULL) receives each candidate's median
 * milliseconds, or -1 for a candidate that could not launch.  The counters of
 * every sketch named by the jobs are saved first and restored at the end, so
 * tuning leaves them as they were.  Synchronous.
 */
ms_status cs_batch_tune(const cs_batch_job* jobs_host, int count,
                        const cs_batch_tuning* candidates, int ncand, int reps,
                        cs_batch_tuning* best, double* times_ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MS_BATCH_H_ */
