/*
 * ms_server.h -- continuous batching of Count Sketch updates and F2 queries
 * over many device-resident sketches.
 *
 * Not in the paper: the serving pattern applied to Process(x, Delta) and
 * Output of Algorithm count-sketch (Sec. 1.3).  Results are exact: a query
 * returns the same 128-bit F2 estimate as cs_estimate_f2 on a sketch that saw
 * exactly the updates submitted to it before the query (per-sketch FIFO),
 * however requests are batched.
 *
 * Conventions are those of include/ms.h.
 */
#ifndef MS_SERVER_H_
#define MS_SERVER_H_

#include "ms.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_server ms_server;

typedef struct {
    int t, k, b;                  /* rows, polynomial degree + 1, prime 2^b - c */
    uint64_t c;
    int mode;                     /* CS_TWO_FOR_ONE or CS_TWO_POLY (no CS_ANY_R) */
    uint64_t seed_base;           /* sketch i is seeded with seed_base + i */
    int num_sketches;
    const uint32_t* m_per_sketch; /* num_sketches widths (host array, copied) */
    uint64_t staging_bytes;       /* device memory for the payloads of admitted
                                     updates (a ring, freed in completion order) */
    int max_inflight;             /* slot limit: admitted, unfinished requests */
    uint64_t max_batch_keys;      /* a batch closes at this many keys ... */
    int max_batch_requests;       /* ... or this many requests */
    double timeout_s;             /* bound on every blocking host wait */
} ms_server_config;

typedef struct {
    int done;             /* 1 when finished */
    ms_status status;     /* status of the request once done */
    ms_u128 f2;           /* query result */
    double submit_s;      /* monotonic host clock at submission, seconds */
    double done_s;        /* monotonic host clock when completion was observed */
} ms_request_result;

/*
 * ms_server_create -- allocates the sketches (zeroed), the staging ring, the
 * job tables, two streams, and starts the worker thread.
 * Errors: INVALID_ARG (bad sizes or sketch parameters), UNSUPPORTED_PRIME,
 * OOM, CUDA.
 */
ms_status ms_server_create(ms_server** out, const ms_server_config* cfg);

/*
 * ms_server_submit_update -- queue n keys (and int32 weights, or NULL for unit
 * weights) for sketch `sketch_id`.  The host buffers are read when the request
 * is admitted into a batch and must stay valid until it is done.  Page-locked
 * buffers (cudaMallocHost, cudaHostRegister, a pinned torch tensor) are read in
 * place by the update kernel and take no staging space; pageable ones are
 * copied into the staging ring.  Blocks while no slot is free (at most
 * timeout_s, then MS_ERR_TIMEOUT); with try_only != 0 returns MS_ERR_BUSY
 * instead.  A pageable update larger than the whole staging ring is rejected
 * with MS_ERR_OUT_OF_RANGE.  *ticket identifies the request.
 */
ms_status ms_server_submit_update(ms_server* s, int sketch_id, const void* keys_host,
                                  const int32_t* weights_host, uint64_t n, int try_only,
                                  uint64_t* ticket);

/* ms_server_submit_query -- queue an F2 estimate of sketch `sketch_id`. */
ms_status ms_server_submit_query(ms_server* s, int sketch_id, int try_only, uint64_t* ticket);

/* Non-blocking: fills *res (res->done tells whether the request finished). */
ms_status ms_server_poll(ms_server* s, uint64_t ticket, ms_request_result* res);

/* Blocks until every submitted request is done (at most timeout_s). */
ms_status ms_server_drain(ms_server* s);

/* Copies sketch i's t*m int64 counters to the host (drains first). */
ms_status ms_server_sketch_counters(ms_server* s, int sketch_id, int64_t* counters_host);

/* Counts since creation: requests done, keys applied, batches launched. */
ms_status ms_server_stats(ms_server* s, uint64_t* requests_done, uint64_t* keys_done,
                          uint64_t* batches);

/* Stops the worker (after draining, bounded by timeout_s) and frees everything. */
ms_status ms_server_destroy(ms_server* s);

/*
 * ms_server_run_load -- an open-loop load generator for measuring a server:
 * `count` requests arrive as a Poisson process of `rate_per_s` requests per
 * second (exponential gaps from SplitMix64 words of `seed`).  A request is a
 * query with probability query_fraction (on a uniform sketch), else an update
 * of floor(exp(U ln(max_keys/min_keys)) * min_keys) keys -- log-uniform in
 * [min_keys, max_keys] -- taken from a random offset of the caller's host key
 * pool (unit weights).  The calling thread submits each request at its
 * arrival time (blocking admission counts as latency), then drains.
 * Latency = completion - scheduled arrival.  Fills the result arrays.
 */
typedef struct {
    uint64_t seed;
    uint64_t count;
    double rate_per_s;
    double query_fraction;
    uint64_t min_keys, max_keys;
    const void* key_pool_host;  /* pool of keys of the server's key type */
    uint64_t pool_keys;         /* must be >= max_keys */
} ms_load_spec;

typedef struct {
    double wall_s;              /* first arrival to last completion */
    double keys_per_s;          /* keys applied / wall_s */
    double update_p50_ms, update_p99_ms;
    double query_p50_ms, query_p99_ms;
    uint64_t updates, queries, keys, batches;
    double offered_keys_per_s;  /* rate_per_s * (1 - query_fraction) * mean size */
} ms_load_result;

ms_status ms_server_run_load(ms_server* s, const ms_load_spec* spec, ms_load_result* out);

#ifdef __cplusplus
}
#endif

#endif /* MS_SERVER_H_ */
