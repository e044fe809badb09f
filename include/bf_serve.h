/*
 * bf_serve.h -- continuous-batching request loop over resident operators
 * (see bf.h for conventions).
 *
 * A server keeps several factored operators resident on one GPU (admitted
 * against an HBM budget) and serves matvec requests g = K_op f for them.  A
 * scheduler thread forms batches continuously: whenever one of its S slots (a
 * stream with its own staging buffers and workspace) is free, it takes the
 * oldest pending request's operator and packs as many of that operator's
 * pending requests as fit (column-concatenated right-hand sides) into one
 * apply (a priority slot takes the oldest small request and packs up to the
 * small-batch size); requests that arrive while slots are busy wait for the next free
 * slot; the S slots' batches run concurrently on the device.  A batch of 2..64
 * requests and at most 1024 right-hand sides moves each request's rows in one
 * contiguous host<->device copy and interleaves the column blocks on the
 * device; larger batches copy each request's column block with a strided 2-D
 * copy (slow for narrow blocks).  Each request's
 * result is bit-identical to applying its operator to that request alone
 * (columns never mix).  The paper has no serving component: this rests on its
 * observation (Sec. 1 footnote) that the factorisation is built once and then
 * applied to many vectors.
 */
#ifndef BF_SERVE_H
#define BF_SERVE_H

#include "bf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_server bf_server;

typedef struct {
    int n_slots;            /* concurrent batches on the device (default 4)                     */
    int64_t hbm_budget;     /* bytes for resident factors + slot buffers (0: 60% of free memory) */
    int64_t max_batch_rhs;  /* right-hand sides per batch at most (default 256)                  */
    int precision;          /* BF_PREC_F32 (default) or BF_PREC_F64                              */
    int per_request;        /* 1: no batching, one request per apply (the plain per-request form) */
    int device;             /* CUDA device (default 0)                                           */
    int n_priority_slots;   /* slots on highest-priority streams that take only small batches
                               (default n_slots / 2; 0: none).  Their kernels' CTAs are
                               scheduled ahead of the other slots', so small requests do not
                               queue behind large applies                                       */
    int64_t small_units;    /* a batch is small if N * (its right-hand sides) <= this
                               (default 2^21)                                                   */
    int method;             /* 0 (default): the butterfly apply for every operator; 1 (auto,
                               BF_PREC_F32 without per_request): Sec. 3's choice per operator --
                               the NUFFT of Eq. tg3 (bf_nufft_prepare / bf_nufft_apply) where the
                               phase is rank 1 on the column halves, the butterfly otherwise     */
    double nufft_eps;       /* tolerance of the NUFFT plans that method 1 prepares (default 1e-6) */
} bf_server_options;

typedef struct {
    int64_t submitted, completed, pending, in_flight;
    int64_t launches;          /* batched applies issued                              */
    double mean_batch_rhs;     /* right-hand sides per apply                          */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit-to-completion latency            */
    double units_per_s;        /* sum N*m of completed requests / wall time since reset */
    double wall_s;             /* seconds since start / last reset                    */
    double device_busy_ms;     /* device time (CUDA events, copies included) covered by at
                                  least one completed batch since reset (the first 2^20
                                  batches after a reset are counted)                   */
    double overlap_ms;         /* ... covered by two or more slots' batches at once     */
    int64_t nufft_operators;   /* operators evaluated by the NUFFT (method 1)          */
} bf_server_stats;

bf_status bf_server_default_options(bf_server_options* opt);
bf_status bf_server_create(const bf_server_options* opt, bf_server** out);

/* Make a factored plan resident (uploads it) if its device factors fit in the
 * remaining HBM budget (else BF_ERR_NOMEM).  The server does not own the
 * plan; it must outlive the server.  *op_id receives the operator index. */
bf_status bf_server_add_operator(bf_server* srv, bf_plan* plan, int* op_id);

/* Allocate the slots (staging + workspace sized from the remaining budget)
 * and start the scheduler thread.  Operators are added before start. */
bf_status bf_server_start(bf_server* srv);

/* Queue G = K_op F for m right-hand sides.  F, G: HOST buffers [N][m]
 * (c64 for F32, c128 for F64; page-locked memory gives the best copy
 * speed); they must stay valid until the request completes.  Non-blocking.
 * Errors: BF_ERR_ARG (bad op, m < 1 or larger than the operator's batch
 * width), BF_ERR_STATE (not started). */
bf_status bf_server_submit(bf_server* srv, int op_id, const void* F, int64_t m, void* G, uint64_t* req_id);

/* Wait until request req_id completes (timeout_ms < 0: no limit); then
 * forget it.  *latency_ms (nullable): submit-to-completion time.
 * Errors: BF_ERR_TIMEOUT, BF_ERR_ARG (unknown id), or the request's own
 * failure status. */
bf_status bf_server_wait(bf_server* srv, uint64_t req_id, double timeout_ms, double* latency_ms);

/* Block until every submitted request has completed (or timeout_ms passed). */
bf_status bf_server_drain(bf_server* srv, double timeout_ms);

bf_status bf_server_get_stats(bf_server* srv, bf_server_stats* stats);
/* Clear latencies and counters (the clock of units_per_s restarts). */
bf_status bf_server_reset_stats(bf_server* srv);

/* Stop the scheduler (in-flight batches finish), free slot buffers.  NULL-safe. */
void bf_server_destroy(bf_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* BF_SERVE_H */
