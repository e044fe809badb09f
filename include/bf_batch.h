/*
 * bf_batch.h -- batched uneven apply, CUDA-graph capture and the column-slice
 * autotuner of the butterfly-factorisation library (see bf.h for conventions).
 *
 * A batch applies many operators g_i = K_i f_i (each a plan of bf.h, of its own
 * N_i, with its own m_i right-hand sides).  By default (mode 0, bf_batch_set_mode
 * has the others) it does so in ONE persistent launch: every CTA
 * takes work items from an atomic counter in the order [front tiles of op 0]
 * [back tiles of op 0] [front tiles of op 1] ... (front = V, H levels and
 * switch; back = G levels and U); a back tile of operator i waits (bounded)
 * until all front tiles of i are finished.  Each operator computes exactly
 * what bf_apply(plan_i, BF_PREC_F32, ...) computes, bit for bit.  The paper applies one operator to one vector at a time
 * (Sec. 5); batching is this library's addition, resting on the footnote of
 * Sec. 1 that the precomputed factorisation is reused across many f.
 */
#ifndef BF_BATCH_H
#define BF_BATCH_H

#include "bf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_batch bf_batch;

/* One operator of a batch: G = K F with K = plan (FP32 fused apply).
 * F, G: device, [N][m] c64, caller-owned, must stay valid for the batch's
 * lifetime (launches and graph replays read/write them). */
typedef struct {
    bf_plan* plan;
    const void* F;
    void* G;
    int64_t m;
} bf_batch_item;

/* Build a batch (uploads plans, allocates one workspace per item and the work
 * list).  All plans must share r and device and be unsplit (split == 1).  The
 * batch keeps device addresses of the plans' factors: the plans must stay alive
 * and uploaded, and must not be refactored, while the batch exists.
 * Errors: BF_ERR_ARG, BF_ERR_UNSUPPORTED, BF_ERR_NOMEM, BF_ERR_CUDA. */
bf_status bf_batch_create(const bf_batch_item* items, int n, bf_batch** out);

/* Enqueue the batch on `stream`: a reset of the work counters, then one
 * persistent launch (grid = resident CTAs per SM x SMs). */
bf_status bf_batch_run(bf_batch* batch, void* stream);

/* Capture bf_batch_run into a CUDA graph on `stream` (a created, non-default
 * stream) and instantiate it; bf_batch_replay then launches the graph. */
bf_status bf_batch_capture_graph(bf_batch* batch, void* stream);
bf_status bf_batch_replay(bf_batch* batch, void* stream);

/* Synchronise `stream` and report device-side failures of earlier runs:
 * BF_ERR_TIMEOUT if a back tile stopped waiting for its front tiles. */
bf_status bf_batch_status(bf_batch* batch, void* stream);

/* Total work items, persistent grid size, workspace bytes, shared memory per CTA. */
bf_status bf_batch_get_info(const bf_batch* batch, int64_t* work_items, int* grid, int64_t* ws_bytes,
                            int64_t* smem);

/* Polls a back tile makes before giving up (default 2^24, about 2-4 s). */
bf_status bf_batch_set_spin_limit(bf_batch* batch, long long polls);

/* Test hook for the failure path: with on != 0, back tiles wait for one more
 * front completion than exists, so every wait runs out after the spin limit,
 * the tile is skipped and bf_batch_status reports BF_ERR_TIMEOUT.  G is then
 * not written.  Nothing faults or hangs: each wait is bounded. */
bf_status bf_batch_debug_hold(bf_batch* batch, int on);

/* How the batch runs (the results are bitwise the same either way):
 *   0 (default): one persistent launch over all work items of all operators, a back tile
 *      waiting (bounded) for its operator's fronts -- the form described above;
 *   1: two launches, one over every operator's front tiles and one over every back tile,
 *      one CTA per work item, operators by decreasing work, each launch with its own
 *      shared-memory size and the tile bodies inlined (no waits: bf_batch_debug_hold has
 *      no effect);
 *   2: each operator's own fused apply (the kernels and tile shapes bf_apply uses for it)
 *      on one of four streams forked from and joined to the caller's stream, operators by
 *      decreasing work, each on the stream with the least work so far, so that one
 *      operator's last wave runs beside the next ones' tiles (no waits either).
 * Changing the mode drops a captured graph (capture again).  Errors: BF_ERR_ARG. */
bf_status bf_batch_set_mode(bf_batch* batch, int mode);
bf_status bf_batch_get_mode(const bf_batch* batch, int* mode);
/* Time the three modes on `stream` (one warm-up and three timed runs each; the operators'
 * G are written) and keep the fastest.  *mode_out (nullable) receives it, ms_out
 * (nullable, 2 doubles) the mean milliseconds of modes 0 and 1 (all three:
 * bf_batch_tune_times).  Synchronises the stream; call it before bf_batch_capture_graph. */
bf_status bf_batch_tune(bf_batch* batch, void* stream, int* mode_out, double* ms_out);
/* The mean milliseconds of modes 0, 1, 2 from the last bf_batch_tune (zeros before one):
 * the first min(n, 3) into ms.  Errors: BF_ERR_ARG. */
bf_status bf_batch_tune_times(const bf_batch* batch, double* ms, int n);

void bf_batch_destroy(bf_batch* batch); /* NULL-safe */

/* Choose the level-tile shapes of the FP32 fused apply (the tiling of Algorithm
 * 4.1's levels, Sec. 4) for this plan and m by timing candidates on the GPU:
 * the column-slice width mr (right-hand sides per tile, a power of two), the
 * most levels a pass closes over one tile when long H or G level ranges are
 * split into passes through HBM, the front tiles per CTA, and the T_Omega
 * chunks a back CTA processes together.  The fields are searched one after the
 * other (each against the built-in rule too), 4 timed applies per candidate.
 * Every candidate computes the same result bitwise.  The choice is kept in the
 * plan (bf_apply, bf_apply_host, bf_batch_create and the sharded apply use it).
 * cache_path (nullable): a text cache; an entry for this (N, r, r_alpha,
 * split, m) is used without timing, and new results are appended.
 * *mr_out (nullable) receives the chosen mr.  Allocates temporaries. */
bf_status bf_autotune(bf_plan* plan, int64_t m, const char* cache_path, int* mr_out);

/* The level-tile shapes bf_apply uses for this plan and m (the autotuner's
 * choice, else the built-in rules): mr, the most levels per pass, front tiles
 * per CTA and back chunks per CTA (each pointer nullable).  Errors: BF_ERR_ARG,
 * BF_ERR_STATE (plan not uploaded). */
bf_status bf_autotune_get(const bf_plan* plan, int64_t m, int* mr, int* levels_per_pass, int* tpc_front,
                          int* tpc_back);

/* One right-hand-side block of bf_apply_batched: G = K F, device [N][m] c64,
 * caller-owned, G not aliasing F. */
typedef struct {
    const void* F;
    void* G;
    int64_t m;
} bf_apply_item;

/* One-call batched apply: G_i = K_{plans[i]} F_i for every i < n_items, in one
 * persistent launch on `stream` (FP32 fused apply; the many-vector apply of the
 * precomputed factorisation, Sec. 1 and Sec. 4, for operators of different N).
 * Asynchronous.  The calling thread keeps the batch it built for the last
 * (plans, m) list: a call with the same list reuses its workspace and work list,
 * replacing only the F and G pointers (uploaded on `stream`), so it allocates
 * nothing; a different list rebuilds it (freeing the old one synchronizes the
 * device).  Calls that reuse the kept batch are ordered by the caller (same
 * stream, or the previous call's stream waited on).  Same restrictions as
 * bf_batch_create.  Errors: BF_ERR_ARG (NULL pointers, n_items < 1, m < 1), and
 * those of bf_batch_create and bf_batch_run. */
bf_status bf_apply_batched(bf_plan* const* plans, const bf_apply_item* items, int n_items, void* stream);

/* Free the batch bf_apply_batched keeps for the calling thread (synchronizes the
 * device).  NULL-safe to call when there is none. */
void bf_apply_batched_release(void);

#ifdef __cplusplus
}
#endif
#endif /* BF_BATCH_H */
