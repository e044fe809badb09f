/*
 * bf_shard.h -- one operator applied by G shards (ranks), each holding 1/G of
 * the rows of F and of G (see bf.h for conventions).
 *
 * The butterfly's levels before the switch depend only on the xi side and the
 * levels after it only on the x side (Sec. 4: a pair (A, B) at level l combines
 * parent(A) with the children of B, Eqs. 2 and 3).  So shard s applies the
 * front half (V, the H levels and the switch, Eqs. 1 and 2 and step 4) to the
 * T_Omega nodes at level L-h under its xi rows, one all-to-all exchanges the
 * switch-level coefficients, and shard d applies the back half (G levels and
 * U, Eqs. 3 and bf3) to the x-nodes at level h over its x rows -- the
 * transpose of a distributed FFT.  The exchange is the caller's (e.g. NCCL
 * all-to-all with equal splits); these calls only launch the two halves.
 *
 * Shard s owns F rows xi in [s N/G, (s+1) N/G) and G rows x in the same range.
 * Buffers (device, c64): F_rows [N/G][m], G_rows [N/G][m], W_send and W_recv
 * [G][chunk] with chunk = *chunk_elems from bf_shard_info; W_send block d goes
 * to shard d, W_recv block s came from shard s.
 *
 * Requirements: the plan is factored, unsplit (split == 1), with a fused FP32
 * kernel for its r; G a power of two with G <= 2^l1 and G <= 2^h.  FP32 only.
 * With G = 1 the two calls are bf_apply's FP32 fused path, and for any G every
 * output element is bitwise the same as bf_apply's.
 * The paper has no distributed form; this partitions its Algorithm 4.1.
 */
#ifndef BF_SHARD_H
#define BF_SHARD_H

#include "bf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Elements (c64) of one peer block of W_send / W_recv for (plan, G, m).
 * Uploads the plan if needed.  Errors: BF_ERR_ARG (G not allowed, m < 1),
 * BF_ERR_STATE (not factored), BF_ERR_UNSUPPORTED (split plan or r). */
bf_status bf_shard_info(bf_plan* plan, int nshard, int64_t m, int64_t* chunk_elems);

/* Front half of shard `shard`: reads F_rows, writes all G blocks of W_send.
 * Asynchronous on `stream`.  Errors: as bf_shard_info, BF_ERR_CUDA. */
bf_status bf_apply_shard_front(bf_plan* plan, int nshard, int shard, const void* F_rows, int64_t m, void* W_send,
                               void* stream);

/* Back half of shard `shard`: reads W_recv (every shard's block), writes G_rows
 * (overwritten).  Asynchronous on `stream`.  Errors: as bf_apply_shard_front. */
bf_status bf_apply_shard_back(bf_plan* plan, int nshard, int shard, const void* W_recv, int64_t m, void* G_rows,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BF_SHARD_H */
