/*
 * fr_gemm.h -- batched multiplication of small matrices with non-blocking
 * dynamic tuning: the paper's second dynamic-tuning workload (the batched
 * GEMM of Sec. 4.2.5, dynamically tuned while the matrix sizes change at run
 * time, Sec. 5.2).
 *
 *   for b in [0, batch):  C[b] = A[b] B[b]
 *   A[b]: m x k, B[b]: k x n, C[b]: m x n, float32, row-major, the batch's
 *   instances stored one after the other (A: batch * m * k floats, ...).
 *   2 <= m, n, k <= 32.
 *
 * Two kernel families make up the configuration space (Sec. 4.2.5 tunes
 * work-item coarsening, instances per work-group and local-memory staging):
 *   - cooperative copies: Y, the rows of C one thread computes, Z, the
 *     instances one CTA computes, and C staged in shared memory for
 *     coalesced stores, or a persistent variant prefetching the next group
 *     with cp.async (72 configurations);
 *   - bulk copies: persistent CTAs stream groups of instances through a ring
 *     of shared-memory stages filled by the bulk-copy engine (cp.async.bulk
 *     with mbarrier completion), each thread computing a TY x TX register
 *     tile of C, the group's C written back by one bulk store; tuned over TY,
 *     TX in {1, 2, 4}, the rounds of the CTA's threads per group (1, 2, 4,
 *     8) and the CTA size cap (128, 256) (72 configurations).
 * Any 4-byte aligned A, B, C are accepted (the bulk copies move the 16-byte
 * aligned interior of each block and plain loads and stores the ends).
 * The tuner is the insertion's non-blocking scheme (Sec. 3.2): a call with
 * tuning on splits its batch into sub-batches, each computed with the next
 * configuration of the search and timed with CUDA events, harvested without
 * blocking on later calls; a size (m, n, k) not seen before starts a new
 * search.  Stop rule (Sec. 5.2): the search of a size ends when a measured
 * configuration reaches `bw_frac` of `bw_gbs` (memory throughput counted as
 * 4 (m k + k n + m n) bytes per instance), when `budget` configurations have
 * been measured, or when the space is exhausted.
 *
 * All pointers are device pointers owned by the caller; work is enqueued on
 * `stream` (a cudaStream_t as void*).  Returns an fr_status (fr.h).
 */
#ifndef FR_GEMM_H
#define FR_GEMM_H

#include "fr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fr_gemm_ctx fr_gemm_ctx;

/* Tuner state.  Defaults: tuning on, FR_SEARCH_RANDOM, budget 20,
 * bw_gbs 0 (no bandwidth criterion), bw_frac 0.75, 2 tuning steps per call. */
int fr_gemm_create(fr_gemm_ctx **out);
int fr_gemm_destroy(fr_gemm_ctx *ctx);
/* search: FR_SEARCH_EXHAUSTIVE, FR_SEARCH_RANDOM, FR_SEARCH_ANNEALING or
 * FR_SEARCH_MCMC; budget >= 1; steps >= 1 sub-batches per tuning call;
 * bw_gbs >= 0 (0: no bandwidth criterion); 0 < bw_frac <= 1. */
int fr_gemm_set_tuning(fr_gemm_ctx *ctx, int tuning, int search, int budget, int steps,
                       double bw_gbs, double bw_frac, uint64_t seed);
/* C = A B for `batch` instances of size (m, n, k), tuned dynamically per size.
 * 0 <= batch <= 2^26. */
int fr_gemm_run(fr_gemm_ctx *ctx, int m, int n, int k, const float *A, const float *B, float *C,
                int batch, void *stream);
/* The same with a fixed configuration (FR_ERR_UNSUPPORTED if it cannot run
 * for this size). */
int fr_gemm_run_config(int config, int m, int n, int k, const float *A, const float *B, float *C,
                       int batch, void *stream);
/* Device-side status of the bulk-copy kernels: FR_ERR_TIMEOUT if, since the
 * last call, a launch's bounded wait for a bulk copy gave up (after 1 s of
 * the global timer; the results of that launch are invalid), else FR_OK.
 * Waits for the device; clears the status.  FR_ERR_CUDA if it cannot be read. */
int fr_gemm_device_status(void);
/* Test hook (fault injection from the host): the limit of the bulk-copy
 * kernels' waits for their copies, in ns of the global timer, for launches
 * enqueued after the call (default 1e9).  A wait gives up when a poll finds
 * its copy incomplete ns or more after the wait began; 0 makes every wait give
 * up at once, which exercises the timeout path deterministically: the CTA
 * records FR_ERR_TIMEOUT, waits (with the default limit) for its copies in
 * flight and ends; the launch's results are invalid.
 * 0 <= ns <= 1e10; synchronous.  FR_ERR_INVALID_ARG or FR_ERR_CUDA on
 * failure. */
int fr_gemm_set_wait_limit(long long ns);
/* Configuration space: count, description, validity for a size. */
int fr_gemm_num_configs(void);
int fr_gemm_describe_config(int id, char *buf, int len);
int fr_gemm_config_valid(int id, int m, int n, int k);
/* Tuning state of size (m, n, k): tuned (0/1), configurations measured, best
 * configuration (-1 if none), its measured throughput (GB/s) and the time of
 * all this size's timed launches over the images they processed, relative
 * to the best (Eq. (performance) of Sec. 5.4, as 100 (rp - 1)).  Harvests
 * finished timings; does not block. */
int fr_gemm_report(fr_gemm_ctx *ctx, int m, int n, int k, int *tuned, int *evaluated, int *best,
                   double *best_gbs, double *overhead_pct);

#ifdef __cplusplus
}
#endif

#endif /* FR_GEMM_H */
