/*
 * fr_noalloc.h -- insertion entry point that allocates no device memory.
 *
 * The paper has no counterpart of this call: it is a service entry point of
 * this library.  It runs the same insertion as fr_insert (the definition is
 * written out in fr.h) through the atomic scatter kernel, whose scratch
 * volume is a fixed array in the library's static device memory instead of a
 * cudaMalloc'd buffer.
 *
 * Who needs it: callers that must not enter the device allocator for the
 * duration of the call.  cudaMalloc and cudaFree can synchronise the device
 * (cudaFree waits for all outstanding work), which stalls every other stream
 * of a latency-bound pipeline; and a process whose memory is held by its own
 * pool allocator (for example a framework's caching allocator running close
 * to the memory limit) may have no room for, or may not allow, a separate
 * allocation.  fr_create allocates its accumulators and therefore cannot serve
 * those callers; this call needs no context and allocates nothing on the
 * device or on the host: no cudaMalloc/cudaFree, no allocating library
 * routine.
 */
#ifndef FR_NOALLOC_H
#define FR_NOALLOC_H

#include "fr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest image side fr_insert_noalloc accepts.  Its scratch array holds one
 * float4 per accumulator voxel for S = 64 and any a < 3: 65 x 65 x 35 cells,
 * 2.37 MB of static device memory. */
#define FR_NOALLOC_MAX_S 64

/* Add the contribution of n images to caller-owned V and W.
 *   S          image side, even, 8 <= S <= FR_NOALLOC_MAX_S.  A larger S
 *              returns FR_ERR_NOALLOC_LIMIT and enqueues nothing; an odd S
 *              returns FR_ERR_UNSUPPORTED, S < 8 FR_ERR_INVALID_ARG.
 *   a, alpha   blob radius (0 < a < 3) and taper (0 <= alpha <= 40); the
 *              weights are evaluated on the fly (Abramowitz & Stegun 9.8.1 /
 *              9.8.2 for I0).
 *   images     device, [n][S][S/2+1] complex of `dtype` (layout of fr.h),
 *              16-byte aligned.
 *   rotations  device, [n][9] float32 (layout of fr.h).
 *   n          0 <= n <= 2^24; n = 0 enqueues nothing and returns FR_OK.
 *   V, W       device, (S+1)^3 complex64 / float32 in the layout of fr.h.
 *              The batch's sums are ADDED to them in FP32: they must hold
 *              zeros before the first call for a new volume, and they are
 *              plain FP32 running sums (fr_create / fr_insert keep a
 *              compensated sum instead).
 *   stream     cudaStream_t as void*; all device work is enqueued on it.
 *
 * The scratch array is cleared by the call itself (cudaMemsetAsync on
 * `stream`) before its first use, so nothing about its earlier contents
 * matters; only V and W must start at zero.
 *
 * There is ONE scratch array per device.  Two calls whose device work
 * overlaps in time (different streams, or different host threads, on the
 * same device) race on it and both results are wrong: the caller must order
 * them (one stream, or events between streams).
 *
 * The first call on each device performs a one-time setup: it looks up the
 * scratch array's address with cudaGetSymbolAddress (which also loads the
 * library's device code on that device if lazy loading has not done so yet)
 * while that device is current, and caches it.  Make that first call before
 * any stream capture begins.
 *
 * The batch is added in sub-batches of 1024 images, each merged into V and W
 * before the next: if a launch fails part way (FR_ERR_CUDA), the sub-batches
 * before it have been added and the rest have not, so V and W are then
 * unspecified and must be rebuilt from zero.  The argument checks all come
 * before any device work: every other error leaves V and W untouched.
 *
 * Returns FR_OK, FR_ERR_INVALID_ARG (null pointer, misaligned images, n or a
 * or alpha out of range, bad dtype), FR_ERR_UNSUPPORTED, FR_ERR_NOALLOC_LIMIT,
 * or FR_ERR_CUDA (the symbol lookup or a launch failed; see
 * fr_last_cuda_error). */
int fr_insert_noalloc(int S, float a, float alpha, const void *images, fr_dtype dtype,
                      const float *rotations, int n, void *V, float *W, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FR_NOALLOC_H */
