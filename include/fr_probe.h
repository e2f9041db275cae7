/*
 * fr_probe.h -- measured FP32 fused multiply-add peak of the current device.
 *
 * The paper has no counterpart of this call: it is a measurement service of
 * this library.  The insertion is bounded by the FP32 arithmetic units (it
 * is not a dense contraction and moves less than one byte of device memory
 * per voxel update), so its roofline denominator is the FP32 FMA rate:
 * SMs x 128 FP32 lanes x 2 flops x SM clock.  This call checks that figure
 * by measurement: every thread of a grid that fills every SM runs 8 (or 8
 * packed pairs of) independent dependent chains of fused multiply-adds, and
 * the call times the launch with CUDA events.
 */
#ifndef FR_PROBE_H
#define FR_PROBE_H

#include "fr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Run the FMA-chain kernel `repeats` times (after one untimed launch) on
 * `stream` and report the fastest launch.
 *   packed   0: scalar fma.rn.f32 chains; 1: packed two-lane fma.rn.f32x2
 *            chains (two FP32 fused multiply-adds per instruction).
 *   repeats  1 <= repeats <= 100.
 *   tflops   out: FP32 flops (2 per fused multiply-add) / fastest launch, in
 *            TFLOP/s.
 *   ms       out (may be NULL): the fastest launch's duration.
 *   stream   cudaStream_t as void*.  The call synchronises it.
 * Each thread runs 8192 steps of its chains and the grid is 4 CTAs of 512
 * threads per SM: 4.1e10 flops (8.2e10 packed) per launch on 152 SMs, about
 * half a millisecond.  The kernel touches no device memory beyond one
 * conditional store that never executes for the chains' values.  The call
 * allocates nothing on the device.
 * Returns FR_OK, FR_ERR_INVALID_ARG (packed not 0/1, repeats out of range,
 * tflops NULL) or FR_ERR_CUDA. */
int fr_probe_fp32_peak(int packed, int repeats, double *tflops, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FR_PROBE_H */
