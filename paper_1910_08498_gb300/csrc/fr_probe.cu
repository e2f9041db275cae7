// fr_probe.cu -- fr_probe_fp32_peak: a measured check of the FP32 FMA peak
// (SMs x 128 lanes x 2 flops x clock) that bounds the insertion kernels.
// Each thread runs CHAINS independent dependent chains a <- a * b + c; with
// 16 resident warps per scheduler and 8 chains per warp the FMA latency is
// hidden and the launch is limited by the FP32 pipes alone.
#include <cuda_runtime.h>

#include <algorithm>

#include "fr_internal.h"
#include "fr_probe.h"

static __device__ float g_probe_sink;

namespace fr {
namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 512;
constexpr int BLOCKS_PER_SM = 4;
constexpr int STEPS = 8192;  // chain steps per thread

template <int PACKED>
__global__ void __launch_bounds__(THREADS, BLOCKS_PER_SM)
fma_chain_kernel(const float b, const float c, const int steps) {
  const float seed = 1e-3f * (float)(threadIdx.x & 31);
  float s = 0.f;
  if constexpr (PACKED) {
    float2 acc[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc[k] = make_float2(seed + k, seed - k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll 16
    for (int i = 0; i < steps; ++i) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) acc[k] = __ffma2_rn(acc[k], bb, cc);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += acc[k].x + acc[k].y;
  } else {
    float acc[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc[k] = seed + k;
#pragma unroll 16
    for (int i = 0; i < steps; ++i) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) acc[k] = fmaf(acc[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += acc[k];
  }
  // the chains converge to c / (1 - b) = 1 and never reach this value; the
  // store keeps the compiler from removing them
  if (s == -12345.f) g_probe_sink = s;
}

int probe_status(cudaError_t e) {
  fr_note_cuda_error((int)e);
  return FR_ERR_CUDA;
}

}  // namespace
}  // namespace fr

extern "C" int fr_probe_fp32_peak(int packed, int repeats, double *tflops, double *ms,
                                  void *stream) {
  using namespace fr;
  if ((packed != 0 && packed != 1) || repeats < 1 || repeats > 100 || !tflops)
    return FR_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return probe_status(e);
  const dim3 grid((unsigned)(sms * BLOCKS_PER_SM));
  const float b = 0.999f, c = 0.001f;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float best = 0.f;
  for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {
    e = cudaEventRecord(ev[0], st);
    if (e != cudaSuccess) break;
    if (packed)
      fma_chain_kernel<1><<<grid, THREADS, 0, st>>>(b, c, STEPS);
    else
      fma_chain_kernel<0><<<grid, THREADS, 0, st>>>(b, c, STEPS);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
    if (e == cudaSuccess && r > 0 && (best == 0.f || t < best)) best = t;  // launch 0 is untimed
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return probe_status(e);
  const double flops = (double)grid.x * THREADS * CHAINS * STEPS * 2.0 * (packed ? 2.0 : 1.0);
  *tflops = best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
  if (ms) *ms = best;
  return FR_OK;
}
