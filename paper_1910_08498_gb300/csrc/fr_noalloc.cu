// fr_noalloc.cu -- fr_insert_noalloc: the atomic scatter insertion with its
// scratch volume in a fixed array of static device memory, for callers that
// must not enter the device allocator (they may be sharing the device with
// latency-bound streams that a cudaMalloc/cudaFree would synchronise, or hold
// all device memory in their own pool allocator).  Nothing here allocates:
// no cudaMalloc, no cudaFree, no allocating library routine; the scratch
// address is looked up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "fr_device.cuh"
#include "fr_internal.h"
#include "fr_noalloc.h"

// One float4 {w re, w im, w, 0} per accumulator voxel of the largest volume:
// D x D x NXa with D = 65 and NXa = S/2 + floor(a) + 1 <= 35 (a < 3); 2.37 MB.
static constexpr size_t NOALLOC_CELLS = (size_t)(FR_NOALLOC_MAX_S + 1) *
                                        (FR_NOALLOC_MAX_S + 1) * (FR_NOALLOC_MAX_S / 2 + 3);
static __device__ __align__(256) float4 g_noalloc_scratch[NOALLOC_CELLS];

namespace fr {
namespace {

constexpr int NOALLOC_SUB = 1024;  // images per scatter launch (span of one FP32 atomic sum)
constexpr int MAX_DEVICES = 64;

struct DeviceSlot {
  bool ready = false;
  float4 *scratch = nullptr;
};
std::mutex g_mu;
DeviceSlot g_slots[MAX_DEVICES];

// Add the scratch sums to V and W (full (S+1)^3 grid) and clear the cells read.
__global__ void noalloc_add_kernel(const Geom g, float4 *__restrict__ scratch,
                                   float2 *__restrict__ V, float *__restrict__ W) {
  const size_t cells = (size_t)g.D * g.D * g.NXa;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < cells;
       v += (size_t)gridDim.x * blockDim.x) {
    const float4 s = scratch[v];
    if (s.x != 0.f || s.y != 0.f || s.z != 0.f) {
      const size_t zy = v / g.NXa;
      const int x = (int)(v - zy * g.NXa) + g.xa0;  // >= -floor(a) > -S/2
      const size_t o = zy * g.D + (size_t)(x + g.H);
      float2 cur = V[o];
      cur.x += s.x;
      cur.y += s.y;
      V[o] = cur;
      W[o] += s.z;
      scratch[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

int cuda_status(cudaError_t e) {
  fr_note_cuda_error((int)e);
  return FR_ERR_CUDA;
}

}  // namespace
}  // namespace fr

extern "C" int fr_insert_noalloc(int S, float a, float alpha, const void *images, fr_dtype dtype,
                                 const float *rotations, int n, void *V, float *W, void *stream) {
  using namespace fr;
  if (S < 8) return FR_ERR_INVALID_ARG;
  if (S & 1) return FR_ERR_UNSUPPORTED;
  if (S > FR_NOALLOC_MAX_S) return FR_ERR_NOALLOC_LIMIT;
  if (!(a > 0.f) || !(alpha >= 0.f && alpha <= 40.f)) return FR_ERR_INVALID_ARG;
  if (!(a < 3.f)) return FR_ERR_UNSUPPORTED;
  if (n < 0 || n > (1 << 24) || (dtype != FR_F32 && dtype != FR_F16)) return FR_ERR_INVALID_ARG;
  if (!V || !W) return FR_ERR_INVALID_ARG;
  if (n == 0) return FR_OK;
  if (!images || !rotations || ((uintptr_t)images & 15)) return FR_ERR_INVALID_ARG;

  // one-time setup per device, with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= MAX_DEVICES) return FR_ERR_INVALID_ARG;
  float4 *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSlot &slot = g_slots[dev];
    if (!slot.ready) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_status(e);
      slot.scratch = static_cast<float4 *>(p);
      slot.ready = true;
    }
    scratch = slot.scratch;
  }

  Geom g{};
  g.S = S;
  g.H = S / 2;
  g.NX = S / 2 + 1;
  g.D = S + 1;
  g.a = a;
  g.a2 = a * a;
  g.alpha = alpha;
  g.xa0 = -(int)std::floor(a);
  g.NXa = g.H - g.xa0 + 1;
  g.KB = a < 2.0f ? 4 : 6;
  const size_t cells = (size_t)g.D * g.D * g.NXa;  // <= NOALLOC_CELLS by the checks above
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  InsertArgs args{};
  args.g = g;
  args.f16 = dtype == FR_F16 ? 1 : 0;
  args.inv_i0a = (float)(1.0 / std::cyl_bessel_i(0.0, (double)alpha));
  args.inv_pa = otf_inv_pa((double)alpha);
  args.err = nullptr;
  args.scratch = scratch;

  e = cudaMemsetAsync(scratch, 0, cells * sizeof(float4), st);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t img_bytes = (size_t)S * g.NX * (dtype == FR_F16 ? 4 : 8);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_status(e);
  const int add_threads = 256;
  const int add_blocks = (int)std::min<size_t>((cells + add_threads - 1) / add_threads,
                                               (size_t)sms * 8);
  for (int i0 = 0; i0 < n; i0 += NOALLOC_SUB) {
    args.n = std::min(NOALLOC_SUB, n - i0);
    args.images = static_cast<const unsigned char *>(images) + (size_t)i0 * img_bytes;
    args.rot = rotations + (size_t)i0 * 9;
    e = launch_scatter(256, W_OTF, args, st, 0, nullptr);
    if (e != cudaSuccess) return cuda_status(e);
    noalloc_add_kernel<<<add_blocks, add_threads, 0, st>>>(g, scratch, static_cast<float2 *>(V), W);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
  }
  return FR_OK;
}
