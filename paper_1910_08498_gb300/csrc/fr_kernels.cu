// fr_kernels.cu -- the scatter-with-atomics insertion variant and the small
// kernels around the insertion: scratch merge, finalize, update count, and
// test hooks for the fold predicate and the blob weights.
#include <cuda_runtime.h>

#include <algorithm>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

// q = R (kx, ky, 0) component as an unevaluated pair hi + lo (Dot2 of two
// products), so that v - q keeps ~1e-7 absolute accuracy at any |k|.
__device__ __forceinline__ void rk_dd(float r0, float r1, float kx, float ky, float &hi,
                                      float &lo) {
  float p0 = r0 * kx, e0 = fmaf(r0, kx, -p0);
  float p1 = r1 * ky, e1 = fmaf(r1, ky, -p1);
  float t;
  two_sum(p0, p1, hi, t);
  lo = (e0 + e1) + t;
}

// ---------------------------------------------------------------- scatter (A4')
//
// One thread per stored pixel: fold, then visit the KB^3 lattice box around
// q and add {w p.re, w p.im, w} with one 16-byte atomic per voxel into the
// float4 scratch volume.  The scratch is merged into the double-float
// accumulators after each sub-batch (see launch_merge_scratch), so a plain
// FP32 atomic sum never runs over more than one sub-batch of images.
template <int WMODE, int KB>
__global__ void scatter_kernel(const InsertArgs args) {
  const Geom &g = args.g;
  extern __shared__ __align__(16) float2 s_lut[];
  if (WMODE == W_LUT) {
    for (int i = threadIdx.x; i < args.lut_n; i += blockDim.x) s_lut[i] = args.lut[i];
    __syncthreads();
  }
  const float a = g.a, a2 = g.a2, inv_a2 = 1.0f / a2;
  const int npx = g.S * g.NX;           // stored pixels per image
  const int total = args.n * npx;       // < 2^31: sub-batches hold at most 1024 images
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x) {
    const int i = idx / npx;
    const int px = idx - i * npx;
    const int row = px / g.NX;
    const int kx = px - row * g.NX;
    const int ky = row < g.H ? row : row - g.S;
    const float *R = args.rot + 9 * (size_t)i;
    const float R00 = __ldg(R + 0), R01 = __ldg(R + 1), R10 = __ldg(R + 3), R11 = __ldg(R + 4),
                R20 = __ldg(R + 6), R21 = __ldg(R + 7);
    float2 p = load_pixel(args.images, args.f16, idx);
    float qxh, qxl, qyh, qyl, qzh, qzl;
    rk_dd(R00, R01, (float)kx, (float)ky, qxh, qxl);
    rk_dd(R10, R11, (float)kx, (float)ky, qyh, qyl);
    rk_dd(R20, R21, (float)kx, (float)ky, qzh, qzl);
    const bool folded = fold_pred(R00, R01, kx, ky);
    if (folded) {
      qxh = -qxh; qxl = -qxl; qyh = -qyh; qyl = -qyl; qzh = -qzh; qzl = -qzl; p.y = -p.y;
    }
    // box origin shifted down by a small margin when the box has a spare cell,
    // so a voxel at distance exactly a is never lost to rounding of q
    const float a_box = KB > (int)floorf(2.0f * a) + 1 ? a + 1e-4f : a;
    const int x0 = (int)ceilf((qxh + qxl) - a_box);
    const int y0 = (int)ceilf((qyh + qyl) - a_box);
    const int z0 = (int)ceilf((qzh + qzl) - a_box);
#pragma unroll 1
    for (int dz = 0; dz < KB; ++dz) {
      const int z = z0 + dz;
      const float fz = ((float)z - qzh) - qzl;
      const float rz = fz * fz;
      if (z < -g.H || z > g.H || rz > a2 * (1.0f + 2e-5f)) continue;
#pragma unroll 1
      for (int dy = 0; dy < KB; ++dy) {
        const int y = y0 + dy;
        const float fy = ((float)y - qyh) - qyl;
        const float ryz = fmaf(fy, fy, rz);
        if (y < -g.H || y > g.H || ryz > a2 * (1.0f + 2e-5f)) continue;
        float4 *rowp = args.scratch + ((size_t)(z + g.H) * g.D + (size_t)(y + g.H)) * g.NXa - g.xa0;
#pragma unroll
        for (int dx = 0; dx < KB; ++dx) {
          const int x = x0 + dx;
          const float fx = ((float)x - qxh) - qxl;
          const float r2 = fmaf(fx, fx, ryz);
          bool in = r2 <= a2;
          if (fabsf(r2 - a2) <= 1e-5f * a2) {
            // within rounding of the blob edge: decide as the real numbers do
            const float sg = folded ? -1.f : 1.f;
            in = exact_r2_le_a2(x, y, z, sg * R00, sg * R10, sg * R20, sg * R01, sg * R11,
                                sg * R21, kx, ky, a);
          }
          if (in && x <= g.H && x >= g.xa0) {
            const float w = blob_w<WMODE>(s_lut, r2, args, inv_a2);
            atomicAdd(rowp + x, make_float4(w * p.x, w * p.y, w, 0.f));
          }
        }
      }
    }
  }
}

// Fold the float4 scratch into the double-float accumulators and clear it.
__global__ void merge_scratch_kernel(const InsertArgs args) {
  const size_t n = args.plane;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (size_t)gridDim.x * blockDim.x) {
    float4 s = args.scratch[v];
    if (s.z != 0.f || s.x != 0.f || s.y != 0.f) {
      float add[3] = {s.x, s.y, s.z};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float h = args.acc[c * n + v], l = args.acc[(3 + c) * n + v];
        dd_add(h, l, add[c]);
        args.acc[c * n + v] = h;
        args.acc[(3 + c) * n + v] = l;
      }
      args.scratch[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// ---------------------------------------------------------------- finalize (A9)
__global__ void finalize_kernel(const Geom g, const float *__restrict__ acc, size_t plane,
                                float2 *__restrict__ V, float *__restrict__ W) {
  const size_t total = (size_t)g.D * g.D * g.D;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(o % g.D);
    const size_t zy = o / g.D;
    const int x = ix - g.H;
    float2 v = make_float2(0.f, 0.f);
    float w = 0.f;
    if (x >= g.xa0) {
      const size_t s = zy * g.NXa + (size_t)(x - g.xa0);
      v.x = acc[s] + acc[3 * plane + s];
      v.y = acc[plane + s] + acc[4 * plane + s];
      w = acc[2 * plane + s] + acc[5 * plane + s];
    }
    V[o] = v;
    W[o] = w;
  }
}

// ---------------------------------------------------------------- update count
//
// Number of (pixel, voxel) pairs the definition performs.  The decision is
// taken in FP32 with the compensated q; candidates within 1e-3 of the
// boundary are re-decided exactly as the FP64 definition states (products of
// an FP32 entry and an integer are exact in FP64), so the count equals the
// definition's.  This is a measurement helper, not part of the insertion.
// Exact number of (pixel, voxel) updates of a batch (the metric's unit).
// Images along grid y, pixels along grid x (32-bit index arithmetic); a row
// of candidates whose own distance already exceeds a is skipped; r <= a is
// decided in FP32 away from the edge and, within 1e-5 a^2 of it, with the
// definition's own FP64 operations.
__global__ void count_kernel(const Geom g, const float *rot, int n, unsigned long long *out) {
  const float a = g.a, a2 = g.a2;
  const float a2_row = a2 * (1.0f + 1e-4f);
  const double a2d = (double)g.a * (double)g.a;
  const int npx = g.S * g.NX;
  const int span = (int)floorf(2.f * a) + 3;
  unsigned long long cnt = 0;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const float *R = rot + 9 * (size_t)i;
    float Rv[6] = {__ldg(R + 0), __ldg(R + 1), __ldg(R + 3), __ldg(R + 4), __ldg(R + 6),
                   __ldg(R + 7)};
    for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < npx; px += gridDim.x * blockDim.x) {
      const int row = px / g.NX;
      const int kx = px - row * g.NX;
      const int ky = row < g.H ? row : row - g.S;
      float qh[3], ql[3];
      for (int c = 0; c < 3; ++c) rk_dd(Rv[2 * c], Rv[2 * c + 1], (float)kx, (float)ky, qh[c], ql[c]);
      float sg = 1.f;
      if (fold_pred(Rv[0], Rv[1], kx, ky)) sg = -1.f;
      for (int c = 0; c < 3; ++c) { qh[c] *= sg; ql[c] *= sg; }
      const int lo0 = (int)ceilf((qh[0] + ql[0]) - a) - 1, lo1 = (int)ceilf((qh[1] + ql[1]) - a) - 1,
                lo2 = (int)ceilf((qh[2] + ql[2]) - a) - 1;
      unsigned c32 = 0;
      for (int z = lo2; z < lo2 + span; ++z) {
        if (z < -g.H || z > g.H) continue;
        const float fz = ((float)z - qh[2]) - ql[2];
        const float rz = fz * fz;
        if (rz > a2_row) continue;
        for (int y = lo1; y < lo1 + span; ++y) {
          if (y < -g.H || y > g.H) continue;
          const float fy = ((float)y - qh[1]) - ql[1];
          const float ryz = fy * fy + rz;
          if (ryz > a2_row) continue;
          for (int x = lo0; x < lo0 + span; ++x) {
            if (x < -g.H || x > g.H) continue;
            const float fx = ((float)x - qh[0]) - ql[0];
            const float r2 = fx * fx + ryz;
            bool in;
            // FP32 r^2 is within a few 1e-6 of the exact value (q kept as a
            // double-float pair): outside a band of 1e-5 a^2 it decides,
            // inside it the definition's FP64 evaluation does
            if (fabsf(r2 - a2) > 1e-5f * a2) {
              in = r2 <= a2;
            } else {
              // same operations and order as the definition, no contraction
              double s = (double)sg;
              double qx = s * __dadd_rn((double)Rv[0] * kx, (double)Rv[1] * ky);
              double qy = s * __dadd_rn((double)Rv[2] * kx, (double)Rv[3] * ky);
              double qz = s * __dadd_rn((double)Rv[4] * kx, (double)Rv[5] * ky);
              double dx = x - qx, dy = y - qy, dz = z - qz;
              double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
              in = d2 <= a2d;
            }
            c32 += in;
          }
        }
      }
      cnt += c32;
    }
  }
  // warp reduce, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// ---------------------------------------------------------------- test hooks
__global__ void debug_fold_kernel(const float *r, const int *k, int m, int *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = fold_pred(r[2 * i], r[2 * i + 1], k[2 * i], k[2 * i + 1]) ? 1 : 0;
}

__global__ void debug_blob_kernel(const InsertArgs args, const float *r2, int m, int mode,
                                  float *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  float v = r2[i];
  if (!(v >= 0.f && v <= args.g.a2)) { out[i] = 0.f; return; }
  const float inv_a2 = 1.0f / args.g.a2;
  out[i] = mode == 0 ? blob_lut(args.lut, v, args.lut_scale)
         : mode == 1 ? blob_otf(v, inv_a2, args.g.alpha, args.inv_i0a, args.inv_pa)
                     : blob_poly(v, 2.0f * inv_a2, args.poly);
}

// ---------------------------------------------------------------- launchers

static int grid_for(size_t work, int threads, int max_blocks) {
  size_t b = (work + threads - 1) / threads;
  if (b > (size_t)max_blocks) b = max_blocks;
  if (b < 1) b = 1;
  return (int)b;
}

static int sm_count() { return device_sm_count(); }

template <int WMODE, int KB>
static cudaError_t launch_scatter_t(int threads, const InsertArgs &a, cudaStream_t st,
                                    int query_only, KernelInfo *info) {
  auto fn = scatter_kernel<WMODE, KB>;
  size_t smem = WMODE == W_LUT ? (size_t)a.lut_n * sizeof(float2) : 0;
  if (info) { info->fn = (const void *)fn; info->threads = threads; info->smem = smem; }
  if (smem) {
    cudaError_t e = allow_dynamic_smem((const void *)fn, smem);
    if (e != cudaSuccess) return e;
  }
  if (query_only) return cudaSuccess;
  if (a.n <= 0) return cudaSuccess;
  const long long work = (long long)a.n * a.g.S * a.g.NX;
  if (work >= (1LL << 31)) return cudaErrorInvalidValue;
  int blocks = grid_for((size_t)work, threads, sm_count() * (2048 / threads));
  fn<<<blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter(int threads, int wmode, const InsertArgs &a, cudaStream_t st,
                           int query_only, KernelInfo *info) {
  if (a.g.KB == 4) {
    if (wmode == W_LUT) return launch_scatter_t<W_LUT, 4>(threads, a, st, query_only, info);
    if (wmode == W_POLY) return launch_scatter_t<W_POLY, 4>(threads, a, st, query_only, info);
    return launch_scatter_t<W_OTF, 4>(threads, a, st, query_only, info);
  }
  if (wmode == W_LUT) return launch_scatter_t<W_LUT, 6>(threads, a, st, query_only, info);
  if (wmode == W_POLY) return launch_scatter_t<W_POLY, 6>(threads, a, st, query_only, info);
  return launch_scatter_t<W_OTF, 6>(threads, a, st, query_only, info);
}

cudaError_t launch_merge_scratch(const InsertArgs &a, cudaStream_t st) {
  int threads = 256;
  merge_scratch_kernel<<<grid_for(a.plane, threads, sm_count() * 8), threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Geom &g, const float *acc, size_t plane, float2 *V, float *W,
                            cudaStream_t st) {
  size_t total = (size_t)g.D * g.D * g.D;
  int threads = 256;
  finalize_kernel<<<grid_for(total, threads, sm_count() * 8), threads, 0, st>>>(g, acc, plane, V, W);
  return cudaGetLastError();
}

cudaError_t launch_count(const Geom &g, const float *rot, int n, unsigned long long *out,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int npx = g.S * g.NX;
  const int bx = std::max(1, std::min((npx + threads - 1) / threads, 64));
  const int by = std::max(1, std::min(n, (sm_count() * 8 + bx - 1) / bx * 4));
  count_kernel<<<dim3(bx, std::min(by, 65535)), threads, 0, st>>>(g, rot, n, out);
  return cudaGetLastError();
}

cudaError_t launch_debug_fold(const float *r, const int *k, int m, int *out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  debug_fold_kernel<<<(m + 255) / 256, 256, 0, st>>>(r, k, m, out);
  return cudaGetLastError();
}

cudaError_t launch_debug_blob(const InsertArgs &a, const float *r2, int m, int mode, float *out,
                              cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  debug_blob_kernel<<<(m + 255) / 256, 256, 0, st>>>(a, r2, m, mode, out);
  return cudaGetLastError();
}

}  // namespace fr
