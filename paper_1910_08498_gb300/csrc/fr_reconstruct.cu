// fr_reconstruct.cu -- the FFT steps of Algorithm 1 (Sec. 5.3.1) around the
// insertion, on the GPU: the forward transforms of the images (the step the
// paper runs on the CPU before uploading), staged into the insertion's input
// layout and dtype, and the last step, applying the weights W to G and
// transforming back.  The staging and weighting kernels are this library's;
// the FFTs are the vendor's plain R2C / C2R transforms (cuFFT), loaded at run
// time so that libfr.so does not depend on them.
//
// Last step:
//   Vs(v) = V(v) + conj(V(-v)),  Ws(v) = W(v) + W(-v)   (undo the half-space fold)
//   F(k)  = Vs(k) / max(Ws(k), w_clip) / S^3              k in [-S/2, S/2)^3,
//           0 on the Nyquist planes k_x = S/2, k_y = -S/2, k_z = -S/2
//   f     = inverse DFT of F (real, S^3, origin at index 0)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cufft.h>
#include <dlfcn.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/fr.h"
#include "fr_ctx.h"
#include "fr_internal.h"

namespace fr {
namespace {

// Half spectrum in C2R order: [kz][ky][kx], kz and ky in FFT order (index j
// is frequency j for j < S/2, j - S otherwise), kx = 0 .. S/2.
__global__ void weight_kernel(const Geom g, const float *__restrict__ acc, size_t plane,
                              float w_clip, float inv_n, float2 *__restrict__ F) {
  const int NXh = g.H + 1;
  const size_t total = (size_t)g.S * g.S * NXh;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(o % NXh);
    const size_t r = o / NXh;
    const int jy = (int)(r % g.S), jz = (int)(r / g.S);
    const int ky = jy < g.H ? jy : jy - g.S, kz = jz < g.H ? jz : jz - g.S;
    float2 out = make_float2(0.f, 0.f);
    if (kx != g.H && ky != -g.H && kz != -g.H) {
      const size_t v = ((size_t)(kz + g.H) * g.D + (size_t)(ky + g.H)) * g.NXa + (size_t)(kx - g.xa0);
      float re = acc[v] + acc[3 * plane + v];
      float im = acc[plane + v] + acc[4 * plane + v];
      float w = acc[2 * plane + v] + acc[5 * plane + v];
      if (-kx >= g.xa0) {  // -v is stored too: its conjugate joins
        const size_t m =
            ((size_t)(-kz + g.H) * g.D + (size_t)(-ky + g.H)) * g.NXa + (size_t)(-kx - g.xa0);
        re += acc[m] + acc[3 * plane + m];
        im -= acc[plane + m] + acc[4 * plane + m];
        w += acc[2 * plane + m] + acc[5 * plane + m];
      }
      const float s = inv_n / fmaxf(w, w_clip);
      out = make_float2(re * s, im * s);
    }
    F[o] = out;
  }
}

}  // namespace

// cuFFT entry points, resolved once
struct Cufft {
  bool tried = false, ok = false;
  cufftResult (*plan3d)(cufftHandle *, int, int, int, cufftType) = nullptr;
  cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
  cufftResult (*exec_c2r)(cufftHandle, cufftComplex *, cufftReal *) = nullptr;
  cufftResult (*destroy)(cufftHandle) = nullptr;
  cufftResult (*plan_many)(cufftHandle *, int, int *, int *, int, int, int *, int, int, cufftType,
                           int) = nullptr;
  cufftResult (*exec_r2c)(cufftHandle, cufftReal *, cufftComplex *) = nullptr;
};
std::mutex g_fft_mu;
Cufft g_fft;

const Cufft &cufft() {
  std::lock_guard<std::mutex> lk(g_fft_mu);
  if (g_fft.tried) return g_fft;
  g_fft.tried = true;
  const char *names[] = {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"};
  void *h = nullptr;
  for (const char *n : names)
    if ((h = dlopen(n, RTLD_NOW | RTLD_GLOBAL)) != nullptr) break;
  if (!h) return g_fft;
  g_fft.plan3d = reinterpret_cast<decltype(g_fft.plan3d)>(dlsym(h, "cufftPlan3d"));
  g_fft.set_stream = reinterpret_cast<decltype(g_fft.set_stream)>(dlsym(h, "cufftSetStream"));
  g_fft.exec_c2r = reinterpret_cast<decltype(g_fft.exec_c2r)>(dlsym(h, "cufftExecC2R"));
  g_fft.destroy = reinterpret_cast<decltype(g_fft.destroy)>(dlsym(h, "cufftDestroy"));
  g_fft.plan_many = reinterpret_cast<decltype(g_fft.plan_many)>(dlsym(h, "cufftPlanMany"));
  g_fft.exec_r2c = reinterpret_cast<decltype(g_fft.exec_r2c)>(dlsym(h, "cufftExecR2C"));
  g_fft.ok = g_fft.plan3d && g_fft.set_stream && g_fft.exec_c2r && g_fft.destroy &&
             g_fft.plan_many && g_fft.exec_r2c;
  return g_fft;
}

void reconstruct_release(fr_ctx *c) {
  if (c->fft_plan >= 0 && g_fft.ok) g_fft.destroy((cufftHandle)c->fft_plan);
  c->fft_plan = -1;
  cudaFree(c->spec);
  c->spec = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (c->prep_plan[k] >= 0 && g_fft.ok) g_fft.destroy((cufftHandle)c->prep_plan[k]);
    c->prep_plan[k] = -1;
    c->prep_batch[k] = 0;
  }
  cudaFree(c->prep_ws);
  c->prep_ws = nullptr;
}

namespace {

// The R2C output of a chunk of images, [m][S][S/2+1] float2 in rfft2 order,
// into the insertion input: multiplied by (-1)^(kx + j) when centring (the
// image origin moved from pixel (0, 0) to (S/2, S/2)), stored as float2 or
// half2.  Two entries per thread (16-byte loads; `total` is even since S is).
// Entry o = (image * S + j) * NX + kx; when NX = S/2 + 1 is odd (S a multiple
// of 4) the parity of kx + j is that of o, so the sign needs no division.
template <int F16>
__global__ void stage_kernel(const float2 *__restrict__ spec, size_t total, int NX, int center,
                             void *__restrict__ out) {
  const size_t pairs = total / 2;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs;
       i += (size_t)gridDim.x * blockDim.x) {
    float4 v = reinterpret_cast<const float4 *>(spec)[i];
    if (center) {
      bool neg0 = false, neg1 = true;  // entry 2i is even, 2i + 1 odd
      if (!(NX & 1)) {
        const size_t o = 2 * i, row = o / (size_t)NX;
        const int kx = (int)(o - row * NX);
        neg0 = ((kx + (int)(row & 1)) & 1) != 0;
        neg1 = kx + 1 < NX ? !neg0 : ((row + 1) & 1) != 0;  // entry 2i + 1 opens row + 1
      }
      if (neg0) v.x = -v.x, v.y = -v.y;
      if (neg1) v.z = -v.z, v.w = -v.w;
    }
    if (F16) {
      const __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
      uint2 u;
      u.x = *reinterpret_cast<const unsigned int *>(&h0);
      u.y = *reinterpret_cast<const unsigned int *>(&h1);
      reinterpret_cast<uint2 *>(out)[i] = u;
    } else {
      reinterpret_cast<float4 *>(out)[i] = v;
    }
  }
}

// plan for m images of S x S (slot 0: full chunks, slot 1: the tail)
int prep_plan(fr_ctx *c, int slot, int m) {
  const Cufft &fft = g_fft;
  if (c->prep_plan[slot] >= 0 && c->prep_batch[slot] == m) return FR_OK;
  if (c->prep_plan[slot] >= 0) fft.destroy((cufftHandle)c->prep_plan[slot]);
  c->prep_plan[slot] = -1;
  int dims[2] = {c->S, c->S};
  cufftHandle h = 0;
  if (fft.plan_many(&h, 2, dims, nullptr, 1, c->S * c->S, nullptr, 1, c->S * (c->S / 2 + 1),
                    CUFFT_R2C, m) != CUFFT_SUCCESS)
    return FR_ERR_CUDA;
  c->prep_plan[slot] = (int)h;
  c->prep_batch[slot] = m;
  return FR_OK;
}

}  // namespace

}  // namespace fr

using namespace fr;

extern "C" int fr_reconstruct(fr_ctx *c, float *out, float w_clip, void *stream) {
  if (!c || !out || !(w_clip > 0.f)) return FR_ERR_INVALID_ARG;
  const Cufft &fft = cufft();
  if (!fft.ok) return FR_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Geom &g = c->g;
  const size_t nspec = (size_t)g.S * g.S * (g.H + 1);
  if (!c->spec) {
    cudaError_t e = cudaMalloc(&c->spec, nspec * sizeof(float2));
    if (e != cudaSuccess) {
      fr_note_cuda_error((int)e);
      return FR_ERR_OOM;
    }
  }
  if (c->fft_plan < 0) {
    cufftHandle h = 0;
    if (fft.plan3d(&h, g.S, g.S, g.S, CUFFT_C2R) != CUFFT_SUCCESS) return FR_ERR_CUDA;
    c->fft_plan = (int)h;
  }
  // the insertions enqueued on another stream must be complete
  if (c->last_stream && c->last_stream != st) {
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e != cudaSuccess) {
      fr_note_cuda_error((int)e);
      return FR_ERR_CUDA;
    }
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  const size_t want = (nspec + threads - 1) / threads;
  const int blocks = (int)std::min<size_t>(want, (size_t)std::max(sms, 1) * 8);
  const float inv_n = 1.0f / ((float)g.S * (float)g.S * (float)g.S);
  weight_kernel<<<blocks, threads, 0, st>>>(g, c->acc, c->plane, w_clip, inv_n, c->spec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fr_note_cuda_error((int)e);
    return FR_ERR_CUDA;
  }
  if (fft.set_stream((cufftHandle)c->fft_plan, st) != CUFFT_SUCCESS) return FR_ERR_CUDA;
  if (fft.exec_c2r((cufftHandle)c->fft_plan, reinterpret_cast<cufftComplex *>(c->spec), out) !=
      CUFFT_SUCCESS)
    return FR_ERR_CUDA;
  c->last_stream = st;
  return FR_OK;
}

extern "C" int fr_prepare_images(fr_ctx *c, const float *real, int n, int center, void *out,
                                 fr_dtype dtype, void *stream) {
  if (!c || n < 0 || n > (1 << 24) || (dtype != FR_F32 && dtype != FR_F16)) return FR_ERR_INVALID_ARG;
  if (n == 0) return FR_OK;
  if (!real || !out || ((uintptr_t)out & 15) || ((uintptr_t)real & 15)) return FR_ERR_INVALID_ARG;
  const Cufft &fft = cufft();
  if (!fft.ok) return FR_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int S = c->S, NX = S / 2 + 1;
  const size_t px_real = (size_t)S * S, px_spec = (size_t)S * NX;
  // images per transform: about 256 MB of spectra per cuFFT launch (fewer,
  // larger launches measured faster than chunks of 256 images at S = 256),
  // and at least 256 images
  const int CHUNK = (int)std::max<size_t>(256, ((size_t)256 << 20) / (px_spec * sizeof(float2)));
  const bool direct = dtype == FR_F32;  // FP32: transform straight into out
  if (!direct && !c->prep_ws) {
    cudaError_t e = cudaMalloc(&c->prep_ws, (size_t)CHUNK * px_spec * sizeof(float2));
    if (e != cudaSuccess) {
      fr_note_cuda_error((int)e);
      return FR_ERR_OOM;
    }
  }
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int i0 = 0; i0 < n; i0 += CHUNK) {
    const int m = std::min(CHUNK, n - i0);
    const int slot = m == CHUNK ? 0 : 1;
    int rc = prep_plan(c, slot, m);
    if (rc != FR_OK) return rc;
    const cufftHandle h = (cufftHandle)c->prep_plan[slot];
    float2 *dst = direct ? reinterpret_cast<float2 *>(out) + (size_t)i0 * px_spec : c->prep_ws;
    if (fft.set_stream(h, st) != CUFFT_SUCCESS ||
        fft.exec_r2c(h, const_cast<cufftReal *>(real + (size_t)i0 * px_real),
                     reinterpret_cast<cufftComplex *>(dst)) != CUFFT_SUCCESS)
      return FR_ERR_CUDA;
    if (!direct || center) {
      const size_t total = (size_t)m * px_spec;
      const int threads = 256;
      const int blocks = (int)std::min<size_t>((total / 2 + threads - 1) / threads, (size_t)std::max(sms, 1) * 8);
      if (direct)
        stage_kernel<0><<<blocks, threads, 0, st>>>(dst, total, NX, center, dst);
      else
        stage_kernel<1><<<blocks, threads, 0, st>>>(
            dst, total, NX, center, reinterpret_cast<__half2 *>(out) + (size_t)i0 * px_spec);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        fr_note_cuda_error((int)e);
        return FR_ERR_CUDA;
      }
    }
  }
  return FR_OK;
}

