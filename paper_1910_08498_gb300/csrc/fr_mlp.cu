// fr_mlp.cu -- the learned cost model of the tuner: a 16-64-64-1 ReLU MLP in
// FP32 with hand-written forward, backward (mean-squared error) and Adam
// kernels, its on-GPU training loop, and the model-ranked search order.
//
// Parameter vector (5313 floats): W1[64][16], b1[64], W2[64][64], b2[64],
// W3[64], b3 -- W[out][in].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "fr_ctx.h"
#include "fr_internal.h"
#include "fr_tuner.h"

namespace fr {

constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_H;
static_assert(OFF_B3 + 1 == MLP_NPARAM, "parameter layout");

constexpr int ROWS = 32;  // rows per CTA; one CTA of MLP_H threads (one per hidden unit)

struct MlpSmem {
  float P[MLP_NPARAM];
  float x[ROWS][MLP_IN];
  float h1[ROWS][MLP_H];
  float h2[ROWS][MLP_H];
  float d2[ROWS][MLP_H];  // dL/dz2
  float d1[ROWS][MLP_H];  // dL/dz1
  float y[ROWS];
  float dy[ROWS];
};

__device__ void mlp_tile_forward(MlpSmem &s, int nrows) {
  const int j = threadIdx.x;  // hidden unit
  for (int r = 0; r < nrows; ++r) {
    float z = s.P[OFF_B1 + j];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) z = fmaf(s.P[OFF_W1 + j * MLP_IN + k], s.x[r][k], z);
    s.h1[r][j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  for (int r = 0; r < nrows; ++r) {
    float z = s.P[OFF_B2 + j];
#pragma unroll 16
    for (int k = 0; k < MLP_H; ++k) z = fmaf(s.P[OFF_W2 + j * MLP_H + k], s.h1[r][k], z);
    s.h2[r][j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  if (j < nrows) {
    float z = s.P[OFF_B3];
    for (int k = 0; k < MLP_H; ++k) z = fmaf(s.P[OFF_W3 + k], s.h2[j][k], z);
    s.y[j] = z;
  }
  __syncthreads();
}

__device__ void load_tile(MlpSmem &s, const float *P, const float *X, int r0, int nrows) {
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) s.P[i] = P[i];
  for (int i = threadIdx.x; i < ROWS * MLP_IN; i += blockDim.x) {
    int r = i / MLP_IN, k = i % MLP_IN;
    s.x[r][k] = r < nrows ? X[(size_t)(r0 + r) * MLP_IN + k] : 0.f;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(MLP_H) mlp_forward_kernel(const float *P, const float *X, int m,
                                                            float *Y) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem &s = *reinterpret_cast<MlpSmem *>(raw);
  const int r0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, m - r0);
  load_tile(s, P, X, r0, nrows);
  mlp_tile_forward(s, nrows);
  if ((int)threadIdx.x < nrows) Y[r0 + threadIdx.x] = s.y[threadIdx.x];
}

// Per-CTA partial gradient (and partial loss) of L = (1/m) sum (y - t)^2 into
// work[blockIdx.x][MLP_NPARAM + 1]; summed in fixed order by mlp_reduce_kernel.
__global__ void __launch_bounds__(MLP_H) mlp_backward_kernel(const float *P, const float *X,
                                                             const float *T, int m, float *work) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem &s = *reinterpret_cast<MlpSmem *>(raw);
  const int r0 = blockIdx.x * ROWS;
  const int nrows = min(ROWS, m - r0);
  const int j = threadIdx.x;
  load_tile(s, P, X, r0, nrows);
  mlp_tile_forward(s, nrows);
  float *G = work + (size_t)blockIdx.x * (MLP_NPARAM + 1);
  const float inv_m = 1.0f / (float)m;
  if (j < nrows) {
    float e = s.y[j] - T[r0 + j];
    s.dy[j] = 2.f * e * inv_m;
    s.y[j] = e * e * inv_m;  // reuse as the per-row loss term
  }
  __syncthreads();
  // output layer
  {
    float gw3 = 0.f;
    for (int r = 0; r < nrows; ++r) gw3 = fmaf(s.dy[r], s.h2[r][j], gw3);
    G[OFF_W3 + j] = gw3;
    const float w3 = s.P[OFF_W3 + j];
    for (int r = 0; r < nrows; ++r) s.d2[r][j] = s.h2[r][j] > 0.f ? s.dy[r] * w3 : 0.f;
  }
  if (j == 0) {
    float gb3 = 0.f, l = 0.f;
    for (int r = 0; r < nrows; ++r) { gb3 += s.dy[r]; l += s.y[r]; }
    G[OFF_B3] = gb3;
    G[MLP_NPARAM] = l;
  }
  __syncthreads();
  // hidden layer 2: dW2[j][k] = sum_r d2[r][j] h1[r][k]; dz1[r][k] = [h1>0] sum_j W2[j][k] d2[r][j]
  {
    float gb2 = 0.f;
    for (int r = 0; r < nrows; ++r) gb2 += s.d2[r][j];
    G[OFF_B2 + j] = gb2;
    for (int k = 0; k < MLP_H; ++k) {
      float g = 0.f;
      for (int r = 0; r < nrows; ++r) g = fmaf(s.d2[r][j], s.h1[r][k], g);
      G[OFF_W2 + j * MLP_H + k] = g;
    }
    // thread j now plays input unit k = j of layer 2
    for (int r = 0; r < nrows; ++r) {
      float d = 0.f;
      for (int o = 0; o < MLP_H; ++o) d = fmaf(s.P[OFF_W2 + o * MLP_H + j], s.d2[r][o], d);
      s.d1[r][j] = s.h1[r][j] > 0.f ? d : 0.f;
    }
  }
  __syncthreads();
  // hidden layer 1
  {
    float gb1 = 0.f;
    for (int r = 0; r < nrows; ++r) gb1 += s.d1[r][j];
    G[OFF_B1 + j] = gb1;
    for (int k = 0; k < MLP_IN; ++k) {
      float g = 0.f;
      for (int r = 0; r < nrows; ++r) g = fmaf(s.d1[r][j], s.x[r][k], g);
      G[OFF_W1 + j * MLP_IN + k] = g;
    }
  }
}

__global__ void mlp_reduce_kernel(const float *work, int nblk, float *grad, float *loss) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > MLP_NPARAM) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += work[(size_t)b * (MLP_NPARAM + 1) + i];
  if (i < MLP_NPARAM) grad[i] = s;
  else if (loss) *loss = s;
}

__global__ void mlp_adam_kernel(float *P, const float *G, float *M1, float *M2, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NPARAM) return;
  float g = G[i];
  float m1 = fmaf(b1, M1[i], (1.f - b1) * g);
  float m2 = fmaf(b2, M2[i], (1.f - b2) * g * g);
  M1[i] = m1;
  M2[i] = m2;
  float mh = m1 / c1, vh = m2 / c2;
  P[i] -= lr * mh / (sqrtf(vh) + eps);
}

static size_t smem_bytes() { return sizeof(MlpSmem); }

static bool set_attrs() {
  return allow_dynamic_smem((const void *)mlp_forward_kernel, smem_bytes()) == cudaSuccess &&
         allow_dynamic_smem((const void *)mlp_backward_kernel, smem_bytes()) == cudaSuccess;
}

size_t mlp_work_floats(int m) { return (size_t)((m + ROWS - 1) / ROWS) * (MLP_NPARAM + 1); }

cudaError_t mlp_forward(const float *params, const float *x, int m, float *y, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if (!set_attrs()) return cudaGetLastError();
  mlp_forward_kernel<<<(m + ROWS - 1) / ROWS, MLP_H, smem_bytes(), st>>>(params, x, m, y);
  return cudaGetLastError();
}

cudaError_t mlp_backward(const float *params, const float *x, const float *t, int m, float *grad,
                         float *loss, float *work, cudaStream_t st) {
  if (m <= 0) return cudaErrorInvalidValue;
  if (!set_attrs()) return cudaGetLastError();
  int nblk = (m + ROWS - 1) / ROWS;
  mlp_backward_kernel<<<nblk, MLP_H, smem_bytes(), st>>>(params, x, t, m, work);
  mlp_reduce_kernel<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(work, nblk, grad, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, const float *grad, float *m1, float *m2, int t, float lr,
                     float b1, float b2, float eps, cudaStream_t st) {
  float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
  mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(params, grad, m1, m2, lr, b1, b2, eps,
                                                            c1, c2);
  return cudaGetLastError();
}

// He-uniform initialisation on the host from a seed.
static void init_params(std::vector<float> &p, unsigned long long seed) {
  std::mt19937_64 rng(seed);
  p.assign(MLP_NPARAM, 0.f);
  auto fill = [&](int off, int nout, int nin) {
    float lim = std::sqrt(6.f / (float)nin);
    std::uniform_real_distribution<float> u(-lim, lim);
    for (int i = 0; i < nout * nin; ++i) p[off + i] = u(rng);
  };
  fill(OFF_W1, MLP_H, MLP_IN);
  fill(OFF_W2, MLP_H, MLP_H);
  fill(OFF_W3, 1, MLP_H);
}

// Model-ranked search order: predicted time ascending, ties by configuration id.
std::vector<int> learned_order(fr_ctx *c, const TuneKey &k, const std::vector<int> &valid,
                               int *predicted_best) {
  std::vector<int> order = valid;
  const int m = (int)valid.size();
  if (m == 0 || !c->d_mlp) return order;
  std::vector<float> feat((size_t)m * MLP_IN), pred(m);
  const int n_repr = (int)std::min<long long>(1LL << 24, (3LL << k.nb) / 2);  // bucket middle
  for (int i = 0; i < m; ++i)
    config_features(config_space()[valid[i]], k.S, n_repr, k.a, &feat[(size_t)i * MLP_IN]);
  float *dx = nullptr, *dy = nullptr;
  if (cudaMalloc(&dx, feat.size() * sizeof(float)) != cudaSuccess) return order;
  if (cudaMalloc(&dy, m * sizeof(float)) != cudaSuccess) { cudaFree(dx); return order; }
  cudaMemcpy(dx, feat.data(), feat.size() * sizeof(float), cudaMemcpyHostToDevice);
  mlp_forward(c->d_mlp, dx, m, dy, 0);
  cudaMemcpy(pred.data(), dy, m * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  std::vector<int> idx(m);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (pred[a] != pred[b]) return pred[a] < pred[b];
    return valid[a] < valid[b];
  });
  for (int i = 0; i < m; ++i) order[i] = valid[idx[i]];
  if (predicted_best) *predicted_best = order[0];
  return order;
}

}  // namespace fr

using namespace fr;

extern "C" {

int fr_mlp_num_params(void) { return MLP_NPARAM; }

int fr_mlp_forward(const float *params, const float *x, int m, float *y, void *stream) {
  if (m < 0 || (m > 0 && (!params || !x || !y))) return FR_ERR_INVALID_ARG;
  return mlp_forward(params, x, m, y, (cudaStream_t)stream) == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}

int fr_mlp_backward(const float *params, const float *x, const float *target, int m, float *grad,
                    float *loss, void *stream) {
  if (m < 1 || !params || !x || !target || !grad || !loss) return FR_ERR_INVALID_ARG;
  float *work = nullptr;
  if (cudaMallocAsync(&work, mlp_work_floats(m) * sizeof(float), (cudaStream_t)stream) !=
      cudaSuccess)
    return FR_ERR_OOM;
  cudaError_t e = mlp_backward(params, x, target, m, grad, loss, work, (cudaStream_t)stream);
  cudaFreeAsync(work, (cudaStream_t)stream);
  return e == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}

int fr_mlp_adam(float *params, const float *grad, float *m1, float *m2, int t, float lr,
                float beta1, float beta2, float eps, void *stream) {
  if (!params || !grad || !m1 || !m2 || t < 1) return FR_ERR_INVALID_ARG;
  return mlp_adam(params, grad, m1, m2, t, lr, beta1, beta2, eps, (cudaStream_t)stream) ==
                 cudaSuccess
             ? FR_OK
             : FR_ERR_CUDA;
}

int fr_mlp_train(fr_ctx *c, const float *feat, const float *logt, int m, int epochs, float lr,
                 uint64_t seed, float *final_loss) {
  if (!c || !feat || !logt || m < 1 || epochs < 0) return FR_ERR_INVALID_ARG;
  std::vector<float> p;
  init_params(p, seed);
  if (!c->d_mlp && cudaMalloc(&c->d_mlp, MLP_NPARAM * sizeof(float)) != cudaSuccess)
    return FR_ERR_OOM;
  float *X = nullptr, *T = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr, *W = nullptr,
        *L = nullptr;
  size_t wn = mlp_work_floats(m);
  bool ok = cudaMalloc(&X, (size_t)m * MLP_IN * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&T, (size_t)m * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&G, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M1, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M2, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&W, wn * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&L, sizeof(float)) == cudaSuccess;
  int rc = FR_OK;
  if (!ok) rc = FR_ERR_OOM;
  if (rc == FR_OK) {
    cudaMemcpy(c->d_mlp, p.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(X, feat, (size_t)m * MLP_IN * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(T, logt, (size_t)m * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(M1, 0, MLP_NPARAM * sizeof(float));
    cudaMemset(M2, 0, MLP_NPARAM * sizeof(float));
    cudaMemset(L, 0, sizeof(float));
    for (int t = 1; t <= epochs; ++t) {
      if (mlp_backward(c->d_mlp, X, T, m, G, L, W, 0) != cudaSuccess ||
          mlp_adam(c->d_mlp, G, M1, M2, t, lr, 0.9f, 0.999f, 1e-8f, 0) != cudaSuccess) {
        rc = FR_ERR_CUDA;
        break;
      }
    }
    if (rc == FR_OK) {
      // loss of the final parameters
      if (mlp_backward(c->d_mlp, X, T, m, G, L, W, 0) != cudaSuccess) rc = FR_ERR_CUDA;
      float l = 0.f;
      if (cudaMemcpy(&l, L, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) rc = FR_ERR_CUDA;
      if (final_loss) *final_loss = l;
    }
  }
  cudaFree(X); cudaFree(T); cudaFree(G); cudaFree(M1); cudaFree(M2); cudaFree(W); cudaFree(L);
  if (rc == FR_OK) {
    c->mlp_trained = true;
    c->tuner.retune(true);
  }
  return rc;
}

int fr_mlp_get(const fr_ctx *c, float *params_host) {
  if (!c || !params_host) return FR_ERR_INVALID_ARG;
  if (!c->d_mlp) return FR_ERR_STATE;
  return cudaMemcpy(params_host, c->d_mlp, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? FR_OK
             : FR_ERR_CUDA;
}

int fr_mlp_set(fr_ctx *c, const float *params_host) {
  if (!c || !params_host) return FR_ERR_INVALID_ARG;
  if (!c->d_mlp && cudaMalloc(&c->d_mlp, MLP_NPARAM * sizeof(float)) != cudaSuccess)
    return FR_ERR_OOM;
  if (cudaMemcpy(c->d_mlp, params_host, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return FR_ERR_CUDA;
  c->mlp_trained = true;
  c->tuner.retune(true);
  return FR_OK;
}

}  // extern "C"
