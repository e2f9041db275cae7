// fr_gemm.cu -- batched multiplication of small matrices (Sec. 4.2.5) with
// the non-blocking dynamic tuning of Sec. 3.2 under matrix-size changes
// (Sec. 5.2); the C ABI of include/fr_gemm.h.
//
// Kernels: a CTA computes Z consecutive instances.  It copies their A and B
// blocks (contiguous in memory) into shared memory with coalesced loads;
// thread (j, ty, tz) then computes column j of rows ty*Y .. ty*Y+Y-1 of
// instance tz, with a sequential FMA over the inner dimension.  With STAGE,
// the CTA's C block is assembled in shared memory and written back with
// coalesced stores; otherwise each thread stores its Y values directly.  The
// pipelined variant keeps a grid of resident CTAs that prefetch their next
// group of instances with cp.async while computing the current one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <numeric>
#include <random>
#include <set>
#include <tuple>
#include <vector>

#include "../../include/fr.h"
#include "../../include/fr_gemm.h"
#include "fr_internal.h"
#include "fr_search.h"

namespace fr {
namespace {

struct GemmConfig {
  int y, z, stage, pipe;  // pipe: persistent CTAs, next group prefetched with cp.async
};

const std::vector<GemmConfig> &gemm_space() {
  static const std::vector<GemmConfig> v = [] {
    std::vector<GemmConfig> c;
    for (int y : {1, 2, 4, 8})
      for (int z : {1, 2, 4, 8, 16, 32}) {
        for (int st : {0, 1}) c.push_back(GemmConfig{y, z, st, 0});
        c.push_back(GemmConfig{y, z, 0, 1});
      }
    return c;
  }();
  return v;
}

int gemm_threads(const GemmConfig &c, int m, int n) { return n * ((m + c.y - 1) / c.y) * c.z; }

size_t gemm_smem(const GemmConfig &c, int m, int n, int k) {
  if (c.pipe)  // two buffers of A and B, each with 16 B of alignment slack
    return 2 * ((size_t)c.z * ((size_t)m * k + (size_t)k * n) * sizeof(float) + 32);
  return (size_t)c.z * ((size_t)m * k + (size_t)k * n + (c.stage ? (size_t)m * n : 0)) * sizeof(float);
}

bool gemm_valid(int id, int m, int n, int k) {
  if (id < 0 || id >= (int)gemm_space().size()) return false;
  if (m < 2 || m > 32 || n < 2 || n > 32 || k < 2 || k > 32) return false;
  const GemmConfig &c = gemm_space()[id];
  const int t = gemm_threads(c, m, n);
  if (c.y > m) return false;  // no thread would get a full strip
  return t >= 32 && t <= 1024 && gemm_smem(c, m, n, k) <= 48 * 1024;
}

// dst[i] = src[i] for i < count (src in global memory): 16-byte loads over the
// 16-byte aligned middle, scalar loads for the ends
__device__ __forceinline__ void copy_to_smem(float *dst, const float *src, int count) {
  const int head = (int)(((16 - (reinterpret_cast<uintptr_t>(src) & 15)) & 15) >> 2);
  const int h = min(head, count);
  for (int i = threadIdx.x; i < h; i += blockDim.x) dst[i] = __ldg(src + i);
  const int nv = (count - h) >> 2;
  const float4 *s4 = reinterpret_cast<const float4 *>(src + h);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const float4 x = __ldg(s4 + v);
    float *d = dst + h + 4 * v;
    d[0] = x.x;
    d[1] = x.y;
    d[2] = x.z;
    d[3] = x.w;
  }
  for (int i = h + 4 * nv + threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
}

template <int Y, int STAGE>
__global__ void bgemm_kernel(int m, int n, int k, int z, const float *__restrict__ A,
                             const float *__restrict__ B, float *__restrict__ C, int batch) {
  extern __shared__ float sm[];
  const long long b0 = (long long)blockIdx.x * z;
  const int nb = (int)min((long long)z, batch - b0);
  const int mk = m * k, kn = k * n, mn = m * n;
  float *sA = sm, *sB = sA + z * mk, *sC = sB + z * kn;
  const int T = blockDim.x;
  const float *gA = A + b0 * mk;
  const float *gB = B + b0 * kn;
  copy_to_smem(sA, gA, nb * mk);
  copy_to_smem(sB, gB, nb * kn);
  __syncthreads();
  const int my = (m + Y - 1) / Y;
  const int j = threadIdx.x % n, t = threadIdx.x / n;
  const int ty = t % my, tz = t / my;
  if (tz < nb) {
    float acc[Y];
#pragma unroll
    for (int r = 0; r < Y; ++r) acc[r] = 0.f;
    const float *a = sA + tz * mk + ty * Y * k;
    const float *bb = sB + tz * kn + j;
    for (int p = 0; p < k; ++p) {
      const float bv = bb[p * n];
#pragma unroll
      for (int r = 0; r < Y; ++r)
        if (ty * Y + r < m) acc[r] = fmaf(a[r * k + p], bv, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < Y; ++r) {
      const int row = ty * Y + r;
      if (row < m) {
        if (STAGE)
          sC[tz * mn + row * n + j] = acc[r];
        else
          C[(b0 + tz) * mn + row * n + j] = acc[r];
      }
    }
  }
  if (STAGE) {
    __syncthreads();
    float *gC = C + b0 * mn;
    for (int i = threadIdx.x; i < nb * mn; i += T) gC[i] = sC[i];
  }
}

// Asynchronous copy of count floats from global src to shared dst, where
// dst and src have the same address modulo 16: 16-byte copies over the
// aligned middle, 4-byte copies at the ends.
__device__ __forceinline__ void async_copy(float *dst, const float *src, int count) {
  const int head = (int)(((16 - (reinterpret_cast<uintptr_t>(src) & 15)) & 15) >> 2);
  const int h = min(head, count);
  const uint32_t d0 = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  for (int i = threadIdx.x; i < h; i += blockDim.x)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d0 + 4 * i), "l"(src + i) : "memory");
  const int nv = (count - h) >> 2;
  for (int v = threadIdx.x; v < nv; v += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 4 * (h + 4 * v)),
                 "l"(src + h + 4 * v)
                 : "memory");
  for (int i = h + 4 * nv + threadIdx.x; i < count; i += blockDim.x)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d0 + 4 * i), "l"(src + i) : "memory");
}

// Persistent variant: CTA c computes the groups c, c + gridDim.x, ... of z
// instances; while it computes one group, the next one's A and B are copied
// into the other shared-memory buffer (two-stage pipeline, cp.async).
template <int Y>
__global__ void bgemm_pipe_kernel(int m, int n, int k, int z, const float *__restrict__ A,
                                  const float *__restrict__ B, float *__restrict__ C, int batch) {
  extern __shared__ __align__(16) float sm[];
  const int mk = m * k, kn = k * n, mn = m * n;
  const int buf_floats = z * (mk + kn) + 8;  // + slack to match the source alignment
  const long long groups = ((long long)batch + z - 1) / z;
  const int my = (m + Y - 1) / Y;
  const int j = threadIdx.x % n, t = threadIdx.x / n;
  const int ty = t % my, tz = t / my;
  // p moved up by 0..3 floats to the same address modulo 16 as src
  auto align_like = [](float *p, const float *src) -> float * {
    const uintptr_t d = (reinterpret_cast<uintptr_t>(src) - reinterpret_cast<uintptr_t>(p)) & 15;
    return p + (d >> 2);
  };
  // where group g's A and B land in buffer s
  auto bases = [&](long long g, int s, float *&sA, float *&sB) {
    sA = align_like(sm + s * buf_floats, A + g * z * mk);
    sB = align_like(sA + z * mk, B + g * z * kn);
  };
  auto issue = [&](long long g, int s) {
    const long long b0 = g * z;
    const int nb = (int)min((long long)z, batch - b0);
    float *sA, *sB;
    bases(g, s, sA, sB);
    async_copy(sA, A + b0 * mk, nb * mk);
    async_copy(sB, B + b0 * kn, nb * kn);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  long long g = blockIdx.x;
  int s = 0;
  if (g < groups) issue(g, 0);
  for (; g < groups; g += gridDim.x, s ^= 1) {
    const long long gn = g + gridDim.x;
    if (gn < groups) {
      issue(gn, s ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const long long b0 = g * z;
    const int nb = (int)min((long long)z, batch - b0);
    float *sA, *sB;
    bases(g, s, sA, sB);
    if (tz < nb) {
      float acc[Y];
#pragma unroll
      for (int r = 0; r < Y; ++r) acc[r] = 0.f;
      const float *a = sA + tz * mk + ty * Y * k;
      const float *bb = sB + tz * kn + j;
      for (int p = 0; p < k; ++p) {
        const float bv = bb[p * n];
#pragma unroll
        for (int r = 0; r < Y; ++r)
          if (ty * Y + r < m) acc[r] = fmaf(a[r * k + p], bv, acc[r]);
      }
#pragma unroll
      for (int r = 0; r < Y; ++r) {
        const int row = ty * Y + r;
        if (row < m) C[(b0 + tz) * mn + row * n + j] = acc[r];
      }
    }
    __syncthreads();  // buffer s is refilled two groups later
  }
}

template <int Y, int STAGE>
cudaError_t launch_t(const GemmConfig &c, int m, int n, int k, const float *A, const float *B,
                     float *C, int batch, cudaStream_t st) {
  const int threads = gemm_threads(c, m, n);
  const size_t smem = gemm_smem(c, m, n, k);
  const long long blocks = ((long long)batch + c.z - 1) / c.z;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  bgemm_kernel<Y, STAGE><<<(unsigned)blocks, threads, smem, st>>>(m, n, k, c.z, A, B, C, batch);
  return cudaGetLastError();
}

template <int Y>
cudaError_t launch_pipe(const GemmConfig &c, int m, int n, int k, const float *A, const float *B,
                        float *C, int batch, cudaStream_t st) {
  const int threads = gemm_threads(c, m, n);
  const size_t smem = gemm_smem(c, m, n, k);
  auto fn = bgemm_pipe_kernel<Y>;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (e != cudaSuccess) return e;
  const long long groups = ((long long)batch + c.z - 1) / c.z;
  const long long grid = std::min<long long>(groups, (long long)std::max(per_sm, 1) * sms);
  fn<<<(unsigned)grid, threads, smem, st>>>(m, n, k, c.z, A, B, C, batch);
  return cudaGetLastError();
}

cudaError_t gemm_launch(int id, int m, int n, int k, const float *A, const float *B, float *C,
                        int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const GemmConfig &c = gemm_space()[id];
  if (c.pipe) {
    switch (c.y) {
      case 1: return launch_pipe<1>(c, m, n, k, A, B, C, batch, st);
      case 2: return launch_pipe<2>(c, m, n, k, A, B, C, batch, st);
      case 4: return launch_pipe<4>(c, m, n, k, A, B, C, batch, st);
      case 8: return launch_pipe<8>(c, m, n, k, A, B, C, batch, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (c.y * 2 + c.stage) {
    case 2: return launch_t<1, 0>(c, m, n, k, A, B, C, batch, st);
    case 3: return launch_t<1, 1>(c, m, n, k, A, B, C, batch, st);
    case 4: return launch_t<2, 0>(c, m, n, k, A, B, C, batch, st);
    case 5: return launch_t<2, 1>(c, m, n, k, A, B, C, batch, st);
    case 8: return launch_t<4, 0>(c, m, n, k, A, B, C, batch, st);
    case 9: return launch_t<4, 1>(c, m, n, k, A, B, C, batch, st);
    case 16: return launch_t<8, 0>(c, m, n, k, A, B, C, batch, st);
    case 17: return launch_t<8, 1>(c, m, n, k, A, B, C, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

double instance_bytes(int m, int n, int k) { return 4.0 * ((double)m * k + (double)k * n + (double)m * n); }

// ---------------------------------------------------------------- tuner

struct GemmMeas {
  double ns = 0, inst = 0;
  double gbs(double bytes) const { return ns > 0 ? inst * bytes / ns : 0; }
};

struct GemmKey {
  std::vector<int> order;
  size_t next = 0;
  bool adaptive = false;
  Walker walker;
  int proposed = 0;
  std::map<int, GemmMeas> meas;
  int pending = 0;
  bool tuned = false;
  int best = -1;
  double all_ns = 0, all_inst = 0;
};

struct GemmPending {
  cudaEvent_t a, b;
  std::tuple<int, int, int> key;
  int config;
  int inst;
  bool tuning;
};

}  // namespace
}  // namespace fr

using namespace fr;

struct fr_gemm_ctx {
  int tuning = 1, search = FR_SEARCH_RANDOM, budget = 20, steps = 2;
  double bw_gbs = 0, bw_frac = 0.75;
  uint64_t seed = 1;
  std::map<std::tuple<int, int, int>, GemmKey> keys;
  std::vector<GemmPending> pending;
  std::vector<cudaEvent_t> pool;
  std::mutex mu;

  cudaEvent_t event() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void update_best(GemmKey &ks, double bytes) {
    int best = -1;
    double bg = 0;
    for (auto &m : ks.meas)
      if (m.second.inst > 0 && m.second.gbs(bytes) > bg) {
        bg = m.second.gbs(bytes);
        best = m.first;
      }
    ks.best = best;
  }
  void finish_if_done(GemmKey &ks, int m, int n, int k) {
    if (ks.tuned) return;
    const double bytes = instance_bytes(m, n, k);
    update_best(ks, bytes);
    const int evaluated = (int)ks.meas.size();
    const bool fast_enough =
        bw_gbs > 0 && ks.best >= 0 && ks.meas[ks.best].gbs(bytes) >= bw_frac * bw_gbs;
    const bool exhausted = ks.adaptive ? ks.proposed >= budget || ks.walker.proposed.size() >= ks.walker.valid.size()
                                       : ks.next >= ks.order.size();
    if (ks.pending == 0 && ks.best >= 0 && (fast_enough || evaluated >= budget || exhausted))
      ks.tuned = true;
  }
  void harvest() {
    size_t w = 0;
    for (size_t i = 0; i < pending.size(); ++i) {
      GemmPending &p = pending[i];
      if (cudaEventQuery(p.b) == cudaErrorNotReady) {
        pending[w++] = p;
        continue;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, p.a, p.b);
      pool.push_back(p.a);
      pool.push_back(p.b);
      auto it = keys.find(p.key);
      if (it == keys.end()) continue;
      GemmKey &ks = it->second;
      ks.all_ns += 1e6 * ms;
      ks.all_inst += p.inst;
      if (p.tuning) {
        GemmMeas &mm = ks.meas[p.config];
        mm.ns += 1e6 * ms;
        mm.inst += p.inst;
        --ks.pending;
        finish_if_done(ks, std::get<0>(p.key), std::get<1>(p.key), std::get<2>(p.key));
      }
    }
    pending.resize(w);
  }
  GemmKey &state(int m, int n, int k) {
    auto key = std::make_tuple(m, n, k);
    auto it = keys.find(key);
    if (it != keys.end()) return it->second;
    GemmKey &ks = keys[key];
    std::vector<int> valid;
    for (int i = 0; i < (int)gemm_space().size(); ++i)
      if (gemm_valid(i, m, n, k)) valid.push_back(i);
    std::mt19937_64 rng(seed ^ ((uint64_t)m << 32) ^ ((uint64_t)n << 16) ^ (uint64_t)k);
    if (search == FR_SEARCH_ANNEALING || search == FR_SEARCH_MCMC) {
      ks.adaptive = true;
      ks.walker.valid = valid;
      ks.walker.nbr.assign(gemm_space().size(), {});
      // neighbours: configurations that differ in one tuning dimension
      for (int a : valid)
        for (int b : valid) {
          const GemmConfig &x = gemm_space()[a], &y = gemm_space()[b];
          if ((x.y != y.y) + (x.z != y.z) + (x.stage != y.stage) + (x.pipe != y.pipe) == 1)
            ks.walker.nbr[a].push_back(b);
        }
      ks.walker.anneal = search == FR_SEARCH_ANNEALING;
      ks.walker.T = ks.walker.anneal ? 0.2 : 0.1;
      ks.walker.rng.seed(rng());
      const int start = valid.empty() ? -1 : valid[rng() % valid.size()];
      if (start >= 0) {
        ks.walker.proposed.insert(start);
        ks.walker.undecided.push_back(start);
        ks.walker.pending_start_ = start;
      }
    } else {
      ks.order = valid;
      if (search != FR_SEARCH_EXHAUSTIVE) std::shuffle(ks.order.begin(), ks.order.end(), rng);
    }
    return ks;
  }
};

extern "C" {

int fr_gemm_create(fr_gemm_ctx **out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = new (std::nothrow) fr_gemm_ctx();
  return *out ? FR_OK : FR_ERR_OOM;
}

int fr_gemm_destroy(fr_gemm_ctx *c) {
  if (!c) return FR_OK;
  for (auto &p : c->pending) {
    cudaEventSynchronize(p.b);
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  delete c;
  return FR_OK;
}

int fr_gemm_set_tuning(fr_gemm_ctx *c, int tuning, int search, int budget, int steps, double bw_gbs,
                       double bw_frac, uint64_t seed) {
  if (!c || budget < 1 || steps < 1 || bw_gbs < 0 || !(bw_frac > 0 && bw_frac <= 1)) return FR_ERR_INVALID_ARG;
  if (search != FR_SEARCH_EXHAUSTIVE && search != FR_SEARCH_RANDOM && search != FR_SEARCH_ANNEALING &&
      search != FR_SEARCH_MCMC)
    return FR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->tuning = tuning;
  c->search = search;
  c->budget = budget;
  c->steps = steps;
  c->bw_gbs = bw_gbs;
  c->bw_frac = bw_frac;
  c->seed = seed;
  c->keys.clear();
  return FR_OK;
}

int fr_gemm_num_configs(void) { return (int)gemm_space().size(); }

int fr_gemm_describe_config(int id, char *buf, int len) {
  if (id < 0 || id >= (int)gemm_space().size() || !buf || len < 1) return FR_ERR_INVALID_ARG;
  const GemmConfig &c = gemm_space()[id];
  std::snprintf(buf, len, "bgemm y=%d z=%d %s", c.y, c.z,
                c.pipe ? "pipelined" : (c.stage ? "stage=1" : "stage=0"));
  return FR_OK;
}

int fr_gemm_config_valid(int id, int m, int n, int k) { return gemm_valid(id, m, n, k) ? 1 : 0; }

int fr_gemm_run_config(int id, int m, int n, int k, const float *A, const float *B, float *C,
                       int batch, void *stream) {
  if (batch < 0 || batch > (1 << 26)) return FR_ERR_INVALID_ARG;
  if (batch == 0) return FR_OK;
  if (!A || !B || !C) return FR_ERR_INVALID_ARG;
  if (!gemm_valid(id, m, n, k)) return FR_ERR_UNSUPPORTED;
  cudaError_t e = gemm_launch(id, m, n, k, A, B, C, batch, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    fr_note_cuda_error((int)e);
    return FR_ERR_CUDA;
  }
  return FR_OK;
}

int fr_gemm_run(fr_gemm_ctx *c, int m, int n, int k, const float *A, const float *B, float *C,
                int batch, void *stream) {
  if (!c || batch < 0 || batch > (1 << 26)) return FR_ERR_INVALID_ARG;
  if (m < 2 || m > 32 || n < 2 || n > 32 || k < 2 || k > 32) return FR_ERR_INVALID_ARG;
  if (batch == 0) return FR_OK;
  if (!A || !B || !C) return FR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(c->mu);
  c->harvest();
  GemmKey &ks = c->state(m, n, k);
  // this call's steps: (configuration, instances, tuning?)
  std::vector<std::tuple<int, int, bool>> steps;
  const int fallback = ks.best >= 0 ? ks.best : -1;
  if (c->tuning && !ks.tuned) {
    std::vector<int> cfgs;
    const int want = std::min(c->steps, batch);
    if (ks.adaptive) {
      ks.walker.decide([&](int i) -> double {
        auto it = ks.meas.find(i);
        // the walk compares times per instance
        return it == ks.meas.end() || it->second.inst <= 0 ? 0.0 : it->second.ns / it->second.inst;
      });
      for (int i = 0; i < want && ks.proposed < c->budget; ++i) {
        const int p = ks.walker.propose();
        if (p < 0) break;
        cfgs.push_back(p);
        ++ks.proposed;
      }
    } else {
      while ((int)cfgs.size() < want && ks.next < ks.order.size() &&
             (int)ks.meas.size() + ks.pending + (int)cfgs.size() < c->budget)
        cfgs.push_back(ks.order[ks.next++]);
    }
    const int mcfg = (int)cfgs.size();
    for (int i = 0; i < mcfg; ++i) {
      const int lo = (int)((long long)batch * i / mcfg), hi = (int)((long long)batch * (i + 1) / mcfg);
      steps.emplace_back(cfgs[i], hi - lo, true);
    }
  }
  if (steps.empty()) {
    int cfg = fallback;
    if (cfg < 0)
      for (int i = 0; i < (int)gemm_space().size() && cfg < 0; ++i)
        if (gemm_valid(i, m, n, k)) cfg = i;
    if (cfg < 0) return FR_ERR_UNSUPPORTED;
    steps.emplace_back(cfg, batch, false);
  }
  long long off = 0;
  const auto key = std::make_tuple(m, n, k);
  for (auto &s : steps) {
    const int cfg = std::get<0>(s), cnt = std::get<1>(s);
    const bool tun = std::get<2>(s);
    GemmPending p{c->event(), c->event(), key, cfg, cnt, tun};
    cudaEventRecord(p.a, st);
    cudaError_t e = gemm_launch(cfg, m, n, k, A + off * m * k, B + off * k * n, C + off * m * n, cnt, st);
    cudaEventRecord(p.b, st);
    if (e != cudaSuccess) {
      fr_note_cuda_error((int)e);
      return FR_ERR_CUDA;
    }
    c->pending.push_back(p);
    if (tun) ++ks.pending;
    off += cnt;
  }
  return FR_OK;
}

int fr_gemm_report(fr_gemm_ctx *c, int m, int n, int k, int *tuned, int *evaluated, int *best,
                   double *best_gbs, double *overhead_pct) {
  if (!c) return FR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->harvest();
  auto it = c->keys.find(std::make_tuple(m, n, k));
  if (it == c->keys.end()) {
    if (tuned) *tuned = 0;
    if (evaluated) *evaluated = 0;
    if (best) *best = -1;
    if (best_gbs) *best_gbs = 0;
    if (overhead_pct) *overhead_pct = 0;
    return FR_OK;
  }
  GemmKey &ks = it->second;
  const double bytes = instance_bytes(m, n, k);
  c->update_best(ks, bytes);
  if (tuned) *tuned = ks.tuned ? 1 : 0;
  if (evaluated) *evaluated = (int)ks.meas.size();
  if (best) *best = ks.best;
  const double bg = ks.best >= 0 ? ks.meas[ks.best].gbs(bytes) : 0;
  if (best_gbs) *best_gbs = bg;
  if (overhead_pct)
    *overhead_pct = (bg > 0 && ks.all_inst > 0) ? 100.0 * (ks.all_ns * bg / (ks.all_inst * bytes) - 1.0) : 0;
  return FR_OK;
}

}  // extern "C"
