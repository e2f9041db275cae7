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
// group of instances with cp.async while computing the current one.  The
// bulk-copy family (bgemm_bulk_kernel, below) moves the blocks with the
// bulk-copy engine instead and computes register tiles of C.
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

// set by a bulk-copy kernel whose bounded wait gave up (fr_gemm_device_status)
static __device__ unsigned int g_gemm_error;
// limit of a bulk-copy kernel's waits for its copies, in ns of the global timer
// (fr_gemm_set_wait_limit; 1 s by default)
static __device__ long long g_gemm_wait_ns = 1000000000LL;

namespace fr {
namespace {

struct BulkGeom {
  int m, n, k, mk, kn, mn;
  int Z;             // instances per group
  int zt;            // instances computed at once (threads = zt * tiles)
  int tiles, tcols;  // register tiles per instance, tiles per row of C
  int ns;            // pipeline stages
  int sa, sb, sc;    // floats per stage buffer of A, B and of the C buffer (incl. 4 of slack)
  long long groups;
  int batch;
};

struct GemmConfig {
  int y, z, stage, pipe;  // pipe: persistent CTAs, next group prefetched with cp.async
  // bulk-copy family (bulk = 1): y x tx register tiles, r rounds of the CTA's
  // threads per group, at most cap threads per CTA
  int bulk = 0, tx = 1, r = 1, cap = 0;
};

const std::vector<GemmConfig> &gemm_space() {
  static const std::vector<GemmConfig> v = [] {
    std::vector<GemmConfig> c;
    for (int y : {1, 2, 4, 8})
      for (int z : {1, 2, 4, 8, 16, 32}) {
        for (int st : {0, 1}) c.push_back(GemmConfig{y, z, st, 0});
        c.push_back(GemmConfig{y, z, 0, 1});
      }
    for (int ty : {1, 2, 4})
      for (int tx : {1, 2, 4})
        for (int r : {1, 2, 4, 8})
          for (int cap : {128, 256}) c.push_back(GemmConfig{ty, 0, 0, 0, 1, tx, r, cap});
    return c;
  }();
  return v;
}

int gemm_threads(const GemmConfig &c, int m, int n) { return n * ((m + c.y - 1) / c.y) * c.z; }

// Launch geometry of a bulk-copy configuration for size (m, n, k); false if
// it cannot run (too many tiles, fewer than 32 threads, too much shared memory).
constexpr size_t BULK_SMEM_MAX = 226 * 1024;  // dynamic; static shared memory comes on top
bool bulk_plan(const GemmConfig &c, int m, int n, int k, long long batch, BulkGeom *g,
               size_t *smem, int *threads) {
  BulkGeom q{};
  q.m = m, q.n = n, q.k = k, q.mk = m * k, q.kn = k * n, q.mn = m * n;
  q.tcols = (n + c.tx - 1) / c.tx;
  q.tiles = ((m + c.y - 1) / c.y) * q.tcols;
  if (q.tiles > c.cap) return false;
  q.zt = c.cap / q.tiles;
  const int t = q.zt * q.tiles;
  if (t < 32) return false;
  q.Z = q.zt * c.r;
  auto round4 = [](long long f) { return (int)((f + 4 + 3) & ~3LL); };  // + shift slack
  q.sa = round4((long long)q.Z * q.mk);
  q.sb = round4((long long)q.Z * q.kn);
  q.sc = round4((long long)q.Z * q.mn);
  auto bytes = [&](int ns) { return 64 + 4 * ((size_t)ns * (q.sa + q.sb) + q.sc); };
  // two stages: a deeper ring holds more shared memory per CTA and so fewer
  // CTAs per SM, which measured slower (the compute phase needs the warps)
  q.ns = 2;
  if (bytes(q.ns) > BULK_SMEM_MAX) return false;
  q.batch = (int)batch;
  q.groups = (batch + q.Z - 1) / q.Z;
  if (g) *g = q;
  if (smem) *smem = bytes(q.ns);
  if (threads) *threads = t;
  return true;
}

size_t gemm_smem(const GemmConfig &c, int m, int n, int k) {
  if (c.pipe)  // two buffers of A and B, each with 16 B of alignment slack
    return 2 * ((size_t)c.z * ((size_t)m * k + (size_t)k * n) * sizeof(float) + 32);
  return (size_t)c.z * ((size_t)m * k + (size_t)k * n + (c.stage ? (size_t)m * n : 0)) * sizeof(float);
}

bool gemm_valid(int id, int m, int n, int k) {
  if (id < 0 || id >= (int)gemm_space().size()) return false;
  if (m < 2 || m > 32 || n < 2 || n > 32 || k < 2 || k > 32) return false;
  const GemmConfig &c = gemm_space()[id];
  if (c.bulk) return c.y <= m && c.tx <= n && bulk_plan(c, m, n, k, 1, nullptr, nullptr, nullptr);
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

// ------------------------------------------------------------ bulk-copy family
//
// Persistent CTAs stream groups of Z consecutive instances through a ring of
// two shared-memory stages.  One thread moves each group's A and B blocks (both
// contiguous in memory) with the bulk-copy engine (cp.async.bulk, completion
// counted in bytes on the stage's mbarrier), so the copy costs no per-element
// instructions; the 16-byte-aligned interior of a block goes by bulk copy and
// its at most 3 + 3 ragged floats by plain loads, each float landing at the
// same address modulo 16 as in global memory.  Compute: a thread owns a
// TY x TX register tile of C (TY rows interleaved with the other row tiles,
// clamped at the matrix edge), reading TY
// values of A and TX values of B per step of the inner dimension.  The
// group's C block is assembled in shared memory and written back by one bulk
// store (ragged ends by plain stores).  Every mbarrier wait is bounded by
// g_gemm_wait_ns of the global timer (GEMM_WAIT_NS unless a test sets it with
// fr_gemm_set_wait_limit); a wait that gives up records
// FR_ERR_TIMEOUT in g_gemm_error (fr_gemm_device_status) and the CTA stops
// after waiting (bounded by GEMM_WAIT_NS) for its copies still in flight.

constexpr long long GEMM_WAIT_NS = 1000000000LL;  // 1 s

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// true once the phase with the given parity has completed; false once a poll
// finds it incomplete limit_ns or more after the start, and at once for a
// limit of 0 (the fault-injection setting).  Between polls try_wait suspends
// the thread for a bounded, hardware-defined time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit_ns) {
  if (limit_ns <= 0) return false;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((long long)(global_ns() - t0) >= limit_ns) return false;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
}

__device__ __forceinline__ void bulk_load(float *dst, const float *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_store(float *dst, const float *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the bulk-copy engine
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A contiguous block of `count` floats at global address src, as the bulk
// copy sees it: `shift` = (src / 4) mod 4 (element e sits at buf[shift + e]),
// the 16-byte aligned interior [lo, hi) of element indices and its bytes.
struct BlockSpan {
  int shift, lo, hi;
  __device__ BlockSpan(const float *src, int count) {
    shift = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
    lo = min(count, (4 - shift) & 3);
    hi = max(lo, ((shift + count) & ~3) - shift);
  }
  __device__ uint32_t bytes() const { return 4u * (uint32_t)(hi - lo); }
};


template <int TY, int TX>
__global__ void __launch_bounds__(256) bgemm_bulk_kernel(const BulkGeom g, const float *__restrict__ A,
                                                          const float *__restrict__ B,
                                                          float *__restrict__ C) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw);          // g.ns barriers
  float *sbase = reinterpret_cast<float *>(smraw + 64);          // 16-byte aligned
  float *sC = sbase + (size_t)g.ns * (g.sa + g.sb);
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const long long wait_ns = tid == 0 ? g_gemm_wait_ns : 0;
  if (tid == 0) {
    for (int s = 0; s < g.ns; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
    s_abort = 0;
  }
  __syncthreads();

  auto stageA = [&](int s) { return sbase + (size_t)s * (g.sa + g.sb); };
  auto stageB = [&](int s) { return sbase + (size_t)s * (g.sa + g.sb) + g.sa; };
  // thread 0: start the bulk copies of group gi into stage s
  auto issue = [&](long long gi, int s) {
    const long long b0 = gi * g.Z;
    const int nb = (int)min((long long)g.Z, (long long)g.batch - b0);
    const float *a = A + b0 * g.mk, *b = B + b0 * g.kn;
    const BlockSpan sa(a, nb * g.mk), sb(b, nb * g.kn);
    mbar_arrive_expect_tx(&bar[s], sa.bytes() + sb.bytes());
    if (sa.hi > sa.lo) bulk_load(stageA(s) + sa.shift + sa.lo, a + sa.lo, sa.bytes(), &bar[s]);
    if (sb.hi > sb.lo) bulk_load(stageB(s) + sb.shift + sb.lo, b + sb.lo, sb.bytes(), &bar[s]);
  };
  // all threads: the ragged ends of group gi's blocks by plain loads
  auto edges_in = [&](long long gi, int s) {
    if (tid >= 32) return;
    const long long b0 = gi * g.Z;
    const int nb = (int)min((long long)g.Z, (long long)g.batch - b0);
    const bool isA = tid < 16;
    const float *src = isA ? A + b0 * g.mk : B + b0 * g.kn;
    const int cnt = nb * (isA ? g.mk : g.kn);
    float *dst = isA ? stageA(s) : stageB(s);
    const BlockSpan sp(src, cnt);
    const int q = tid & 15;  // q < 4: head element, 4 <= q < 8: tail element
    int e = -1;
    if (sp.hi > sp.lo) {
      if (q < 4 && q < sp.lo) e = q;
      else if (q >= 4 && q < 8 && sp.hi + (q - 4) < cnt) e = sp.hi + (q - 4);
    } else if (q < cnt) {  // no interior (fewer than 8 floats): all by plain loads
      e = q;
    }
    if (e >= 0) dst[sp.shift + e] = __ldg(src + e);
  };

  const long long G = g.groups;
  if (tid == 0)
    for (int s = 0; s < g.ns; ++s) {
      const long long gi = blockIdx.x + (long long)s * gridDim.x;
      if (gi < G) issue(gi, s);
    }
  const int tile = tid % g.tiles, tz = tid / g.tiles;
  const int tr = tile / g.tcols, tc = tile - tr * g.tcols;
  // a thread's rows are tr, tr + rt, ... (rt row tiles), not TY consecutive
  // rows: the A rows that a warp's lanes read at one step then lie k floats
  // apart instead of TY k, which spreads them over the shared-memory banks
  // when TY k is a multiple of 32 (k = 8, 16, 24, 32); +8 % on average over
  // 8 sizes, +39 % at 16 x 16 x 16
  const int rt = g.tiles / g.tcols;
  const int r0 = tr, c0 = tc * TX;
  const bool active = tz < g.zt;
  int i = 0;
  for (long long gi = blockIdx.x; gi < G; gi += gridDim.x, ++i) {
    const int s = i % g.ns;
    const uint32_t parity = (uint32_t)((i / g.ns) & 1);
    edges_in(gi, s);
    if (tid == 0) {
      bulk_wait_read_all();  // the previous group's C store has read sC
      if (!mbar_wait_bounded(&bar[s], parity, wait_ns)) s_abort = 1;
    }
    __syncthreads();
    if (s_abort) break;
    const long long b0 = gi * g.Z;
    const int nb = (int)min((long long)g.Z, (long long)g.batch - b0);
    const float *gA = A + b0 * g.mk, *gB = B + b0 * g.kn;
    float *gC = C + b0 * g.mn;
    const BlockSpan spA(gA, nb * g.mk), spB(gB, nb * g.kn), spC(gC, nb * g.mn);
    const float *sA = stageA(s) + spA.shift, *sB = stageB(s) + spB.shift;
    float *sCc = sC + spC.shift;
    if (active) {
      int arow[TY], bcol[TX];
#pragma unroll
      for (int r = 0; r < TY; ++r) arow[r] = min(r0 + r * rt, g.m - 1) * g.k;
      // columns past n are not clamped: they read at most TX - 1 floats past a
      // row of B, which stays inside this CTA's shared memory (the buffer's
      // slack, or the next region), and their results are never stored
#pragma unroll
      for (int c = 0; c < TX; ++c) bcol[c] = c0 + c;
      for (int t = tz; t < nb; t += g.zt) {
        const float *a = sA + t * g.mk, *b = sB + t * g.kn;
        float acc[TY][TX];
#pragma unroll
        for (int r = 0; r < TY; ++r)
#pragma unroll
          for (int c = 0; c < TX; ++c) acc[r][c] = 0.f;
#pragma unroll 2
        for (int p = 0; p < g.k; ++p) {
          float av[TY], bv[TX];
#pragma unroll
          for (int r = 0; r < TY; ++r) av[r] = a[arow[r] + p];
#pragma unroll
          for (int c = 0; c < TX; ++c) bv[c] = b[p * g.n + bcol[c]];
#pragma unroll
          for (int r = 0; r < TY; ++r)
#pragma unroll
            for (int c = 0; c < TX; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
        float *cc = sCc + t * g.mn;
#pragma unroll
        for (int r = 0; r < TY; ++r)
          if (r0 + r * rt < g.m)
#pragma unroll
            for (int c = 0; c < TX; ++c)
              if (c0 + c < g.n) cc[(r0 + r * rt) * g.n + c0 + c] = acc[r][c];
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (spC.hi > spC.lo) {
        bulk_store(gC + spC.lo, sCc + spC.lo, spC.bytes());
        bulk_commit();
      }
      const long long gn = gi + (long long)g.ns * gridDim.x;
      if (gn < G) issue(gn, s);
    }
    // ragged ends of C by plain stores (sC is not rewritten before the next barrier)
    if (tid < 8) {
      const int q = tid;
      const int cnt = nb * g.mn;
      int e = -1;
      if (spC.hi > spC.lo) {
        if (q < 4 && q < spC.lo) e = q;
        else if (q >= 4 && spC.hi + (q - 4) < cnt) e = spC.hi + (q - 4);
      } else if (q < cnt) {
        e = q;
      }
      if (e >= 0) gC[e] = sCc[e];
    }
  }
  if (tid == 0) {
    if (s_abort) {
      atomicOr(&g_gemm_error, 1u);
      // bounded waits for the copies still in flight (groups i .. i + ns - 1),
      // so that none lands after the CTA's shared memory is released
      for (int j = 0; j < g.ns; ++j) {
        const long long gj = blockIdx.x + (long long)(i + j) * gridDim.x;
        if (gj < G)
          mbar_wait_bounded(&bar[(i + j) % g.ns], (uint32_t)(((i + j) / g.ns) & 1), GEMM_WAIT_NS);
      }
    }
    bulk_wait_all();
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

template <int TY, int TX>
cudaError_t launch_bulk(const GemmConfig &c, int m, int n, int k, const float *A, const float *B,
                        float *C, int batch, cudaStream_t st) {
  BulkGeom g;
  size_t smem = 0;
  int threads = 0;
  if (!bulk_plan(c, m, n, k, batch, &g, &smem, &threads)) return cudaErrorInvalidValue;
  auto fn = bgemm_bulk_kernel<TY, TX>;
  cudaError_t e = allow_dynamic_smem((const void *)fn, BULK_SMEM_MAX, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const int per_sm = resident_ctas((const void *)fn, threads, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long grid = std::min<long long>(g.groups, (long long)per_sm * sms);
  fn<<<(unsigned)grid, threads, smem, st>>>(g, A, B, C);
  return cudaGetLastError();
}

cudaError_t gemm_launch(int id, int m, int n, int k, const float *A, const float *B, float *C,
                        int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const GemmConfig &c = gemm_space()[id];
  if (c.bulk) {
    switch (c.y * 8 + c.tx) {
      case 9: return launch_bulk<1, 1>(c, m, n, k, A, B, C, batch, st);
      case 10: return launch_bulk<1, 2>(c, m, n, k, A, B, C, batch, st);
      case 12: return launch_bulk<1, 4>(c, m, n, k, A, B, C, batch, st);
      case 17: return launch_bulk<2, 1>(c, m, n, k, A, B, C, batch, st);
      case 18: return launch_bulk<2, 2>(c, m, n, k, A, B, C, batch, st);
      case 20: return launch_bulk<2, 4>(c, m, n, k, A, B, C, batch, st);
      case 33: return launch_bulk<4, 1>(c, m, n, k, A, B, C, batch, st);
      case 34: return launch_bulk<4, 2>(c, m, n, k, A, B, C, batch, st);
      case 36: return launch_bulk<4, 4>(c, m, n, k, A, B, C, batch, st);
      default: return cudaErrorInvalidValue;
    }
  }
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

// Neighbours for the annealing and Metropolis walks: configurations of one
// family that differ in exactly one tuning dimension; across the two families
// (the family being one more dimension), those with the same row coarsening.
bool gemm_neighbours(const GemmConfig &x, const GemmConfig &y) {
  if (x.bulk != y.bulk) return x.y == y.y;
  if (x.bulk)
    return (x.y != y.y) + (x.tx != y.tx) + (x.r != y.r) + (x.cap != y.cap) == 1;
  return (x.y != y.y) + (x.z != y.z) + (x.stage != y.stage) + (x.pipe != y.pipe) == 1;
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
          if (gemm_neighbours(x, y)) ks.walker.nbr[a].push_back(b);
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

int fr_gemm_device_status(void) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_gemm_error, sizeof(v));
  if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_gemm_error, &zero, sizeof(zero));
  if (e != cudaSuccess) {
    fr_note_cuda_error((int)e);
    return FR_ERR_CUDA;
  }
  return v ? FR_ERR_TIMEOUT : FR_OK;
}

int fr_gemm_set_wait_limit(long long ns) {
  if (ns < 0 || ns > 10000000000LL) return FR_ERR_INVALID_ARG;
  const cudaError_t e = cudaMemcpyToSymbol(g_gemm_wait_ns, &ns, sizeof(ns));
  if (e != cudaSuccess) {
    fr_note_cuda_error((int)e);
    return FR_ERR_CUDA;
  }
  return FR_OK;
}

int fr_gemm_num_configs(void) { return (int)gemm_space().size(); }

int fr_gemm_describe_config(int id, char *buf, int len) {
  if (id < 0 || id >= (int)gemm_space().size() || !buf || len < 1) return FR_ERR_INVALID_ARG;
  const GemmConfig &c = gemm_space()[id];
  if (c.bulk)
    std::snprintf(buf, len, "bgemm bulk ty=%d tx=%d r=%d t=%d", c.y, c.tx, c.r, c.cap);
  else
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
