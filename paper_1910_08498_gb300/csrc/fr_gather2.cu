// fr_gather2.cu -- shared-memory sizing, per-device attribute cache and
// dispatch of the direct-drain gather (fr_gather2.cuh); the kernels are
// instantiated per brick shape in fr_gather2_s<k>.cu.
#include <mutex>
#include <vector>

#include "fr_gather2.cuh"

namespace fr {

// The dynamic shared memory a kernel may use is a per-device attribute:
// remember, per device and kernel, the size already allowed.
cudaError_t allow_dynamic_smem(const void *fn, size_t smem, int carveout) {
  struct Entry { int dev; const void *fn; size_t smem; };
  static std::mutex mu;
  static std::vector<Entry> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  for (const Entry &d : done)
    if (d.dev == dev && d.fn == fn && d.smem >= smem) return cudaSuccess;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  // the opt-in limit covers static and dynamic shared memory together
  if (smem + fa.sharedSizeBytes > (size_t)optin) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && carveout >= 0)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
  if (e != cudaSuccess) return e;
  for (Entry &d : done)
    if (d.dev == dev && d.fn == fn) { d.smem = smem; return cudaSuccess; }
  done.push_back(Entry{dev, fn, smem});
  return cudaSuccess;
}

int device_sm_count() {
  static std::mutex mu;
  static std::vector<int> n;  // by device ordinal
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)n.size() <= dev) n.resize(dev + 1, 0);
  if (n[dev] <= 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

int resident_ctas(const void *fn, int threads, size_t smem) {
  struct Entry { int dev; const void *fn; int threads; size_t smem; int ctas; };
  static std::mutex mu;
  static std::vector<Entry> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry &d : done)
      if (d.dev == dev && d.fn == fn && d.threads == threads && d.smem == smem) return d.ctas;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
    return 0;
  std::lock_guard<std::mutex> lk(mu);
  done.push_back(Entry{dev, fn, threads, smem, per_sm});
  return per_sm;
}

cudaError_t launch_multi(const void *fn, const MultiLaunch &p, int threads, size_t smem,
                         cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)p.nitems);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = p.priority;
  cfg.attrs = attr;
  cfg.numAttrs = p.priority != 0 ? 1 : 0;
  void *params[] = {const_cast<MultiLaunch *>(&p)};
  return cudaLaunchKernelExC(&cfg, fn, params);
}

size_t gather2_smem_bytes(const GatherShape &sh, int chunk) {
  const int nw = sh.bx * sh.by / 32;
  return (size_t)nw * (sh.zc == 8 ? gather2_warp_smem<8>(chunk) : gather2_warp_smem<16>(chunk));
}

// brick shapes: columns in x, columns in y, voxels per column (z)
static const GatherShape kShapes2[] = {{16, 16, 8}, {16, 8, 8}, {16, 8, 16}};

int num_gather2_shapes() { return (int)(sizeof(kShapes2) / sizeof(kShapes2[0])); }

GatherShape gather2_shape(int id) {
  return id >= 0 && id < num_gather2_shapes() ? kShapes2[id] : GatherShape{0, 0, 0};
}

cudaError_t launch_gather2_shape0(int minw, const InsertArgs &a, cudaStream_t st, int query_only,
                                  KernelInfo *info);
cudaError_t launch_gather2_shape1(int minw, const InsertArgs &a, cudaStream_t st, int query_only,
                                  KernelInfo *info);
cudaError_t launch_gather2_shape2(int minw, const InsertArgs &a, cudaStream_t st, int query_only,
                                  KernelInfo *info);

cudaError_t launch_gather2_multi_shape0(int minw, int f16, const MultiLaunch &p, cudaStream_t st);
cudaError_t launch_gather2_multi_shape1(int minw, int f16, const MultiLaunch &p, cudaStream_t st);
cudaError_t launch_gather2_multi_shape2(int minw, int f16, const MultiLaunch &p, cudaStream_t st);

cudaError_t launch_gather2_multi(int shape_id, int minw, int f16, const MultiLaunch &p,
                                 cudaStream_t st) {
  if (p.base.chunk > 64 || p.base.g.KB != 4) return cudaErrorInvalidValue;
  switch (shape_id) {
    case 0: return launch_gather2_multi_shape0(minw, f16, p, st);
    case 1: return launch_gather2_multi_shape1(minw, f16, p, st);
    case 2: return launch_gather2_multi_shape2(minw, f16, p, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gather2(int shape_id, int minw, const InsertArgs &a, cudaStream_t st,
                           int query_only, KernelInfo *info) {
  if (a.g.KB != 4 || a.chunk > 64) return cudaErrorInvalidValue;
  // two-pixel row loads: the images must be 16-byte aligned (fr_insert checks it)
  if (reinterpret_cast<uintptr_t>(a.images) & 15u) return cudaErrorInvalidValue;
  switch (shape_id) {
    case 0: return launch_gather2_shape0(minw, a, st, query_only, info);
    case 1: return launch_gather2_shape1(minw, a, st, query_only, info);
    case 2: return launch_gather2_shape2(minw, a, st, query_only, info);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fr
