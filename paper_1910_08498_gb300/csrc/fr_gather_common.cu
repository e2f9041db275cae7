// fr_gather_common.cu -- shape table, shared-memory sizing and dispatch of
// the gather kernel family.
#include "fr_gather.cuh"
#include "fr_gather_shapes.h"

namespace fr {

#define FR_DECL(id, bx, by, zc)                                                             \
  cudaError_t launch_gather_shape##id##_kb4(int wmode, const InsertArgs &a, cudaStream_t st, \
                                            int query_only, KernelInfo *info);              \
  cudaError_t launch_gather_shape##id##_kb6(int wmode, const InsertArgs &a, cudaStream_t st, \
                                            int query_only, KernelInfo *info);              \
  cudaError_t launch_gather_persistent_shape##id##_kb4(int f16, const PersistentLaunch &p,   \
                                                       cudaStream_t st);                    \
  cudaError_t launch_gather_persistent_shape##id##_kb6(int f16, const PersistentLaunch &p,   \
                                                       cudaStream_t st);
FR_GATHER_SHAPES(FR_DECL)
#undef FR_DECL

int num_gather_shapes() { return FR_NUM_GATHER_SHAPES; }

GatherShape gather_shape(int id) {
#define FR_CASE(i, bx, by, zc) \
  if (id == i) return GatherShape{bx, by, zc};
  FR_GATHER_SHAPES(FR_CASE)
#undef FR_CASE
  return GatherShape{0, 0, 0};
}

static size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

size_t gather_smem_bytes(const GatherShape &sh, int wmode, int lut_n, int chunk) {
  const int nw = sh.bx * sh.by / 32;
  size_t b = 0;
  if (wmode == W_LUT) b += up16((size_t)lut_n * sizeof(float2));
  // per warp: image list, partial sums, item queues
  b += (size_t)nw * gather_warp_smem(sh.zc, chunk);
  return b;
}

size_t gather_persistent_smem_bytes(const GatherShape &sh, int chunk) {
  const int nw = sh.bx * sh.by / 32;
  return GATHER_ARGS_BYTES + (size_t)nw * gather_warp_smem(sh.zc, chunk);
}

cudaError_t launch_gather(int shape_id, int wmode, const InsertArgs &a, cudaStream_t st,
                          int query_only, KernelInfo *info) {
  switch (shape_id) {
#define FR_SW(i, bx, by, zc)                                                   \
  case i:                                                                      \
    return a.g.KB == 4 ? launch_gather_shape##i##_kb4(wmode, a, st, query_only, info) \
                       : launch_gather_shape##i##_kb6(wmode, a, st, query_only, info);
    FR_GATHER_SHAPES(FR_SW)
#undef FR_SW
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gather_persistent(int shape_id, int kb, int f16, const PersistentLaunch &p,
                                     cudaStream_t st) {
  switch (shape_id) {
#define FR_SWP(i, bx, by, zc)                                                  \
  case i:                                                                      \
    return kb == 4 ? launch_gather_persistent_shape##i##_kb4(f16, p, st)       \
                   : launch_gather_persistent_shape##i##_kb6(f16, p, st);
    FR_GATHER_SHAPES(FR_SWP)
#undef FR_SWP
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fr
