// fr_gather_fold.cu -- the per-voxel gather instantiated for the fold
// columns x <= floor(a) (InsertArgs::fold_only): bricks one 8-column
// footprint wide (8 x 16 x 8), so that every warp of a CTA holds fold columns,
// 4 x 4 boxes (a < 2), polynomial weights.  Launched beside the direct-drain
// gather, which covers x >= floor(a) + 1: for one batch, or for the work
// items of several batches in one launch.
#include "fr_gather.cuh"

namespace fr {

GatherShape fold_shape() { return GatherShape{8, 16, 8}; }

template <int F16>
static cudaError_t launch_fold(const InsertArgs &a, cudaStream_t st) {
  auto fn = gather_kernel<8, 16, 8, W_POLY, 4, F16>;
  const size_t smem = (size_t)(8 * 16 / 32) * gather_warp_smem(8, a.chunk);
  cudaError_t e = allow_dynamic_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  if (a.nunits <= 0) return cudaSuccess;
  fn<<<a.nunits, 8 * 16, smem, st>>>(a);
  return cudaGetLastError();
}

template <int F16>
static cudaError_t launch_fold_multi(const MultiLaunch &p, cudaStream_t st) {
  auto fn = gather_multi_kernel<8, 16, 8, W_POLY, 4, F16>;
  const size_t smem = GATHER_ARGS_BYTES + (size_t)(8 * 16 / 32) * gather_warp_smem(8, p.base.chunk);
  cudaError_t e = allow_dynamic_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  if (p.nitems <= 0) return cudaSuccess;
  return launch_multi((const void *)fn, p, 8 * 16, smem, st);
}

cudaError_t launch_gather_fold_multi(int f16, const MultiLaunch &p, cudaStream_t st) {
  if (p.base.g.KB != 4 || !p.base.fold_only) return cudaErrorInvalidValue;
  return f16 ? launch_fold_multi<1>(p, st) : launch_fold_multi<0>(p, st);
}

cudaError_t launch_gather_fold(const InsertArgs &a, cudaStream_t st) {
  if (a.g.KB != 4 || !a.fold_only) return cudaErrorInvalidValue;
  return a.f16 ? launch_fold<1>(a, st) : launch_fold<0>(a, st);
}

}  // namespace fr
