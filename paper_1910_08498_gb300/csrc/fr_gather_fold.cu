// fr_gather_fold.cu -- the direct-drain gather instantiated for the fold
// columns |x| <= floor(a) (FOLD): bricks one 4-column footprint wide
// (4 x 32 x 8, four 4 x 8 warp footprints stacked in y), the fold predicate
// tested per candidate, 4 x 4 boxes (a < 2), polynomial weights.  Launched
// beside the main direct-drain launch, which covers x >= floor(a) + 1: for one
// batch, or for the work items of several batches in one launch.
#include "fr_gather2.cuh"

namespace fr {

namespace {
constexpr int FBX = 4, FBY = 32, FZC = 8, FFW = 4;
constexpr int FOLD_MINW = 16;  // resident warps per SM the registers allow
constexpr size_t fold_smem(int chunk) { return (size_t)(FBX * FBY / 32) * gather2_warp_smem<FZC>(chunk); }
}  // namespace

GatherShape fold_shape() { return GatherShape{FBX, FBY, FZC}; }

template <int F16>
static cudaError_t launch_fold(const InsertArgs &a, cudaStream_t st) {
  auto fn = gather2_kernel<FBX, FBY, FZC, F16, FOLD_MINW, FFW, 1>;
  const size_t smem = fold_smem(a.chunk);
  cudaError_t e = allow_dynamic_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  if (a.nunits <= 0) return cudaSuccess;
  fn<<<a.nunits, FBX * FBY, smem, st>>>(a);
  return cudaGetLastError();
}

template <int F16>
static cudaError_t launch_fold_multi(const MultiLaunch &p, cudaStream_t st) {
  auto fn = gather2_multi_kernel<FBX, FBY, FZC, F16, FOLD_MINW, FFW, 1>;
  const size_t smem = GATHER_ARGS_BYTES + fold_smem(p.base.chunk);
  cudaError_t e = allow_dynamic_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  if (p.nitems <= 0) return cudaSuccess;
  return launch_multi((const void *)fn, p, FBX * FBY, smem, st);
}

cudaError_t launch_gather_fold_multi(int f16, const MultiLaunch &p, cudaStream_t st) {
  if (p.base.g.KB != 4 || p.base.chunk > 64) return cudaErrorInvalidValue;
  return f16 ? launch_fold_multi<1>(p, st) : launch_fold_multi<0>(p, st);
}

cudaError_t launch_gather_fold(const InsertArgs &a, cudaStream_t st) {
  if (a.g.KB != 4 || a.chunk > 64) return cudaErrorInvalidValue;
  if (reinterpret_cast<uintptr_t>(a.images) & 15u) return cudaErrorInvalidValue;
  return a.f16 ? launch_fold<1>(a, st) : launch_fold<0>(a, st);
}

}  // namespace fr
