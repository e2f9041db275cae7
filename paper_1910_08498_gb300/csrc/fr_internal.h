// fr_internal.h -- types shared by the kernels and the host runtime of libfr.
//
// Accumulator layout in HBM.  Folding puts every insertion point at q_x >= 0,
// so a voxel with x < -floor(a) is never touched; the context stores only
// x in [xa0, S/2] with xa0 = -floor(a).  Six float planes, each
// [z][y][x - xa0] (x fastest), hold a double-float (hi + lo) running sum of
// V.re, V.im and W:  plane p at acc + p * plane_elems, order
// {Vre_hi, Vim_hi, W_hi, Vre_lo, Vim_lo, W_lo}.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace fr {

// blob weights: table staged in shared memory (precomputed), Abramowitz &
// Stegun Bessel approximations evaluated per pixel, or a Chebyshev polynomial
// in r^2 held in registers (both on the fly)
enum WeightMode { W_LUT = 0, W_OTF = 1, W_POLY = 2 };
constexpr int POLY_N = 12;  // coefficients of the degree-11 weight polynomial
enum Algo { ALGO_GATHER = 0, ALGO_SCATTER = 1, ALGO_GATHER2 = 2 };

struct Geom {
  int S;      // image side (even)
  int H;      // S / 2
  int NX;     // stored columns per row, S / 2 + 1
  int D;      // volume side, S + 1
  int xa0;    // first stored accumulator x coordinate, -floor(a)
  int NXa;    // stored accumulator x extent, H - xa0 + 1
  float a;    // blob radius
  float a2;   // a * a
  float alpha;
  int KB;     // candidate box width per axis: floor(2a) + 1 rounded up to 4 or 6
};

// Per-launch arguments of the insertion kernels.
struct InsertArgs {
  Geom g;
  const void *images;   // [n][S][NX] complex, FP32 (float2) or FP16 (half2)
  int f16;              // 1 if images are FP16
  const float *rot;     // [n][9]
  int n;                // images in this launch
  float *acc;           // 6 planes (see above)
  size_t plane;         // elements per plane
  const float2 *lut;    // blob table: (value at node i, value[i+1] - value[i]), lut_n entries
  int lut_n;
  float lut_scale;      // (lut_n - 1) / a^2
  float inv_i0a;        // 1 / I0(alpha) (on-the-fly weights)
  float inv_pa;         // 1 / (A&S 9.8.2 polynomial at 3.75 / alpha) (on-the-fly weights)
  float poly[POLY_N];   // b as a polynomial in x = 2 r^2 / a^2 - 1, power basis (W_POLY)
  float2 poly2[POLY_N]; // the same coefficients as pairs (c_k, c_k) for packed FP32x2 FMAs
  int *err;             // device error word
  // gather geometry
  int nbx, nby, nbz;    // bricks per axis
  int chunk;            // capacity of a warp's image list
  const int4 *units;    // work units: (brick x, y, z, split | nsplit << 16), one per CTA
  int nunits;
  int any_split;        // 1 if some unit shares its brick with other units
  unsigned long long *phase;  // optional per-phase cycle and item counters (PH_*), or null
  // scatter
  float4 *scratch;      // [z][y][x - xa0] (re, im, w, 0)
};

// Per-phase counters of the gather kernel (diagnostics, enabled by
// fr_options.debug bit 1): SM clock cycles spent by warps in each phase and
// item counts.
enum PhaseCounter {
  PH_CULL = 0, PH_QUEUE, PH_DRAIN_FAST, PH_DRAIN_EDGE, PH_DRAIN_CAREFUL, PH_FLUSH,
  PH_ITEMS_FAST, PH_ITEMS_EDGE, PH_ITEMS_CAREFUL, PH_LIST_IMAGES, PH_WARP_CYCLES, PH_ROUNDS,
  PH_DRAIN_FOLD, PH_ITEMS_FOLD,
  PH_COUNT = 16
};

// Error bits written to the device error word.
enum DevErr { DERR_RANGE = 1, DERR_TIMEOUT = 2 };

struct KernelInfo {
  const void *fn;       // __global__ function pointer
  int threads;          // block size
  size_t smem;          // dynamic shared memory for the launch
};

// ---- gather family: template parameters of one instantiation
struct GatherShape {
  int bx, by, zc;       // brick: bx x by columns of zc voxels (one column per thread)
};

// launchers implemented in the .cu files
cudaError_t launch_gather(int shape_id, int wmode, const InsertArgs &a, cudaStream_t st,
                          int query_only, KernelInfo *info);
// direct-drain gather (fr_gather2.cuh): brick shape id of gather2_shape(),
// register budget for minw (16, 20, 24) resident warps per SM
int num_gather2_shapes();
GatherShape gather2_shape(int id);
cudaError_t launch_gather2(int shape_id, int minw, const InsertArgs &a, cudaStream_t st,
                           int query_only, KernelInfo *info);
size_t gather2_smem_bytes(const GatherShape &sh, int chunk);
// allow a kernel `smem` bytes of dynamic shared memory on the current device
// (and, if carveout >= 0, set its preferred shared-memory carveout in percent);
// remembered per device and kernel; thread-safe
cudaError_t allow_dynamic_smem(const void *fn, size_t smem, int carveout = -1);
// SM count of the current device (cached per device; thread-safe)
int device_sm_count();
// resident CTAs per SM of kernel fn with `threads` threads and `smem` bytes
// of dynamic shared memory on the current device (cached per device, kernel
// and size; thread-safe); 0 if it cannot run
int resident_ctas(const void *fn, int threads, size_t smem);
cudaError_t launch_scatter(int threads, int wmode, const InsertArgs &a, cudaStream_t st,
                           int query_only, KernelInfo *info);
cudaError_t launch_merge_scratch(const InsertArgs &a, cudaStream_t st);
// 1 / (A&S 9.8.2 polynomial at 3.75 / alpha): the constant of the on-the-fly weights
float otf_inv_pa(double alpha);
// record a CUDA error for fr_last_cuda_error
void fr_note_cuda_error(int e);
cudaError_t launch_finalize(const Geom &g, const float *acc, size_t plane, float2 *V, float *W,
                            cudaStream_t st);
cudaError_t launch_count(const Geom &g, const float *rot, int n, unsigned long long *out,
                         cudaStream_t st);
cudaError_t launch_debug_fold(const float *r, const int *k, int m, int *out, cudaStream_t st);
cudaError_t launch_debug_blob(const InsertArgs &a, const float *r2, int m, int mode, float *out,
                              cudaStream_t st);

// number of gather shapes and their geometry
int num_gather_shapes();
GatherShape gather_shape(int id);
// the direct-drain gather over the fold columns |x| <= floor(a) only, in
// bricks of fold_shape() (one 4-column footprint wide), polynomial weights
GatherShape fold_shape();
cudaError_t launch_gather_fold(const InsertArgs &a, cudaStream_t st);
// dynamic shared memory a gather launch needs
size_t gather_smem_bytes(const GatherShape &sh, int wmode, int lut_n, int chunk);
size_t gather_persistent_smem_bytes(const GatherShape &sh, int chunk);

// One persistent gather launch over the work items of several batches.
struct PersistentLaunch {
  const InsertArgs *descs;  // device, one per batch
  const int4 *items;        // device, {bx | by << 10 | bz << 20, split word, batch, 0}, one per unit
  int nitems;
  int chunk;                // image-list capacity per warp, common to all batches
  unsigned *counter;        // device, zero at launch
};
cudaError_t launch_gather_persistent(int shape_id, int kb, int f16, const PersistentLaunch &p,
                                     cudaStream_t st);

// One launch over the work items of several batches, one CTA per item (the
// hardware block scheduler hands out the items, heaviest first).  The
// batches of one launch share S, blob, dtype and configuration: what they
// share stays in the kernel parameters (base), the rest is read per batch.
constexpr int MULTI_MAX = 64;  // batches per multi-batch launch
struct MultiLaunch {
  InsertArgs base;           // common arguments: geometry, weights, list capacity
  const InsertArgs *descs;   // device, one per batch (images, rot, n, acc, scratch, err)
  const int4 *items;         // device, {bx | by << 10 | bz << 20, split word, batch, slot}
  int nitems;
  int priority;              // launch priority (cudaLaunchAttributePriority), 0 = the stream's
  const void *images[MULTI_MAX];  // images of the launch's batches, by slot (read in the inner loop)
};
// launch kernel fn (taking one MultiLaunch) with p.nitems CTAs, at p.priority
cudaError_t launch_multi(const void *fn, const MultiLaunch &p, int threads, size_t smem,
                         cudaStream_t st);
// the direct-drain gather (fold columns excluded), FP32 or FP16 images
cudaError_t launch_gather2_multi(int shape_id, int minw, int f16, const MultiLaunch &p,
                                 cudaStream_t st);
// the direct-drain gather over the fold columns
cudaError_t launch_gather_fold_multi(int f16, const MultiLaunch &p, cudaStream_t st);

// MLP kernels
cudaError_t mlp_forward(const float *params, const float *x, int m, float *y, cudaStream_t st);
cudaError_t mlp_backward(const float *params, const float *x, const float *t, int m, float *grad,
                         float *loss, float *work, cudaStream_t st);
cudaError_t mlp_adam(float *params, const float *grad, float *m1, float *m2, int t, float lr,
                     float b1, float b2, float eps, cudaStream_t st);
size_t mlp_work_floats(int m);

constexpr int MLP_IN = 16, MLP_H = 64;
constexpr int MLP_NPARAM = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;

}  // namespace fr
