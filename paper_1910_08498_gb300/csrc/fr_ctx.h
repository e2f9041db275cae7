// fr_ctx.h -- the context object behind the opaque fr_ctx handle.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/fr.h"
#include "fr_internal.h"
#include "fr_tuner.h"

struct fr_ctx {
  int S = 0;
  fr_blob blob{};
  fr::Geom g{};
  int device = 0;
  float *acc = nullptr;
  size_t plane = 0;
  float2 *lut = nullptr;
  int lut_n = 0;
  float lut_scale = 0.f;
  float inv_i0a = 0.f, inv_pa = 0.f;
  float poly[fr::POLY_N] = {};
  double poly_err = 1.0;  // max |poly - b| measured on the host (FP32 Horner)
  float4 *scratch = nullptr;
  int *d_err = nullptr;
  unsigned long long *d_count = nullptr;
  fr_options opt{};
  cudaStream_t last_stream = nullptr;
  unsigned long long images = 0;
  int launches = 0;
  int alloc_countdown = 0;  // fault injection: allocations left before the injected failure
  fr::Tuner tuner;
  // gather work-unit lists, keyed by (brick shape, n); most recent first
  struct Units {
    int shape = -1, n = -1, count = 0, any_split = 0, algo = 0;
    int4 *dev = nullptr;
    // direct-drain gather: the units of its fold-column launch (|x| <=
    // floor(a)), stored after the main units in dev
    int fold_count = 0, fold_split = 0;
    const int4 *fold = nullptr;
  };
  Units units[8];
  unsigned long long *d_phase = nullptr;  // gather phase counters (debug bit 1)
  // side stream (highest priority) and fork/join events: the direct-drain
  // gather's fold-column launch runs beside its main launch
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // cost model
  float *d_mlp = nullptr;
  bool mlp_trained = false;
  // reconstruction (Algorithm 1's last step): weighted half spectrum and the
  // inverse-FFT plan, created on first use
  float2 *spec = nullptr;
  int fft_plan = -1;
  // image transforms: batched R2C plans (full chunk, tail) and the FP16 staging buffer
  int prep_plan[2] = {-1, -1};
  int prep_batch[2] = {0, 0};
  float2 *prep_ws = nullptr;
};


namespace fr {
int key_bucket(int n);
InsertArgs base_args(const fr_ctx *c);
// allocate the context's float4 scratch volume if it has none yet
int ensure_scratch(fr_ctx *c);
// create the context's side stream and fork/join events if it has none yet
int ensure_side_stream(fr_ctx *c);
// gather work unit with its expected load (images it scans)
struct UnitLoad {
  double load;
  int4 unit;  // brick x, y, z; split | nsplit << 16
};
double gather_unit_loads(const fr_ctx *c, int shape, int n, double target,
                         std::vector<UnitLoad> &out, int &any_split);
// work units of bricks of shape sh tiling x in [x0, x1] (all y, z), split so
// that no unit exceeds `target` expected images (target <= 0: the total over
// per_sm units per SM, at least UNIT_MIN_LOAD), into at most 64 units of at
// least SPLIT_MIN_IMAGES images per brick; returns the total expected load
constexpr double UNIT_MIN_LOAD = 16.0;
constexpr int SPLIT_MIN_IMAGES = 8;
// units per SM of the direct-drain gather's main launch and of its fold-column
// launch (the fold bricks are few and every plane crosses the central ones:
// fine splits keep that launch's serial path inside the main launch's time)
constexpr int MAIN_UNITS_PER_SM = 32;
constexpr int FOLD_UNITS_PER_SM = 8;
double brick_unit_loads(const fr_ctx *c, const GatherShape &sh, int x0, int x1, int n,
                        double target, int per_sm, std::vector<UnitLoad> &out, int &any_split);
// drop cached batched-insertion plans that refer to c (called by fr_destroy)
void batched_forget(const fr_ctx *c);
// release the reconstruction buffers of c (called by fr_destroy)
void reconstruct_release(fr_ctx *c);
int do_insert_ctx(fr_ctx *c, const void *images, fr_dtype dtype, const float *rot, int n,
                  cudaStream_t st);
}  // namespace fr
