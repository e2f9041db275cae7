// fr_runtime.cu -- host runtime of libfr: contexts, the configuration space,
// the non-blocking dynamic tuner (Sec. 3.2, Sec. 5.3), tuning-cache
// persistence and the C ABI declared in include/fr.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "../../include/fr.h"
#include "fr_internal.h"
#include "fr_ctx.h"
#include "fr_tuner.h"

using namespace fr;

namespace {

std::atomic<int> g_last_cuda{0};

inline int cuda_fail(cudaError_t e) {
  g_last_cuda.store((int)e);
  if (e == cudaErrorMemoryAllocation) return FR_ERR_OOM;
  return FR_ERR_CUDA;
}

#define FR_CUDA(call)                         \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// Host evaluation of the A&S 9.8.2 polynomial (same coefficients as the device).
double as_982_host(double u) {
  const double c[9] = {0.39894228, 0.01328592, 0.00225319, -0.00157565, 0.00916281,
                       -0.02057706, 0.02635537, -0.01647633, 0.00392377};
  double r = c[8];
  for (int k = 7; k >= 0; --k) r = r * u + c[k];
  return r;
}

// Chebyshev interpolant of degree POLY_N-1 of f on [-1, 1] at the first-kind
// nodes x_k = cos((k + 1/2) pi / N) (Mason & Handscomb, Chebyshev Polynomials,
// 2003, Sec. 6.3: c_j = (2/N) sum_k f(x_k) T_j(x_k), c_0 halved), converted to
// the power basis with T_{j+1} = 2 x T_j - T_{j-1}.
template <class F>
void chebyshev_power_basis(F f, double *mono) {
  const int N = POLY_N;
  const double pi = 3.14159265358979323846;
  double fx[N], cheb[N];
  for (int k = 0; k < N; ++k) fx[k] = f(std::cos(pi * (k + 0.5) / N));
  for (int j = 0; j < N; ++j) {
    double s = 0;
    for (int k = 0; k < N; ++k) s += fx[k] * std::cos(pi * j * (k + 0.5) / N);
    cheb[j] = 2.0 * s / N;
  }
  cheb[0] *= 0.5;
  double tprev[N] = {0}, tcur[N] = {0}, tnext[N];
  tprev[0] = 1.0;  // T_0
  tcur[1] = 1.0;   // T_1
  for (int i = 0; i < N; ++i) mono[i] = cheb[0] * tprev[i] + (N > 1 ? cheb[1] * tcur[i] : 0.0);
  for (int j = 2; j < N; ++j) {
    for (int i = 0; i < N; ++i) tnext[i] = (i ? 2.0 * tcur[i - 1] : 0.0) - tprev[i];
    for (int i = 0; i < N; ++i) mono[i] += cheb[j] * tnext[i];
    for (int i = 0; i < N; ++i) { tprev[i] = tcur[i]; tcur[i] = tnext[i]; }
  }
}

}  // namespace

namespace fr {

InsertArgs base_args(const fr_ctx *c) {
  InsertArgs a{};
  a.g = c->g;
  a.acc = c->acc;
  a.plane = c->plane;
  a.lut = c->lut;
  a.lut_n = c->lut_n;
  a.lut_scale = c->lut_scale;
  a.inv_i0a = c->inv_i0a;
  a.inv_pa = c->inv_pa;
  for (int k = 0; k < POLY_N; ++k) {
    a.poly[k] = c->poly[k];
    a.poly2[k] = make_float2(c->poly[k], c->poly[k]);
  }
  a.err = c->d_err;
  a.scratch = c->scratch;
  a.phase = (c->opt.debug & 2) ? c->d_phase : nullptr;
  return a;
}

void fr_note_cuda_error(int e) { g_last_cuda.store(e); }

float otf_inv_pa(double alpha) {
  return alpha > 3.75 ? (float)(1.0 / as_982_host(3.75 / alpha)) : 1.0f;
}

// host-side fault injection (fr_options.fault_alloc): true for the allocation
// that is to fail
bool alloc_fault(fr_ctx *c) {
  if (c->alloc_countdown <= 0) return false;
  if (--c->alloc_countdown) return false;
  c->opt.fault_alloc = 0;  // one shot: a later fr_set_options from fr_get_options does not re-arm it
  return true;
}

int ensure_side_stream(fr_ctx *c) {
  if (c->side) return FR_OK;
  int lo = 0, hi = 0;
  FR_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  FR_CUDA(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi));
  FR_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  FR_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  return FR_OK;
}

int ensure_scratch(fr_ctx *c) {
  if (c->scratch) return FR_OK;
  if (alloc_fault(c)) return FR_ERR_OOM;
  FR_CUDA(cudaMalloc(&c->scratch, c->plane * sizeof(float4)));
  FR_CUDA(cudaMemset(c->scratch, 0, c->plane * sizeof(float4)));
  return FR_OK;
}

// Work units of a gather launch.  A brick at distance d from the centre is
// crossed, within a + (brick radius) r, by a fraction min(1, (a + r) / d) of
// uniformly oriented planes through the origin, so its expected image count is
// n min(1, (a + r) / d).  Bricks whose count exceeds a target share are split
// into several units, each taking a contiguous range of the images.  `target`
// <= 0 selects the share of one launch of this batch alone (total load over
// per_sm units per SM, at least UNIT_MIN_LOAD).  Every plane crosses the
// bricks at the centre, whose warps take the images of their unit one after
// another: the split floor bounds that serial path (at most 64 units per
// brick, at least SPLIT_MIN_IMAGES images each).  Returns the units with
// their expected loads, unsorted.
double brick_unit_loads(const fr_ctx *c, const GatherShape &sh, int x0, int x1, int n,
                        double target, int per_sm, std::vector<UnitLoad> &out, int &any_split) {
  const Geom &g = c->g;
  const int nbx = (x1 - x0 + sh.bx) / sh.bx, nby = (g.D + sh.by - 1) / sh.by,
            nbz = (g.D + sh.zc - 1) / sh.zc;
  const double hx = 0.5 * (sh.bx - 1), hy = 0.5 * (sh.by - 1), hz = 0.5 * (sh.zc - 1);
  const double rb = std::sqrt(hx * hx + hy * hy + hz * hz);
  const double reach = std::sqrt(2.0) * (g.H + g.a) + rb;
  std::vector<double> load((size_t)nbx * nby * nbz);
  double total = 0;
  for (int bz = 0; bz < nbz; ++bz)
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) {
        const double cx = x0 + bx * sh.bx + hx, cy = -g.H + by * sh.by + hy,
                     cz = -g.H + bz * sh.zc + hz;
        const double d = std::sqrt(cx * cx + cy * cy + cz * cz);
        double f = d <= g.a + rb ? 1.0 : (g.a + rb) / d;
        if (d - rb > reach) f = 0.0;
        const double l = n * f + 0.02 * n;  // images kept, plus the cull scan
        load[((size_t)bz * nby + by) * nbx + bx] = l;
        total += l;
      }
  if (target <= 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    target = std::max(UNIT_MIN_LOAD, total / (std::max(sms, 1) * (double)per_sm));
  }
  out.clear();
  out.reserve(load.size() + 64);
  any_split = 0;
  for (int bz = 0; bz < nbz; ++bz)
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) {
        const double l = load[((size_t)bz * nby + by) * nbx + bx];
        int ns = (int)std::ceil(l / target);
        ns = std::max(1, std::min(ns, std::min(64, std::max(1, n / SPLIT_MIN_IMAGES))));
        if (ns > 1) any_split = 1;
        for (int s = 0; s < ns; ++s)
          out.push_back(UnitLoad{l / ns, make_int4(bx, by, bz, s | (ns << 16))});
      }
  return total;
}

double gather_unit_loads(const fr_ctx *c, int shape, int n, double target,
                         std::vector<UnitLoad> &out, int &any_split) {
  return brick_unit_loads(c, gather_shape(shape), c->g.xa0, c->g.H, n, target, 32, out,
                          any_split);
}

// Work units of a gather launch of this batch alone, heaviest first (so the
// largest ones start first), cached on the device per (shape, n).
static int gather_units(fr_ctx *c, const Config &cfg, int n, InsertArgs &a,
                        const int4 **fold = nullptr, int *nfold = nullptr, int *fold_split = nullptr) {
  const int algo = cfg.algo == ALGO_GATHER2 ? ALGO_GATHER2 : ALGO_GATHER;
  for (int k = 0; k < 8; ++k) {
    fr_ctx::Units &u = c->units[k];
    if (u.dev && u.shape == cfg.shape && u.n == n && u.algo == algo) {
      a.units = u.dev;
      a.nunits = u.count;
      a.any_split = u.any_split;
      if (fold) { *fold = u.fold; *nfold = u.fold_count; *fold_split = u.fold_split; }
      return FR_OK;
    }
  }
  if (alloc_fault(c)) return FR_ERR_OOM;
  std::vector<UnitLoad> us, fs;
  int any_split = 0, fsplit = 0;
  if (algo == ALGO_GATHER2) {
    // the direct-drain gather's bricks tile x in [floor(a) + 1, H]; the fold
    // columns x in [-floor(a), floor(a)] go to its fold-column launch in
    // bricks one footprint wide, split finely (they are few and heavy)
    brick_unit_loads(c, gather2_shape(cfg.shape), 1 - c->g.xa0, c->g.H, n, 0.0, MAIN_UNITS_PER_SM,
                     us, any_split);
    brick_unit_loads(c, fold_shape(), c->g.xa0, -c->g.xa0, n, 0.0, FOLD_UNITS_PER_SM, fs, fsplit);
  } else {
    gather_unit_loads(c, cfg.shape, n, 0.0, us, any_split);
  }
  auto heavy_first = [](const UnitLoad &p, const UnitLoad &q) { return p.load > q.load; };
  std::stable_sort(us.begin(), us.end(), heavy_first);
  std::stable_sort(fs.begin(), fs.end(), heavy_first);
  std::vector<int4> host;
  host.reserve(us.size() + fs.size());
  for (const UnitLoad &x : us) host.push_back(x.unit);
  for (const UnitLoad &x : fs) host.push_back(x.unit);
  // replace the oldest cached list
  fr_ctx::Units &slot = c->units[7];
  cudaFree(slot.dev);
  for (int k = 7; k > 0; --k) c->units[k] = c->units[k - 1];
  c->units[0] = fr_ctx::Units{};
  fr_ctx::Units &u = c->units[0];
  FR_CUDA(cudaMalloc(&u.dev, host.size() * sizeof(int4)));
  FR_CUDA(cudaMemcpy(u.dev, host.data(), host.size() * sizeof(int4), cudaMemcpyHostToDevice));
  u.shape = cfg.shape;
  u.algo = algo;
  u.n = n;
  u.count = (int)us.size();
  u.any_split = any_split;
  u.fold = u.dev + us.size();
  u.fold_count = (int)fs.size();
  u.fold_split = fsplit;
  a.units = u.dev;
  a.nunits = u.count;
  a.any_split = any_split;
  if (fold) { *fold = u.fold; *nfold = u.fold_count; *fold_split = u.fold_split; }
  return FR_OK;
}

// Fill the launch geometry of configuration `cfg` into `a`.
static void gather_geometry(const fr_ctx *c, const Config &cfg, InsertArgs &a) {
  GatherShape sh = cfg.algo == ALGO_GATHER2 ? gather2_shape(cfg.shape) : gather_shape(cfg.shape);
  a.chunk = cfg.chunk;
  a.nbx = (c->g.NXa + sh.bx - 1) / sh.bx;
  a.nby = (c->g.D + sh.by - 1) / sh.by;
  a.nbz = (c->g.D + sh.zc - 1) / sh.zc;
}

// Allocate and upload whatever a launch of configuration id on n images
// needs (work units, scratch), so that the launch itself only enqueues work.
int prepare_config(fr_ctx *c, int id, int n) {
  const Config &cfg = config_space()[id];
  InsertArgs a = base_args(c);
  if (cfg.algo == ALGO_GATHER || cfg.algo == ALGO_GATHER2) {
    const int4 *fold = nullptr;
    int nfold = 0, fold_split = 0;
    int rc = gather_units(c, cfg, n, a, &fold, &nfold, &fold_split);
    if (rc) return rc;
    if (cfg.algo == ALGO_GATHER2) {
      rc = ensure_side_stream(c);
      if (rc) return rc;
    }
    return (a.any_split || fold_split) ? ensure_scratch(c) : FR_OK;
  }
  return ensure_scratch(c);
}

// Enqueue the insertion of n images with configuration id; no timing.
int run_config(fr_ctx *c, int id, const void *images, int f16, const float *rot, int n,
               cudaStream_t st) {
  const Config &cfg = config_space()[id];
  InsertArgs a = base_args(c);
  a.images = images;
  a.f16 = f16;
  a.rot = rot;
  a.n = n;
  if (cfg.algo == ALGO_GATHER || cfg.algo == ALGO_GATHER2) {
    gather_geometry(c, cfg, a);
    const int4 *fold = nullptr;
    int nfold = 0, fold_split = 0;
    int rc = gather_units(c, cfg, n, a, &fold, &nfold, &fold_split);
    if (rc) return rc;
    if (cfg.algo == ALGO_GATHER2) a.any_split |= fold_split;
    if (a.any_split) {
      rc = ensure_scratch(c);
      if (rc) return rc;
      a.scratch = c->scratch;
    }
    cudaError_t e;
    if (cfg.algo == ALGO_GATHER2) {
      // the fold columns: the fold-column instantiation, on the side stream
      // so that its few heavy units run beside the main launch (disjoint
      // voxels; split units add to the scratch with atomics, merged after both)
      rc = ensure_side_stream(c);
      if (rc) return rc;
      InsertArgs f = a;
      f.units = fold;
      f.nunits = nfold;
      e = cudaEventRecord(c->ev_fork, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
      if (e == cudaSuccess) e = launch_gather_fold(f, c->side);
      if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
      if (e != cudaSuccess) return cuda_fail(e);
      e = launch_gather2(cfg.shape, cfg.minw, a, st, 0, nullptr);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_join, 0);
    } else {
      e = launch_gather(cfg.shape, cfg.wmode, a, st, 0, nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (a.any_split) {
      e = launch_merge_scratch(a, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    return FR_OK;
  }
  int rc = ensure_scratch(c);
  if (rc) return rc;
  a.scratch = c->scratch;
  const size_t px = (size_t)c->g.S * c->g.NX;
  const size_t bytes = f16 ? 4 : 8;
  for (int off = 0; off < n; off += cfg.sub) {
    int m = std::min(cfg.sub, n - off);
    InsertArgs b = a;
    b.images = (const char *)images + (size_t)off * px * bytes;
    b.rot = rot + 9 * (size_t)off;
    b.n = m;
    cudaError_t e = launch_scatter(cfg.threads, cfg.wmode, b, st, 0, nullptr);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_merge_scratch(b, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return FR_OK;
}

int config_valid(const fr_ctx *c, int id) {
  if (id < 0 || id >= (int)config_space().size()) return 0;
  const Config &cfg = config_space()[id];
  // the polynomial is offered only where it is as accurate as the table
  if (cfg.wmode == W_POLY && c && !(c->poly_err < 1e-6)) return 0;
  int dev = c ? c->device : 0;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int lut_n = c ? c->lut_n : 10000;
  if (cfg.algo == ALGO_GATHER) {
    GatherShape sh = gather_shape(cfg.shape);
    size_t smem = gather_smem_bytes(sh, cfg.wmode, lut_n, cfg.chunk) + 1024;
    return optin == 0 || (int)smem <= optin;
  }
  if (cfg.algo == ALGO_GATHER2) {
    // 4 x 4 candidate boxes (a < 2) and at least one column inside every box
    if (c && (c->g.KB != 4 || c->g.H < 4)) return 0;
    GatherShape sh = gather2_shape(cfg.shape);
    size_t smem = gather2_smem_bytes(sh, cfg.chunk) + 1024;
    return optin == 0 || (int)smem <= optin;
  }
  size_t smem = cfg.wmode == W_LUT ? (size_t)lut_n * sizeof(float2) : 0;
  return optin == 0 || (int)smem <= optin;
}

}  // namespace fr

// ------------------------------------------------------------------ tuner glue

int fr::key_bucket(int n) {
  int b = 0;
  while ((2LL << b) <= n) ++b;
  return b;
}

int fr::do_insert_ctx(fr_ctx *c, const void *images, fr_dtype dtype, const float *rot, int n,
                      cudaStream_t st) {
  const int f16 = dtype == FR_F16;
  const size_t px_bytes = (size_t)c->g.S * c->g.NX * (f16 ? 4 : 8);
  TuneKey key{c->S, key_bucket(n), c->g.a, (int)dtype};
  c->tuner.harvest();
  KeyState &ks = c->tuner.state(key, c);
  std::vector<Step> plan;
  if (c->opt.forced_config >= 0) {
    plan.push_back(Step{c->opt.forced_config, n, false});
  } else {
    plan = c->tuner.plan(ks, n, c->opt);
  }
  int status = FR_OK;
  int off = 0;
  for (const Step &s : plan) {
    if (s.images <= 0) continue;
    const void *img = (const char *)images + (size_t)off * px_bytes;
    const float *r = rot + 9 * (size_t)off;
    // optional NVTX range per step (debug bit 2); a no-op unless a tool is attached
    const bool nvtx = (c->opt.debug & 4) != 0;
    if (nvtx) {
      char name[96];
      std::snprintf(name, sizeof(name), "fr_insert S=%d images=%d %s", c->S, s.images,
                    describe(config_space()[s.config]).c_str());
      nvtxRangePushA(name);
    }
    // host-side fault injection (test hook): report a failed launch, enqueue nothing
    int rc = (c->opt.fault_config > 0 && s.config == c->opt.fault_config - 1) ? FR_ERR_LAUNCH : FR_OK;
    // host work of the step (work-unit list, scratch) before the timed region,
    // so that a configuration's first use is timed like its later ones
    if (rc == FR_OK) rc = prepare_config(c, s.config, s.images);
    Timing tm = c->tuner.begin(st);
    if (rc == FR_OK) rc = run_config(c, s.config, img, f16, r, s.images, st);
    if (rc != FR_OK) {
      // the configuration could not launch: mark it and redo the work with the default
      cudaGetLastError();
      ks.invalid.insert(s.config);
      int fb = default_config(c);
      rc = run_config(c, fb, img, f16, r, s.images, st);
      if (rc != FR_OK) {
        c->tuner.abandon(tm);
        if (nvtx) nvtxRangePop();
        return rc;
      }
      c->tuner.end(tm, ks, fb, s.images, false, st);
      status = FR_ERR_LAUNCH;
    } else {
      c->tuner.end(tm, ks, s.config, s.images, s.tuning, st, s.full);
    }
    if (nvtx) nvtxRangePop();
    ks.last_config = s.config;
    off += s.images;
    ++c->launches;
    if (c->opt.debug) {
      FR_CUDA(cudaStreamSynchronize(st));
      int h = 0;
      FR_CUDA(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (h) return (h & DERR_TIMEOUT) ? FR_ERR_TIMEOUT : FR_ERR_DEVICE_ASSERT;
    }
  }
  c->images += (unsigned long long)n;
  c->last_stream = st;
  return status;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

int fr_create(int S, const fr_blob *blob, fr_ctx **out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!blob) return FR_ERR_INVALID_ARG;
  if (S < 8 || S > 512) return FR_ERR_INVALID_ARG;
  if (S & 1) return FR_ERR_UNSUPPORTED;
  if (blob->order != 0) return FR_ERR_UNSUPPORTED;
  if (!(blob->a > 0.f)) return FR_ERR_INVALID_ARG;
  if (!(blob->a < 3.f)) return FR_ERR_UNSUPPORTED;
  if (!(blob->alpha >= 0.f && blob->alpha <= 40.f)) return FR_ERR_INVALID_ARG;
  if (blob->table_size < 2 || blob->table_size > 16384) return FR_ERR_INVALID_ARG;

  fr_ctx *c = new (std::nothrow) fr_ctx();
  if (!c) return FR_ERR_OOM;
  c->S = S;
  c->blob = *blob;
  cudaGetDevice(&c->device);
  Geom &g = c->g;
  g.S = S;
  g.H = S / 2;
  g.NX = S / 2 + 1;
  g.D = S + 1;
  g.a = blob->a;
  g.a2 = blob->a * blob->a;
  g.alpha = blob->alpha;
  g.xa0 = -(int)std::floor(blob->a);
  g.NXa = g.H - g.xa0 + 1;
  g.KB = blob->a < 2.0f ? 4 : 6;
  c->plane = (size_t)g.D * g.D * g.NXa;
  c->opt.tuning = 1;
  c->opt.search = FR_SEARCH_EXHAUSTIVE;
  c->opt.budget = 0;
  c->opt.steps_per_insert = 0;  // automatic
  c->opt.forced_config = -1;
  c->opt.seed = 1;
  c->opt.debug = 0;

  auto fail = [&](int rc) {
    fr_destroy(c);
    return rc;
  };
  cudaError_t e = cudaMalloc(&c->acc, 6 * c->plane * sizeof(float));
  if (e != cudaSuccess) return fail(cuda_fail(e));
  e = cudaMemset(c->acc, 0, 6 * c->plane * sizeof(float));
  if (e != cudaSuccess) return fail(cuda_fail(e));
  e = cudaMalloc(&c->d_err, sizeof(int));
  if (e != cudaSuccess) return fail(cuda_fail(e));
  cudaMemset(c->d_err, 0, sizeof(int));
  e = cudaMalloc(&c->d_count, sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(cuda_fail(e));
  e = cudaMalloc(&c->d_phase, PH_COUNT * sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(cuda_fail(e));
  cudaMemset(c->d_phase, 0, PH_COUNT * sizeof(unsigned long long));

  // blob table: b at r^2 = i a^2 / (N - 1), (value, next - value); I0 from the
  // C++17 special-function library in double precision
  const int N = blob->table_size;
  c->lut_n = N;
  c->lut_scale = (float)((double)(N - 1) / ((double)g.a * (double)g.a));
  const double a2 = (double)g.a * (double)g.a, alpha = (double)g.alpha;
  const double i0a = std::cyl_bessel_i(0.0, alpha);
  std::vector<double> b(N);
  for (int i = 0; i < N; ++i) {
    double t = std::max(0.0, 1.0 - ((double)i * a2 / (N - 1)) / a2);
    b[i] = std::cyl_bessel_i(0.0, alpha * std::sqrt(t)) / i0a;
  }
  std::vector<float2> tab(N);
  for (int i = 0; i < N; ++i) {
    float v = (float)b[i];
    float nxt = i + 1 < N ? (float)b[i + 1] : v;
    tab[i] = make_float2(v, (float)((double)nxt - (double)v));
  }
  e = cudaMalloc(&c->lut, N * sizeof(float2));
  if (e != cudaSuccess) return fail(cuda_fail(e));
  e = cudaMemcpy(c->lut, tab.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  c->inv_i0a = (float)(1.0 / i0a);
  c->inv_pa = alpha > 3.75 ? (float)(1.0 / as_982_host(3.75 / alpha)) : 1.0f;

  // polynomial weights: b as a function of x = 2 r^2 / a^2 - 1 in [-1, 1]
  {
    auto bx = [&](double x) {
      double t = std::min(1.0, std::max(0.0, 0.5 * (x + 1.0)));  // (r/a)^2
      return std::cyl_bessel_i(0.0, alpha * std::sqrt(1.0 - t)) / i0a;
    };
    double mono[POLY_N];
    chebyshev_power_basis(bx, mono);
    for (int k = 0; k < POLY_N; ++k) c->poly[k] = (float)mono[k];
    // measured error of the FP32 even/odd evaluation the device performs
    double worst = 0;
    for (int i = 0; i <= 20000; ++i) {
      const float x = -1.0f + 2.0f * (float)i / 20000.0f;
      const float y = x * x;
      float e = c->poly[POLY_N - 2], o = c->poly[POLY_N - 1];
      for (int k = POLY_N / 2 - 2; k >= 0; --k) {
        e = std::fma(e, y, c->poly[2 * k]);
        o = std::fma(o, y, c->poly[2 * k + 1]);
      }
      const float p = std::fma(o, x, e);
      worst = std::max(worst, std::fabs((double)p - bx((double)x)));
    }
    c->poly_err = worst;
  }

  c->tuner.init(c);
  *out = c;
  return FR_OK;
}

int fr_destroy(fr_ctx *c) {
  if (!c) return FR_OK;
  cudaDeviceSynchronize();
  batched_forget(c);
  reconstruct_release(c);
  c->tuner.release();
  cudaFree(c->acc);
  cudaFree(c->lut);
  cudaFree(c->scratch);
  cudaFree(c->d_err);
  cudaFree(c->d_count);
  cudaFree(c->d_phase);
  cudaFree(c->d_mlp);
  for (auto &u : c->units) cudaFree(u.dev);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
  return FR_OK;
}

int fr_reset(fr_ctx *c, void *stream) {
  if (!c) return FR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FR_CUDA(cudaMemsetAsync(c->acc, 0, 6 * c->plane * sizeof(float), st));
  c->images = 0;
  c->last_stream = st;
  return FR_OK;
}

int fr_insert(fr_ctx *c, const void *images, fr_dtype dtype, const float *rotations, int n,
              void *stream) {
  if (!c) return FR_ERR_INVALID_ARG;
  if (n < 0 || n > (1 << 24)) return FR_ERR_INVALID_ARG;
  if (dtype != FR_F32 && dtype != FR_F16) return FR_ERR_INVALID_ARG;
  if (n == 0) return FR_OK;
  if (!images || !rotations) return FR_ERR_INVALID_ARG;
  if (((uintptr_t)images & 15) != 0 || ((uintptr_t)rotations & 3) != 0) return FR_ERR_INVALID_ARG;
  return do_insert_ctx(c, images, dtype, rotations, n, (cudaStream_t)stream);
}

int fr_insert_batched(fr_ctx *const *ctxs, const void *const *images, const fr_dtype *dtypes,
                      const float *const *rotations, const int *n, int nb, int capture,
                      void *stream) {
  if (nb < 0 || (nb > 0 && (!ctxs || !images || !dtypes || !rotations || !n)))
    return FR_ERR_INVALID_ARG;
  return fr::insert_batched(ctxs, images, (const int *)dtypes, rotations, n, nb, capture,
                            (cudaStream_t)stream);
}

int fr_finalize(fr_ctx *c, void *V, float *W, void *stream) {
  if (!c || !V || !W) return FR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FR_CUDA(cudaStreamSynchronize(st));
  if (c->last_stream && c->last_stream != st) FR_CUDA(cudaStreamSynchronize(c->last_stream));
  int h = 0;
  FR_CUDA(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  cudaError_t e = launch_finalize(c->g, c->acc, c->plane, (float2 *)V, W, st);
  if (e != cudaSuccess) return cuda_fail(e);
  c->last_stream = st;
  if (h) return (h & DERR_TIMEOUT) ? FR_ERR_TIMEOUT : FR_ERR_DEVICE_ASSERT;
  return FR_OK;
}

size_t fr_state_bytes(const fr_ctx *c) { return c ? 6 * c->plane * sizeof(float) : 0; }

static int state_copy(fr_ctx *c, void *dst, const void *src) {
  if (c->last_stream) FR_CUDA(cudaStreamSynchronize(c->last_stream));
  FR_CUDA(cudaDeviceSynchronize());
  FR_CUDA(cudaMemcpy(dst, src, fr_state_bytes(c), cudaMemcpyDefault));
  return FR_OK;
}

int fr_state_save(fr_ctx *c, void *dst) {
  if (!c || !dst) return FR_ERR_INVALID_ARG;
  return state_copy(c, dst, c->acc);
}

int fr_state_load(fr_ctx *c, const void *src) {
  if (!c || !src) return FR_ERR_INVALID_ARG;
  return state_copy(c, c->acc, src);
}

int fr_retune(fr_ctx *c, int all) {
  if (!c) return FR_ERR_INVALID_ARG;
  c->tuner.harvest();
  c->tuner.retune(all != 0);
  return FR_OK;
}

int fr_set_options(fr_ctx *c, const fr_options *o) {
  if (!c || !o) return FR_ERR_INVALID_ARG;
  if (o->search < 0 || o->search > FR_SEARCH_MCMC || o->budget < 0 || o->steps_per_insert < 0)
    return FR_ERR_INVALID_ARG;
  if (o->forced_config >= (int)config_space().size()) return FR_ERR_INVALID_ARG;
  if (o->fault_config < 0 || o->fault_config > (int)config_space().size()) return FR_ERR_INVALID_ARG;
  if (o->fault_alloc < 0) return FR_ERR_INVALID_ARG;
  if (o->forced_config >= 0 && !config_valid(c, o->forced_config)) return FR_ERR_UNSUPPORTED;
  bool search_changed = o->search != c->opt.search || o->budget != c->opt.budget ||
                        o->seed != c->opt.seed;
  c->opt = *o;
  c->alloc_countdown = o->fault_alloc;
  if (search_changed) c->tuner.retune(true);
  return FR_OK;
}

int fr_get_options(const fr_ctx *c, fr_options *o) {
  if (!c || !o) return FR_ERR_INVALID_ARG;
  *o = c->opt;
  return FR_OK;
}

int fr_tuning_report(fr_ctx *c, fr_report *r) {
  if (!c || !r) return FR_ERR_INVALID_ARG;
  c->tuner.harvest();
  std::memset(r, 0, sizeof(*r));
  c->tuner.report(r);
  r->S = c->S;
  r->launches = c->launches;
  r->images = c->images;
  return FR_OK;
}

int fr_tuning_measurements(fr_ctx *c, int *cfg, double *ns, double *images, int cap) {
  if (!c || cap < 0) return -FR_ERR_INVALID_ARG;
  c->tuner.harvest();
  return c->tuner.measurements(cfg, ns, images, cap);
}

int fr_tuning_save(const fr_ctx *c, const char *path) {
  if (!c || !path) return FR_ERR_INVALID_ARG;
  return const_cast<fr_ctx *>(c)->tuner.save(path);
}

int fr_tuning_load(fr_ctx *c, const char *path) {
  if (!c || !path) return FR_ERR_INVALID_ARG;
  return c->tuner.load(path);
}

int fr_num_configs(void) { return (int)config_space().size(); }

int fr_describe_config(int id, char *buf, int len) {
  if (id < 0 || id >= (int)config_space().size() || !buf || len <= 0) return -FR_ERR_INVALID_ARG;
  std::string s = describe(config_space()[id]);
  std::snprintf(buf, (size_t)len, "%s", s.c_str());
  return (int)config_space().size();
}

int fr_config_valid(const fr_ctx *c, int id) { return config_valid(c, id); }

int fr_config_features(int id, int S, int n, float a, float *out16) {
  if (id < 0 || id >= (int)config_space().size() || !out16) return FR_ERR_INVALID_ARG;
  config_features(config_space()[id], S, n, a, out16);
  return FR_OK;
}

int fr_insert_launches(fr_ctx *c, int id, int n, int *out) {
  if (!c || !out || n < 1 || id < 0 || id >= (int)config_space().size())
    return FR_ERR_INVALID_ARG;
  const Config &cfg = config_space()[id];
  if (cfg.algo == ALGO_SCATTER) {
    *out = 2 * ((n + cfg.sub - 1) / cfg.sub);  // scatter + merge per sub-batch
    return FR_OK;
  }
  InsertArgs a = base_args(c);
  const int4 *fold = nullptr;
  int nfold = 0, fold_split = 0;
  int rc = gather_units(c, cfg, n, a, &fold, &nfold, &fold_split);
  if (rc) return rc;
  if (cfg.algo == ALGO_GATHER2)  // main launch, fold-column launch, merge if split
    *out = 2 + ((a.any_split || fold_split) ? 1 : 0);
  else
    *out = 1 + (a.any_split ? 1 : 0);
  return FR_OK;
}

int fr_count_updates(fr_ctx *c, const float *rot, int n, void *stream, unsigned long long *out) {
  if (!c || !out || n < 0 || (n > 0 && !rot)) return FR_ERR_INVALID_ARG;
  *out = 0;
  if (n == 0) return FR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  FR_CUDA(cudaMemsetAsync(c->d_count, 0, sizeof(unsigned long long), st));
  cudaError_t e = launch_count(c->g, rot, n, c->d_count, st);
  if (e != cudaSuccess) return cuda_fail(e);
  FR_CUDA(cudaMemcpyAsync(out, c->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  FR_CUDA(cudaStreamSynchronize(st));
  return FR_OK;
}

double fr_relative_performance(double s, double t_avg, double t_well, double n) {
  return relative_performance(s, t_avg, t_well, n);
}
double fr_invocations_to_amortize(double rp, double s, double t_avg, double t_well) {
  return invocations_to_amortize(rp, s, t_avg, t_well);
}
double fr_random_search_steps(double r, double p) { return random_search_steps(r, p); }

const char *fr_error_string(int s) {
  switch (s) {
    case FR_OK: return "ok";
    case FR_ERR_INVALID_ARG: return "invalid argument";
    case FR_ERR_UNSUPPORTED: return "unsupported parameters";
    case FR_ERR_OOM: return "out of memory";
    case FR_ERR_CUDA: return "CUDA runtime error";
    case FR_ERR_LAUNCH: return "configuration failed to launch; work re-run with the fallback";
    case FR_ERR_DEVICE_ASSERT: return "device range check failed";
    case FR_ERR_TIMEOUT: return "device wait timed out";
    case FR_ERR_IO: return "tuning file I/O error";
    case FR_ERR_STATE: return "invalid state";
    case FR_ERR_NOALLOC_LIMIT:
      return "size exceeds the fixed scratch of fr_insert_noalloc (S <= 64)";
    default: return "unknown status";
  }
}

int fr_last_device_error(fr_ctx *c) {
  if (!c) return FR_ERR_INVALID_ARG;
  if (c->last_stream) FR_CUDA(cudaStreamSynchronize(c->last_stream));
  else FR_CUDA(cudaDeviceSynchronize());
  int h = 0;
  FR_CUDA(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  FR_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
  if (!h) return FR_OK;
  return (h & DERR_TIMEOUT) ? FR_ERR_TIMEOUT : FR_ERR_DEVICE_ASSERT;
}

int fr_last_cuda_error(void) { return g_last_cuda.load(); }

int fr_debug_phase_counters(fr_ctx *c, unsigned long long *out, int cap) {
  if (!c || !out || cap < 0) return FR_ERR_INVALID_ARG;
  FR_CUDA(cudaDeviceSynchronize());
  unsigned long long h[PH_COUNT];
  FR_CUDA(cudaMemcpy(h, c->d_phase, sizeof h, cudaMemcpyDeviceToHost));
  FR_CUDA(cudaMemset(c->d_phase, 0, sizeof h));
  for (int k = 0; k < cap && k < PH_COUNT; ++k) out[k] = h[k];
  return FR_OK;
}

int fr_debug_fold(const float *r, const int *k, int m, int *out, void *stream) {
  if (m < 0 || (m > 0 && (!r || !k || !out))) return FR_ERR_INVALID_ARG;
  cudaError_t e = launch_debug_fold(r, k, m, out, (cudaStream_t)stream);
  return e == cudaSuccess ? FR_OK : cuda_fail(e);
}

int fr_debug_blob(const fr_ctx *c, const float *r2, int m, int mode, float *out, void *stream) {
  if (!c || m < 0 || (m > 0 && (!r2 || !out)) || mode < 0 || mode > 2)
    return FR_ERR_INVALID_ARG;
  InsertArgs a = base_args(c);
  cudaError_t e = launch_debug_blob(a, r2, m, mode, out, (cudaStream_t)stream);
  return e == cudaSuccess ? FR_OK : cuda_fail(e);
}

}  // extern "C"
