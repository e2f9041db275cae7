// fr_batched.cu -- insertion of many uneven batches (differing S and n), one
// batch per context, in a few launches that each cover the work units of
// several batches (A8), optionally captured into a CUDA graph.
//
// A call is turned into a plan, cached by (contexts, image and rotation
// pointers, sizes, dtypes, configurations).  Every batch runs with its
// context's configuration (the tuned best for its key, else the default):
//   * batches are grouped by what one kernel instantiation needs in common
//     (kernel family, brick shape, register budget, candidate-box width,
//     image dtype, list capacity, and for the direct-drain gather the weight
//     polynomial, which stays a kernel parameter);
//   * each group's work units (bricks and image splits, with expected loads)
//     are pooled over its batches with one splitting target and ordered
//     heaviest first.  A direct-drain group is one launch with a CTA per item,
//     plus one launch of its fold-column instantiation over the items of the
//     fold columns on a high-priority side stream beside it; a per-voxel gather
//     group is one persistent launch whose CTAs take items from a device
//     counter;
//   * the per-batch launch arguments and the items are uploaded once into a
//     device buffer the plan owns;
//   * after the groups, the float4 scratch of every context that received
//     split (or shared) units is merged.
// A context that appears in several batches of one call has all of its units
// routed through its scratch (atomics), so concurrent units never race on its
// accumulators.  Batches whose configuration no multi-batch kernel takes
// (scatter, tabulated weights, a context whose polynomial weights are not
// accurate enough) run their own configuration's launches, in order, after
// the groups.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <list>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "fr_ctx.h"
#include "fr_gather.cuh"
#include "fr_internal.h"
#include "fr_tuner.h"

namespace fr {

namespace {

struct PlanKey {
  std::vector<const void *> ptrs;
  std::vector<int> ints;
  bool operator<(const PlanKey &o) const { return std::tie(ptrs, ints) < std::tie(o.ptrs, o.ints); }
};

struct Group {
  int algo = ALGO_GATHER, shape = 0, kb = 4, f16 = 0, chunk = 64, minw = 0;
  PersistentLaunch launch{};  // per-voxel gather: persistent launch
  MultiLaunch main{}, fold{};  // direct-drain gather: main and fold-column launches
  int lane = 0;               // direct-drain gather: the stream its main launch runs on
};

constexpr int MAX_LANES = 4;

struct Plan {
  PlanKey key;
  std::vector<const fr_ctx *> ctxs;  // contexts the plan refers to
  void *dev = nullptr;               // descriptors, items, counters (owned)
  std::vector<Group> groups;
  std::vector<InsertArgs> merges;    // scratch merges after the groups
  std::vector<int> sequential;       // batches run with their own launches
  // direct-drain groups: their main launches on up to MAX_LANES streams side
  // by side, the fold-column launches on a highest-priority stream; forked
  // from and joined back into the caller's stream
  std::vector<cudaStream_t> lanes;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;  // one per lane, then the side stream's
  cudaGraphExec_t exec = nullptr;
};

std::mutex g_mu;
std::list<Plan> g_plans;  // most recently used first
constexpr size_t MAX_PLANS = 32;

void free_plan(Plan &p) {
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.ev_fork) cudaEventDestroy(p.ev_fork);
  for (cudaEvent_t e : p.ev_join) cudaEventDestroy(e);
  for (cudaStream_t l : p.lanes) cudaStreamDestroy(l);
  if (p.side) cudaStreamDestroy(p.side);
  cudaFree(p.dev);
  p.exec = nullptr;
  p.dev = nullptr;
  p.side = nullptr;
  p.ev_fork = nullptr;
  p.ev_join.clear();
  p.lanes.clear();
}

// configuration a batch runs with: the forced one, else the context's tuned
// best for its key, else its default
int batched_config(fr_ctx *c, int n, int dtype) {
  if (c->opt.forced_config >= 0) return c->opt.forced_config;
  TuneKey k{c->S, key_bucket(n), c->g.a, dtype};
  const int best = c->tuner.best_for(k);
  return best >= 0 ? best : default_config(c);
}

int cuda_err(cudaError_t e) {
  fr_note_cuda_error((int)e);
  return e == cudaErrorMemoryAllocation ? FR_ERR_OOM : FR_ERR_CUDA;
}

// Build the plan of one call: groups, pooled and ordered items, uploads.
int build_plan(Plan &pl, fr_ctx *const *ctxs, const void *const *images, const int *dtypes,
               const float *const *rotations, const int *n, int nb, const std::vector<int> &cfg) {
  std::map<const fr_ctx *, int> uses;
  for (int b = 0; b < nb; ++b)
    if (n[b] > 0) ++uses[ctxs[b]];
  // group the batches a multi-batch kernel can take: the direct-drain gather
  // by (configuration, dtype, S, blob), the persistent per-voxel gather by
  // (shape, box width, dtype, list capacity)
  using GKey = std::tuple<int, int, int, int, int, int, int, float, float>;
  std::map<GKey, std::vector<int>> groups;
  for (int b = 0; b < nb; ++b) {
    if (n[b] == 0) continue;
    fr_ctx *c = ctxs[b];
    const Config &k = config_space()[cfg[b]];
    const int f16 = dtypes[b] == FR_F16 ? 1 : 0;
    const bool poly_ok = c->poly_err < 1e-6;
    if (k.algo == ALGO_GATHER2 && poly_ok && c->g.KB == 4) {
      groups[GKey(ALGO_GATHER2, k.shape, 4, f16, k.chunk, k.minw, c->S, c->g.a, c->g.alpha)]
          .push_back(b);
    } else if (k.algo == ALGO_GATHER && k.wmode == W_POLY && poly_ok) {
      groups[GKey(ALGO_GATHER, k.shape, c->g.KB, f16, k.chunk, 0, 0, 0.f, 0.f)].push_back(b);
    } else {
      // its own launches: units, scratch and side stream ready before any capture
      int rc = prepare_config(c, cfg[b], n[b]);
      if (rc != FR_OK) return rc;
      pl.sequential.push_back(b);
    }
  }
  const int sms = std::max(device_sm_count(), 1);

  std::vector<InsertArgs> descs(nb);  // each batch's own arguments
  std::vector<std::vector<int4>> items;  // per group: main items, then (gather2) fold items
  std::set<const fr_ctx *> merge_ctx;
  struct It { double load; int4 v; };
  auto order = [](std::vector<It> &its) {
    std::stable_sort(its.begin(), its.end(), [](const It &p, const It &q) { return p.load > q.load; });
    std::vector<int4> v(its.size());
    for (size_t i = 0; i < its.size(); ++i) v[i] = its[i].v;
    return v;
  };
  // a direct-drain launch takes at most MULTI_MAX batches (its image pointers
  // are kernel parameters)
  std::vector<std::pair<GKey, std::vector<int>>> glist;
  for (auto &kv : groups) {
    const size_t cap = std::get<0>(kv.first) == ALGO_GATHER2 ? MULTI_MAX : kv.second.size();
    for (size_t i = 0; i < kv.second.size(); i += cap)
      glist.push_back({kv.first, std::vector<int>(kv.second.begin() + i,
                                                  kv.second.begin() + std::min(kv.second.size(), i + cap))});
  }
  int greatest = 0, least = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  int n_g2 = 0;
  for (auto &kv : glist) {
    Group gr;
    int S_ = 0;
    float a_ = 0.f, alpha_ = 0.f;
    std::tie(gr.algo, gr.shape, gr.kb, gr.f16, gr.chunk, gr.minw, S_, a_, alpha_) = kv.first;
    const bool g2 = gr.algo == ALGO_GATHER2;
    const GatherShape sh = g2 ? gather2_shape(gr.shape) : gather_shape(gr.shape);
    auto main_loads = [&](const fr_ctx *c, int nn, double target, std::vector<UnitLoad> &out,
                          int &split) {
      return g2 ? brick_unit_loads(c, sh, 1 - c->g.xa0, c->g.H, nn, target, MAIN_UNITS_PER_SM, out,
                                   split)
                : brick_unit_loads(c, sh, c->g.xa0, c->g.H, nn, target, 32, out, split);
    };
    auto fold_loads = [&](const fr_ctx *c, int nn, double target, std::vector<UnitLoad> &out,
                          int &split) {
      return brick_unit_loads(c, fold_shape(), c->g.xa0, -c->g.xa0, nn, target, FOLD_UNITS_PER_SM,
                              out, split);
    };
    // pooled splitting target of the main items: total expected load over
    // 32 items per SM; the fold-column items are split as in a launch of
    // their batch alone (8 per SM: the few heavy bricks every plane crosses
    // set the fold launch's length)
    double total = 0;
    std::vector<UnitLoad> tmp;
    int any = 0;
    for (int b : kv.second) total += main_loads(ctxs[b], n[b], 1e300, tmp, any);
    const double target = std::max(UNIT_MIN_LOAD, total / (sms * (double)MAIN_UNITS_PER_SM));
    std::vector<It> its, fits;
    for (size_t slot = 0; slot < kv.second.size(); ++slot) {
      const int b = kv.second[slot];
      fr_ctx *c = ctxs[b];
      int split = 0, fsplit = 0;
      const bool shared = uses[c] > 1;
      const int shared_bit = shared ? (1 << 30) : 0;
      main_loads(c, n[b], target, tmp, split);
      for (const UnitLoad &u : tmp)
        its.push_back(It{u.load, make_int4(u.unit.x | (u.unit.y << 10) | (u.unit.z << 20),
                                           u.unit.w | shared_bit, b, (int)slot)});
      if (g2) {
        fold_loads(c, n[b], 0.0, tmp, fsplit);
        for (const UnitLoad &u : tmp)
          fits.push_back(It{u.load, make_int4(u.unit.x | (u.unit.y << 10) | (u.unit.z << 20),
                                              u.unit.w | shared_bit, b, (int)slot)});
        gr.main.images[slot] = gr.fold.images[slot] = images[b];
      }
      if (split || fsplit || shared) {
        int rc = ensure_scratch(c);
        if (rc != FR_OK) return rc;
        merge_ctx.insert(c);
      }
      InsertArgs a = base_args(c);
      a.images = images[b];
      a.f16 = gr.f16;
      a.rot = rotations[b];
      a.n = n[b];
      a.chunk = gr.chunk;
      a.phase = nullptr;
      a.units = nullptr;
      a.scratch = c->scratch;
      descs[b] = a;
    }
    items.push_back(order(its));
    if (g2) {
      items.push_back(order(fits));
      // the arguments the group's batches share (geometry, weights, list
      // capacity): those of its first batch; the kernels read the rest per batch
      InsertArgs base = descs[kv.second.front()];
      gr.main.base = base;
      gr.fold.base = base;
      gr.fold.priority = greatest;
      gr.lane = n_g2++ % MAX_LANES;
    }
    pl.groups.push_back(gr);
  }
  // device buffer: descriptors | items of each group | one counter per group
  size_t off = (size_t)nb * sizeof(InsertArgs);
  off = (off + 15) & ~(size_t)15;
  std::vector<size_t> item_off;
  for (auto &v : items) {
    item_off.push_back(off);
    off += v.size() * sizeof(int4);
  }
  const size_t counter_off = off;
  off += pl.groups.size() * sizeof(unsigned) + 16;
  cudaError_t e = cudaMalloc(&pl.dev, off);
  if (e != cudaSuccess) return cuda_err(e);
  unsigned char *d = static_cast<unsigned char *>(pl.dev);
  e = cudaMemcpy(d, descs.data(), descs.size() * sizeof(InsertArgs), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(e);
  for (size_t i = 0; i < items.size(); ++i) {
    if (items[i].empty()) continue;
    e = cudaMemcpy(d + item_off[i], items[i].data(), items[i].size() * sizeof(int4),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(e);
  }
  size_t ii = 0;
  for (size_t gi = 0; gi < pl.groups.size(); ++gi) {
    Group &gr = pl.groups[gi];
    if (gr.algo == ALGO_GATHER2) {
      gr.main.descs = gr.fold.descs = reinterpret_cast<const InsertArgs *>(d);
      gr.main.items = reinterpret_cast<const int4 *>(d + item_off[ii]);
      gr.main.nitems = (int)items[ii].size();
      gr.fold.items = reinterpret_cast<const int4 *>(d + item_off[ii + 1]);
      gr.fold.nitems = (int)items[ii + 1].size();
      ii += 2;
    } else {
      PersistentLaunch &L = gr.launch;
      L.descs = reinterpret_cast<const InsertArgs *>(d);
      L.items = reinterpret_cast<const int4 *>(d + item_off[ii]);
      L.nitems = (int)items[ii].size();
      L.chunk = gr.chunk;
      L.counter = reinterpret_cast<unsigned *>(d + counter_off) + gi;
      ii += 1;
    }
  }
  if (n_g2 > 0) {
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&pl.side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl.ev_fork, cudaEventDisableTiming);
    const int nl = std::min(n_g2, MAX_LANES);
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
      cudaStream_t s = nullptr;
      e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e == cudaSuccess) pl.lanes.push_back(s);
    }
    for (int l = 0; l <= nl && e == cudaSuccess; ++l) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) pl.ev_join.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (const fr_ctx *c : merge_ctx) pl.merges.push_back(base_args(c));
  for (int b = 0; b < nb; ++b) pl.ctxs.push_back(ctxs[b]);
  return FR_OK;
}

// Enqueue one execution of the plan on st.
int enqueue_plan(const Plan &pl, fr_ctx *const *ctxs, const void *const *images, const int *dtypes,
                 const float *const *rotations, const int *n, const std::vector<int> &cfg,
                 cudaStream_t st) {
  // direct-drain groups: fork the lanes and the side stream off st; the
  // fold-column launches first, on the side stream (disjoint voxels; split
  // and shared units add to the scratch with atomics, merged after the join)
  cudaError_t e = cudaSuccess;
  const int nl = (int)pl.lanes.size();
  if (pl.side) {
    e = cudaEventRecord(pl.ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pl.side, pl.ev_fork, 0);
    for (int l = 0; l < nl && e == cudaSuccess; ++l)
      e = cudaStreamWaitEvent(pl.lanes[l], pl.ev_fork, 0);
    for (const Group &gr : pl.groups)
      if (e == cudaSuccess && gr.algo == ALGO_GATHER2)
        e = launch_gather_fold_multi(gr.f16, gr.fold, pl.side);
    for (const Group &gr : pl.groups)
      if (e == cudaSuccess && gr.algo == ALGO_GATHER2)
        e = launch_gather2_multi(gr.shape, gr.minw, gr.f16, gr.main, pl.lanes[gr.lane]);
    for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaEventRecord(pl.ev_join[l], pl.lanes[l]);
    if (e == cudaSuccess) e = cudaEventRecord(pl.ev_join[nl], pl.side);
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (const Group &gr : pl.groups) {
    if (gr.algo == ALGO_GATHER2) continue;
    e = cudaMemsetAsync(gr.launch.counter, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = launch_gather_persistent(gr.shape, gr.kb, gr.f16, gr.launch, st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  if (pl.side) {
    for (int l = 0; l <= nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(st, pl.ev_join[l], 0);
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (const InsertArgs &m : pl.merges) {
    e = launch_merge_scratch(m, st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (int b : pl.sequential) {
    int rc = run_config(ctxs[b], cfg[b], images[b], dtypes[b] == FR_F16, rotations[b], n[b], st);
    if (rc != FR_OK) return rc;
  }
  return FR_OK;
}

// One-time host-side setup of every kernel the plan launches (shared-memory
// attributes, occupancy), done before a capture so that the captured
// sequence holds launches, memsets and event records only.
int prime_plan(const Plan &pl, fr_ctx *const *ctxs, const int *dtypes, const std::vector<int> &cfg) {
  for (const Group &gr : pl.groups) {
    cudaError_t e;
    if (gr.algo == ALGO_GATHER2) {
      MultiLaunch q = gr.main;
      q.nitems = 0;
      e = launch_gather2_multi(gr.shape, gr.minw, gr.f16, q, nullptr);
      q = gr.fold;
      q.nitems = 0;
      if (e == cudaSuccess) e = launch_gather_fold_multi(gr.f16, q, nullptr);
    } else {
      PersistentLaunch q = gr.launch;
      q.nitems = 0;
      e = launch_gather_persistent(gr.shape, gr.kb, gr.f16, q, nullptr);
    }
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (int b : pl.sequential) {
    const Config &k = config_space()[cfg[b]];
    InsertArgs a = base_args(ctxs[b]);
    a.f16 = dtypes[b] == FR_F16;
    a.chunk = k.chunk;
    cudaError_t e = cudaSuccess;
    if (k.algo == ALGO_GATHER) {
      e = launch_gather(k.shape, k.wmode, a, nullptr, 1, nullptr);
    } else if (k.algo == ALGO_GATHER2) {
      e = launch_gather2(k.shape, k.minw, a, nullptr, 1, nullptr);
      InsertArgs f = a;
      f.nunits = 0;
      if (e == cudaSuccess) e = launch_gather_fold(f, nullptr);
    } else {
      e = launch_scatter(k.threads, k.wmode, a, nullptr, 1, nullptr);
    }
    if (e != cudaSuccess) return cuda_err(e);
  }
  return FR_OK;
}

}  // namespace

void batched_forget(const fr_ctx *c) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (std::find(it->ctxs.begin(), it->ctxs.end(), c) != it->ctxs.end()) {
      free_plan(*it);
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
}

int insert_batched(fr_ctx *const *ctxs, const void *const *images, const int *dtypes,
                   const float *const *rotations, const int *n, int nb, int capture,
                   cudaStream_t st) {
  for (int b = 0; b < nb; ++b) {
    if (!ctxs[b] || n[b] < 0 || n[b] > (1 << 24)) return FR_ERR_INVALID_ARG;
    if (n[b] > 0 && (!images[b] || !rotations[b])) return FR_ERR_INVALID_ARG;
    if (n[b] > 0 && (((uintptr_t)images[b] & 15) != 0 || ((uintptr_t)rotations[b] & 3) != 0))
      return FR_ERR_INVALID_ARG;
    if (dtypes[b] != FR_F32 && dtypes[b] != FR_F16) return FR_ERR_INVALID_ARG;
    if (ctxs[b]->device != ctxs[0]->device) return FR_ERR_INVALID_ARG;
  }
  if (nb == 0) return FR_OK;
  std::vector<int> cfg(nb);
  PlanKey key;
  for (int b = 0; b < nb; ++b) {
    cfg[b] = batched_config(ctxs[b], n[b], dtypes[b]);
    key.ptrs.push_back(ctxs[b]);
    key.ptrs.push_back(images[b]);
    key.ptrs.push_back(rotations[b]);
    key.ints.push_back(n[b]);
    key.ints.push_back(dtypes[b]);
    key.ints.push_back(cfg[b]);
  }
  key.ints.push_back(capture);

  std::lock_guard<std::mutex> lk(g_mu);
  auto it = std::find_if(g_plans.begin(), g_plans.end(),
                         [&](const Plan &p) { return !(p.key < key) && !(key < p.key); });
  if (it == g_plans.end()) {
    Plan pl;
    pl.key = key;
    int rc = build_plan(pl, ctxs, images, dtypes, rotations, n, nb, cfg);
    if (rc != FR_OK) {
      free_plan(pl);
      return rc;
    }
    if (capture) {
      rc = prime_plan(pl, ctxs, dtypes, cfg);
      if (rc != FR_OK) {
        free_plan(pl);
        return rc;
      }
      // capture on a library-owned stream (the caller's may be a default
      // stream, which cannot be captured); the graph is launched on st
      static cudaStream_t cap = nullptr;
      cudaError_t e = cudaSuccess;
      if (!cap) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        free_plan(pl);
        return cuda_err(e);
      }
      rc = enqueue_plan(pl, ctxs, images, dtypes, rotations, n, cfg, cap);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cap, &graph);
      if (rc == FR_OK && e == cudaSuccess) e = cudaGraphInstantiate(&pl.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (rc != FR_OK || e != cudaSuccess) {
        free_plan(pl);
        return rc != FR_OK ? rc : cuda_err(e);
      }
    }
    if (g_plans.size() >= MAX_PLANS) {
      // the evicted plan's buffers may still be read by queued work
      cudaDeviceSynchronize();
      free_plan(g_plans.back());
      g_plans.pop_back();
    }
    g_plans.push_front(std::move(pl));
    it = g_plans.begin();
  } else if (it != g_plans.begin()) {
    g_plans.splice(g_plans.begin(), g_plans, it);
    it = g_plans.begin();
  }
  if (it->exec) {
    cudaError_t e = cudaGraphLaunch(it->exec, st);
    if (e != cudaSuccess) return cuda_err(e);
  } else {
    int rc = enqueue_plan(*it, ctxs, images, dtypes, rotations, n, cfg, st);
    if (rc != FR_OK) return rc;
  }
  for (int b = 0; b < nb; ++b) {
    ctxs[b]->images += (unsigned long long)n[b];
    ctxs[b]->last_stream = st;
    ++ctxs[b]->launches;
  }
  return FR_OK;
}

}  // namespace fr
