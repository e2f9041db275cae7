// fr_batched.cu -- insertion of many uneven batches (differing S and n), one
// batch per context, in persistent gather launches fed by a device work
// counter (A8), optionally captured into a CUDA graph.
//
// A call is turned into a plan, cached by (contexts, image and rotation
// pointers, sizes, dtypes, configurations):
//   * batches are grouped by what one kernel instantiation needs in common
//     (brick shape, candidate-box width, image dtype, list capacity);
//   * each group's work units (bricks and image splits, with expected loads)
//     are pooled over its batches with one splitting target and ordered
//     heaviest first; a CTA of the persistent kernel takes one unit at a time;
//   * the per-batch launch arguments and the items are uploaded once into a
//     device buffer the plan owns;
//   * a launch clears each group's counter, runs the group's persistent
//     kernel, and merges the float4 scratch of every context that received
//     split (or shared) units.
// A context that appears in several batches of one call has all of its units
// routed through its scratch (atomics), so concurrent units never race on its
// accumulators.  Batches the persistent kernel cannot take (scatter choices
// are mapped to the default gather; a context whose polynomial weights are
// not accurate enough) run one launch per batch, in order, after the groups.
#include <cuda_runtime.h>

#include <algorithm>
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
  int shape = 0, kb = 4, f16 = 0, chunk = 64;
  PersistentLaunch launch{};
};

struct Plan {
  PlanKey key;
  std::vector<const fr_ctx *> ctxs;  // contexts the plan refers to
  void *dev = nullptr;               // descriptors, items, counters (owned)
  std::vector<Group> groups;
  std::vector<InsertArgs> merges;    // scratch merges after the groups
  std::vector<int> sequential;       // batches run one launch each
  cudaGraphExec_t exec = nullptr;
};

std::mutex g_mu;
std::list<Plan> g_plans;  // most recently used first
constexpr size_t MAX_PLANS = 32;

void free_plan(Plan &p) {
  if (p.exec) cudaGraphExecDestroy(p.exec);
  cudaFree(p.dev);
  p.exec = nullptr;
  p.dev = nullptr;
}

// configuration a batch runs with: the context's tuned best for its key, else
// its default; scatter configurations are mapped to the default gather
int batched_config(fr_ctx *c, int n, int dtype) {
  TuneKey k{c->S, key_bucket(n), c->g.a, dtype};
  int best = c->tuner.best_for(k);
  if (c->opt.forced_config >= 0) best = c->opt.forced_config;
  if (best < 0 || config_space()[best].algo != ALGO_GATHER) best = default_gather_config(c);
  return best;
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
  // group the batches the persistent kernel can take
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
  for (int b = 0; b < nb; ++b) {
    if (n[b] == 0) continue;
    const fr_ctx *c = ctxs[b];
    const Config &k = config_space()[cfg[b]];
    if (!(c->poly_err < 1e-6)) {
      pl.sequential.push_back(b);
      continue;
    }
    groups[std::make_tuple(k.shape, c->g.KB, dtypes[b] == FR_F16 ? 1 : 0, k.chunk)].push_back(b);
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctxs[0]->device);
  sms = std::max(sms, 1);

  std::vector<InsertArgs> descs(nb);
  std::vector<std::vector<int4>> items;
  std::set<const fr_ctx *> merge_ctx;
  for (auto &kv : groups) {
    Group gr;
    std::tie(gr.shape, gr.kb, gr.f16, gr.chunk) = kv.first;
    // pooled splitting target: total expected load over 32 items per SM
    double total = 0;
    std::vector<UnitLoad> tmp;
    int any = 0;
    for (int b : kv.second) total += gather_unit_loads(ctxs[b], gr.shape, n[b], 1e300, tmp, any);
    const double target = std::max(64.0, total / (sms * 32.0));
    struct It { double load; int4 v; };
    std::vector<It> its;
    for (int b : kv.second) {
      fr_ctx *c = ctxs[b];
      int any_split = 0;
      gather_unit_loads(c, gr.shape, n[b], target, tmp, any_split);
      const bool shared = uses[c] > 1;
      if (any_split || shared) {
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
      a.scratch = c->scratch;
      a.phase = nullptr;
      a.units = nullptr;
      descs[b] = a;
      for (const UnitLoad &u : tmp) {
        const int w = u.unit.w | (shared ? (1 << 30) : 0);
        its.push_back(It{u.load, make_int4(u.unit.x | (u.unit.y << 10) | (u.unit.z << 20), w, b, 0)});
      }
    }
    std::stable_sort(its.begin(), its.end(), [](const It &p, const It &q) { return p.load > q.load; });
    std::vector<int4> v(its.size());
    for (size_t i = 0; i < its.size(); ++i) v[i] = its[i].v;
    items.push_back(std::move(v));
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
  e = cudaMemcpy(d, descs.data(), (size_t)nb * sizeof(InsertArgs), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(e);
  for (size_t gi = 0; gi < pl.groups.size(); ++gi) {
    e = cudaMemcpy(d + item_off[gi], items[gi].data(), items[gi].size() * sizeof(int4),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(e);
    PersistentLaunch &L = pl.groups[gi].launch;
    L.descs = reinterpret_cast<const InsertArgs *>(d);
    L.items = reinterpret_cast<const int4 *>(d + item_off[gi]);
    L.nitems = (int)items[gi].size();
    L.chunk = pl.groups[gi].chunk;
    L.counter = reinterpret_cast<unsigned *>(d + counter_off) + gi;
  }
  for (const fr_ctx *c : merge_ctx) pl.merges.push_back(base_args(c));
  for (int b = 0; b < nb; ++b) pl.ctxs.push_back(ctxs[b]);
  return FR_OK;
}

// Enqueue one execution of the plan on st.
int enqueue_plan(const Plan &pl, fr_ctx *const *ctxs, const void *const *images, const int *dtypes,
                 const float *const *rotations, const int *n, const std::vector<int> &cfg,
                 cudaStream_t st) {
  for (const Group &gr : pl.groups) {
    cudaError_t e = cudaMemsetAsync(gr.launch.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_err(e);
    e = launch_gather_persistent(gr.shape, gr.kb, gr.f16, gr.launch, st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (const InsertArgs &m : pl.merges) {
    cudaError_t e = launch_merge_scratch(m, st);
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
// sequence holds launches and memsets only.
int prime_plan(const Plan &pl, fr_ctx *const *ctxs, const int *dtypes, const std::vector<int> &cfg) {
  for (const Group &gr : pl.groups) {
    PersistentLaunch q = gr.launch;
    q.nitems = 0;
    cudaError_t e = launch_gather_persistent(gr.shape, gr.kb, gr.f16, q, nullptr);
    if (e != cudaSuccess) return cuda_err(e);
  }
  for (int b : pl.sequential) {
    const Config &k = config_space()[cfg[b]];
    InsertArgs a = base_args(ctxs[b]);
    a.f16 = dtypes[b] == FR_F16;
    a.chunk = k.chunk;
    cudaError_t e = launch_gather(k.shape, k.wmode, a, nullptr, 1, nullptr);
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
    if (dtypes[b] != FR_F32 && dtypes[b] != FR_F16) return FR_ERR_INVALID_ARG;
    if (ctxs[b]->device != ctxs[0]->device) return FR_ERR_INVALID_ARG;
  }
  if (nb == 0) return FR_OK;
  std::vector<int> cfg(nb);
  PlanKey key;
  for (int b = 0; b < nb; ++b) {
    cfg[b] = batched_config(ctxs[b], n[b], dtypes[b]);
    if (n[b] > 0 && config_space()[cfg[b]].algo == ALGO_GATHER) {
      // the sequential fallback needs the context's own units and scratch ready
      int rc = prepare_config(ctxs[b], cfg[b], n[b]);
      if (rc != FR_OK) return rc;
    }
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
