// fr_batched.cu -- insertion of many uneven batches (differing S and n), one
// batch per context, with the launch sequence captured into a CUDA graph.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fr_ctx.h"
#include "fr_internal.h"
#include "fr_tuner.h"

namespace fr {

namespace {
struct GraphKey {
  std::vector<const void *> ptrs;
  std::vector<int> ints;
  bool operator<(const GraphKey &o) const {
    return std::tie(ptrs, ints) < std::tie(o.ptrs, o.ints);
  }
};
std::mutex g_graph_mu;
std::map<GraphKey, cudaGraphExec_t> g_graphs;
}  // namespace

// configuration a batch runs with: the context's tuned best for its key, else
// its default; scatter configurations need the scratch volume and are mapped
// to the default so the captured sequence allocates nothing
static int batched_config(fr_ctx *c, int n, int dtype) {
  TuneKey k{c->S, key_bucket(n), c->g.a, dtype};
  int best = c->tuner.best_for(k);
  if (c->opt.forced_config >= 0) best = c->opt.forced_config;
  if (best < 0 || config_space()[best].algo != ALGO_GATHER) best = default_config(c);
  return best;
}

int insert_batched(fr_ctx *const *ctxs, const void *const *images, const int *dtypes,
                   const float *const *rotations, const int *n, int nb, int capture,
                   cudaStream_t st) {
  for (int b = 0; b < nb; ++b) {
    if (!ctxs[b] || n[b] < 0 || n[b] > (1 << 24)) return FR_ERR_INVALID_ARG;
    if (n[b] > 0 && (!images[b] || !rotations[b])) return FR_ERR_INVALID_ARG;
    if (dtypes[b] != FR_F32 && dtypes[b] != FR_F16) return FR_ERR_INVALID_ARG;
  }
  if (nb == 0) return FR_OK;
  std::vector<int> cfg(nb);
  for (int b = 0; b < nb; ++b) {
    cfg[b] = batched_config(ctxs[b], n[b], dtypes[b]);
    if (n[b] > 0) {
      int rc = prepare_config(ctxs[b], cfg[b], n[b]);
      if (rc != FR_OK) return rc;
    }
  }
  auto enqueue = [&]() -> int {
    for (int b = 0; b < nb; ++b) {
      if (n[b] == 0) continue;
      int rc = run_config(ctxs[b], cfg[b], images[b], dtypes[b] == FR_F16, rotations[b], n[b], st);
      if (rc != FR_OK) return rc;
    }
    return FR_OK;
  };
  if (!capture) {
    int rc = enqueue();
    if (rc != FR_OK) return rc;
  } else {
    GraphKey key;
    for (int b = 0; b < nb; ++b) {
      key.ptrs.push_back(ctxs[b]);
      key.ptrs.push_back(images[b]);
      key.ptrs.push_back(rotations[b]);
      key.ints.push_back(n[b]);
      key.ints.push_back(dtypes[b]);
      key.ints.push_back(cfg[b]);
    }
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_graph_mu);
      auto it = g_graphs.find(key);
      if (it != g_graphs.end()) exec = it->second;
    }
    if (!exec) {
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return FR_ERR_CUDA;
      int rc = enqueue();
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &graph);
      if (rc != FR_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (e != cudaSuccess) return FR_ERR_CUDA;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return FR_ERR_CUDA;
      std::lock_guard<std::mutex> lk(g_graph_mu);
      g_graphs[key] = exec;
    }
    if (cudaGraphLaunch(exec, st) != cudaSuccess) return FR_ERR_CUDA;
  }
  for (int b = 0; b < nb; ++b) {
    ctxs[b]->images += (unsigned long long)n[b];
    ctxs[b]->last_stream = st;
    ++ctxs[b]->launches;
  }
  return FR_OK;
}

}  // namespace fr
