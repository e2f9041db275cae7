// fr_tuner.h -- configuration space and the non-blocking dynamic tuner.
//
// Tuning follows the non-blocking dynamic mode of Sec. 3.2: every tuning step
// is a real insertion of real images (a sub-batch of the caller's batch), run
// with the next configuration of the search order and timed with CUDA events;
// the output is kept, so the volume is the same whatever the tuner does.
// Timings are harvested without blocking (cudaEventQuery) on later calls.
// Once every configuration of the search order has a timing, the key is
// tuned and later inserts run the fastest configuration (the paper's
// tuneKernelByStep behaviour once the space is exhausted).
//
// Sub-batch steps favour kernels whose cost has no fixed part: a gather
// launch carries a per-launch cost (the serial path of the bricks every plane
// crosses, the scratch merge) that a 50-image step does not amortise, so
// ranking kernel families on sub-batches can pick a family that is slower at
// the batch's own size.  When the screening ran in sub-batch steps, the
// fastest configuration of each kernel family is therefore run once more on
// a whole insert, and the key's best is the fastest of those whole-insert
// timings (within a family the per-launch costs are alike, so the
// sub-batch ranking stands).
//
// A key is (S, batch-size bucket, blob radius, image dtype): a change of image
// size or of batch shape starts a new search (or reuses a cached one), which
// is the runtime re-tuning of Sec. 5.3.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <set>
#include <string>
#include <vector>

#include "fr_search.h"

struct fr_ctx;
struct fr_options;
struct fr_report;

namespace fr {

struct Config {
  int algo;     // ALGO_GATHER or ALGO_SCATTER
  int shape;    // gather brick shape id
  int wmode;    // W_LUT, W_OTF or W_POLY
  int chunk;    // gather: capacity of a warp's shared-memory image list
  int threads;  // scatter: block size
  int sub;      // scatter: images per atomic sub-batch (merged after each)
  int minw = 0; // direct-drain gather: resident warps per SM the registers allow (16, 20, 24)
};

const std::vector<Config> &config_space();
std::string describe(const Config &c);
unsigned long long space_hash();
// 16 normalised features of (configuration, S, n, a) for the cost model
void config_features(const Config &c, int S, int n, float a, float *out16);
int default_config(const fr_ctx *c);
// the per-voxel gather's default (the persistent batched launches run that family)
int default_gather_config(const fr_ctx *c);
int config_valid(const fr_ctx *c, int id);
int run_config(fr_ctx *c, int id, const void *images, int f16, const float *rot, int n,
               cudaStream_t st);
int prepare_config(fr_ctx *c, int id, int n);

// Eq. (performance), Eq. (invocations), Eq. (samples) of Sec. 5.4
double relative_performance(double s, double t_avg, double t_well, double n);
double invocations_to_amortize(double rp, double s, double t_avg, double t_well);
double random_search_steps(double r, double p);

struct TuneKey {
  int S;
  int nb;
  float a;
  int dtype;
  bool operator<(const TuneKey &o) const {
    if (S != o.S) return S < o.S;
    if (nb != o.nb) return nb < o.nb;
    if (a != o.a) return a < o.a;
    return dtype < o.dtype;
  }
};

struct Meas {
  double ns = 0;      // summed kernel time
  double images = 0;  // summed images
  int launches = 0;
  double per_image() const { return images > 0 ? ns / images : 0; }
};

struct KeyState {
  TuneKey key{};
  std::vector<int> order;  // configurations to measure, in search order
  size_t next = 0;
  std::map<int, Meas> meas;
  std::set<int> invalid;
  int pending = 0;
  bool tuned = false;
  int best = -1;
  int last_config = -1;
  double all_ns = 0, all_images = 0;  // every timed launch of this key
  int space_size = 0;
  int predicted_best = -1;            // learned search: the model's first choice
  // adaptive searches (annealing, Metropolis): configurations are proposed
  // one step at a time from the measurements known so far
  bool adaptive = false;
  int budget = 0, proposed = 0;
  Walker walker;
  // confirmation on whole inserts (see the file comment)
  bool sub_steps = false;       // some screening step took part of an insert
  bool confirming = false, confirmed = false;
  std::vector<int> finalists;   // the fastest screened configuration of each family
  size_t fin_next = 0;
  int fin_pending = 0;
  std::map<int, Meas> full;     // whole-insert timings of the finalists
};

struct Step {
  int config;
  int images;
  bool tuning;
  bool full = false;  // a finalist's whole-insert timing
};

struct Timing {
  cudaEvent_t start = nullptr, stop = nullptr;
};

class Tuner {
 public:
  void init(fr_ctx *c) { ctx_ = c; }
  void release();
  KeyState &state(const TuneKey &k, fr_ctx *c);
  std::vector<Step> plan(KeyState &ks, int n, const fr_options &opt);
  Timing begin(cudaStream_t st);
  void end(Timing t, KeyState &ks, int config, int images, bool tuning, cudaStream_t st,
           bool full = false);
  void abandon(Timing t);
  void harvest();
  void retune(bool all);
  void report(fr_report *r);
  int measurements(int *cfg, double *ns, double *images, int cap);
  int save(const char *path);
  int load(const char *path);
  int retunes() const { return retunes_; }
  // best configuration of a finished or partly measured key, -1 if unknown
  int best_for(const TuneKey &k) const {
    auto it = keys_.find(k);
    return it == keys_.end() ? -1 : it->second.best;
  }

 private:
  struct Pending {
    Timing t;
    KeyState *ks;
    int config;
    int images;
    bool tuning;
    bool full;
  };
  void finish_if_done(KeyState &ks);
  void update_best(KeyState &ks);
  std::vector<int> search_order(const TuneKey &k, fr_ctx *c);
  cudaEvent_t get_event();

  fr_ctx *ctx_ = nullptr;
  std::map<TuneKey, KeyState> keys_;
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> pool_;
  KeyState *current_ = nullptr;
  int retunes_ = 0;
};

// batched insertion (fr_insert_batched)
int insert_batched(fr_ctx *const *ctxs, const void *const *images, const int *dtypes,
                   const float *const *rotations, const int *n, int nb, int capture,
                   cudaStream_t st);

}  // namespace fr
