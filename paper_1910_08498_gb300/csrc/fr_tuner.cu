// fr_tuner.cu -- configuration space, search orders, event-timed
// non-blocking tuning steps, amortisation arithmetic and the JSON tuning cache.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <sstream>
#include <string>
#include <vector>

#include "fr_ctx.h"
#include "fr_internal.h"
#include "fr_tuner.h"

namespace fr {

// ------------------------------------------------------------------ space
//
// Dimensions (the Fourier row of the paper's tuning space, Sec. 4.2.10,
// re-derived for this kernel family): algorithm (gather / atomic scatter),
// brick shape = work-group size and coarsening, image-tile depth (images
// staged in shared memory per barrier), blob weights from the shared-memory
// table or on the fly, scatter block size and atomic sub-batch.
const std::vector<Config> &config_space() {
  static const std::vector<Config> v = [] {
    std::vector<Config> c;
    for (int shape = 0; shape < num_gather_shapes(); ++shape)
      for (int w : {W_LUT, W_POLY, W_OTF})
        for (int ch : {32, 64, 128}) c.push_back(Config{ALGO_GATHER, shape, w, ch, 0, 0});
    for (int th : {128, 256})
      for (int w : {W_LUT, W_POLY})
        for (int sub : {256, 1024}) c.push_back(Config{ALGO_SCATTER, -1, w, 0, th, sub});
    for (int shape = 0; shape < num_gather2_shapes(); ++shape)
      for (int minw : {16, 20, 24})
        c.push_back(Config{ALGO_GATHER2, shape, W_POLY, 64, 0, 0, minw});
    for (int minw : {20, 24}) c.push_back(Config{ALGO_GATHER2, 2, W_POLY, 32, 0, 0, minw});
    return c;
  }();
  return v;
}

std::string describe(const Config &c) {
  char b[128];
  if (c.algo == ALGO_GATHER) {
    GatherShape s = gather_shape(c.shape);
    std::snprintf(b, sizeof b, "gather bx=%d by=%d zc=%d chunk=%d w=%s", s.bx, s.by, s.zc, c.chunk,
                  c.wmode == W_LUT ? "lut" : c.wmode == W_POLY ? "poly" : "otf");
  } else if (c.algo == ALGO_GATHER2) {
    GatherShape s = gather2_shape(c.shape);
    std::snprintf(b, sizeof b, "gather2 bx=%d by=%d zc=%d chunk=%d warps=%d w=poly", s.bx, s.by,
                  s.zc, c.chunk, c.minw);
  } else {
    std::snprintf(b, sizeof b, "scatter threads=%d sub=%d w=%s", c.threads, c.sub,
                  c.wmode == W_LUT ? "lut" : c.wmode == W_POLY ? "poly" : "otf");
  }
  return b;
}

unsigned long long space_hash() {
  unsigned long long h = 1469598103934665603ULL;  // FNV-1a
  for (const Config &c : config_space())
    for (char ch : describe(c)) {
      h ^= (unsigned char)ch;
      h *= 1099511628211ULL;
    }
  return h;
}

void config_features(const Config &c, int S, int n, float a, float *f) {
  for (int i = 0; i < 16; ++i) f[i] = 0.f;
  f[0] = c.algo == ALGO_SCATTER ? 1.f : (c.algo == ALGO_GATHER2 ? 0.5f : 0.f);
  if (c.algo == ALGO_GATHER || c.algo == ALGO_GATHER2) {
    if (c.algo == ALGO_GATHER && c.shape >= 0 && c.shape < 4) f[1 + c.shape] = 1.f;
    GatherShape s = c.algo == ALGO_GATHER2 ? gather2_shape(c.shape) : gather_shape(c.shape);
    f[6] = std::log2((float)c.chunk / 32.f) / 2.f;
    f[13] = s.zc / 16.f;
    f[14] = (float)(s.bx * s.by * s.zc) / 2048.f;
    f[15] = (float)(s.bx * s.by) / 256.f;
    if (c.algo == ALGO_GATHER2) f[8] = c.minw / 24.f;
  } else {
    f[7] = c.threads / 256.f;
    f[8] = c.sub / 1024.f;
  }
  f[5] = c.wmode == W_OTF ? 1.f : 0.f;
  f[12] = c.wmode == W_POLY ? 1.f : 0.f;
  f[9] = S / 256.f;
  f[10] = std::log2((float)std::max(n, 1)) / 13.f;
  f[11] = a / 2.5f;
}

int default_gather_config(const fr_ctx *c) {
  // the per-voxel gather, 16 x 16 x 8 CTA, polynomial weights, 64-image warp lists
  const auto &sp = config_space();
  for (int i = 0; i < (int)sp.size(); ++i)
    if (sp[i].algo == ALGO_GATHER && sp[i].shape == 0 && sp[i].wmode == W_POLY &&
        sp[i].chunk == 64 && config_valid(c, i))
      return i;
  for (int i = 0; i < (int)sp.size(); ++i)
    if (sp[i].algo == ALGO_GATHER && config_valid(c, i)) return i;
  return 0;
}

int default_config(const fr_ctx *c) {
  // the direct-drain gather, 16 x 8 x 8 CTA, registers for 24 warps per SM;
  // where it cannot run (a >= 2), the per-voxel gather default
  const auto &sp = config_space();
  for (int i = 0; i < (int)sp.size(); ++i)
    if (sp[i].algo == ALGO_GATHER2 && sp[i].shape == 1 && sp[i].minw == 24 && sp[i].chunk == 64 &&
        config_valid(c, i))
      return i;
  for (int i = 0; i < (int)sp.size(); ++i)
    if (sp[i].algo == ALGO_GATHER && sp[i].shape == 0 && sp[i].wmode == W_POLY &&
        sp[i].chunk == 64 && config_valid(c, i))
      return i;
  for (int i = 0; i < (int)sp.size(); ++i)
    if (config_valid(c, i)) return i;
  return 0;
}

// ------------------------------------------------------------------ Sec. 5.4 arithmetic

double relative_performance(double s, double t_avg, double t_well, double n) {
  return (s * t_avg + (n - s) * t_well) / (n * t_well);
}

double invocations_to_amortize(double rp, double s, double t_avg, double t_well) {
  return rp * s * (t_avg / t_well - 1.0) / (1.0 - rp);
}

double random_search_steps(double r, double p) { return std::log(1.0 - p) / std::log(1.0 - r); }

// ------------------------------------------------------------------ tuner

void Tuner::release() {
  for (auto &p : pending_) {
    cudaEventSynchronize(p.t.stop);
    cudaEventDestroy(p.t.start);
    cudaEventDestroy(p.t.stop);
  }
  pending_.clear();
  for (cudaEvent_t e : pool_) cudaEventDestroy(e);
  pool_.clear();
}

cudaEvent_t Tuner::get_event() {
  if (!pool_.empty()) {
    cudaEvent_t e = pool_.back();
    pool_.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// learned ordering lives in fr_mlp.cu
std::vector<int> learned_order(fr_ctx *c, const TuneKey &k, const std::vector<int> &valid,
                               int *predicted_best);

std::vector<int> Tuner::search_order(const TuneKey &k, fr_ctx *c) {
  std::vector<int> valid;
  for (int i = 0; i < (int)config_space().size(); ++i)
    if (config_valid(c, i)) valid.push_back(i);
  const fr_options &o = c->opt;
  std::mt19937_64 rng(o.seed ^ ((unsigned long long)k.S << 20) ^ ((unsigned long long)k.nb << 8) ^
                      (unsigned long long)k.dtype);
  std::vector<int> order = valid;
  if (o.search == FR_SEARCH_ANNEALING || o.search == FR_SEARCH_MCMC) {
    // adaptive: proposals are made step by step (plan); the order stays empty
    KeyState &ks = keys_[k];
    ks.adaptive = true;
    ks.budget = o.budget > 0 ? o.budget : std::max(1, (int)(valid.size() / 10));
    ks.walker.init(valid, default_config(c), o.search == FR_SEARCH_ANNEALING, rng());
    return {};
  }
  if (o.search == FR_SEARCH_LEARNED && c->mlp_trained) {
    int pb = -1;
    order = learned_order(c, k, valid, &pb);
    // default budget: at most a tenth of the valid space
    int budget = o.budget > 0 ? o.budget : std::max(1, (int)(valid.size() / 10));
    if ((int)order.size() > budget) order.resize(budget);
    keys_[k].predicted_best = pb;
    return order;
  }
  std::shuffle(order.begin(), order.end(), rng);
  if (o.search == FR_SEARCH_RANDOM && o.budget > 0 && (int)order.size() > o.budget)
    order.resize(o.budget);
  return order;
}

KeyState &Tuner::state(const TuneKey &k, fr_ctx *c) {
  auto it = keys_.find(k);
  if (it == keys_.end()) {
    KeyState &ks = keys_[k];
    ks.key = k;
    ks.order = search_order(k, c);
    ks.space_size = 0;
    for (int i = 0; i < (int)config_space().size(); ++i) ks.space_size += config_valid(c, i);
    if (current_ != nullptr) ++retunes_;
    current_ = &ks;
    return ks;
  }
  if (current_ != &it->second && current_ != nullptr && !it->second.tuned) ++retunes_;
  current_ = &it->second;
  return it->second;
}

// Tuning steps one insert may take.  Automatic (steps_per_insert = 0): each
// step gets at least AUTO_STEP_UPDATES estimated voxel updates (pixels per
// image x the blob's lattice volume 4/3 pi a^3), which keeps a step's kernel
// near 0.1 ms or longer so its event timing is accurate; at most AUTO_STEPS_MAX.
// Smaller steps put fewer images through slow configurations: over a stream of
// 20 batches of 5000 images at S = 256, 32 steps per insert cost 20 % over the
// oraculum where 4 steps cost 92 %, with the same configuration chosen.
static int steps_for(const fr_ctx *c, int n, const fr_options &opt) {
  if (opt.steps_per_insert > 0) return opt.steps_per_insert;
  constexpr double AUTO_STEP_UPDATES = 2e7;
  constexpr int AUTO_STEPS_MAX = 32;
  const double per_image = (double)c->S * (c->S / 2 + 1) * (4.0 / 3.0) * 3.14159265358979 *
                           (double)c->g.a * c->g.a * c->g.a;
  const double k = std::floor((double)n * per_image / AUTO_STEP_UPDATES);
  return (int)std::max(1.0, std::min((double)AUTO_STEPS_MAX, k));
}

std::vector<Step> Tuner::plan(KeyState &ks, int n, const fr_options &opt) {
  std::vector<Step> steps;
  const int kmax = steps_for(ctx_, n, opt);
  const int fallback = ks.best >= 0 ? ks.best : default_config(ctx_);
  if (!opt.tuning || ks.tuned) {
    steps.push_back(Step{fallback, n, false});
    return steps;
  }
  if (ks.confirming) {
    // the finalists, one whole insert each; then the best so far until
    // their timings are harvested
    if (ks.fin_next < ks.finalists.size())
      steps.push_back(Step{ks.finalists[ks.fin_next++], n, true, true});
    else
      steps.push_back(Step{fallback, n, false});
    return steps;
  }
  if (ks.adaptive) {
    // decide the proposals whose times are known, then propose this insert's steps
    ks.walker.decide([&](int c) -> double {
      if (ks.invalid.count(c)) return -1.0;
      auto it = ks.meas.find(c);
      return it == ks.meas.end() || it->second.images <= 0 ? 0.0 : it->second.per_image();
    });
    std::vector<int> cfgs;
    const int k = std::min(std::min(kmax, ks.budget - ks.proposed), n);
    for (int i = 0; i < k; ++i) {
      const int c = ks.walker.propose();
      if (c < 0) break;
      cfgs.push_back(c);
    }
    if (cfgs.empty()) {
      ks.budget = ks.proposed;  // nothing left to propose
      steps.push_back(Step{fallback, n, false});
      return steps;
    }
    ks.proposed += (int)cfgs.size();
    const int m = (int)cfgs.size();
    if (m > 1) ks.sub_steps = true;
    const int base = n / m, extra = n % m;
    for (int i = 0; i < m; ++i) steps.push_back(Step{cfgs[i], base + (i < extra ? 1 : 0), true});
    return steps;
  }
  // skip configurations found invalid
  while (ks.next < ks.order.size() && ks.invalid.count(ks.order[ks.next])) ++ks.next;
  const int remaining = (int)(ks.order.size() - ks.next);
  if (remaining <= 0) {
    steps.push_back(Step{fallback, n, false});
    return steps;
  }
  int k = std::min(std::min(kmax, remaining), n);
  if (k > 1) ks.sub_steps = true;
  int base = n / k, extra = n % k;
  for (int i = 0; i < k; ++i) {
    int cfg = ks.order[ks.next++];
    steps.push_back(Step{cfg, base + (i < extra ? 1 : 0), true});
  }
  return steps;
}

Timing Tuner::begin(cudaStream_t st) {
  Timing t;
  t.start = get_event();
  t.stop = get_event();
  cudaEventRecord(t.start, st);
  return t;
}

void Tuner::end(Timing t, KeyState &ks, int config, int images, bool tuning, cudaStream_t st,
                bool full) {
  cudaEventRecord(t.stop, st);
  pending_.push_back(Pending{t, &ks, config, images, tuning, full});
  if (full)
    ++ks.fin_pending;
  else if (tuning)
    ++ks.pending;
}

void Tuner::abandon(Timing t) {
  pool_.push_back(t.start);
  pool_.push_back(t.stop);
}

static int fastest(const std::map<int, Meas> &meas, const std::set<int> &invalid, int algo) {
  int best = -1;
  double bt = 0;
  for (auto &m : meas) {
    if (m.second.images <= 0 || invalid.count(m.first)) continue;
    if (algo >= 0 && config_space()[m.first].algo != algo) continue;
    double t = m.second.per_image();
    if (best < 0 || t < bt) { best = m.first; bt = t; }
  }
  return best;
}

// the best so far: the fastest screened configuration, or the fastest
// finalist once confirmed; final once the key is tuned
void Tuner::update_best(KeyState &ks) {
  if (ks.tuned) return;
  int best = ks.confirmed ? fastest(ks.full, ks.invalid, -1) : -1;
  if (best < 0) best = fastest(ks.meas, ks.invalid, -1);
  ks.best = best;
}

void Tuner::finish_if_done(KeyState &ks) {
  if (ks.tuned) return;
  const bool exhausted = ks.adaptive ? ks.proposed >= ks.budget : ks.next >= ks.order.size();
  if (!exhausted || ks.pending != 0) return;
  if (!ks.confirming) {
    update_best(ks);
    ks.finalists.clear();
    if (ks.sub_steps) {
      std::vector<std::pair<double, int>> fam;
      for (int algo : {ALGO_GATHER2, ALGO_GATHER, ALGO_SCATTER}) {
        const int f = fastest(ks.meas, ks.invalid, algo);
        if (f >= 0) fam.push_back({ks.meas[f].per_image(), f});
      }
      std::sort(fam.begin(), fam.end());
      for (auto &x : fam) ks.finalists.push_back(x.second);
    }
    if (ks.finalists.size() > 1) {
      ks.confirming = true;
      return;
    }
    ks.tuned = ks.best >= 0;
    return;
  }
  if (ks.fin_next < ks.finalists.size() || ks.fin_pending > 0) return;
  ks.confirmed = true;
  update_best(ks);
  ks.tuned = ks.best >= 0;
}

void Tuner::harvest() {
  size_t w = 0;
  for (size_t i = 0; i < pending_.size(); ++i) {
    Pending &p = pending_[i];
    cudaError_t q = cudaEventQuery(p.t.stop);
    if (q == cudaErrorNotReady) {
      pending_[w++] = p;
      continue;
    }
    float ms = 0.f;
    if (q == cudaSuccess && cudaEventElapsedTime(&ms, p.t.start, p.t.stop) == cudaSuccess) {
      double ns = (double)ms * 1e6;
      p.ks->all_ns += ns;
      p.ks->all_images += p.images;
      if (p.full || p.tuning) {
        Meas &m = p.full ? p.ks->full[p.config] : p.ks->meas[p.config];
        m.ns += ns;
        m.images += p.images;
        m.launches += 1;
      }
    } else {
      cudaGetLastError();
    }
    if (p.full)
      --p.ks->fin_pending;
    else if (p.tuning)
      --p.ks->pending;
    pool_.push_back(p.t.start);
    pool_.push_back(p.t.stop);
    update_best(*p.ks);
    finish_if_done(*p.ks);
  }
  pending_.resize(w);
  for (auto &kv : keys_) finish_if_done(kv.second);
}

void Tuner::retune(bool all) {
  // keep pending timings consistent: drop those of the keys being forgotten
  for (auto &p : pending_) {
    cudaEventSynchronize(p.t.stop);
    pool_.push_back(p.t.start);
    pool_.push_back(p.t.stop);
  }
  pending_.clear();
  if (all) {
    keys_.clear();
    current_ = nullptr;
  } else if (current_) {
    TuneKey k = current_->key;
    keys_.erase(k);
    current_ = nullptr;
  }
  ++retunes_;
}

// predicted-best configuration of a learned search, exposed in reserved[0]
static void reserved_hint(fr_report *r, const KeyState &ks) { r->reserved[0] = ks.predicted_best; }

void Tuner::report(fr_report *r) {
  r->best_config = -1;
  r->last_config = -1;
  r->retunes = retunes_;
  if (!current_) return;
  KeyState &ks = *current_;
  r->n_bucket = ks.key.nb;
  r->space_size = ks.space_size;
  r->evaluated = (int)ks.meas.size();
  r->tuned = ks.tuned ? 1 : 0;
  r->best_config = ks.best;
  r->last_config = ks.last_config;
  if (ks.best >= 0) {
    auto f = ks.full.find(ks.best);
    r->best_ns_per_image = ks.confirmed && f != ks.full.end() && f->second.images > 0
                               ? f->second.per_image()
                               : ks.meas[ks.best].per_image();
  }
  double sum = 0;
  int cnt = 0;
  for (auto &m : ks.meas)
    if (m.second.images > 0) { sum += m.second.per_image(); ++cnt; }
  r->mean_ns_per_image = cnt ? sum / cnt : 0;
  if (ks.best >= 0 && ks.all_images > 0 && r->best_ns_per_image > 0) {
    double rp = ks.all_ns / (ks.all_images * r->best_ns_per_image);
    r->tuning_overhead_pct = 100.0 * (rp - 1.0);
  }
  reserved_hint(r, ks);
}

int Tuner::measurements(int *cfg, double *ns, double *images, int cap) {
  if (!current_) return 0;
  int k = 0;
  for (auto &m : current_->meas) {
    if (k < cap) {
      if (cfg) cfg[k] = m.first;
      if (ns) ns[k] = m.second.per_image();
      if (images) images[k] = m.second.images;
    }
    ++k;
  }
  return k;
}

// ------------------------------------------------------------------ persistence

static std::string device_name(int dev, int *sms) {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    *sms = 0;
    return "unknown";
  }
  *sms = p.multiProcessorCount;
  return p.name;
}

int Tuner::save(const char *path) {
  harvest();
  int sms = 0;
  std::string dev = device_name(ctx_->device, &sms);
  FILE *f = std::fopen(path, "w");
  if (!f) return FR_ERR_IO;
  std::fprintf(f, "{\"version\": 1, \"device\": \"%s\", \"sms\": %d, \"space_hash\": \"%016llx\",\n",
               dev.c_str(), sms, space_hash());
  std::fprintf(f, " \"entries\": [");
  bool first = true;
  for (auto &kv : keys_) {
    const KeyState &ks = kv.second;
    if (ks.meas.empty()) continue;
    std::fprintf(f, "%s\n  {\"S\": %d, \"nb\": %d, \"a\": %.9g, \"dtype\": %d, \"tuned\": %d, "
                 "\"best\": %d, \"meas\": [", first ? "" : ",", ks.key.S, ks.key.nb,
                 (double)ks.key.a, ks.key.dtype, ks.tuned ? 1 : 0, ks.best);
    bool f2 = true;
    for (auto &m : ks.meas) {
      std::fprintf(f, "%s[%d, %.6f, %.1f]", f2 ? "" : ", ", m.first, m.second.ns,
                   m.second.images);
      f2 = false;
    }
    std::fprintf(f, "]}");
    first = false;
  }
  std::fprintf(f, "\n ]}\n");
  return std::fclose(f) == 0 ? FR_OK : FR_ERR_IO;
}

// Minimal reader for the format written above.
static bool read_file(const char *path, std::string &out) {
  FILE *f = std::fopen(path, "rb");
  if (!f) return false;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) out.append(buf, n);
  std::fclose(f);
  return true;
}

static bool find_num(const std::string &s, size_t from, size_t to, const char *key, double *v) {
  std::string k = std::string("\"") + key + "\":";
  size_t p = s.find(k, from);
  if (p == std::string::npos || p >= to) return false;
  *v = std::strtod(s.c_str() + p + k.size(), nullptr);
  return true;
}

int Tuner::load(const char *path) {
  std::string s;
  if (!read_file(path, s)) return FR_ERR_IO;
  int sms = 0;
  std::string dev = device_name(ctx_->device, &sms);
  char hash[32];
  std::snprintf(hash, sizeof hash, "%016llx", space_hash());
  if (s.find(std::string("\"device\": \"") + dev + "\"") == std::string::npos) return FR_OK;
  if (s.find(std::string("\"space_hash\": \"") + hash + "\"") == std::string::npos) return FR_OK;
  double v = 0;
  if (!find_num(s, 0, s.size(), "sms", &v) || (int)v != sms) return FR_OK;
  size_t pos = s.find("\"entries\"");
  if (pos == std::string::npos) return FR_ERR_IO;
  while (true) {
    size_t b = s.find("{\"S\":", pos);
    if (b == std::string::npos) break;
    size_t e = s.find("]}", b);
    if (e == std::string::npos) return FR_ERR_IO;
    double S, nb, a, dt, tuned, best;
    if (!find_num(s, b, e, "S", &S) || !find_num(s, b, e, "nb", &nb) ||
        !find_num(s, b, e, "a", &a) || !find_num(s, b, e, "dtype", &dt) ||
        !find_num(s, b, e, "tuned", &tuned) || !find_num(s, b, e, "best", &best))
      return FR_ERR_IO;
    TuneKey k{(int)S, (int)nb, (float)a, (int)dt};
    KeyState &ks = keys_[k];
    ks = KeyState();
    ks.key = k;
    ks.space_size = 0;
    for (int i = 0; i < (int)config_space().size(); ++i) ks.space_size += config_valid(ctx_, i);
    size_t m = s.find("\"meas\": [", b);
    size_t p = m + 9;
    while (p < e) {
      size_t lb = s.find('[', p);
      if (lb == std::string::npos || lb >= e) break;
      char *q = nullptr;
      int cfg = (int)std::strtol(s.c_str() + lb + 1, &q, 10);
      double ns = std::strtod(q + 1, &q);
      double im = std::strtod(q + 1, &q);
      if (cfg >= 0 && cfg < (int)config_space().size()) {
        Meas &mm = ks.meas[cfg];
        mm.ns = ns;
        mm.images = im;
        mm.launches = 1;
      }
      p = (size_t)(q - s.c_str()) + 1;
    }
    // a loaded key is finished if it was finished when saved; otherwise the
    // unmeasured configurations are searched next
    std::vector<int> order;
    for (int i = 0; i < (int)config_space().size(); ++i)
      if (config_valid(ctx_, i) && !ks.meas.count(i)) order.push_back(i);
    ks.order = tuned > 0 ? std::vector<int>() : order;
    ks.next = 0;
    update_best(ks);
    // a finished key keeps the best it was saved with (it may have been
    // decided by whole-insert timings, which are not saved)
    const int saved = (int)best;
    if (tuned > 0 && saved >= 0 && saved < (int)config_space().size() && config_valid(ctx_, saved))
      ks.best = saved;
    ks.tuned = tuned > 0 && ks.best >= 0;
    pos = e + 2;
  }
  return FR_OK;
}

}  // namespace fr
