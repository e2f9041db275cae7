// fr_search.cu -- neighbourhoods and proposals of the adaptive searchers
// (simulated annealing, Metropolis walk), and a host-only simulation of every
// search order over a table of known times (fr_search_simulate) so that the
// searchers can be compared at equal budgets on measured sweeps.
#include <cmath>

#include <algorithm>
#include <numeric>

#include "../../include/fr.h"
#include "fr_internal.h"
#include "fr_search.h"
#include "fr_tuner.h"

namespace fr {

std::vector<std::vector<int>> config_neighbours(const std::vector<int> &valid) {
  const auto &sp = config_space();
  std::vector<std::vector<int>> nbr(sp.size());
  for (int i : valid)
    for (int j : valid) {
      if (i == j) continue;
      const Config &a = sp[i], &b = sp[j];
      bool adj = false;
      if (a.algo == b.algo) {
        int diff = 0;
        if (a.algo == ALGO_GATHER)
          diff = (a.shape != b.shape) + (a.wmode != b.wmode) + (a.chunk != b.chunk);
        else if (a.algo == ALGO_GATHER2)
          diff = (a.shape != b.shape) + (a.minw != b.minw);
        else
          diff = (a.threads != b.threads) + (a.wmode != b.wmode) + (a.sub != b.sub);
        adj = diff == 1;
      } else if (a.algo == ALGO_GATHER2 || b.algo == ALGO_GATHER2) {
        // the direct-drain gather neighbours the per-voxel gather of its brick
        // shape and list capacity with polynomial weights (and nothing else)
        const Config &g2 = a.algo == ALGO_GATHER2 ? a : b, &o = a.algo == ALGO_GATHER2 ? b : a;
        adj = o.algo == ALGO_GATHER && o.shape == g2.shape && o.chunk == g2.chunk &&
              o.wmode == W_POLY && g2.minw == 16;
      } else {
        adj = a.wmode == b.wmode;  // gather <-> scatter with the same weights
      }
      if (adj) nbr[i].push_back(j);
    }
  return nbr;
}

void Walker::init(const std::vector<int> &valid_cfgs, int start, bool annealing,
                  unsigned long long seed) {
  valid = valid_cfgs;
  nbr = config_neighbours(valid);
  anneal = annealing;
  T = annealing ? 0.2 : 0.1;
  proposed.clear();
  undecided.clear();
  current = -1;
  cur_t = 0;
  rng.seed(seed);
  if (std::find(valid.begin(), valid.end(), start) == valid.end() && !valid.empty())
    start = valid[rng() % valid.size()];
  if (start >= 0) {
    proposed.insert(start);
    undecided.push_back(start);
    pending_start_ = start;
  }
}

int Walker::propose() {
  if (pending_start_ >= 0) {
    const int s = pending_start_;
    pending_start_ = -1;
    return s;
  }
  if (proposed.size() >= valid.size()) return -1;
  std::vector<int> cand;
  const int from = current >= 0 ? current : (proposed.empty() ? -1 : *proposed.begin());
  if (from >= 0)
    for (int j : nbr[from])
      if (!proposed.count(j)) cand.push_back(j);
  if (cand.empty())
    for (int j : valid)
      if (!proposed.count(j)) cand.push_back(j);
  if (cand.empty()) return -1;
  const int c = cand[rng() % cand.size()];
  proposed.insert(c);
  undecided.push_back(c);
  return c;
}

}  // namespace fr

using namespace fr;

extern "C" int fr_search_simulate(int search, const double *ns_per_image, int nconfig, int budget,
                                  uint64_t seed, int start, int *order) {
  const auto &sp = config_space();
  if (!ns_per_image || !order || nconfig != (int)sp.size() || budget < 1) return -FR_ERR_INVALID_ARG;
  std::vector<int> valid;
  for (int i = 0; i < nconfig; ++i)
    if (ns_per_image[i] > 0) valid.push_back(i);
  const int k = std::min(budget, (int)valid.size());
  if (search == FR_SEARCH_EXHAUSTIVE || search == FR_SEARCH_RANDOM) {
    std::vector<int> o = valid;
    std::mt19937_64 rng(seed);
    if (search == FR_SEARCH_RANDOM) std::shuffle(o.begin(), o.end(), rng);
    for (int i = 0; i < k; ++i) order[i] = o[i];
    return k;
  }
  if (search != FR_SEARCH_ANNEALING && search != FR_SEARCH_MCMC) return -FR_ERR_INVALID_ARG;
  Walker w;
  w.init(valid, start, search == FR_SEARCH_ANNEALING, seed);
  int m = 0;
  while (m < k) {
    const int c = w.propose();
    if (c < 0) break;
    order[m++] = c;
    w.decide([&](int i) { return ns_per_image[i]; });  // measured at once
  }
  return m;
}
