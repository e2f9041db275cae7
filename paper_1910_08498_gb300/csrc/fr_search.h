// fr_search.h -- adaptive searchers of the tuning space: simulated annealing
// and a Metropolis (MCMC) walk over neighbouring configurations.
#pragma once

#include <cmath>
#include <random>
#include <set>
#include <vector>

namespace fr {

// Neighbours of configuration i among `valid`: the configurations of the same
// algorithm that differ from it in exactly one tuning dimension, and for a
// gather configuration the scatter ones with the same weights (and back).
std::vector<std::vector<int>> config_neighbours(const std::vector<int> &valid);

// A walk over the space.  The state is the current configuration and its
// time; a proposal is a not yet proposed neighbour of the current one (a
// not yet proposed configuration anywhere once the neighbourhood is used
// up).  When a proposal's time is known it is accepted if faster, else with
// probability exp(-(t_new / t_cur - 1) / T).  Simulated annealing lowers T
// geometrically after every decision; the Metropolis walk keeps it constant.
struct Walker {
  bool anneal = true;
  double T = 0.2, decay = 0.7;
  std::vector<int> valid;
  std::vector<std::vector<int>> nbr;  // indexed like config_space()
  std::set<int> proposed;
  std::vector<int> undecided;  // proposals whose acceptance is still open, in order
  int current = -1;
  double cur_t = 0;
  std::mt19937_64 rng;
  int pending_start_ = -1;  // the starting configuration, proposed first

  void init(const std::vector<int> &valid_cfgs, int start, bool annealing, unsigned long long seed);
  // next configuration to measure, or -1 when every valid one was proposed
  int propose();
  // decide the open proposals whose times are known (time(c) > 0: ns per
  // image; 0: not yet measured; < 0: invalid)
  template <class F>
  void decide(F time) {
    while (!undecided.empty()) {
      const int c = undecided.front();
      const double t = time(c);
      if (t == 0) break;  // wait for it: decisions are taken in proposal order
      undecided.erase(undecided.begin());
      if (t < 0) continue;
      if (current < 0 || cur_t <= 0) {
        current = c;
        cur_t = t;
      } else {
        const double d = t / cur_t - 1.0;
        std::uniform_real_distribution<double> u(0.0, 1.0);
        if (d < 0 || u(rng) < std::exp(-d / T)) {
          current = c;
          cur_t = t;
        }
      }
      if (anneal) T *= decay;
    }
  }
};

}  // namespace fr
