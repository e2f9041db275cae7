"""Host-side pieces of the learned-tuner evaluation (no GPU): the exact
expected regret of random search, the per-workload relative log-time targets
and the feature rows, and the shipped model and sweeps are well formed."""
import json
import math

import numpy as np
import pytest

from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import costmodel as cm


@pytest.fixture(scope="module", autouse=True)
def lib():
    import os
    if not os.path.exists(L.LIB_PATH):
        from paper_1910_08498_gb300.build import build
        build()
    return L.lib()


def test_random_expected_regret_closed_form():
    # best of k = 1 draw from {1, 2, 3, 4}: mean regret (0 + 1 + 2 + 3) / 4
    assert cm.random_expected_regret([1, 2, 3, 4], 1) == pytest.approx(1.5)
    # k = 2 of 4: P(best is the fastest) = 3/6, second 2/6, third 1/6
    assert cm.random_expected_regret([4, 3, 2, 1], 2) == pytest.approx(2 / 6 * 1 + 1 / 6 * 2)
    assert cm.random_expected_regret([5, 7], 2) == 0.0


def test_random_expected_regret_matches_enumeration():
    rng = np.random.default_rng(3)
    t = rng.uniform(1, 3, 9)
    import itertools
    for k in (1, 2, 4):
        subsets = list(itertools.combinations(range(9), k))
        brute = np.mean([min(t[list(s)]) / t.min() - 1 for s in subsets])
        assert cm.random_expected_regret(t, k) == pytest.approx(brute, rel=1e-12)


def test_training_targets_are_relative_log_times():
    wl = {(64, 1.9, 500): {0: 100.0, 1: 400.0}, (128, 1.9, 500): {0: 50.0, 36: 50.0}}
    X, y = cm.training_set(wl)
    assert X.shape == (4, 16)
    assert y[:2] == pytest.approx([-math.log(2), math.log(2)], abs=1e-6)
    assert y[2:] == pytest.approx([0.0, 0.0], abs=1e-6)
    assert X[0][9] == pytest.approx(64 / 256) and X[2][9] == pytest.approx(128 / 256)


def test_shipped_model_and_sweeps_are_well_formed():
    p = json.load(open(cm.PRETRAINED))
    assert len(p) == L.MLP_NPARAM and all(math.isfinite(x) for x in p)
    for name in ("sweep_gb300_train.json", "sweep_gb300_heldout.json"):
        d = json.load(open(f"{cm.DATA}/{name}"))
        space = [L.fr_describe_config(i) for i in range(L.fr_num_configs())]
        assert d["space"] == space  # measured on the current configuration space
        wl = cm.workloads(d["rows"])
        assert all(len(t) >= 10 and min(t.values()) > 0 for t in wl.values())
        # every valid configuration of each workload was measured: all of the
        # space where the direct-drain gather runs (a < 2), the rest otherwise
        for (S, a, n), t in wl.items():
            g2 = [i for i, s in enumerate(space) if s.startswith("gather2")]
            assert (set(g2) <= set(t)) == (a < 2.0), (S, a, n)


def test_search_simulate_orders():
    N = L.fr_num_configs()
    rng = np.random.default_rng(5)
    t = list(rng.uniform(1, 3, N))
    t[7] = 0.0   # invalid
    t[40] = -1.0  # invalid
    valid = [c for c in range(N) if t[c] > 0]
    assert L.fr_search_simulate(L.FR_SEARCH_EXHAUSTIVE, t, N) == valid
    r = L.fr_search_simulate(L.FR_SEARCH_RANDOM, t, 10, seed=3)
    assert len(r) == 10 and len(set(r)) == 10 and set(r) <= set(valid)
    for s in (L.FR_SEARCH_ANNEALING, L.FR_SEARCH_MCMC):
        o = L.fr_search_simulate(s, t, 12, seed=4, start=4)
        assert o[0] == 4 and len(o) == 12 and len(set(o)) == 12 and set(o) <= set(valid)
        full = L.fr_search_simulate(s, t, N, seed=4, start=4)
        assert sorted(full) == valid          # a walk eventually proposes every valid one
    with pytest.raises(L.FrError):
        L.fr_search_simulate(L.FR_SEARCH_LEARNED, t, 4)


def test_walks_beat_random_on_a_smooth_landscape():
    """Time = 1 + (number of tuning dimensions that differ from a fixed
    optimum): neighbours of the current configuration are one step closer or
    farther, so the walks descend; random search does not use that."""
    N = L.fr_num_configs()
    desc = [L.fr_describe_config(c) for c in range(N)]
    opt = desc.index("gather bx=32 by=8 zc=4 chunk=128 w=otf")

    def dims(d):
        return dict(x.split("=") for x in d.split()[1:]) | {"algo": d.split()[0]}

    o = dims(desc[opt])
    t = [1.0 + sum(dims(d).get(k) != v for k, v in o.items()) for d in desc]
    wl = {(256, 1.9, 5000): {c: t[c] for c in range(N)}}
    # the optimum is three improving moves from the start; with 19 evaluations
    # the walks almost always reach it, random draws rarely do
    rows = cm.compare_searchers(wl, frac=0.45, seeds=50, start=4)
    assert rows[0]["annealing"] < 0.2 and rows[0]["mcmc"] < 0.2
    assert rows[0]["random"] > 0.5
