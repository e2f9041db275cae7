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
        assert d["space"] == [L.fr_describe_config(i) for i in range(L.fr_num_configs())]
        wl = cm.workloads(d["rows"])
        assert all(len(t) >= 10 and min(t.values()) > 0 for t in wl.values())
