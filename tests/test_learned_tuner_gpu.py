"""The learned search order of the tuner (A7) on the GPU.

* On a synthetic cost table over the real configuration space (a known
  nonlinear function of the 16 features plus seeded noise), the cost model
  trained with the library's kernels on five image sizes picks, on two
  held-out sizes and with a tenth of the space as budget, configurations
  within 5 % of the best on average, and does better than random search with
  the same budget (whose expected regret is computed exactly).
* On the measured GB300 sweeps shipped with the package (the whole space
  timed on S in {64, 96, 128, 192, 256, 384} x a in {1.5, 1.9, 2.5} x n in
  {500, 2000, 5000} for training, S in {160, 320} held out): trained with
  fr_mlp_train, ranking with fr_mlp_forward, a tenth of the space as budget,
  mean regret <= 5 % on the held-out workloads and below random search's
  exact expected regret at the same budget.
* Online: a context with the shipped GB300 model and the learned search order
  evaluates at most a tenth of the space, settles on a configuration, and
  its volume still matches the FP64 oracle.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import costmodel as cm
from paper_1910_08498_gb300 import inputs
from tests.helpers import TOL_F32, oracle_insert, rel_err

pytestmark = pytest.mark.gpu


def synthetic_cost(cfg, S, n, a, rng):
    f = np.array(L.fr_config_features(cfg, S, n, a), dtype=np.float64)
    g = (1.5 * f[0] * (f[9] - 0.45) ** 2 + 0.8 * f[0] * f[8] - 0.6 * f[12] + 0.4 * f[5] * f[11]
         + 0.3 * (f[6] - 0.5) ** 2 + 0.5 * f[1] * f[9] - 0.4 * f[2] * (1 - f[9]) + 0.2 * f[13] * f[10]
         + 0.25 * f[7] * f[0] + 2.0 * math.log(S) + math.log(a))
    return math.exp(g + rng.normal(0, 0.01))


def synthetic_workloads(S_list, seed):
    rng = np.random.default_rng(seed)
    wl = {}
    ncfg = L.fr_num_configs()
    for S in S_list:
        for a in (1.5, 1.9, 2.5):
            for n in (500, 2000, 5000):
                wl[(S, a, n)] = {c: synthetic_cost(c, S, n, a, rng) for c in range(ncfg)}
    return wl


def test_learned_order_beats_random_on_synthetic_costs():
    train = synthetic_workloads([64, 96, 128, 192, 256, 384], 1)
    held = synthetic_workloads([160, 320], 2)
    ctx = L.fr_create(32)
    try:
        loss = cm.train(ctx, train, epochs=3000, lr=3e-3, seed=1)
        assert loss < 0.05
        res = cm.evaluate(ctx, held)
    finally:
        L.fr_destroy(ctx)
    s = cm.summary(res)
    assert s["evaluations_per_space"] <= 0.10
    assert s["mean_learned_regret"] <= 0.05, s
    assert s["mean_learned_regret"] < s["mean_random_regret"], s


def test_learned_order_on_measured_gb300_sweeps():
    def load(name):
        d = json.load(open(os.path.join(cm.DATA, name)))
        assert d["space"] == [L.fr_describe_config(i) for i in range(L.fr_num_configs())]
        return cm.workloads(d["rows"])
    train, held = load("sweep_gb300_train.json"), load("sweep_gb300_heldout.json")
    assert len(train) == 54 and len(held) == 18
    ctx = L.fr_create(32)
    try:
        loss = cm.train(ctx, train, epochs=3000, lr=3e-3, seed=1)
        res = cm.evaluate(ctx, held)
    finally:
        L.fr_destroy(ctx)
    s = cm.summary(res)
    assert math.isfinite(loss)
    assert s["evaluations_per_space"] <= 0.10
    assert s["mean_learned_regret"] <= 0.05, s
    assert s["mean_learned_regret"] < s["mean_random_regret"], s


def test_online_learned_tuning_with_shipped_model():
    S = 64
    # screening in 2-step inserts, then the kernel families' fastest on whole inserts
    batches = [inputs.make_batch(S, 300, 60 + b) for b in range(8)]
    Vr, Wr, _ = oracle_insert(S, batches)
    ctx = L.fr_create(S)
    try:
        cm.load_pretrained(ctx)
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_LEARNED, steps_per_insert=2, budget=0)
        import torch
        for img, rot in batches:
            L.fr_insert(ctx, img.cuda(), rot.cuda())
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        rep = L.fr_tuning_report(ctx)
        space = sum(L.fr_config_valid(ctx, i) for i in range(L.fr_num_configs()))
    finally:
        L.fr_destroy(ctx)
    assert rep["tuned"] == 1
    assert 1 <= rep["evaluated"] <= max(1, space // 10)
    V = V.cpu().numpy().astype(np.complex128)
    W = W.cpu().numpy().astype(np.float64)
    assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32
