"""Dynamic tuning behaviour on the GPU (Sec. 3.2, Sec. 5.3): a key change
(new batch-size bucket) starts a new tuning key and a return to an old key
reuses its result; fr_retune forgets it; the tuning cache saved to JSON is
restored by a new context, which then runs the cached best without
evaluating anything.  Volumes stay those of the oracle throughout."""
import numpy as np
import pytest
import torch

from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import TOL_F32, oracle_insert, rel_err

pytestmark = pytest.mark.gpu


def _finalize(ctx, S):
    D = S + 1
    V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
    W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
    L.fr_finalize(ctx, V, W)
    torch.cuda.synchronize()
    return V.cpu().numpy().astype(np.complex128), W.cpu().numpy().astype(np.float64)


def _tune_until_done(ctx, img, rot, cap=60):
    for _ in range(cap):
        L.fr_insert(ctx, img, rot)
        if L.fr_tuning_report(ctx)["tuned"]:
            return
    raise AssertionError("tuning did not finish")


def test_key_change_retunes_and_returns_reuse(tmp_path):
    S = 48
    big = [t.cuda() for t in inputs.make_batch(S, 200, 70)]    # bucket floor(log2 200) = 7
    small = [t.cuda() for t in inputs.make_batch(S, 20, 71)]   # bucket 4
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_RANDOM, budget=6, steps_per_insert=3)
        _tune_until_done(ctx, *big)
        r1 = L.fr_tuning_report(ctx)
        assert r1["evaluated"] == 6 and r1["n_bucket"] == 7
        _tune_until_done(ctx, *small)
        r2 = L.fr_tuning_report(ctx)
        assert r2["n_bucket"] == 4 and r2["evaluated"] == 6 and r2["retunes"] >= r1["retunes"]
        L.fr_insert(ctx, *big)          # back to the first key: cached, nothing new measured
        r3 = L.fr_tuning_report(ctx)
        assert r3["n_bucket"] == 7 and r3["tuned"] == 1 and r3["best_config"] == r1["best_config"]
        assert r3["evaluated"] == r1["evaluated"]
        L.fr_retune(ctx, 0)             # forget the current key: tuning starts over
        r4 = L.fr_tuning_report(ctx)
        assert r4["tuned"] == 0
        path = str(tmp_path / "cache.json")
        _tune_until_done(ctx, *big)
        L.fr_tuning_save(ctx, path)
        best = L.fr_tuning_report(ctx)["best_config"]
    finally:
        L.fr_destroy(ctx)

    # a new context restores the cache and runs the cached best at once
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_RANDOM, budget=6, steps_per_insert=3)
        L.fr_tuning_load(ctx, path)
        L.fr_insert(ctx, *big)
        r = L.fr_tuning_report(ctx)
        assert r["tuned"] == 1 and r["best_config"] == best and r["last_config"] == best
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    Vr, Wr, _ = oracle_insert(S, [(big[0].cpu(), big[1].cpu())])
    assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32


def test_tuning_with_every_search_keeps_results():
    S = 40
    batches = [inputs.make_batch(S, 90, 80 + b) for b in range(5)]
    Vr, Wr, _ = oracle_insert(S, batches)
    for search in (L.FR_SEARCH_EXHAUSTIVE, L.FR_SEARCH_RANDOM):
        ctx = L.fr_create(S)
        try:
            L.fr_set_options(ctx, tuning=1, search=search, budget=10, steps_per_insert=4)
            for img, rot in batches:
                L.fr_insert(ctx, img.cuda(), rot.cuda())
            V, W = _finalize(ctx, S)
            assert L.fr_tuning_report(ctx)["images"] == 450
        finally:
            L.fr_destroy(ctx)
        assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32


@pytest.mark.parametrize("search", [L.FR_SEARCH_ANNEALING, L.FR_SEARCH_MCMC])
def test_adaptive_walks_online(search):
    """The adaptive searchers propose from harvested timings, stop at their
    budget, settle on the fastest measured configuration and keep the
    volume the oracle's."""
    S = 40
    batches = [inputs.make_batch(S, 120, 110 + b) for b in range(8)]
    Vr, Wr, _ = oracle_insert(S, batches)
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=search, budget=7, steps_per_insert=2)
        for img, rot in batches:
            L.fr_insert(ctx, img.cuda(), rot.cuda())
        torch.cuda.synchronize()
        rep = L.fr_tuning_report(ctx)
        meas = L.fr_tuning_measurements(ctx)
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    assert rep["tuned"] == 1 and rep["evaluated"] == 7
    # the fastest measured configuration of its kernel family (the families'
    # fastest are then compared on whole inserts)
    fam = _family(rep["best_config"])
    assert rep["best_config"] == min((m for m in meas if _family(m[0]) == fam), key=lambda m: m[1])[0]
    assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32


def _family(cfg):
    return L.fr_describe_config(cfg).split(" ")[0]


def test_whole_insert_confirmation_of_family_bests():
    """Screening in sub-batch steps, then the fastest screened configuration
    of each kernel family runs one whole insert (in screened order), and the
    key's best is the fastest of those whole-insert timings; with one step per
    insert there is no confirmation.  Every image is inserted once."""
    S, n = 48, 160
    batches = [inputs.make_batch(S, n, 140 + b) for b in range(3)]
    Vr, Wr, _ = oracle_insert(S, batches)
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_EXHAUSTIVE, steps_per_insert=16)
        dev = [(i.cuda(), r.cuda()) for i, r in batches]
        lasts = []
        for k in range(40):
            L.fr_insert(ctx, *dev[k % 3])
            torch.cuda.synchronize()
            rep = L.fr_tuning_report(ctx)
            lasts.append(rep["last_config"])
            if rep["tuned"]:
                break
        assert rep["tuned"] == 1
        inserts = len(lasts)
        meas = L.fr_tuning_measurements(ctx)
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    assert len(meas) == rep["space_size"]
    fastest = {}
    for c, t, _ in meas:
        f = _family(c)
        if f not in fastest or t < fastest[f][1]:
            fastest[f] = (c, t)
    finalists = [c for c, _ in sorted(fastest.values(), key=lambda x: x[1])]
    assert len(finalists) == 3
    assert lasts[-len(finalists):] == finalists
    assert rep["best_config"] in finalists
    screen = -(-rep["space_size"] // 16)
    assert inserts == screen + len(finalists)
    # the volume holds every image of every insert exactly once
    reps = [inserts // 3 + (1 if b < inserts % 3 else 0) for b in range(3)]
    Vw = sum(k * v for k, v in zip(reps, [oracle_insert(S, [b])[0] for b in batches]))
    Ww = sum(k * w for k, w in zip(reps, [oracle_insert(S, [b])[1] for b in batches]))
    assert rel_err(V, Vw) <= TOL_F32 and rel_err(W, Ww) <= TOL_F32


def test_single_step_inserts_skip_confirmation():
    S, n = 32, 64
    img, rot = [t.cuda() for t in inputs.make_batch(S, n, 150)]
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_RANDOM, budget=5, steps_per_insert=1)
        for k in range(5):
            L.fr_insert(ctx, img, rot)
        torch.cuda.synchronize()
        rep = L.fr_tuning_report(ctx)
        meas = L.fr_tuning_measurements(ctx)
    finally:
        L.fr_destroy(ctx)
    assert rep["tuned"] == 1 and rep["evaluated"] == 5
    assert rep["best_config"] == min(meas, key=lambda m: m[1])[0]


def test_automatic_tuning_steps():
    """steps_per_insert = 0 (the default): an insert takes as many tuning steps
    as keep each at >= 2e7 estimated voxel updates, at most 32.  S = 128,
    n = 600: 600 x 128 x 65 x (4/3) pi a^3 / 2e7 = 7.2, so 7 configurations
    are measured by the first insert; every image is inserted once."""
    S, n = 128, 600
    img, rot = inputs.make_batch(S, n, 88)
    Vr, Wr, _ = oracle_insert(S, [(img, rot)])
    ctx = L.fr_create(S)
    try:
        assert L.fr_get_options(ctx).steps_per_insert == 0
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_EXHAUSTIVE)
        L.fr_insert(ctx, img.cuda(), rot.cuda())
        torch.cuda.synchronize()
        rep = L.fr_tuning_report(ctx)
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    assert rep["evaluated"] == 7
    assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32
