"""The learned cost model of the tuner: training on configuration sweeps and
the regret of the learned search order on held-out workloads.

Rows of a sweep (see sweep.py) give, per workload (S, a, n) and valid
configuration, the measured ns per image.  The model (the 16-64-64-1 ReLU
network whose forward, backward and Adam kernels live in the library) is
trained with fr_mlp_train on the 16 configuration/workload features of
fr_config_features against the log time relative to the workload's mean
log time (ranking within a workload is all the tuner needs).

Evaluation on a workload with N valid configurations and a budget of
k = max(1, floor(N / 10)) evaluations (the tuner's default learned budget):
  learned   measure the k configurations the model ranks fastest, keep the
            fastest measured;
  random    k configurations drawn uniformly without replacement (the
            expectation is computed exactly from the sorted times: the best
            of the draw is the i-th fastest with probability
            C(N-i, k-1) / C(N, k));
  annealing, mcmc
            the library's adaptive walks over neighbouring configurations,
            simulated on the measured table (fr_search_simulate), mean over
            20 seeds, started from the library's default configuration;
  regret = t(kept) / t(best of all N) - 1.

    python -m paper_1910_08498_gb300.costmodel --train sweep_train.json \
        --test sweep_heldout.json [--epochs 3000] [--save model.json]

The package ships GB300 sweeps (data/sweep_gb300_train.json: S in {64, 96,
128, 192, 256, 384} x a in {1.5, 1.9, 2.5} x n in {500, 2000, 5000};
data/sweep_gb300_heldout.json: S in {160, 320}) and the model trained on the
first (data/costmodel_gb300.json); load_pretrained() installs it in a context.
"""
from __future__ import annotations

import argparse
import json
import math
import os
from collections import defaultdict

import numpy as np

from . import _lib as L


DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
PRETRAINED = os.path.join(DATA, "costmodel_gb300.json")


def load_pretrained(ctx, path: str = PRETRAINED):
    """Install the shipped GB300 cost model in ctx (the learned search order
    then uses it)."""
    L.fr_mlp_set(ctx, np.array(json.load(open(path)), dtype=np.float32))


def workloads(rows):
    """{(S, a, n): {config: ns per image}}."""
    w = defaultdict(dict)
    for r in rows:
        w[(int(r["S"]), float(r["a"]), int(r["n"]))][int(r["config"])] = float(r["ns_per_image"])
    return dict(w)


def features(S, a, n, cfgs):
    return np.array([L.fr_config_features(c, S, n, a) for c in cfgs], dtype=np.float32)


def training_set(wl):
    X, y = [], []
    for (S, a, n), t in wl.items():
        cfgs = sorted(t)
        lt = np.log(np.array([t[c] for c in cfgs]))
        X.append(features(S, a, n, cfgs))
        y.append(lt - lt.mean())
    return np.concatenate(X), np.concatenate(y).astype(np.float32)


def train(ctx, wl, epochs=3000, lr=3e-3, seed=1):
    X, y = training_set(wl)
    return L.fr_mlp_train(ctx, X, y, epochs=epochs, lr=lr, seed=seed)


def predict(ctx, S, a, n, cfgs):
    import torch
    params = torch.tensor(L.fr_mlp_get(ctx), dtype=torch.float32, device="cuda")
    x = torch.from_numpy(features(S, a, n, cfgs)).cuda()
    out = torch.empty(len(cfgs), dtype=torch.float32, device="cuda")
    L.fr_mlp_forward(params, x, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def random_expected_regret(times, k):
    """Expected regret of the best of k distinct uniform draws among times."""
    t = np.sort(np.asarray(times, dtype=np.float64))
    N = len(t)
    tot = math.comb(N, k)
    return sum(math.comb(N - i, k - 1) / tot * (t[i - 1] / t[0] - 1.0) for i in range(1, N - k + 2))


def evaluate(ctx, wl, frac=0.10):
    out = []
    for (S, a, n), t in sorted(wl.items()):
        cfgs = sorted(t)
        k = max(1, int(frac * len(cfgs) + 1e-9))
        pred = predict(ctx, S, a, n, cfgs)
        top = [cfgs[i] for i in np.argsort(pred, kind="stable")[:k]]
        best = min(t.values())
        chosen = min(t[c] for c in top)
        out.append({"S": S, "a": a, "n": n, "configs": len(cfgs), "budget": k,
                    "learned_regret": chosen / best - 1.0,
                    "random_expected_regret": random_expected_regret(list(t.values()), k),
                    "best": L.fr_describe_config(min(t, key=t.get)),
                    "learned_pick": L.fr_describe_config(min(top, key=lambda c: t[c]))})
    return out


DEFAULT_CONFIGS = ("gather2 bx=16 by=8 zc=8 chunk=64 warps=24 w=poly",
                   "gather bx=16 by=16 zc=8 chunk=64 w=poly")


def default_start(t):
    """The library's default configuration among the measured ones of a
    workload: the direct-drain gather 16 x 8 x 8 where it runs (a < 2), else
    the per-voxel gather 16 x 16 x 8."""
    desc = {L.fr_describe_config(c): c for c in t}
    for d in DEFAULT_CONFIGS:
        if d in desc:
            return desc[d]
    return min(t)


def compare_searchers(wl, frac=0.10, seeds=20, start=None, learned=None):
    """Regret at equal budget k = max(1, floor(frac N)) of the random search
    (exact expectation), simulated annealing and the Metropolis walk (mean
    over `seeds` seeds, started from `start`, default: the library's default
    configuration) and, if given, the learned ranking ({workload: regret})."""
    ncfg = L.fr_num_configs()
    rows = []
    for key, t in sorted(wl.items()):
        table = [t.get(c, 0.0) for c in range(ncfg)]
        st = default_start(t) if start is None else start
        k = max(1, int(frac * len(t) + 1e-9))
        best = min(t.values())
        row = {"S": key[0], "a": key[1], "n": key[2], "budget": k, "configs": len(t),
               "random": random_expected_regret(list(t.values()), k)}
        for name, search in (("annealing", L.FR_SEARCH_ANNEALING), ("mcmc", L.FR_SEARCH_MCMC)):
            regs = []
            for sd in range(seeds):
                o = L.fr_search_simulate(search, table, k, seed=1000 + sd, start=st)
                regs.append(min(table[c] for c in o) / best - 1.0)
            row[name] = float(np.mean(regs))
        if learned is not None and key in learned:
            row["learned"] = learned[key]
        rows.append(row)
    return rows


def summary(res):
    lr = np.array([r["learned_regret"] for r in res])
    rr = np.array([r["random_expected_regret"] for r in res])
    return {"workloads": len(res), "mean_learned_regret": float(lr.mean()),
            "max_learned_regret": float(lr.max()), "mean_random_regret": float(rr.mean()),
            "share_within_5pct": float(np.mean(lr <= 0.05)),
            "evaluations_per_space": float(np.mean([r["budget"] / r["configs"] for r in res]))}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--train", required=True)
    p.add_argument("--test", required=True)
    p.add_argument("--epochs", type=int, default=3000)
    p.add_argument("--lr", type=float, default=3e-3)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--save", default=None, help="write the trained parameters (JSON list)")
    p.add_argument("--out", default=None, help="write the per-workload evaluation (JSON)")
    args = p.parse_args(argv)
    tr = workloads(json.load(open(args.train))["rows"])
    te = workloads(json.load(open(args.test))["rows"])
    ctx = L.fr_create(32)
    try:
        loss = train(ctx, tr, args.epochs, args.lr, args.seed)
        res_in, res_out = evaluate(ctx, tr), evaluate(ctx, te)
        rep = {"final_loss": loss, "train": summary(res_in), "heldout": summary(res_out),
               "heldout_rows": res_out}
        # the other searchers at the same budget (simulated on the measured tables)
        learned = {(r["S"], r["a"], r["n"]): r["learned_regret"] for r in res_out}
        cmp_rows = compare_searchers(te, learned=learned)
        rep["searchers_heldout"] = {
            name: {"mean_regret": float(np.mean([r[name] for r in cmp_rows])),
                   "max_regret": float(np.max([r[name] for r in cmp_rows])),
                   "within_5pct": float(np.mean([r[name] <= 0.05 for r in cmp_rows]))}
            for name in ("random", "annealing", "mcmc", "learned")}
        if args.save:
            json.dump([float(x) for x in L.fr_mlp_get(ctx)], open(args.save, "w"))
    finally:
        L.fr_destroy(ctx)
    print(json.dumps({k: v for k, v in rep.items() if k not in ("heldout_rows",)}, indent=1))
    if args.out:
        json.dump(rep, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
