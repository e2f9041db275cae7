"""Configuration sweeps: the time of every valid configuration of the tuning
space on a grid of workloads (image side S, blob radius a, batch size n).

This is the training and evaluation data of the learned cost model (the
16-64-64-1 network of the tuner's learned search order).  Each workload is a
seeded synthetic batch (uniform rotations, N(0,1)/(1+|k|) pixels, the input
recipe of the insertion tests); each configuration is forced on a fresh
context with tuning off, run once untimed, then timed with CUDA events over
enough inserts to reach about 20 ms (at least two).

    python -m paper_1910_08498_gb300.sweep --out sweep.json \
        --S 64,96,128,192,256,384 --a 1.5,1.9,2.5 --n 500,2000,5000 --seed 4
"""
from __future__ import annotations

import argparse
import json
import math
import time

from . import _lib as L
from . import inputs


def time_config(ctx, cfg, img, rot, target_ms=20.0, max_reps=20):
    """ns per image of configuration cfg on one resident batch."""
    import torch
    L.fr_set_options(ctx, tuning=0, forced_config=cfg)
    L.fr_insert(ctx, img, rot, allow_fallback=False)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    L.fr_insert(ctx, img, rot, allow_fallback=False)
    e.record()
    torch.cuda.synchronize()
    first = s.elapsed_time(e)
    reps = max(2, min(max_reps, int(math.ceil(target_ms / max(first, 1e-3)))))
    s.record()
    for _ in range(reps):
        L.fr_insert(ctx, img, rot, allow_fallback=False)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / reps
    return 1e6 * ms / rot.shape[0]


def sweep(S_list, a_list, n_list, seed, alpha=15.0, log=print):
    import torch
    dev = torch.device("cuda", 0)
    L.lib()
    ncfg = L.fr_num_configs()
    rows = []
    for S in S_list:
        for a in a_list:
            a32 = float(torch.tensor(a, dtype=torch.float32))
            for n in n_list:
                img, rot = inputs.make_batch(S, n, seed * 100000 + S * 100 + int(round(10 * a)),
                                             device=dev)
                ctx = L.fr_create(S, a32, alpha, 0, 10000)
                t0 = time.time()
                try:
                    for cfg in range(ncfg):
                        if not L.fr_config_valid(ctx, cfg):
                            continue
                        try:
                            ns = time_config(ctx, cfg, img, rot)
                        except L.FrError as err:
                            log(f"S={S} a={a} n={n} config {cfg}: {err}")
                            continue
                        rows.append({"S": S, "a": a32, "n": n, "config": cfg, "ns_per_image": ns})
                finally:
                    L.fr_destroy(ctx)
                del img, rot
                log(f"S={S} a={a} n={n}: {time.time() - t0:.1f} s")
    props = torch.cuda.get_device_properties(dev)
    return {"device": props.name, "sms": props.multi_processor_count, "alpha": alpha, "seed": seed,
            "space": [L.fr_describe_config(i) for i in range(ncfg)], "rows": rows}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--out", required=True)
    p.add_argument("--S", default="64,96,128,192,256,384")
    p.add_argument("--a", default="1.5,1.9,2.5")
    p.add_argument("--n", default="500,2000,5000")
    p.add_argument("--seed", type=int, default=4)
    args = p.parse_args(argv)
    res = sweep([int(x) for x in args.S.split(",")], [float(x) for x in args.a.split(",")],
                [int(x) for x in args.n.split(",")], args.seed)
    with open(args.out, "w") as f:
        json.dump(res, f)
    print(f"{len(res['rows'])} measurements -> {args.out}")


if __name__ == "__main__":
    main()
