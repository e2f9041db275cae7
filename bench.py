#!/usr/bin/env python
"""Benchmark of the 3D Fourier insertion hot path on GB300.

Workload (stand-in for the large reconstruction of Sec. 5.3.2): S = 256
images (129 x 256 complex half planes), batches of 5000 images, a 257^3
volume, Kaiser-Bessel blob a = 1.9, alpha = 15, 10000-entry table.  A step is
one fr_insert of one resident batch (every step of the path runs in the
library's CUDA kernels).  The metric is voxel-updates/s: one update is one
(pixel, voxel) pair with |v - q| <= a inside the volume, counted exactly by
fr_count_updates.

Phases (one JSON line at the end):
  untuned  the library's default configuration, no tuning;
  tuning   cold-start non-blocking dynamic tuning (exhaustive search, four
           configurations per insert) until the space is exhausted; reports
           the tuning overhead of Eq. (performance) (Sec. 5.4);
  tuned    the configuration the tuner chose -- the headline `value`;
  e2e      the tuned path with host-resident (pinned) inputs copied in every
           step (the next batch on a copy stream while the current one is
           inserted), W at the volume centre read back every step, and the
           final volume downloaded once at the end of the timed region;
  recon    Algorithm 1's last step on the accumulated volume (fr_reconstruct)
           and its image-side step, the images' 2D transforms staged into
           the insertion input (fr_prepare_images);
  fp16     the tuned configuration on FP16-stored copies of the batches;
  stream   20 batches with a switch to S = 192 for batches 8-11 (Sec. 5.3.2
           style): tuning overhead against the oraculum, exhaustive and
           learned search, with and without the tuning cache;
  c2       the cold-start workload (S = 128, 10 batches of 1000 images):
           untuned, tuned, space-average rates and the online-tuning overhead
           of the exhaustive and learned orders;
  batched  the uneven-batch workload (40 batches of S in {64..256}, n in
           [500, 5000]), FP32 and FP16 images, every batch with the
           configuration tuned for its key: one graph replay of the
           multi-batch launches per pass against one fr_insert per batch;
  gemm     the second dynamic-tuning workload (Sec. 5.2): batched small GEMM
           with random size changes, tuned with the paper's stop rule.

--impl reference times the FP64 CPU oracle (the definition, written as a
plain scatter) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Fourier-insertion voxel-updates/s at S=256 (tuned vs untuned); tuning overhead %"
UNIT = "voxel-updates/s"
FLOPS_PER_UPDATE = 16  # algorithmic FP32 flops per update (3 sub, 5 for r^2, 3 table lerp, 5 accumulate)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dtype", default="f32", choices=["f32", "f16"])
    p.add_argument("--S", type=int, default=256)
    p.add_argument("--n", type=int, default=5000)
    p.add_argument("--batches", type=int, default=4, help="distinct resident batches, cycled")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target oracle work for cpu_baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the uneven-batch workload")
    p.add_argument("--no-stream", action="store_true", help="skip the 20-batch stream with an S switch")
    p.add_argument("--no-c2", action="store_true", help="skip the S = 128 cold-start workload")
    p.add_argument("--no-fp16", action="store_true", help="skip the FP16-image measurement")
    p.add_argument("--no-recon", action="store_true", help="skip the reconstruction (last step) timing")
    p.add_argument("--no-gemm", action="store_true", help="skip the batched-GEMM dynamic-tuning study")
    p.add_argument("--only-gemm", action="store_true", help="run only the batched-GEMM study")
    p.add_argument("--only-batched", action="store_true",
                   help="profiling mode: run only the uneven-batch workload and print its result")
    p.add_argument("--seed", type=int, default=5)
    p.add_argument("--profile-config", type=int, default=None,
                   help="profiling mode: time only this configuration id (no tuning, no baselines)")
    p.add_argument("--gemm-profile", default=None, metavar="M,N,K,CONFIG",
                   help="profiling mode: time one batched-GEMM configuration on one size "
                        "(batch of about 512 MB of matrices)")
    p.add_argument("--phases", action="store_true",
                   help="profiling mode: also report the gather kernel's per-phase cycle counters")
    return p.parse_args()


def workload_name(S, n, dtype):
    return f"3D Fourier insertion, S={S} ({S // 2 + 1}x{S} complex {dtype.upper()} half planes), " \
           f"batches of {n} images, {S + 1}^3 volume, blob a=1.9 alpha=15 table 10000"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return res
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                             parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return res
        mx = max(r[1] for r in rows)
        loaded = [r for r in rows if r[2] > 0.25 * max(x[2] for x in rows)] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        res.update(sm_mhz=statistics.median(r[0] for r in loaded), sm_max_mhz=mx, reasons=reasons,
                   samples=len(rows))
        return res


# ------------------------------------------------------------------ distributed helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU oracle timing

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample(S, img_cpu, rot_cpu, target_s, a):
    """Time the FP64 oracle on the first m images, m sized for ~target_s of
    work, on every host core; and on one core, on a sample sized for about a
    sixth of that time."""
    import oracle
    oracle.build()
    nt = oracle.max_threads()
    m0 = 4
    t0 = time.perf_counter()
    _, _, c0 = oracle.insert(S, img_cpu[:m0], rot_cpu[:m0], a=a, alpha=15.0, nthreads=nt)
    dt0 = time.perf_counter() - t0
    m = int(max(m0, min(img_cpu.shape[0], m0 * target_s / max(dt0, 1e-3))))
    t1 = time.perf_counter()
    _, _, c = oracle.insert(S, img_cpu[:m], rot_cpu[:m], a=a, alpha=15.0, nthreads=nt)
    dt = time.perf_counter() - t1
    # one thread: a sample of m1 images sized from the parallel rate
    m1 = int(max(1, min(m, m * target_s / 6.0 / max(dt * nt, 1e-3))))
    t2 = time.perf_counter()
    _, _, c1 = oracle.insert(S, img_cpu[:m1], rot_cpu[:m1], a=a, alpha=15.0, nthreads=1)
    dt1 = time.perf_counter() - t2
    return {"value": c / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "single_thread": {"value": c1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first {m1} images of batch 0 ({c1} updates, {dt1:.1f} s)"},
            "sample": f"first {m} images of batch 0 ({c} updates, {dt:.1f} s, FP64 scatter, OpenMP z-slab "
                      f"ownership, {nt} threads)"}


# ------------------------------------------------------------------ precision (error vs the FP64 oracle)

TOL_F32, TOL_F16 = 2e-5, 2e-3


def sample_voxels(S, seed, k):
    """k voxel coordinates of an (S+1)^3 volume: the centre and its
    neighbourhood (many planes meet there), the fold columns, and random."""
    import numpy as np
    H = S // 2
    rng = np.random.default_rng(seed)
    pts = [(0, 0, 0), (1, 0, 0), (-1, 0, 1), (2, -3, 1)]
    pts += [tuple(int(v) for v in rng.integers(-6, 7, 3)) for _ in range(max(0, k // 4))]
    pts += [(int(rng.integers(-1, 2)), int(rng.integers(-H, H + 1)), int(rng.integers(-H, H + 1)))
            for _ in range(max(0, k // 4))]
    while len(pts) < k:
        pts.append((int(rng.integers(-1, H + 1)), int(rng.integers(-H, H + 1)),
                    int(rng.integers(-H, H + 1))))
    return pts[:k]


def gpu_samples(L, ctx, S, pts, dev):
    """Finalize ctx and read V, W at pts with the grid maxima of |V| and W."""
    import numpy as np
    import torch
    D, H = S + 1, S // 2
    V = torch.empty(D ** 3, dtype=torch.complex64, device=dev)
    W = torch.empty(D ** 3, dtype=torch.float32, device=dev)
    L.fr_finalize(ctx, V, W)
    idx = torch.tensor([((z + H) * D + (y + H)) * D + (x + H) for x, y, z in pts], device=dev)
    out = {"pts": pts, "V": V[idx].cpu().numpy().astype(np.complex128),
           "W": W[idx].cpu().numpy().astype(np.float64),
           "scale_v": V.abs().max().item(), "scale_w": W.max().item()}
    del V, W
    return out


def sample_errors(g, Vo, Wo):
    """err_V, err_W of sampled GPU values against the oracle's, relative to
    the grid maxima of |V| and W."""
    import numpy as np
    return {"err_V": float(np.max(np.abs(g["V"] - Vo)) / g["scale_v"]),
            "err_W": float(np.max(np.abs(g["W"] - Wo)) / g["scale_w"]), "voxels": len(g["pts"])}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1910_08498_gb300 import inputs
    oracle.build()
    S, n = args.S, args.n
    a = float(np.float32(1.9))
    img, rot = inputs.make_batch(S, n, args.seed)
    img, rot = img.numpy(), rot.numpy()
    nt = oracle.max_threads()
    # size one step for ~8 s of oracle work
    t0 = time.perf_counter()
    _, _, c0 = oracle.insert(S, img[:2], rot[:2], a=a, nthreads=nt)
    per_img = (time.perf_counter() - t0) / 2
    m = int(max(1, min(n, 8.0 / max(per_img, 1e-4))))
    times, ups = [], []
    for step in range(args.warmup + args.steps):
        lo = (step * m) % max(1, n - m + 1)
        t = time.perf_counter()
        _, _, c = oracle.insert(S, img[lo:lo + m], rot[lo:lo + m], a=a, nthreads=nt)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
            ups.append(c)
    total_t = sum(times)
    value = sum(ups) / total_t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(S, n, args.dtype), "S": S, "n_per_step": m,
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                             "sample": f"{m} images per step (of a {n}-image batch), FP64 scatter"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch

    from paper_1910_08498_gb300 import _lib as L
    from paper_1910_08498_gb300 import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    L.lib()
    S, n, NB = args.S, args.n, args.batches
    a = float(np.float32(1.9))
    f16 = args.dtype == "f16"
    stream = torch.cuda.current_stream()

    # resident inputs (each batch 1.32 GB in FP32: larger than L2, cycled)
    batches = []
    for b in range(NB):
        gen = torch.Generator(device=dev)
        gen.manual_seed(args.seed * 1000 + 97 * rank + b)
        rot = inputs.random_rotations(n, gen, dev).contiguous()
        img = inputs.random_images(S, n, gen, dev)
        img = inputs.to_half(img) if f16 else img.contiguous()
        batches.append((img, rot))
    ctx = L.fr_create(S, a, 15.0, 0, 10000)
    updates = [L.fr_count_updates(ctx, rot) for _, rot in batches]
    img_bytes = batches[0][0].numel() * batches[0][0].element_size()
    rot_bytes = batches[0][1].numel() * 4

    def timed_steps(k, first=0):
        """k inserts, batches cycled; returns (seconds, updates, per-launch ms list)."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        ups = 0
        for i in range(k):
            img, rot = batches[(first + i) % NB]
            evs[i][0].record(stream)
            L.fr_insert(ctx, img, rot)
            evs[i][1].record(stream)
            ups += updates[(first + i) % NB]
        torch.cuda.synchronize()
        ms = [s.elapsed_time(e) for s, e in evs]
        return sum(ms) / 1e3, ups, ms

    # ---- untuned: default configuration
    L.fr_set_options(ctx, tuning=0, forced_config=-1)
    timed_steps(args.warmup)
    barrier(world)
    torch.cuda.synchronize()
    t_un, u_un, _ = timed_steps(args.steps)
    t_un = max_over_ranks(t_un, world, dev)
    untuned_cfg = L.fr_tuning_report(ctx)["last_config"]

    # ---- tuning: cold start, exhaustive, non-blocking
    L.fr_reset(ctx)
    L.fr_retune(ctx, True)
    L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_EXHAUSTIVE, steps_per_insert=0, forced_config=-1)
    tune_inserts = 0
    t_tune = 0.0
    u_tune = 0
    while True:
        dt, u, _ = timed_steps(1, tune_inserts)
        t_tune += dt
        u_tune += u
        tune_inserts += 1
        rep = L.fr_tuning_report(ctx)
        if rep["tuned"] or tune_inserts >= 200:
            break
    rep_tune = L.fr_tuning_report(ctx)
    meas = L.fr_tuning_measurements(ctx)
    best = rep_tune["best_config"]
    space_avg_ns = rep_tune["mean_ns_per_image"]

    # ---- tuning with the learned search order (the shipped GB300 cost model;
    # budget: a tenth of the space), same cold start
    from paper_1910_08498_gb300 import costmodel
    L.fr_reset(ctx)
    L.fr_retune(ctx, True)
    costmodel.load_pretrained(ctx)
    L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_LEARNED, steps_per_insert=0, forced_config=-1,
                     budget=0)
    ln_inserts, t_ln, u_ln = 0, 0.0, 0
    while True:
        dt, u, _ = timed_steps(1, ln_inserts)
        t_ln += dt
        u_ln += u
        ln_inserts += 1
        if L.fr_tuning_report(ctx)["tuned"] or ln_inserts >= 200:
            break
    rep_ln = L.fr_tuning_report(ctx)
    best_ln = rep_ln["best_config"]
    # the learned choice against the exhaustive one, both timed on whole
    # inserts of the resident batches (the tuners' own step timings are taken
    # at different step sizes)
    regret_ln = 0.0
    if best_ln != best and best_ln >= 0:
        tt = {}
        for c in (best, best_ln):
            L.fr_set_options(ctx, tuning=0, forced_config=c)
            timed_steps(1)
            tt[c], _, _ = timed_steps(max(2, NB))
        regret_ln = tt[best_ln] / tt[best] - 1.0

    # back to the exhaustive choice for the headline
    L.fr_reset(ctx)
    L.fr_set_options(ctx, tuning=0, forced_config=best)

    # ---- tuned (headline)
    timed_steps(args.warmup)
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t0 = time.perf_counter()
    t_tu, u_tu, ms_list = timed_steps(args.steps)
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    t_tu_max = max_over_ranks(t_tu, world, dev)
    u_all = sum_over_ranks(u_tu, world, dev)
    value = u_all / t_tu_max
    rep_tuned = L.fr_tuning_report(ctx)

    # ---- precision of the timed configuration: batch 0 alone into a fresh
    # context, sampled voxels (compared with the FP64 oracle in the
    # cpu_baseline leg, after the timed regions)
    prec_pts = sample_voxels(S, 11, 32)
    prec_gpu = {}
    ctxp = L.fr_create(S, a, 15.0, 0, 10000)
    L.fr_set_options(ctxp, tuning=0, forced_config=best)
    L.fr_insert(ctxp, *batches[0])
    prec_gpu["f32" if not f16 else "f16"] = gpu_samples(L, ctxp, S, prec_pts, dev)
    L.fr_destroy(ctxp)

    # ---- e2e: pinned host inputs copied in every step
    e2e = None
    if not args.no_e2e:
        hosts = []
        for b in range(min(2, NB)):
            hi = torch.empty_like(batches[b][0], device="cpu").pin_memory()
            hi.copy_(batches[b][0])
            hr = torch.empty_like(batches[b][1], device="cpu").pin_memory()
            hr.copy_(batches[b][1])
            hosts.append((hi, hr))
        # two device buffers: the next batch is copied on a copy stream while
        # the current one is inserted (the overlap Algorithm 1's loop uses)
        d_img = [torch.empty_like(batches[0][0]) for _ in range(2)]
        d_rot = [torch.empty_like(batches[0][1]) for _ in range(2)]
        cstream = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device=dev)
        W = torch.empty(D ** 3, dtype=torch.float32, device=dev)
        centre = ((S // 2) * D + S // 2) * D + S // 2
        w_h = torch.zeros(max(args.steps, args.warmup), dtype=torch.float32).pin_memory()
        Vh = torch.empty(D ** 3, dtype=torch.complex64).pin_memory()
        Wh = torch.empty(D ** 3, dtype=torch.float32).pin_memory()

        def e2e_steps(k, start_event=None):
            """k steps: H2D of batch i+1 overlapped with the insertion of batch i."""
            for ev in used:
                ev.record(stream)
            if start_event is not None:
                cstream.wait_event(start_event)
            ups_k = 0

            def h2d(i):
                hi, hr = hosts[i % len(hosts)]
                cstream.wait_event(used[i % 2])
                with torch.cuda.stream(cstream):
                    d_img[i % 2].copy_(hi, non_blocking=True)
                    d_rot[i % 2].copy_(hr, non_blocking=True)
                copied[i % 2].record(cstream)

            h2d(0)
            for i in range(k):
                if i + 1 < k:
                    h2d(i + 1)
                stream.wait_event(copied[i % 2])
                L.fr_insert(ctx, d_img[i % 2], d_rot[i % 2])
                used[i % 2].record(stream)
                L.fr_finalize(ctx, V, W)
                w_h[i:i + 1].copy_(W[centre:centre + 1], non_blocking=True)
                ups_k += updates[i % len(hosts)]
            return ups_k

        L.fr_reset(ctx)
        e2e_steps(args.warmup)
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ups = e2e_steps(args.steps, start_event=e0)
        Vh.copy_(V, non_blocking=True)
        Wh.copy_(W, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
        e2e = {"value": sum_over_ranks(ups, world, dev) / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": img_bytes + rot_bytes, "d2h_bytes_per_step": 4,
               "d2h_bytes_end": Vh.numel() * 8 + Wh.numel() * 4,
               "note": "per step: pinned H2D of the next batch and its rotations on a copy stream, "
                       "overlapped with fr_insert of the current one, then fr_finalize and a D2H of W "
                       "at the volume centre; at the end: D2H of the full V and W; the timed region "
                       "starts before the first copy and ends after the last download"}

    # ---- roofline of the dominant kernel (the tuned insertion launch)
    per_launch_s = t_tu / args.steps
    ups_per_launch = u_tu / args.steps
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    achieved = FLOPS_PER_UPDATE * ups_per_launch / per_launch_s / 1e12
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            if tj.get("config") == L.fr_describe_config(best) and tj.get("S") == S and \
                    tj.get("source_hash") == source_hash():
                traffic = tj["bytes_per_launch"]
        except Exception:
            traffic = None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": traffic,
            "kernel": L.fr_describe_config(best), "flops_per_update": FLOPS_PER_UPDATE,
            "peak_note": f"FP32 FMA peak: {sms} SMs x 128 lanes x 2 flops x {max_mhz:.0f} MHz (max SM clock)",
            "avg_launch_ms": 1e3 * per_launch_s, "updates_per_launch": ups_per_launch}
    # measured check of the denominator: FMA-chain kernels that fill every SM
    # (run after the timed region; fastest of 5 launches each)
    tf1, _ = L.fr_probe_fp32_peak(False, 5)
    tf2, _ = L.fr_probe_fp32_peak(True, 5)
    roof["probe_tflops"] = {"fma_f32": tf1, "fma_f32x2": tf2,
                            "note": "fr_probe_fp32_peak: 8 independent FMA chains per thread, "
                                    "4 x 512 threads per SM, scalar and packed two-lane FMAs"}

    # ---- Algorithm 1's last step on the accumulated volume: symmetrise,
    # weight, inverse FFT (fr_reconstruct)
    recon = None
    if not args.no_recon:
        out = torch.empty(S ** 3, dtype=torch.float32, device=dev)
        L.fr_reconstruct(ctx, out, 1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, args.steps)
        e0.record(stream)
        for _ in range(k):
            L.fr_reconstruct(ctx, out, 1.0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        nspec = S * S * (S // 2 + 1)
        recon = {"ms_per_call": ms, "S": S, "spectrum_entries": nspec,
                 "weighting_bytes": nspec * (24 + 8),
                 "note": "weighting kernel (reads the double-float sums, writes the half spectrum) "
                         "+ cuFFT C2R of S^3"}
        del out

    # ---- the image-side step: 2D transforms of n real images staged into the
    # insertion input (fr_prepare_images), FP32 and FP16 output
    prep = None
    if not args.no_recon:
        gen = torch.Generator(device=dev)
        gen.manual_seed(args.seed * 1000 + 900 + rank)
        real = torch.randn(n, S, S, generator=gen, device=dev, dtype=torch.float32)
        prep = {"images": n, "S": S}
        for name, buf in (("f32", torch.empty(n, S, S // 2 + 1, dtype=torch.complex64, device=dev)),
                          ("f16", torch.empty(n, S, S // 2 + 1, 2, dtype=torch.float16, device=dev))):
            L.fr_prepare_images(ctx, real, buf, center=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                L.fr_prepare_images(ctx, real, buf, center=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            byts = real.numel() * 4 + buf.numel() * buf.element_size()
            prep[name] = {"ms_per_batch": ms, "images_per_s": n / (ms * 1e-3),
                          "hbm_gbs_min_traffic": byts / (ms * 1e-3) / 1e9}
            del buf
        del real

    # ---- FP16-stored images, the tuned configuration
    fp16 = None
    if not f16 and not args.no_fp16:
        h16 = [(inputs.to_half(img), rot) for img, rot in batches[:2]]
        ctx16 = L.fr_create(S, a, 15.0, 0, 10000)
        L.fr_set_options(ctx16, tuning=0, forced_config=best)
        for i in range(args.warmup):
            L.fr_insert(ctx16, *h16[i % 2])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            L.fr_insert(ctx16, *h16[i % 2])
        e1.record(stream)
        torch.cuda.synchronize()
        t16 = e0.elapsed_time(e1) / 1e3
        fp16 = {"value": sum(updates[i % 2] for i in range(args.steps)) / t16, "unit": UNIT,
                "config": L.fr_describe_config(best), "ms_per_step": 1e3 * t16 / args.steps}
        L.fr_reset(ctx16)
        L.fr_insert(ctx16, *h16[0])
        prec_gpu["f16"] = gpu_samples(L, ctx16, S, prec_pts, dev)
        L.fr_destroy(ctx16)
        del h16

    stream_exp = None
    if not args.no_stream:
        stream_exp = run_stream(L, inputs, costmodel, dev, stream, batches, updates, n, f16,
                                args.seed * 1000 + 500 + rank)
    c2 = None
    if not args.no_c2:
        c2 = run_c2(L, inputs, costmodel, dev, stream, f16, args.seed * 1000 + 700 + rank)

    gemm_dyn = None
    if not args.no_gemm:
        gemm_dyn = run_gemm_dynamic(L, dev, stream)

    batched = None
    c3_samples = None
    if not args.no_batched:
        batched, c3_samples = {}, {}
        for dt in ("f32", "f16"):
            batched[dt], c3_samples[dt] = run_batched(L, inputs, dev, stream, max(2, args.steps // 3),
                                                      1, dt == "f16")

    cpu = None
    precision = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        img0, rot0 = batches[0]
        m = min(n, 2000)
        imgc = (inputs.half_values(img0[:m]) if f16 else img0[:m]).cpu().numpy()
        cpu = oracle_sample(S, imgc, rot0[:m].cpu().numpy(), args.cpu_seconds, a)
        precision = run_precision(prec_gpu, batches[0], S, a, f16, c3_samples, dev, inputs)

    rep = rep_tune
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_tu_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": workload_name(S, n, args.dtype), "S": S, "n_per_step": n,
                   "resident_batches": NB, "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 ({img_bytes / 1e9:.2f} GB per batch, {NB} batches cycled)"},
        "untuned": {"value": sum_over_ranks(u_un, world, dev) / t_un, "config": L.fr_describe_config(untuned_cfg)},
        "tuning": {"inserts": tune_inserts, "evaluated": rep["evaluated"], "space": rep["space_size"],
                   "best": L.fr_describe_config(best), "best_ns_per_image": rep["best_ns_per_image"],
                   "space_avg_ns_per_image": space_avg_ns,
                   "space_avg_value": (ups_per_launch / n) / (space_avg_ns * 1e-9) if space_avg_ns else None,
                   "overhead_pct": rep["tuning_overhead_pct"],
                   "tuning_phase_value": u_tune / t_tune,
                   "per_config_ns_per_image": {L.fr_describe_config(c): round(ns, 1)
                                               for c, ns, _ in sorted(meas, key=lambda x: x[1])}},
        "tuning_learned": {
            "inserts": ln_inserts, "evaluated": rep_ln["evaluated"], "space": rep_ln["space_size"],
            "best": L.fr_describe_config(best_ln), "overhead_pct": rep_ln["tuning_overhead_pct"],
            "tuning_phase_value": u_ln / t_ln,
            "regret_vs_exhaustive": regret_ln,
            "model": "data/costmodel_gb300.json (trained on data/sweep_gb300_train.json)"},
        "stream_overhead_pct": {
            # the paper's overhead over a whole stream of 20 batches (Sec. 5.3.2):
            # tuning inserts as measured, the rest at the tuned rate
            "exhaustive": 100.0 * ((t_tune + max(0, 20 - tune_inserts) * t_tu / args.steps)
                                   / (20 * t_tu / args.steps) - 1.0) if tune_inserts <= 20 else None,
            "learned": 100.0 * ((t_ln + max(0, 20 - ln_inserts) * t_tu / args.steps)
                                / (20 * t_tu / args.steps) - 1.0) if ln_inserts <= 20 else None},
        "roofline": roof,
        "cpu_baseline": cpu,
        "precision": precision,
        "e2e": e2e,
        "fp16": fp16,
        "reconstruct": recon,
        "prepare_images": prep,
        "stream": stream_exp,
        "c2": c2,
        "batched": batched,
        "gemm_dynamic": gemm_dyn,
        "gpu_launches": args.steps * launches_per_insert(L, ctx, best, n),
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "wall_s_timed": wall,
    }
    L.fr_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def tune_batches(L, spec, data, contexts):
    """Online tuning of the uneven-batch workload's keys: per S, one tuning
    context inserts that S's batches with tuning on (exhaustive search) until
    the key (S, n bucket, dtype) of every one of them is tuned; its cache is
    saved and loaded into every context of that S, which then runs the tuned
    best with tuning off.  Returns the chosen configuration per key, the
    tuning inserts and their wall time."""
    import torch
    chosen, inserts = {}, 0
    t0 = time.perf_counter()
    with tempfile.TemporaryDirectory() as tmp:
        for S in sorted({S for S, _, _ in spec}):
            idx = [b for b, (Sb, _, _) in enumerate(spec) if Sb == S]
            t = L.fr_create(S, 1.9, 15.0, 0, 10000)
            L.fr_set_options(t, tuning=1)
            pending = list(idx)
            for _ in range(200):
                if not pending:
                    break
                left = []
                for b in pending:
                    L.fr_insert(t, *data[b])
                    inserts += 1
                    rep = L.fr_tuning_report(t)
                    if rep["tuned"]:
                        chosen[f"S={S} n_bucket={rep['n_bucket']}"] = L.fr_describe_config(rep["best_config"])
                    else:
                        left.append(b)
                pending = left
            torch.cuda.synchronize()
            path = os.path.join(tmp, f"tune_{S}.json")
            L.fr_tuning_save(t, path)
            L.fr_destroy(t)
            for b in idx:
                for lst in contexts:
                    L.fr_tuning_load(lst[b], path)
    return {"configs": chosen, "tuning_inserts": inserts,
            "tuning_wall_s": time.perf_counter() - t0, "search": "exhaustive"}


def run_batched(L, inputs, dev, stream, steps, warmup, f16):
    """The uneven-batch workload (40 batches, S uniform over {64, 96, 128, 192,
    256}, n uniform over [500, 5000], one volume per batch), every batch with
    the configuration the tuner picked for its key (tune_batches, untimed): all
    batches in multi-batch launches replayed from a CUDA graph, against one
    fr_insert per batch with the same configurations."""
    import torch
    spec = inputs.uneven_batches()
    data, ctx_p, ctx_s = [], [], []
    ups = 0
    for S, n, seed in spec:
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        rot = inputs.random_rotations(n, gen, dev).contiguous()
        img = inputs.random_images(S, n, gen, dev)
        img = inputs.to_half(img) if f16 else img.contiguous()
        data.append((img, rot))
        for lst in (ctx_p, ctx_s):
            c = L.fr_create(S, 1.9, 15.0, 0, 10000)
            L.fr_set_options(c, tuning=0, forced_config=-1)
            lst.append(c)
        ups += L.fr_count_updates(ctx_p[-1], rot)
    tuning = tune_batches(L, spec, data, (ctx_p, ctx_s))
    imgs = [d[0] for d in data]
    rots = [d[1] for d in data]

    def persistent(k):
        for _ in range(k):
            L.fr_insert_batched(ctx_p, imgs, rots, capture=1)

    def sequential(k):
        for _ in range(k):
            for c, (img, rot) in zip(ctx_s, data):
                L.fr_insert(c, img, rot)

    out = {}
    for name, fn in (("persistent_graph", persistent), ("per_batch_inserts", sequential)):
        fn(max(1, warmup))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        out[name] = {"value": ups / t, "ms_per_pass": 1e3 * t}
    out["speedup"] = out["persistent_graph"]["value"] / out["per_batch_inserts"]["value"]
    # one persistent pass into cleared volumes, sampled per batch (compared
    # with the FP64 oracle in the cpu_baseline leg)
    for c in ctx_p:
        L.fr_reset(c)
    persistent(1)
    samples = []
    for b, ((S, n, seed), c) in enumerate(zip(spec, ctx_p)):
        samples.append(((S, n, seed), gpu_samples(L, c, S, sample_voxels(S, 100 + b, 6), dev)))
    for c in ctx_p + ctx_s:
        L.fr_destroy(c)
    sizes = sorted({S for S, _, _ in spec})
    return ({"workload": f"{len(spec)} batches, S in {sizes}, n in [500, 5000] (seeded), one volume each, "
                         f"{'FP16' if f16 else 'FP32'} images",
             "updates_per_pass": ups, "images_per_pass": sum(n for _, n, _ in spec),
             "tuning": tuning, **out},
            {"f16": f16, "batches": samples})


def run_precision(prec_gpu, batch0, S, a, f16_run, c3, dev, inputs):
    """The error of the timed configurations against the FP64 oracle, on
    sampled voxels the oracle computes one by one: the S = 256 batch (FP32
    images; FP16 images against the oracle fed the FP32 values and the
    FP16-rounded values) and every batch of the uneven-batch workload."""
    import torch
    import oracle
    oracle.build()
    img0, rot0 = batch0
    rot = rot0.cpu().numpy()
    pts = next(iter(prec_gpu.values()))["pts"]
    vals = (inputs.half_values(img0) if f16_run else img0).cpu().numpy()
    Vo, Wo = oracle.voxels(S, vals, rot, pts, a=a, alpha=15.0)
    out = {"bounds": {"f32": TOL_F32, "f16": TOL_F16},
           "note": "err = max over sampled voxels of |GPU - FP64 oracle| / max over the grid "
                   "(|V| or W); centre, fold columns and random voxels"}
    if "f32" in prec_gpu:
        out["f32"] = sample_errors(prec_gpu["f32"], Vo, Wo)
    if "f16" in prec_gpu:
        if f16_run:
            out["f16"] = {"vs_f16_values": sample_errors(prec_gpu["f16"], Vo, Wo)}
        else:
            Vh, Wh = oracle.voxels(S, inputs.half_values(inputs.to_half(img0)).cpu().numpy(), rot,
                                   pts, a=a, alpha=15.0)
            out["f16"] = {"vs_f32_values": sample_errors(prec_gpu["f16"], Vo, Wo),
                          "vs_f16_values": sample_errors(prec_gpu["f16"], Vh, Wh)}
    for key, c3s in (c3 or {}).items():
        per = []
        for (Sb, n, seed), g in c3s["batches"]:
            gen = torch.Generator(device=dev)
            gen.manual_seed(seed)
            rb = inputs.random_rotations(n, gen, dev)
            ib = inputs.random_images(Sb, n, gen, dev)
            if c3s["f16"]:
                ib = inputs.half_values(inputs.to_half(ib))
            Vb, Wb = oracle.voxels(Sb, ib.cpu().numpy(), rb.cpu().numpy(), g["pts"], a=a, alpha=15.0)
            e = sample_errors(g, Vb, Wb)
            per.append({"S": Sb, "n": n, "err_V": e["err_V"], "err_W": e["err_W"]})
            del ib, rb
        out.setdefault("c3", {})[key] = {
            "images": "FP16 (vs the FP16-rounded values)" if c3s["f16"] else "FP32",
            "batches": len(per), "max_err_V": max(p["err_V"] for p in per),
            "max_err_W": max(p["err_W"] for p in per), "per_batch": per}
        out.setdefault("c3_max", {})[key] = {"err_V": max(p["err_V"] for p in per),
                                             "err_W": max(p["err_W"] for p in per)}
    return out


def run_stream(L, inputs, costmodel, dev, stream, batches256, updates256, n, f16, seed):
    """The paper's stream experiment (Sec. 5.3.2) on synthetic inputs: 20
    batches of n images, S = 256 except batches 8-11 at S = 192.  Each S has
    its own context (its own volume).  T_dyn: cold-start tuning during the
    stream (exhaustive or learned search), with the tuning cache (the S = 256
    context keeps its result over the switch) or without it (its key is
    forgotten when S changes back).  T_oraculum: every batch with the best
    configuration measured for its S from the start.  Overhead =
    T_dyn / T_oraculum - 1."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    b192 = []
    for _ in range(2):
        rot = inputs.random_rotations(n, gen, dev).contiguous()
        img = inputs.random_images(192, n, gen, dev)
        b192.append((inputs.to_half(img) if f16 else img.contiguous(), rot))
    plan = [(256, i % len(batches256)) for i in range(8)] + [(192, i % 2) for i in range(4)] + \
           [(256, (8 + i) % len(batches256)) for i in range(8)]

    def run(ctxs, forget_on_return):
        ev = []
        prev = None
        for S, b in plan:
            c = ctxs[S]
            if forget_on_return and prev == 192 and S == 256:
                L.fr_retune(c, 1)
            img, rot = (batches256 if S == 256 else b192)[b]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.fr_insert(c, img, rot)
            e1.record(stream)
            ev.append((e0, e1))
            prev = S
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    def contexts(search):
        cs = {}
        for S in (256, 192):
            c = L.fr_create(S, 1.9, 15.0, 0, 10000)
            if search == L.FR_SEARCH_LEARNED:
                costmodel.load_pretrained(c)
            L.fr_set_options(c, tuning=1, search=search, steps_per_insert=0, budget=0, forced_config=-1)
            cs[S] = c
        return cs

    out = {}
    best = {}
    for name, search in (("exhaustive", L.FR_SEARCH_EXHAUSTIVE), ("learned", L.FR_SEARCH_LEARNED)):
        for cache in (True, False):
            cs = contexts(search)
            t = run(cs, forget_on_return=not cache)
            for c in cs.values():
                L.fr_destroy(c)
            out[f"{name}_{'cache' if cache else 'no_cache'}_s"] = t
    # oraculum: the exhaustive best of each S (tuned to the end outside the
    # stream) from the first batch
    cs = contexts(L.FR_SEARCH_EXHAUSTIVE)
    for S, c in cs.items():
        img, rot = (batches256 if S == 256 else b192)[0]
        for _ in range(100):
            L.fr_insert(c, img, rot)
            if L.fr_tuning_report(c)["tuned"]:
                break
        best[S] = L.fr_tuning_report(c)["best_config"]
        L.fr_set_options(c, tuning=0, forced_config=best[S])
    run(cs, False)  # warm
    for c in cs.values():
        L.fr_reset(c)
    t_or = run(cs, False)
    for c in cs.values():
        L.fr_destroy(c)
    res = {"batches": len(plan), "images": len(plan) * n, "oraculum_s": t_or,
           "oraculum_configs": {S: L.fr_describe_config(b) for S, b in best.items()}}
    for k, v in out.items():
        res[k] = v
        res[k.replace("_s", "_overhead_pct")] = 100.0 * (v / t_or - 1.0)
    return res


def run_c2(L, inputs, costmodel, dev, stream, f16, seed, S=128, batches=10, n=1000):
    """The cold-start workload of Sec. 5.3.2 (Table 10's setting): S = 128, 10
    batches of 1000 images into one volume, online tuning over the whole
    configuration space from a fresh context.  Reported in voxel updates/s
    over the 10 batches: untuned (the default configuration), tuned (the
    configuration the exhaustive search settles on, from the first batch),
    space average (each valid configuration timed on a whole batch; the mean
    time per image), and the stream with online tuning for the exhaustive and
    the learned search orders: its rate, its overhead against the tuned
    stream, and the tuner's own Eq. (performance) figure (all tuning-step
    time against the best configuration's rate)."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    data = []
    for _ in range(batches):
        rot = inputs.random_rotations(n, gen, dev).contiguous()
        img = inputs.random_images(S, n, gen, dev)
        data.append((inputs.to_half(img) if f16 else img.contiguous(), rot))
    probe = L.fr_create(S, 1.9, 15.0, 0, 10000)
    ups = sum(L.fr_count_updates(probe, r) for _, r in data)

    def stream_s(c):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for img, rot in data:
            L.fr_insert(c, img, rot)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def fresh(**opt):
        c = L.fr_create(S, 1.9, 15.0, 0, 10000)
        L.fr_set_options(c, **opt)
        return c

    out = {"workload": f"S={S}, {batches} batches x {n} images, one volume, a=1.9, "
                       f"{'FP16' if f16 else 'FP32'} images, cold-start tuning",
           "updates": ups}
    # untuned: the default configuration
    c = fresh(tuning=0, forced_config=-1)
    stream_s(c)
    L.fr_reset(c)
    t = stream_s(c)
    out["untuned"] = {"updates_per_s": ups / t, "config": L.fr_describe_config(
        L.fr_tuning_report(c)["last_config"])}
    L.fr_destroy(c)
    # the two online searches, cold start
    chosen = {}
    for name, search in (("exhaustive", L.FR_SEARCH_EXHAUSTIVE), ("learned", L.FR_SEARCH_LEARNED)):
        c = fresh(tuning=1, search=search, steps_per_insert=0, budget=0, forced_config=-1)
        if search == L.FR_SEARCH_LEARNED:
            costmodel.load_pretrained(c)
        t = stream_s(c)
        rep = L.fr_tuning_report(c)
        extra = 0
        while not rep["tuned"] and extra < 100:  # finish the search outside the stream
            L.fr_insert(c, *data[extra % batches])
            torch.cuda.synchronize()
            rep = L.fr_tuning_report(c)
            extra += 1
        chosen[name] = rep["best_config"]
        out[name] = {"updates_per_s": ups / t, "stream_s": t, "evaluated": rep["evaluated"],
                     "space": rep["space_size"], "tuned_within_stream": extra == 0,
                     "config": L.fr_describe_config(rep["best_config"]),
                     "tuner_eq_performance_overhead_pct": rep["tuning_overhead_pct"]}
        L.fr_destroy(c)
    # tuned: the exhaustive choice from the first batch
    c = fresh(tuning=0, forced_config=chosen["exhaustive"])
    stream_s(c)
    L.fr_reset(c)
    t_tuned = stream_s(c)
    out["tuned"] = {"updates_per_s": ups / t_tuned, "config": L.fr_describe_config(chosen["exhaustive"])}
    for name in ("exhaustive", "learned"):
        out[name]["overhead_vs_tuned_pct"] = 100.0 * (out[name]["stream_s"] / t_tuned - 1.0)
    # space average: every valid configuration on one whole batch
    img, rot = data[0]
    per = []
    for cfg in range(L.fr_num_configs()):
        if not L.fr_config_valid(c, cfg):
            continue
        L.fr_set_options(c, tuning=0, forced_config=cfg)
        L.fr_insert(c, img, rot)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.fr_insert(c, img, rot)
        e1.record(stream)
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1) / 1e3 / n)
    L.fr_destroy(c)
    L.fr_destroy(probe)
    t_avg = sum(per) / len(per)
    out["space_average"] = {"updates_per_s": ups / (t_avg * n * batches), "configs": len(per),
                            "best_over_average": t_avg / min(per)}
    return out


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_gemm_dynamic(L, dev, stream, sizes=10, calls=100, seed=7, target_bytes=512e6):
    """The dynamic-tuning study of Sec. 5.2 on the batched small GEMM: sizes
    (m, n, k) drawn uniformly from [2, 32]^3 change every `calls` calls; the
    tuner (random search, at most 20 configurations, stop at 75 % of the
    measured HBM bandwidth) runs inside the calls.  Per size: Maximum = best
    configuration measured offline (every valid one), Restricted = the
    tuner's choice relative to it, Incl. overhead = all calls of the size
    (tuning included) relative to it (the columns of the paper's Table 7)."""
    import torch
    peak, src = measured_hbm_gbs()
    g = torch.Generator().manual_seed(seed)
    ctx = L.fr_gemm_create()
    L.fr_gemm_set_tuning(ctx, tuning=1, search=L.FR_SEARCH_RANDOM, budget=20, steps=2,
                         bw_gbs=peak, bw_frac=0.75, seed=seed)
    rows = []
    try:
        for _ in range(sizes):
            m, n, k = (int(x) for x in torch.randint(2, 33, (3,), generator=g))
            per = 4.0 * (m * k + k * n + m * n)
            batch = int(min(1 << 26, max(1, target_bytes // per)))
            A = torch.randn(batch, m, k, device=dev)
            B = torch.randn(batch, k, n, device=dev)
            C = torch.empty(batch, m, n, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = 0.0
            for cfg in range(L.fr_gemm_num_configs()):
                if not L.fr_gemm_config_valid(cfg, m, n, k):
                    continue
                L.fr_gemm_run_config(cfg, A, B, C)
                e0.record(stream)
                for _ in range(3):
                    L.fr_gemm_run_config(cfg, A, B, C)
                e1.record(stream)
                torch.cuda.synchronize()
                best = max(best, 3 * batch * per / (e0.elapsed_time(e1) * 1e-3) / 1e9)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(calls):
                L.fr_gemm_run(ctx, A, B, C)
            e1.record(stream)
            torch.cuda.synchronize()
            dyn = calls * batch * per / (e0.elapsed_time(e1) * 1e-3) / 1e9
            rep = L.fr_gemm_report(ctx, m, n, k)
            rows.append({"m": m, "n": n, "k": k, "batch": batch, "maximum_gbs": best,
                         "restricted_pct": 100.0 * rep["best_gbs"] / best if best else None,
                         "incl_overhead_pct": 100.0 * dyn / best if best else None,
                         "evaluated": rep["evaluated"], "tuned": rep["tuned"],
                         "config": L.fr_gemm_describe_config(rep["best"]) if rep["best"] >= 0 else None})
            del A, B, C
    finally:
        L.fr_gemm_destroy(ctx)
    import statistics as st
    return {"sizes": rows, "calls_per_size": calls,
            "maximum_gbs_avg": st.mean(r["maximum_gbs"] for r in rows),
            "maximum_pct_of_hbm": 100.0 * st.mean(r["maximum_gbs"] for r in rows) / peak,
            "restricted_pct_avg": st.mean(r["restricted_pct"] for r in rows),
            "incl_overhead_pct_avg": st.mean(r["incl_overhead_pct"] for r in rows),
            "hbm_gbs": peak, "hbm_source": src}


def launches_per_insert(L, ctx, cfg, n):
    """Kernel launches of one insert of n images with configuration cfg (one
    step: tuning is off in the timed region)."""
    return L.fr_insert_launches(ctx, cfg, n)


GATHER_SOURCES = ("fr_device.cuh", "fr_gather.cuh", "fr_gather_common.cu", "fr_gather_launch.inc",
                  "fr_gather_shapes.h", "fr_internal.h", "fr_gather2.cuh", "fr_gather2.cu",
                  "fr_gather2_launch.inc", "fr_gather_fold.cu", "fr_ctx.h")


def source_hash():
    """Hash of the sources that define the gather kernels: a stored DRAM
    traffic figure is reported only while they are unchanged."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_08498_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f in GATHER_SOURCES or ((f.startswith("fr_gather_s") or f.startswith("fr_gather2_s"))
                                   and f.endswith(".cu")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def run_profile(args):
    """Small-case mode for ncu: warm-up then `steps` launches of one configuration."""
    import numpy as np
    import torch

    from paper_1910_08498_gb300 import _lib as L
    from paper_1910_08498_gb300 import inputs
    dev = torch.device("cuda", 0)
    img, rot = inputs.make_batch(args.S, args.n, args.seed, device=dev)
    if args.dtype == "f16":
        img = inputs.to_half(img)
    ctx = L.fr_create(args.S, float(np.float32(1.9)), 15.0, 0, 10000)
    L.fr_set_options(ctx, tuning=0, forced_config=args.profile_config)
    ups = L.fr_count_updates(ctx, rot)
    phases = None
    if args.phases:
        L.fr_set_options(ctx, debug=2)
        L.fr_insert(ctx, img, rot)
        phases = L.fr_debug_phase_counters(ctx)
        L.fr_set_options(ctx, debug=0)
    for _ in range(args.warmup):
        L.fr_insert(ctx, img, rot)
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        L.fr_insert(ctx, img, rot)
    e.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = s.elapsed_time(e) / args.steps
    print(json.dumps({"config": L.fr_describe_config(args.profile_config), "S": args.S, "n": args.n,
                      "ms_per_launch": ms, "updates_per_launch": ups,
                      "updates_per_s": ups / (ms * 1e-3), "phases": phases,
                      "clocks": clocks}), flush=True)
    L.fr_destroy(ctx)
    return 0


def run_gemm_profile(args):
    """Small-case mode for ncu: warm-up then `steps` launches of one batched-GEMM
    configuration on one size; prints its throughput (GB/s of A, B and C)."""
    import torch

    from paper_1910_08498_gb300 import _lib as L
    m, n, k, cfg = (int(x) for x in args.gemm_profile.split(","))
    if not L.fr_gemm_config_valid(cfg, m, n, k):
        raise SystemExit(f"configuration {cfg} cannot run size {m}x{n}x{k}")
    dev = torch.device("cuda", 0)
    per = 4.0 * (m * k + k * n + m * n)
    batch = int(min(1 << 26, max(1, 512e6 // per)))
    g = torch.Generator(device=dev).manual_seed(args.seed)
    A = torch.randn(batch, m, k, device=dev, generator=g)
    B = torch.randn(batch, k, n, device=dev, generator=g)
    C = torch.empty(batch, m, n, device=dev)
    for _ in range(args.warmup):
        L.fr_gemm_run_config(cfg, A, B, C)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        L.fr_gemm_run_config(cfg, A, B, C)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / args.steps
    print(json.dumps({"config": L.fr_gemm_describe_config(cfg), "m": m, "n": n, "k": k, "batch": batch,
                      "ms_per_launch": ms, "gbs": batch * per / (ms * 1e-3) / 1e9,
                      "device_status": L.fr_gemm_device_status()}), flush=True)
    return 0


def main():
    args = parse()
    if args.profile_config is not None:
        return run_profile(args)
    if args.gemm_profile is not None:
        return run_gemm_profile(args)
    if args.only_gemm:
        import torch

        from paper_1910_08498_gb300 import _lib as L
        L.lib()
        print(json.dumps(run_gemm_dynamic(L, torch.device("cuda", 0), torch.cuda.current_stream())),
              flush=True)
        return 0
    if args.only_batched:
        import torch

        from paper_1910_08498_gb300 import _lib as L
        from paper_1910_08498_gb300 import inputs
        dev = torch.device("cuda", 0)
        L.lib()
        res, _ = run_batched(L, inputs, dev, torch.cuda.current_stream(), args.steps, args.warmup,
                             args.dtype == "f16")
        print(json.dumps(res), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
