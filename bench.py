"""Throughput benchmark of the hole-transport step (Eq. 6 pair sum + Fig. 2 step).

Default workload: one event of 1,048,576 holes -- 16 parallel straight
muon-like tracks of 65,536 holes, 30 um apart, crossing the 675 um CCD -- with
the FP32 + Kahan pair sum and FP64 positions.  A "step" is one time step of
the whole path: Eq. 6 pair sum, integrate (Eqs. 1-4, Philox diffusion,
update, collection, binning), compaction and bookkeeping.

Prints ONE JSON line: pair-interactions/s (value) and carrier-steps/s, the
pair kernel's live roofline fraction, the oracle CPU baseline, an end-to-end
figure through the C ABI with host buffers, clocks sampled during the timed
region, the FP64 form timed on a sub-sample of the same workload, and the
batched X-ray workload (4096 events) with its batched-vs-per-event ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_11043_gb300 import inputs  # noqa: E402

FP32_OPS_PER_PAIR = 11  # 3 sub + 3 fma (r^2) + 2 mul (r^-3) + 3 fma (accumulate); rsqrt on MUFU
FP32_LANES_PER_SM = 128
# Coulomb-off step (integrate + compaction), algorithmic HBM bytes per
# carrier-step: integrate reads id 4 + event 4 + FP64 position 24 and writes
# the position 24 (+ 1 keep bit); compaction reads and writes the id (4 + 4).
BYTES_PER_CARRIER_STEP_O_N = 64
METRIC = "pair-interactions/s"
FIELD = "E = 2 z - 1500 V/cm, T = 140 K, dt = 10 ps, eps = 0.01 um"
WORKLOADS = {
    "bundle": ("track-bundle-1M: one event of 1,048,576 holes in 16 straight muon-like tracks "
               "(65,536 holes each, 2.5 mm long, 0.5 um jitter, 30 um apart) across a 675 um CCD; "
               + FIELD + ", 512 x 512 pixels of 15 um"),
    "xray-batch": ("xray-batch-4096: 4096 independent X-ray clouds, E ~ U(1, 18) keV, N = E / 3.75 eV "
                   "(267..4800 holes), sigma 0.3 um, depth ~ U(0, 675) um, seeds 1..4096; " + FIELD
                   + ", 64 x 64 pixels of 15 um per event"),
    "muon": ("muon-200k: one straight 2.5 mm track of 200,000 holes across the 675 um CCD, "
             "0.5 um jitter; " + FIELD + ", 512 x 512 pixels of 15 um"),
    "xray": ("xray-5.9keV: one cloud of 1573 holes, sigma 0.3 um, depth from seed 1; " + FIELD
             + ", 64 x 64 pixels of 15 um"),
    "cloud-256": ("cloud-256: one cloud of 256 holes, sigma 0.5 um, at depth 300 um; " + FIELD
                  + ", 32 x 32 pixels of 15 um"),
}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32k": 2, "fp16x2": 3}
WORKLOAD = WORKLOADS["bundle"]


def make_workload(name: str):
    if name == "bundle":
        return inputs.track_bundle()
    if name == "xray-batch":
        return inputs.xray_batch()
    if name == "muon":
        return inputs.muon_track()
    if name == "xray":
        return inputs.xray_5p9kev()
    if name == "cloud-256":
        return inputs.single_cloud()
    raise ValueError(name)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def aggregate(time_ms: float, work, device="cpu"):
    """Whole-job figures over the ranks of an initialised process group: the
    max of the timed durations and the sum of the work (pairs, carrier-steps).
    Without a group (or with one rank) the inputs come back unchanged."""
    import torch
    import torch.distributed as dist
    work = [float(w) for w in work]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(time_ms), work
    t = torch.tensor([float(time_ms)], dtype=torch.float64, device=device)
    w = torch.tensor(work, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), [float(x) for x in w]


def replica_seeds(seeds, rank: int):
    """Each rank simulates an independent replica of the workload: the event
    seeds are offset by the rank (replicas only; the event is not sharded)."""
    return np.asarray(seeds, dtype=np.uint64) + np.uint64(rank)


def recorded_traffic():
    """DRAM bytes per pair-kernel launch on the track-bundle workload, as
    recorded from one ncu capture in profiles/pair_fp32_track_bundle_traffic.txt
    (key=value lines), only while the kernel source (gc_pair.cuh + pair.cu) is
    the one that was profiled (otherwise None): a recorded figure, not
    measured by this run."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "pair_fp32_track_bundle_traffic.txt")
    try:
        rec = {}
        for line in open(path):
            line = line.split("#", 1)[0].strip()
            if "=" in line:
                k, v = line.split("=", 1)
                rec[k.strip()] = v.strip()
        h = hashlib.sha256()
        for f in ("gc_pair.cuh", "pair.cu"):  # the pair kernel's templates and their instantiation
            h.update(open(os.path.join(ROOT, "paper_2203_11043_gb300", "csrc", f), "rb").read())
    except OSError:
        return None
    if rec.get("kernel_source_sha256") != h.hexdigest():
        return None
    return float(rec["traffic_bytes_per_launch"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


def cpu_baseline(wl, seconds: float = 12.0):
    """The FP64 oracle as it stands, on this host's cores: the Eq. 6 sum plus
    the rest of the step for a bounded sample of carriers of the same event."""
    import oracle as O
    p = O.make_params(img_w=wl.img_w, img_h=wl.img_h)
    src = np.arange(wl.n, dtype=np.int64)
    rng = np.random.default_rng(0)
    m = 8
    while True:
        tg = np.sort(rng.choice(wl.n, size=m, replace=False))
        t0 = time.perf_counter()
        O.step_targets(p, wl.xyz, src, tg, int(wl.seeds[0]), 1)
        dt = time.perf_counter() - t0
        if dt > 0.5 or m >= wl.n:
            break
        m = min(wl.n, m * 4)
    m = int(min(wl.n, max(m, m * seconds / max(dt, 1e-3))))
    tg = np.sort(rng.choice(wl.n, size=m, replace=False))
    t0 = time.perf_counter()
    O.step_targets(p, wl.xyz, src, tg, int(wl.seeds[0]), 1)
    dt = time.perf_counter() - t0
    return {"value": m * wl.n / dt, "unit": "pairs/s", "cores": O.num_threads(), "kind": "oracle",
            "carrier_steps_per_s": m / dt,
            "sample": f"one step (Eq. 6 field from all {wl.n} holes + drift/diffusion/update) for {m} "
                      f"randomly chosen holes of the same event: {m * wl.n:.3e} pair terms in {dt:.1f} s"}


def reference_arm(args):
    """--impl reference: the FP64 CPU oracle on the same workload, bounded steps."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    wl = make_workload(args.workload)
    if args.n_carriers:
        wl = inputs.subsample(wl, args.n_carriers, seed=3)
    per_step = max(2.0, min(4.0, 150.0 / max(1, args.steps + args.warmup)))
    import oracle as O
    p = O.make_params(img_w=wl.img_w, img_h=wl.img_h)
    src = np.arange(wl.n, dtype=np.int64)
    rng = np.random.default_rng(0)
    # size the per-step sample to ~per_step seconds
    m = 16
    t0 = time.perf_counter()
    O.step_targets(p, wl.xyz, src, np.arange(m), int(wl.seeds[0]), 1)
    dt = time.perf_counter() - t0
    m = int(min(wl.n, max(16, m * per_step / max(dt, 1e-3))))
    for _ in range(args.warmup):
        O.step_targets(p, wl.xyz, src, np.sort(rng.choice(wl.n, m, replace=False)), int(wl.seeds[0]), 1)
    total = 0.0
    for s in range(args.steps):
        tg = np.sort(rng.choice(wl.n, m, replace=False))
        t0 = time.perf_counter()
        O.step_targets(p, wl.xyz, src, tg, int(wl.seeds[0]), s + 1)
        total += time.perf_counter() - t0
    pairs = args.steps * m * wl.n
    value = pairs / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "n_carriers": wl.n},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{m} randomly chosen holes per step, field from all {wl.n}"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def to_completion(args):
    """One run of the workload until every hole is collected (CUDA graphs),
    timed with CUDA events; optionally the first M events run one simulation
    each, for the batched-vs-per-event comparison."""
    import torch
    import paper_2203_11043_gb300 as gc
    from paper_2203_11043_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    wl = make_workload(args.workload)
    prec = PRECISIONS[args.precision]

    def timed_run(w):
        p = gc.gc_default_params(precision=prec, img_w=w.img_w, img_h=w.img_h, pair_R=args.pair_R,
                                 coulomb=args.coulomb, stored_charge=args.stored_charge,
                                 tile_frames=args.tile_frames, fuse_small=args.fuse_small)
        with gc.Simulation(p, w.xyz, w.ev_off, w.seeds, w.img_origin, stream=stream.cuda_stream) as s:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            st, steps = s.run(-1)
            b.record(stream)
            torch.cuda.synchronize()
            stats = s.stats()
        return a.elapsed_time(b) / 1e3, steps, stats

    secs, steps, stats = timed_run(wl)
    line = {"metric": METRIC, "value": stats["pair_interactions"] / secs, "unit": "pairs/s",
            "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": 1e3 * secs / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f32", "precision": args.precision,
            "data": "synthetic", "mode": "to completion", "coulomb": args.coulomb,
            "stored_charge": args.stored_charge,
            "tile_frames": args.tile_frames,
            "config": {"workload": WORKLOADS[args.workload], "n_carriers": wl.n,
                       "events": wl.n_events, "pair_R": stats["pair_variant"],
                       "jchunk": stats["jchunk"], "pair_blocks": stats["pair_blocks"],
                       "small_path": stats["fused_path"], "pair_kernel_variant": stats["pair_kernel_variant"]},
            "carrier_steps_per_s": stats["carrier_steps"] / secs, "seconds": secs,
            "pair_interactions": stats["pair_interactions"], "carrier_steps": stats["carrier_steps"]}
    if args.per_event and wl.n_events > 1:
        m = min(args.per_event, wl.n_events)
        sub = inputs.Workload(wl.name, wl.xyz[:wl.ev_off[m]], wl.ev_off[:m + 1].copy(), wl.seeds[:m],
                              wl.img_origin[:m], wl.img_w, wl.img_h)
        bsecs, _, bst = timed_run(sub)
        tot, pairs = 0.0, 0.0
        for e in range(m):
            a, b = int(wl.ev_off[e]), int(wl.ev_off[e + 1])
            ev = inputs.Workload(wl.name, wl.xyz[a:b], np.array([0, b - a], np.int64),
                                 wl.seeds[e:e + 1], wl.img_origin[e:e + 1], wl.img_w, wl.img_h)
            es, _, est = timed_run(ev)
            tot += es
            pairs += est["pair_interactions"]
        line["per_event_launches"] = {"events": m, "batched_pairs_per_s": bst["pair_interactions"] / bsecs,
                                      "per_event_pairs_per_s": pairs / tot,
                                      "batched_over_per_event": (bst["pair_interactions"] / bsecs) / (pairs / tot)}
    print(json.dumps(line), flush=True)
    return 0


def e2e_run(gc, wl, seeds, stream, args):
    """One end-to-end use of the public API with host buffers and default
    parameters: create, load (autotuner), run, collect, image.  Returns
    (seconds, stats, h2d bytes per step, d2h bytes per step, steps)."""
    import torch
    steps = min(args.steps, 20)
    p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=wl.img_w, img_h=wl.img_h,
                             graph_steps=min(32, steps), tile_frames=args.tile_frames)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with gc.Simulation(p, wl.xyz, wl.ev_off, seeds, wl.img_origin, stream=stream.cuda_stream) as s3:
        s3.run(steps)
        res = s3.collect()
        img = s3.image()
        st3 = s3.stats()
    t1 = time.perf_counter()
    h2d = wl.xyz.nbytes + 8 * wl.n  # FP64 positions, active-id list and event map
    d2h = res["final_xy"].nbytes + res["collect_step"].nbytes + img.nbytes
    return t1 - t0, st3, h2d / steps, d2h / steps, steps


def batched_record(gc, stream, peak, steps=20, warmup=3, per_event=64):
    """The batched X-ray workload (4096 independent events of 267..4800 holes,
    Sec. 5.1's X-ray clouds) in one segmented launch per step: pair
    interactions/s over its first `steps` steps (all events active) with the
    pair kernel's own roofline fraction, and the same first `per_event` events
    run to completion once as one batch and once as one simulation per event."""
    import torch
    wl = inputs.xray_batch()
    p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=wl.img_w, img_h=wl.img_h,
                             graph_steps=1, timing=1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin, stream=stream.cuda_stream) as sim:
        for _ in range(warmup):
            sim.run(1)
        torch.cuda.synchronize()
        b = sim.stats()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        with ClockSampler(torch.cuda.current_device()) as clk:
            for a, z in ev:
                flush.zero_()
                a.record(stream)
                sim.run(1)
                z.record(stream)
            torch.cuda.synchronize()
        a_ = sim.stats()
    ms = sum(a.elapsed_time(z) for a, z in ev)
    pairs = a_["pair_interactions"] - b["pair_interactions"]
    launches = a_["pair_kernel_launches"] - b["pair_kernel_launches"]
    pair_ms = a_["pair_kernel_ms"] - b["pair_kernel_ms"]
    achieved = pairs / (pair_ms / 1e3) if pair_ms > 0 else None
    rec = {"workload": WORKLOADS["xray-batch"], "events": wl.n_events, "n_carriers": wl.n,
           "steps": steps, "warmup": warmup, "pairs_per_s": pairs / (ms / 1e3),
           "carrier_steps_per_s": (a_["carrier_steps"] - b["carrier_steps"]) / (ms / 1e3),
           "ms_per_step": ms / steps, "pair_kernel_pairs_per_s": achieved,
           "pair_kernel_frac": achieved / peak if achieved else None,
           "pair_kernel_launches": launches, "pair_R": a_["pair_variant"], "jchunk": a_["jchunk"],
           "pair_blocks": a_["pair_blocks"], "clocks": clk.summary(),
           "l2": "flushed between timed steps (256 MB write)"}

    def to_end(w):
        q = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=w.img_w, img_h=w.img_h)
        with gc.Simulation(q, w.xyz, w.ev_off, w.seeds, w.img_origin, stream=stream.cuda_stream) as s:
            x, y = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            x.record(stream)
            s.run(-1)
            y.record(stream)
            torch.cuda.synchronize()
            return x.elapsed_time(y) / 1e3, s.stats()["pair_interactions"]

    m = min(per_event, wl.n_events)
    sub = inputs.Workload(wl.name, wl.xyz[:wl.ev_off[m]], wl.ev_off[:m + 1].copy(), wl.seeds[:m],
                          wl.img_origin[:m], wl.img_w, wl.img_h)
    bs, bp = to_end(sub)
    tot, pp = 0.0, 0.0
    for e in range(m):
        lo, hi = int(wl.ev_off[e]), int(wl.ev_off[e + 1])
        one = inputs.Workload(wl.name, wl.xyz[lo:hi], np.array([0, hi - lo], np.int64), wl.seeds[e:e + 1],
                              wl.img_origin[e:e + 1], wl.img_w, wl.img_h)
        es, ep = to_end(one)
        tot += es
        pp += ep
    rec["per_event_launches"] = {
        "events": m, "mode": "each to completion, CUDA graphs with the device-side loop",
        "batched_pairs_per_s": bp / bs, "per_event_pairs_per_s": pp / tot,
        "batched_seconds": bs, "per_event_seconds": tot,
        "batched_over_per_event": (bp / bs) / (pp / tot)}
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched X-ray sub-record of the default run")
    ap.add_argument("--n-carriers", type=int, default=0,
                    help="run on a random sub-sample of the bundle (profiling small cases)")
    ap.add_argument("--pair-R", type=int, default=0, help="force the pair-kernel register blocking")
    ap.add_argument("--tile-frames", type=int, default=0, choices=[0, 1],
                    help="FP32 shadow relative to 256-slot tile origins for events of >= 2048 holes")
    ap.add_argument("--workload", default="bundle", choices=sorted(WORKLOADS))
    ap.add_argument("--to-completion", action="store_true",
                    help="time one run until every hole is collected (graphs, no per-step flush)")
    ap.add_argument("--coulomb", type=int, default=1, choices=[0, 1],
                    help="0 runs the O(N) Coulomb-off path (metric: carrier-steps/s)")
    ap.add_argument("--stored-charge", type=int, default=0, choices=[0, 1],
                    help="with --to-completion: 1 adds the field of the charge stored in the pixels")
    ap.add_argument("--per-event", type=int, default=0,
                    help="with --to-completion: also run the first M events one simulation each")
    ap.add_argument("--fuse-small", type=int, default=1, choices=[0, 1, 2, 3, 4, 5],
                    help="small-workload path (gc_params.fuse_small; 1 = automatic)")
    ap.add_argument("--precision", default="fp32k", choices=sorted(PRECISIONS),
                    help="with --to-completion: arithmetic of the pair sum")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if not args.coulomb:  # the O(N) path has its own metric; no end-to-end leg
        args.no_e2e = True
    if args.impl == "reference":
        return reference_arm(args)
    if args.to_completion:
        return to_completion(args)

    import torch
    import paper_2203_11043_gb300 as gc
    from paper_2203_11043_gb300 import build

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    gc.load()
    stream = torch.cuda.current_stream()
    sms, ccmaj, ccmin = gc.gc_device_info()

    if args.workload == "xray-batch" and world > 1:
        # sharded: a global batch of 4096 events per rank, dealt by LPT on
        # N^2 (z0 + 5 um); each rank loads and runs only its events, with no
        # collective in the run (weak scaling: per-rank work fixed)
        from paper_2203_11043_gb300 import shard
        glob = inputs.xray_batch(n_events=4096 * world)
        wl = shard.sub_workload(glob, shard.lpt_partition(shard.event_costs(glob), world)[rank])
        seeds = wl.seeds
        parallelism = f"events sharded x{world} (LPT on N^2 (z0 + 5 um), {glob.n_events} events in all)"
    else:
        wl = make_workload(args.workload)
        if args.n_carriers:
            wl = inputs.subsample(wl, args.n_carriers, seed=3)
        # every rank runs an independent replica of the workload (its seeds
        # differ per rank): one event is not split across GPUs
        seeds = replica_seeds(wl.seeds, rank)
        parallelism = f"replicas x{world}"

    params = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=wl.img_w, img_h=wl.img_h,
                                  graph_steps=1, timing=1, pair_R=args.pair_R, coulomb=args.coulomb,
                                  tile_frames=args.tile_frames)
    cold = e2e_run(gc, wl, seeds, stream, args) if not args.no_e2e else None
    sim = gc.Simulation(params, wl.xyz, wl.ev_off, seeds, wl.img_origin, stream=stream.cuda_stream)
    st0 = sim.stats()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        sim.run(1)
    torch.cuda.synchronize()
    base = sim.stats()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (256 MB > 129 MB L2)
            starts[k].record(stream)
            sim.run(1)
            ends[k].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    after = sim.stats()
    pairs = after["pair_interactions"] - base["pair_interactions"]
    csteps = after["carrier_steps"] - base["carrier_steps"]
    pair_ms = after["pair_kernel_ms"] - base["pair_kernel_ms"]
    pair_launches = after["pair_kernel_launches"] - base["pair_kernel_launches"]
    step_kernels_ms = (after["integrate_kernel_ms"] - base["integrate_kernel_ms"]
                       + after["compact_kernel_ms"] - base["compact_kernel_ms"])
    steps_done = after["steps"] - base["steps"]
    total_ms, (pairs, csteps) = aggregate(total_ms, [pairs, csteps], device="cuda")
    value = pairs / (total_ms / 1e3)
    clocks = clk.summary()

    peaks = measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * FP32_LANES_PER_SM * max_mhz * 1e6 / FP32_OPS_PER_PAIR
    pairs_per_launch = pairs / max(1, pair_launches) / max(1, world)
    achieved = pairs_per_launch / (pair_ms / max(1, pair_launches) / 1e3) if pair_launches else None
    traffic = recorded_traffic() if (args.workload == "bundle" and not args.n_carriers) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "pairs/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "traffic_source": "recorded from one ncu capture of this kernel source "
                                  "(profiles/pair_fp32_track_bundle_traffic.txt), not measured by this run",
                "kernel": "pair_fp32_kernel<R,Kahan>",
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {max_mhz:.0f} MHz "
                              f"(sm_max_mhz of MEASURED_PEAKS.json) / {FP32_OPS_PER_PAIR} FP32 ops per pair",
                "frac_at_sampled_clock": ((achieved / (peak * clocks["sm_mhz"] / max_mhz))
                                          if achieved and clocks.get("sm_mhz") else None),
                "pair_kernel_share_of_step": pair_ms / max(total_ms, 1e-9)}

    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_carriers": wl.n, "events": wl.n_events,
                       "precision": "FP32 pair sum with Kahan across j-tiles; FP64 positions",
                       "frames": "tile (256-slot FP64 origins, Morton order)" if args.tile_frames
                                 else "event centroid",
                       "pair_R": after["pair_variant"], "pair_blocks": after["pair_blocks"],
                       "jchunk": after["jchunk"], "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": parallelism, "device": f"sm_{ccmaj}{ccmin}, {sms} SMs"},
            "carrier_steps_per_s": csteps / (total_ms / 1e3), "steps_done": steps_done,
            "roofline": roofline, "gpu_launches": int(steps_done * after["launches_per_step"]),
            "clocks": clocks}

    if not args.coulomb:  # the O(N) path: carrier-steps/s against the HBM copy bandwidth
        hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
        bw = BYTES_PER_CARRIER_STEP_O_N * csteps / max(world, 1) / (step_kernels_ms / 1e3)
        line.update(metric="carrier-steps/s", value=csteps / (total_ms / 1e3), unit="carrier-steps/s",
                    dtype="f64")
        line["config"]["precision"] = "Coulomb off: FP32 mobility/diffusion, FP64 positions"
        line["roofline"] = {"bound": "hbm", "achieved": bw / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                            "frac": bw / hbm, "traffic": None,
                            "kernel": "integrate_kernel + compact_kernel",
                            "algorithmic_bytes_per_carrier_step": BYTES_PER_CARRIER_STEP_O_N,
                            "peak_basis": "hbm_gbs of MEASURED_PEAKS.json (STREAM-style copy)",
                            "step_kernels_share_of_step": step_kernels_ms / max(total_ms, 1e-9)}
        args.no_fp64 = True
        args.no_e2e = True
    # FP64 form vs FP32 form on one track of the same workload (like for like)
    if not args.no_fp64 and rank == 0:
        sub = inputs.subsample(wl, 65536, seed=3)
        forms = {}
        for name, prec in (("fp64", gc.GC_FP64), ("fp32_kahan", gc.GC_FP32_KAHAN)):
            p = gc.gc_default_params(precision=prec, img_w=wl.img_w, img_h=wl.img_h, graph_steps=1,
                                     timing=1)
            with gc.Simulation(p, sub.xyz, sub.ev_off, sub.seeds, sub.img_origin,
                               stream=stream.cuda_stream) as s2:
                s2.run(2)
                b = s2.stats()
                s2.run(3)
                a = s2.stats()
                forms[name] = (a["pair_interactions"] - b["pair_interactions"]) / (
                    (a["pair_kernel_ms"] - b["pair_kernel_ms"]) / 1e3)
        line["fp64_form"] = {"pair_kernel_pairs_per_s": forms["fp64"],
                             "fp32_kahan_pair_kernel_pairs_per_s": forms["fp32_kahan"],
                             "fp32_over_fp64": forms["fp32_kahan"] / forms["fp64"],
                             "workload": "65,536 holes drawn from the same bundle, 3 steps"}

    # end to end through the C ABI with host buffers (H2D load, steps, D2H results),
    # default parameters (autotuner on): cold = the first load of this workload in
    # the process (it pays the tuning), warm = a later load (cached shape)
    if not args.no_e2e:
        warm = e2e_run(gc, wl, seeds, stream, args)
        e2e_s, (e2e_pairs,) = aggregate(cold[0], [cold[1]["pair_interactions"]], device="cuda")
        w_s, (w_pairs,) = aggregate(warm[0], [warm[1]["pair_interactions"]], device="cuda")
        line["e2e"] = {"value": e2e_pairs / e2e_s, "unit": "pairs/s",
                       "h2d_bytes_per_step": cold[2], "d2h_bytes_per_step": cold[3], "steps": cold[4],
                       "warm_value": w_pairs / w_s, "cold_seconds": cold[0], "warm_seconds": warm[0],
                       "tune_ms_cold": cold[1]["tune_ms"], "tune_candidates": cold[1]["tune_candidates"],
                       "tune_cached_warm": warm[1]["tune_cached"],
                       "shape": {k: warm[1][k] for k in ("pair_variant", "pair_kernel_variant", "pair_blocks",
                                                         "jchunk", "small_n")},
                       "includes": "gc_create + gc_load_carriers (host positions, autotuner) + gc_run + "
                                   "gc_collect + gc_image (host outputs), host wall clock; value = cold "
                                   "(first load of the workload in the process), warm_value = cached shape"}

    if not args.no_batched and rank == 0 and args.coulomb and args.workload == "bundle" \
            and not args.n_carriers:
        line["batched"] = batched_record(gc, stream, peak)

    if not args.no_cpu_baseline and rank == 0 and world == 1 and args.coulomb:
        line["cpu_baseline"] = cpu_baseline(wl)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
