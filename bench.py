#!/usr/bin/env python
"""Benchmark of the GB300 multi-scale MPV stereo matcher.

Workload: one rectified 1280x720 uint8 pair per step, D = 128, 3 pyramid scales,
8 scan paths, p1 = 10, T = 30, N = 5 SSIM windows, left-right check (both views).
The pair is synthetic (slanted planes on Voronoi regions over gradient-noise texture),
standing in for the paper's driving sequences.  Metric: Mdisp-evals/s = W*H*D / frame
time (nominal full-range labels of one view), plus fps and p50/p99 latency.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--variant plain|paper|gradient|paper_gradient|road|learned|learned16]
                  [--workload frame|batch64]

--variant selects, on the same pair, the paper's layered path merge (Section 3.2) and/or
the gradient-weighted TV penalty (Eq. EU, slopes round(p1 e^{-g/16})), the road profile of
Section 3.5 on the matcher's output (road), or the learned window proposal with a 17- or
16-label window (learned, learned16).  --workload batch64 times the 64-pair mixed batch
against the same pairs matched one at a time.

--impl reference times the CPU oracle (single-threaded C) on a bounded sample of the
same workload: the reference arm of this method is the oracle.  Under torchrun every
rank matches its own pair on its own GPU (replicas; no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Load every kernel when the process starts instead of at its first launch: a lazy load
# in the middle of the served streams held the host for tens of milliseconds (set before
# CUDA initialises; an explicit setting in the environment wins).
os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")

W, H, D = 1280, 720, 128
PARAMS = dict(max_disparity=D, num_scales=3, num_paths=8, p1=10, trunc=30, ssim_window=5,
              lr_check=1, lr_tol=1)
METRIC = "Mdisp-evals/s at 1280x720 D=128 (3-scale MPV, 8 paths, left-right check)"
UNIT = "Mdisp-evals/s"
WORKLOAD = ("1280x720 uint8 pair, D=128, 3 scales (factor 2, windows D/4), 8 paths, "
            "p1=10, T=30, N=5, left-right check")
CLOCK_FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
L2_FLUSH_BYTES = 256 << 20
GRAD_SIGMA = 16.0
VARIANTS = {          # merge mode, gradient weighting, learned window (0: pyramid)
    "plain": (0, False, 0),
    "paper": (1, False, 0),
    "gradient": (0, True, 0),
    "paper_gradient": (1, True, 0),
    "road": (0, False, 0),       # plus road detection on every frame's disparity map
    "learned": (0, False, 17),   # learned window proposal, centre +- 8
    "learned16": (0, False, 16),  # learned window proposal, one 16-label stride
}
ROAD_ETA = 8
WEIGHTS = os.path.join(ROOT, "paper_2001_09678_gb300", "weights", "proposal_d128_s3.bin")


def gradient_table(p1=PARAMS["p1"], sigma=GRAD_SIGMA):
    """256 integer slopes round(p1 e^{-g / sigma}): Eq. EU's e^{-|G|} weighting with a scale."""
    import numpy as np
    g = np.arange(256, dtype=np.float64)
    return np.floor(p1 * np.exp(-g / sigma) + 0.5).astype(np.int32)


def variant_names(variant):
    """Metric and workload strings of a variant (the plain matcher keeps the headline's)."""
    if variant == "plain":
        return METRIC, WORKLOAD
    if variant == "road":
        return (METRIC[:-1] + ", + road detection)",
                WORKLOAD + f", + v/u-disparity and road profile (eta={ROAD_ETA})")
    merge, grad, lw = VARIANTS[variant]
    if lw:
        tag = f"learned proposal, {lw}-label finest window"
        return (METRIC.replace("3-scale MPV", "learned-proposal MPV")[:-1] + f", window {lw})",
                WORKLOAD + f", learned window proposal (6-layer CNN at the top level, "
                           f"finest-level window {lw}, intermediate level skipped)")
    tag = " + ".join(t for t, on in (("layered merge", merge), ("gradient TV", grad)) if on)
    return METRIC[:-1] + ", " + tag + ")", WORKLOAD + ", " + tag


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def nominal_units(w=W, h=H, d=D):
    return w * h * d


# ------------------------------------------------------------------------------------
# Algorithmic bytes per stage (one frame, both views)
# ------------------------------------------------------------------------------------

def level_geometry():
    levels = []
    w, h = W, H
    dims = []
    for _ in range(PARAMS["num_scales"]):
        dims.append((w, h))
        w, h = (w + 1) // 2, (h + 1) // 2
    dims = dims[::-1]
    S = PARAMS["num_scales"]
    for l, (w, h) in enumerate(dims):
        sh = S - 1 - l
        Dl = (D + (1 << sh) - 1) >> sh
        Dw = Dl if l == 0 else min(D // 4, Dl)
        levels.append((w, h, Dl, Dw))
    return levels


ALG_NOTE = {
    "cost": "images 2 B/px + cost write 1 B/node (cost stored as uint8: exact, costs <= 255)",
    "aggregate": "cost read 1 B + summed-energy write 2 B per node, window starts 2 B/px "
                 "(the survey's B_alg reads a uint16 cost: 2 B + 2 B, reported as "
                 "frac_at_survey_bytes)",
    "wta": "summed-energy read 2 B/node + window starts and map 2 B/px each",
}


def algorithmic_bytes(views=2, variant="plain", cost_bytes=1):
    """Minimum HBM bytes per frame of each stage: the cost kernel reads both images and
    writes the cost volume (1 B/node: costs are <= 255); the aggregation reads it
    (1 B/node) and writes the uint16 summed volume (2 B/node); winner-take-all reads
    that (2 B/node) and writes the uint16 map.  The layered merge stores each pass
    (2 B/node per direction) and reads the previous layer's pair (4 B/node per
    direction; the first layer reads the cost bytes), and its WTA reads the last pair."""
    merge, grad, lw = VARIANTS[variant]
    layers = PARAMS["num_paths"] // 2
    cost = agg = wta = 0
    nodes = 0
    levels = level_geometry()
    if lw:   # the top level's cost feeds the network; the finest level searches lw labels
        (w0, h0, _, D0), (w2, h2, D2, _) = levels[0], levels[-1]
        cost += views * (w0 * h0 * D0 + 2 * w0 * h0)
        levels = [(w2, h2, D2, lw)]
        nodes = w0 * h0 * D0
    for (w, h, Dl, Dw) in levels:
        n = w * h * Dw
        nodes += n
        cost += views * (cost_bytes * n + 2 * w * h)
        img = 2 * w * h if grad else 0          # the reference image, read by the passes
        if merge:
            agg += views * ((2 * n + 4 * n) + (layers - 1) * (8 * n + 4 * n) + img)
            wta += views * (4 * n + 2 * w * h + 2 * w * h)
        else:
            agg += views * (cost_bytes * n + 2 * n + 2 * w * h + img)
            wta += views * (2 * n + 2 * w * h + 2 * w * h)
    return dict(cost=cost, aggregate=agg, wta=wta), nodes


# ------------------------------------------------------------------------------------
# Clocks
# ------------------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()

    def mark(self, start, end):
        """Wall-clock window (time.time()) of the timed region."""
        self.window = (start, end)

    def summary(self):
        import datetime
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f if ln.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        win = getattr(self, "window", None)
        for r in rows:
            try:
                r = [x.strip() for x in r]
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if win and not (win[0] - 0.06 <= ts <= win[1] + 0.06):
                    continue
                sm.append(float(r[2]))
                smax = max(smax, float(r[3]))
                for nm, v in zip(names, r[6:10]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(value, world, device=None):
    """Max of a per-rank float over all ranks (identity on one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_step, steps, world, slowest_ms):
    """Whole-job Mdisp-evals/s: every rank matched `steps` pairs; time of the slowest."""
    return world * steps * units_per_step / (slowest_ms / 1e3) / 1e6


def code_hash(*paths):
    """sha256 prefix of C/CUDA sources (in the given order) with their comments, trailing
    blanks and empty lines removed: edits to comments leave it unchanged, edits to code do
    not."""
    import hashlib
    import re
    parts = []
    for path in paths:
        text = open(path, encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        parts.append("\n".join(ln for ln in lines if ln))
    return hashlib.sha256("\n".join(parts).encode("utf-8")).hexdigest()[:16]


def measured_counters(kernel):
    """Per-frame device-time-weighted ALU-pipe and issue-slot activity and DRAM bytes of
    `kernel`'s launches from the committed ncu summary, or None when the kernel's code
    changed since the capture (the file's code hash no longer matches)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_counters.txt")
    if not os.path.exists(path):
        return None
    rows, src_ok = [], None
    for line in open(path):
        if line.startswith("#") or "=" not in line:
            continue
        kv = dict(f.split("=", 1) for f in line.split())
        if "code_sha256_16" in kv:
            srcs = [os.path.join(ROOT, f) for f in kv["source"].split(",")]
            src_ok = (all(os.path.exists(f) for f in srcs) and
                      code_hash(*srcs) == kv["code_sha256_16"])
            continue
        rows.append({k: float(v) for k, v in kv.items() if k != "level"})
    if not src_ok or not rows:
        return None
    t = sum(r["us"] for r in rows)
    return {"alu_pipe_active": round(sum(r["alu_pct"] * r["us"] for r in rows) / t / 100, 4),
            "issue_active": round(sum(r["issue_pct"] * r["us"] for r in rows) / t / 100, 4),
            "dram_bytes_per_step": int(sum(r["dram_bytes"] for r in rows)),
            "launches": len(rows),
            "source": f"profiles/{kernel}_counters.txt (ncu, one frame's launches)"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------

def run_mine(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_09678_gb300 import mpv, synth

    L, R, _ = synth.slanted_pair(W, H, seed=rank)
    left = torch.from_numpy(L).to(dev)
    right = torch.from_numpy(R).to(dev)
    disp = torch.empty((H, W), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = mpv.mpv_create(local)
    merge, grad, lw = VARIANTS[args.variant]
    extra = dict(proposal=mpv.MPV_PROPOSAL_LEARNED, window=lw) if lw else {}
    mpv.mpv_set_params(ctx, mpv.mpv_default_params(merge_mode=merge, **extra, **PARAMS))
    if grad:
        mpv.mpv_set_gradient_penalty(ctx, gradient_table())
    if lw:
        mpv.mpv_load_proposal_weights(ctx, WEIGHTS)
    metric, workload = variant_names(args.variant)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    road = args.variant == "road"
    if road:
        vd = torch.empty((H, D), dtype=torch.int32, device=dev)
        ud = torch.empty((W, D), dtype=torch.int32, device=dev)
        prof_r = torch.empty(D, dtype=torch.int32, device=dev)
        en_r = torch.empty(1, dtype=torch.int64, device=dev)

    def step():
        mpv.mpv_match(ctx, left, right, disp, stream)
        if road:
            mpv.mpv_road_detect(ctx, disp, D, ROAD_ETA, vd, prof_r, en_r, udisp=ud,
                                stream=stream)

    for _ in range(args.warmup):
        step()
    mpv.mpv_sync(ctx)
    mpv.mpv_profile_read(ctx)  # reset counters

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        w0 = time.time()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)          # L2 flush between timed steps (not timed)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        wall = time.perf_counter() - t0
        clocks.mark(w0, time.time())
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # stage breakdown and launch count: a separate pass with the per-stage event profiler
    # (the timed frames above replay one CUDA graph per frame, without profiler events)
    prof_steps = min(args.steps, 200)
    mpv.mpv_profile_read(ctx)
    mpv.mpv_profile_enable(ctx, True)
    for i in range(prof_steps):
        flush.fill_(i & 0xFF)
        mpv.mpv_match(ctx, left, right, disp, stream)
    torch.cuda.synchronize(dev)
    prof = mpv.mpv_profile_read(ctx)
    mpv.mpv_profile_enable(ctx, False)
    road_ms = None
    if road:   # the road stage alone, on the last disparity map
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(prof_steps):
            mpv.mpv_road_detect(ctx, disp, D, ROAD_ETA, vd, prof_r, en_r, udisp=ud,
                                stream=stream)
        r1.record(stream)
        torch.cuda.synchronize(dev)
        road_ms = r0.elapsed_time(r1) / prof_steps
    total_ms = reduce_max(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(nominal_units(), args.steps, world, total_ms)

    # end to end through the host entry point: pinned host buffers, copies inside
    hl = torch.from_numpy(L).pin_memory()
    hr = torch.from_numpy(R).pin_memory()
    hd = torch.empty((H, W), dtype=torch.int16).pin_memory()
    for _ in range(max(1, args.warmup)):
        mpv.mpv_match_host(ctx, hl, hr, hd, stream)
    barrier()
    e2e_times = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        mpv.mpv_match_host(ctx, hl, hr, hd, stream)   # synchronizes before returning
        e2e_times.append(time.perf_counter() - t1)
    e2e_s = reduce_max(sum(e2e_times), world, dev)
    e2e_value = replica_throughput(nominal_units(), args.steps, world, 1e3 * e2e_s)
    ok = np.array_equal(hd.numpy(), disp.cpu().numpy())

    # roofline of the dominant kernel (by device time over the timed region)
    alg, nodes = algorithmic_bytes(variant=args.variant)
    alg4, _ = algorithmic_bytes(variant=args.variant, cost_bytes=2)
    stage_ms = {k: v[0] for k, v in prof.items()}
    launches_per_frame = sum(v[1] for v in prof.values()) / prof_steps
    dom = max(("cost", "aggregate", "wta"), key=lambda k: stage_ms[k])
    peak, peak_kind = measured_peaks()
    dom_s = stage_ms[dom] / 1e3
    achieved = alg[dom] * prof_steps / dom_s / 1e9 if dom_s > 0 else 0.0
    achieved4 = alg4[dom] * prof_steps / dom_s / 1e9 if dom_s > 0 else 0.0
    kern_launches = prof[dom][1]
    per_step_launches = kern_launches / prof_steps
    counters = measured_counters(dom) if args.variant == "plain" else None
    traffic_step = counters["dram_bytes_per_step"] if counters else None

    out = None
    if rank == 0:
        clk = clocks.summary()
        out = {
            "metric": metric, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload, "width": W, "height": H, "max_disparity": D,
                       "scales": 3, "paths": 8, "global_batch": world,
                       "parallelism": f"replicas{world}",
                       "l2": "flushed between timed steps (256 MiB device write, untimed)"},
            "fps": round(1e3 / ms_per_step, 1),
            "latency_ms": {"p50": round(statistics.median(step_ms), 4),
                           "p99": round(sorted(step_ms)[min(len(step_ms) - 1,
                                                            int(0.99 * len(step_ms)))], 4),
                           "samples": len(step_ms)},
            "evaluated_nodes_per_view": nodes,
            "stage_ms_per_step": {k: round(v / prof_steps, 4) for k, v in stage_ms.items()},
            "stage_profile": f"{prof_steps} further frames with per-stage events",
            **({"road_ms_per_step": round(road_ms, 4)} if road_ms is not None else {}),
            "roofline": {
                "kernel": dom, "bound": "hbm", "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": peak_kind,
                # traffic and the algorithmic bytes per launch (the frame's launches, one
                # per pyramid level, averaged), and per step with their ratio
                "traffic": (int(traffic_step / per_step_launches) if traffic_step else None),
                "alg_bytes_per_launch": int(alg[dom] / per_step_launches),
                "alg_bytes_per_step": alg[dom], "launches_per_step": per_step_launches,
                "traffic_per_step": traffic_step,
                "traffic_over_alg": (round(traffic_step / alg[dom], 2) if traffic_step else None),
                "alg_bytes_per_node": ALG_NOTE[dom],
                "frac_at_survey_bytes": round(achieved4 / peak, 4),
                # the whole path: every stage's algorithmic bytes of one frame over the
                # frame time (the survey's whole-path figure reads a uint16 cost: the second)
                "whole_path": {"alg_bytes_per_step": int(sum(alg.values())),
                               "frac": round(sum(alg.values()) / (ms_per_step * 1e-3) / 1e9 / peak, 4),
                               "frac_at_survey_bytes": round(sum(alg4.values()) / (ms_per_step * 1e-3)
                                                             / 1e9 / peak, 4)},
                # the integer path's second bound: ALU-pipe and issue-slot activity of the
                # same kernel (ncu, device-time weighted over the frame's launches)
                "int_pipe": (dict(alu_pipe_active=counters["alu_pipe_active"],
                                  issue_active=counters["issue_active"],
                                  source=counters["source"]) if counters else None)},
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": 2 * W * H, "d2h_bytes_per_step": 2 * W * H,
                    "ms_per_step": round(1e3 * e2e_s / args.steps, 4),
                    "matches_device_path": bool(ok)},
            "gpu_launches": int(round(launches_per_frame * args.steps)),
            "clocks": clk,
            "wall_s_timed_region": round(wall, 4),
            "device": device_info(dev),
        }
    mpv.mpv_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0 and world == 1 and not args.no_extras and args.variant == "plain":
        out["extras"] = bench_extras(dev, L, R, ms_per_step)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not lw:
        # (the oracle has no network: the learned variants report no CPU baseline)
        out["cpu_baseline"] = cpu_baseline_full(L, R, args.variant)
        if not args.no_extras:
            out["cpu_baseline"]["per_config"] = oracle_per_config()
    if out is not None:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------
# The oracle on the host
# ------------------------------------------------------------------------------------

def _ora_params(variant="plain"):
    from oracle import ref
    merge, grad, _ = VARIANTS[variant]
    return ref.params(window=0, block=(0, 0, 0, 0), merge_mode=merge,
                      grad_lut=gradient_table() if grad else None, **PARAMS)


def _oracle_pair(job):
    """One full pair through the oracle in a worker process; returns its seconds."""
    L, R, variant = job
    from oracle import ref
    p = _ora_params(variant)
    ref.lib()
    t = time.perf_counter()
    ref.match(L, R, p)
    return time.perf_counter() - t


def device_info(dev):
    """Name, SM count and L2 size (cudaDevAttrL2CacheSize) of the timed GPU."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    return {"name": p.name, "sms": p.multi_processor_count,
            "l2_bytes": getattr(p, "L2_cache_size", None),
            "hbm_bytes": p.total_memory}


def _oracle_job(job):
    """One generated pair of another configuration through the oracle (worker process):
    (kind, W, H, D, seed, scales, paths) -> seconds."""
    kind, w, h, d, seed, scales, paths = job
    from oracle import ref
    from paper_2001_09678_gb300 import synth
    if kind == "bands":
        L, R, _ = synth.bands_pair(w, h, seed=seed)
    else:
        L, R, _ = synth.slanted_pair(w, h, seed=seed, d_max=min(120.0, d - 8.0))
    p = ref.params(window=0, block=(0, 0, 0, 0),
                   **dict(PARAMS, max_disparity=d, num_scales=scales, num_paths=paths))
    ref.lib()
    t = time.perf_counter()
    ref.match(L, R, p)
    return time.perf_counter() - t


def oracle_per_config():
    """Single-core oracle seconds for configuration 1 and for four representative pairs of
    the 64-pair batch (one 640x480 D64, two 1280x720 D128, one 1920x1080 D192), each in
    its own process, run side by side."""
    import multiprocessing as mp
    from paper_2001_09678_gb300 import synth
    specs = synth.mixed_batch_specs()
    pick = []
    for (w, h, d) in ((640, 480, 64), (1280, 720, 128), (1280, 720, 128), (1920, 1080, 192)):
        seed = next(s for s, sw, sh, sd in specs if (sw, sh, sd) == (w, h, d) and
                    all(s != q[4] for q in pick))
        pick.append(("slanted", w, h, d, seed, 3, 8))
    jobs = [("bands", 320, 240, 32, 0, 1, 4)] + pick
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        secs = pool.map(_oracle_job, jobs, chunksize=1)
    return {"config1": {"seconds": round(secs[0], 3), "cores": 1,
                        "value": round(320 * 240 * 32 / secs[0] / 1e6, 3), "unit": UNIT,
                        "sample": "the 320x240 bands pair (seed 0), D=32, 1 scale, 4 paths, LR"},
            "config3_representative": [
                {"width": j[1], "height": j[2], "max_disparity": j[3], "seed": j[4],
                 "seconds": round(s, 2), "cores": 1,
                 "value": round(j[1] * j[2] * j[3] / s / 1e6, 3), "unit": UNIT}
                for j, s in zip(pick, secs[1:])],
            "note": "one process per pair, side by side on the host cores; every pair of the "
                    "64-pair batch is verified against the oracle in the GPU tests"}


def cpu_baseline_full(L, R, variant="plain"):
    """The oracle (single-threaded C) on the machine's host cores: one full pair of the
    workload (both views) on one core, then one full pair in each of nproc independent
    processes at once (their aggregate throughput is the reported value)."""
    import multiprocessing as mp
    dt1 = _oracle_pair((L, R, variant))
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_oracle_pair, [(L[:40], R[:40], variant)] * n)    # workers up, oracle loaded
        t = time.perf_counter()
        per = pool.map(_oracle_pair, [(L, R, variant)] * n, chunksize=1)
        wall = time.perf_counter() - t
    return {"value": round(n * nominal_units() / wall / 1e6, 3), "unit": UNIT, "cores": n,
            "kind": "oracle",
            "sample": f"{n} independent processes (one per host core), each one full "
                      "1280x720 pair, 3 scales, both views",
            "seconds": round(wall, 2), "per_process_s_max": round(max(per), 2),
            "single_core": {"value": round(nominal_units() / dt1 / 1e6, 3), "cores": 1,
                            "seconds": round(dt1, 2),
                            "sample": "one full 1280x720 pair on one core"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if VARIANTS[args.variant][2]:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no network: "
                          "the learned window proposal has no CPU reference"}), flush=True)
        return
    from oracle import ref
    from paper_2001_09678_gb300 import synth
    L, R, _ = synth.slanted_pair(W, H, seed=0)
    # bounded sample: a 1280 x rows strip through the matcher, sized so that the whole
    # run (warm-up + steps) takes about two minutes; at least 20 rows keep the top level
    # of the 3-scale pyramid >= 5 rows high
    rows = int(min(180, max(20, 8000 // max(1, args.steps + args.warmup))))
    y0 = (H - rows) // 2
    Ls, Rs = L[y0:y0 + rows].copy(), R[y0:y0 + rows].copy()
    p = _ora_params(args.variant)
    metric, workload = variant_names(args.variant)
    ref.lib()
    for _ in range(args.warmup):
        ref.match(Ls, Rs, p)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        ref.match(Ls, Rs, p)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    units = W * rows * D
    value = args.steps * units / tot / 1e6
    sample = f"1280x{rows} strip (rows {y0}..{y0 + rows - 1}) of the 1280x720 pair per step"
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": round(value, 3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": workload, "width": W, "height": H, "max_disparity": D,
                   "scales": 3, "paths": 8},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def measure_batch64(steps, warmup, serial=True):
    """The 64-pair mixed-resolution batch (one cached CUDA graph per batch): ms per
    batch, and optionally the same pairs matched one mpv_match at a time."""
    import multiprocessing as mp
    import torch
    from paper_2001_09678_gb300 import synth
    specs = synth.mixed_batch_specs()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        images = pool.map(_gen_pair, specs)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_09678_gb300 import mpv
    dev = torch.device("cuda", 0)
    pairs = []
    units = 0
    for (L, R), (_seed, W, H, D) in zip(images, specs):
        pairs.append(dict(left=torch.from_numpy(L).to(dev), right=torch.from_numpy(R).to(dev),
                          disp=torch.empty((H, W), dtype=torch.int16, device=dev),
                          max_disparity=D))
        units += W * H * D
    ctx = mpv.mpv_create(0)
    mpv.mpv_set_params(ctx, mpv.mpv_default_params(**PARAMS))
    stream = torch.cuda.current_stream(dev)
    t = time.perf_counter()
    mpv.mpv_match_batch(ctx, pairs, stream)     # autotune + capture
    mpv.mpv_sync(ctx)
    setup_s = time.perf_counter() - t
    for _ in range(warmup):
        mpv.mpv_match_batch(ctx, pairs, stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        mpv.mpv_match_batch(ctx, pairs, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    persistent, lanes, queues, cblocks, p_ms, s_ms, occ = mpv.mpv_batch_info(ctx)
    mpv.mpv_destroy(ctx)
    out = {"value": round(units / ms / 1e3, 1), "unit": UNIT, "ms_per_batch": round(ms, 3),
           "pairs_per_s": round(64e3 / ms, 1), "steps": steps, "warmup": warmup,
           "setup_s": round(setup_s, 2),
           # the batch autotuner's measurements: the persistent kernel (best shapes) and the
           # stream graph on this batch, and the path it kept
           "path": "persistent kernel" if persistent else "stream graph",
           "tuner_ms": {"persistent": round(p_ms, 3), "streams": round(s_ms, 3)},
           "persistent_shapes": {"lanes": lanes, "queues": queues, "cost_blocks": cblocks,
                                 "blocks_per_sm": occ}}
    if serial:
        seq_ms = _serial_ms(mpv, pairs, stream, max(1, steps // 4), warmup)
        out.update({"serial_ms_per_64_pairs": round(seq_ms, 3),
                    "batch_speedup": round(seq_ms / ms, 2),
                    "serial": "the same pairs one mpv_match at a time on one stream; per size "
                              "class one context and one input/output buffer set (each pair "
                              "copied in on the device first), so every call replays that "
                              "class's cached graph"})
    return out


def run_batch64(args):
    """Throughput of the 64-pair mixed-resolution batch (one cached CUDA graph)."""
    res = measure_batch64(args.steps, args.warmup)
    print(json.dumps({
        "metric": "Mdisp-evals/s, 64-pair mixed batch", **res,
        "config": {"workload": "16x640x480 D64 + 32x1280x720 D128 + 16x1920x1080 D192, "
                               "3 scales, 8 paths, LR, one CUDA graph per batch"},
    }), flush=True)


def bench_extras(dev, L, R, plain_ms):
    """The other configurations of the workload list, bounded in time and measured on
    the same GPU beside the headline: the learned window proposal (17- and 16-label
    windows, the committed network, its bad-pixel rate against full-range single-scale
    MPV on the bench pair), the 64-pair mixed batch, and the 8-camera served stream
    (plain and with the learned proposal where the network fits)."""
    import numpy as np
    import torch
    from paper_2001_09678_gb300 import mpv, serve
    out = {}
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    left = torch.from_numpy(L).to(dev)
    right = torch.from_numpy(R).to(dev)
    disp = torch.empty((H, W), dtype=torch.int16, device=dev)
    full = mpv.mpv_create(dev.index)
    mpv.mpv_set_params(full, mpv.mpv_default_params(**dict(PARAMS, num_scales=1)))
    mpv.mpv_match(full, left, right, disp, stream)
    mpv.mpv_sync(full)
    ref_map = disp.cpu().numpy().view(np.uint16).copy()
    mpv.mpv_destroy(full)
    for lw in (17, 16):
        ctx = mpv.mpv_create(dev.index)
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(
            proposal=mpv.MPV_PROPOSAL_LEARNED, window=lw, **PARAMS))
        mpv.mpv_load_proposal_weights(ctx, WEIGHTS)
        for _ in range(10):
            mpv.mpv_match(ctx, left, right, disp, stream)
        mpv.mpv_sync(ctx)
        n = 200
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        for a, b in ev:
            flush.fill_(1)
            a.record(stream)
            mpv.mpv_match(ctx, left, right, disp, stream)
            b.record(stream)
        mpv.mpv_sync(ctx)
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        got = disp.cpu().numpy().view(np.uint16)
        both = (got != 0xFFFF) & (ref_map != 0xFFFF)
        bad = float((np.abs(got.astype(int) - ref_map.astype(int)) > 1)[both].mean())
        hits, px = mpv.mpv_proposal_stats(ctx)
        frames, falls = mpv.mpv_proposal_fallbacks(ctx)
        mpv.mpv_destroy(ctx)
        out[f"learned{lw}"] = {
            "ms_per_step": round(sum(ms) / n, 4), "p50_ms": round(ms[n // 2], 4),
            "p99_ms": round(ms[int(0.99 * n)], 4), "samples": n,
            "vs_plain_ms": round(plain_ms, 4),
            "bad_pixel_rate_vs_full_range": round(bad, 5),
            "edge_hit_rate": round(hits / max(1, px), 4),
            "fallbacks": falls, "frames": frames,
            "workload": f"the bench pair, learned proposal (committed network), finest window "
                        f"{lw}, default fallback (pyramid above 15 % edge hits), L2 flushed"}
    # configuration 1: 320x240, D=32, one scale, 4 paths, LR; its 4.9 MB volume stays in
    # L2, so only its latency is reported (no flush between frames)
    from paper_2001_09678_gb300 import synth
    L1, R1, _ = synth.bands_pair(320, 240, seed=0)
    l1, r1 = torch.from_numpy(L1).to(dev), torch.from_numpy(R1).to(dev)
    d1 = torch.empty((240, 320), dtype=torch.int16, device=dev)
    ctx = mpv.mpv_create(dev.index)
    mpv.mpv_set_params(ctx, mpv.mpv_default_params(**dict(PARAMS, max_disparity=32,
                                                          num_scales=1, num_paths=4)))
    for _ in range(20):
        mpv.mpv_match(ctx, l1, r1, d1, stream)
    mpv.mpv_sync(ctx)
    n = 500
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(n)]
    for a, b in ev:
        a.record(stream)
        mpv.mpv_match(ctx, l1, r1, d1, stream)
        b.record(stream)
    mpv.mpv_sync(ctx)
    mpv.mpv_destroy(ctx)
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    out["config1"] = {
        "ms_per_step": round(sum(ms) / n, 4), "p50_ms": round(ms[n // 2], 4),
        "p99_ms": round(ms[int(0.99 * n)], 4), "samples": n,
        "value": round(320 * 240 * 32 / (sum(ms) / n * 1e-3) / 1e6, 1), "unit": UNIT,
        "workload": "320x240 bands pair (seed 0), D=32, 1 scale, 4 paths, p1=10, T=30, LR; "
                    "cost volume L2-resident: latency only, no roofline"}
    out["batch64"] = measure_batch64(5, 2, serial=False)
    out["batch64"]["workload"] = ("16x640x480 D64 + 32x1280x720 D128 + 16x1920x1080 D192, "
                                  "3 scales, 8 paths, LR, one CUDA graph per batch")
    cams = serve.camera_specs()
    pools = serve.frame_pools(sorted({(w, h, d) for _, w, h, d in cams}), 4)
    for name, prop in (("serving", None), ("serving_learned", WEIGHTS)):
        r = serve.run(cams, pools, seconds=3.0, hz=30.0, proposal=prop)
        out[name] = {k: (round(r[k], 4) if isinstance(r[k], float) else r[k])
                     for k in ("frames", "ok", "fps", "p50_ms", "p99_ms", "max_ms",
                               "peak_inflight")}
        out[name]["samples"] = r["ok"]
        out[name]["workload"] = ("8 cameras (2x640x480 D64, 4x1280x720 D128, 2x1920x1080 "
                                 "D192), Poisson 30 Hz each, 3 s, latency arrival to map in "
                                 "host memory" + (", learned proposal on the D128 cameras"
                                                  if prop else ""))
    return out


def _serial_ms(mpv, pairs, stream, steps, warmup):
    """Milliseconds for matching the batch's pairs one after another (single-pair calls)."""
    import torch
    cls = {}
    for p in pairs:
        H, W = p["disp"].shape
        key = (H, W, p["max_disparity"])
        if key not in cls:
            ctx = mpv.mpv_create(0)
            mpv.mpv_set_params(ctx, mpv.mpv_default_params(**dict(PARAMS,
                                                                  max_disparity=key[2])))
            cls[key] = (ctx, torch.empty_like(p["left"]), torch.empty_like(p["right"]),
                        torch.empty_like(p["disp"]))

    def once():
        for p in pairs:
            H, W = p["disp"].shape
            ctx, l, r, d = cls[(H, W, p["max_disparity"])]
            l.copy_(p["left"])
            r.copy_(p["right"])
            mpv.mpv_match(ctx, l, r, d, stream)
    for _ in range(max(1, warmup)):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        once()
    e1.record(stream)
    torch.cuda.synchronize()
    for ctx, *_ in cls.values():
        mpv.mpv_destroy(ctx)
    return e0.elapsed_time(e1) / steps


def _gen_pair(spec):
    from paper_2001_09678_gb300 import synth
    seed, W, H, D = spec
    L, R, _ = synth.slanted_pair(W, H, seed=seed, d_max=min(120.0, D - 8.0))
    return L, R


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=("mine", "reference"), default="mine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the learned, batched and served configurations")
    ap.add_argument("--workload", choices=("frame", "batch64"), default="frame",
                    help="frame: the 1280x720 D=128 pair (default); batch64: the mixed batch")
    ap.add_argument("--variant", choices=tuple(VARIANTS), default="plain",
                    help="layered merge and/or gradient-weighted TV on the frame workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batch64" and args.impl == "mine":
        run_batch64(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
