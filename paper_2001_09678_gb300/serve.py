"""Serving driver: simulated cameras feeding the library's continuous-batching server.

Each camera produces frames as a Poisson process (rate `hz`, its own seed) cycling over
a pool of pre-generated pairs of its size.  Frames are submitted to mpv_server_* (the
native scheduler in libmpv.so) at their arrival times; the server admits them as slots
and device memory allow and runs frames of different cameras concurrently.  Latency is
measured from submission to the map reaching host memory.

    python -m paper_2001_09678_gb300.serve [--seconds 10] [--budget-mb 0]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

from . import mpv, synth

# camera layout of the 8-camera workload: (count, width, height, max disparity)
CAMERAS_8 = ((2, 640, 480, 64), (4, 1280, 720, 128), (2, 1920, 1080, 192))


def camera_specs(layout=CAMERAS_8):
    out, cid = [], 0
    for n, W, H, D in layout:
        for _ in range(n):
            out.append((cid, W, H, D))
            cid += 1
    return out


def arrivals(camera: int, hz: float, seconds: float, seed: int = 0):
    """Poisson arrival times (s) of one camera: exponential gaps from its own stream."""
    n = int(seconds * hz * 2 + 20)
    u = synth.uniform01(seed * 131 + camera, 77, (n,))
    t = np.cumsum(-np.log1p(-u) / hz)
    return t[t < seconds]


def _make_frame(args):
    W, H, D, k = args
    L, R, _ = synth.slanted_pair(W, H, seed=50000 + 97 * W + k, d_max=min(120.0, D - 8.0))
    return L, R


def frame_pools(sizes, per_size: int, workers: int | None = None):
    """{(W, H, D): [(left, right), ...]} generated in a spawn pool."""
    jobs = [(W, H, D, k) for (W, H, D) in sizes for k in range(per_size)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or min(16, os.cpu_count() or 4)) as pool:
        frames = pool.map(_make_frame, jobs)
    pools = {}
    for (W, H, D, _k), fr in zip(jobs, frames):
        pools.setdefault((W, H, D), []).append(fr)
    return pools


def _warm(srv, cams, pools):
    """One frame per camera, not timed: makes every camera's state resident."""
    keep = []
    for cid, W, H, D in cams:
        L, R = pools[(W, H, D)][0]
        disp = np.empty((H, W), np.uint16)
        keep.append(disp)
        mpv.mpv_server_submit(srv, cid, L, R, disp, (1 << 62) + cid)
    done = 0
    while done < len(cams):
        done += len(mpv.mpv_server_poll(srv))
        time.sleep(1e-4)


def run(cams, pools, seconds=5.0, hz=30.0, budget=0, max_inflight=8, params=None,
        keep_outputs=False, seed=0, warm=True, proposal=None):
    """Serves every camera's arrivals for `seconds`; returns latencies and stats.
    proposal: weights of the learned window proposal (cameras whose range fits it)."""
    params = params or mpv.mpv_default_params()
    srv = mpv.mpv_server_create(params, hbm_budget=budget, max_inflight=max_inflight)
    try:
        if proposal:
            mpv.mpv_server_set_proposal(srv, proposal)
        events = []
        for cid, W, H, D in cams:
            mpv.mpv_server_add_camera(srv, cid, W, H, D)
            for k, t in enumerate(arrivals(cid, hz, seconds, seed)):
                events.append((t, cid, k, W, H, D))
        if warm and budget == 0:
            _warm(srv, cams, pools)
        events.sort()
        outputs = {}
        pending = {}
        lat, status, waits, service, sizes, t_arrive = [], [], [], [], [], []
        t0 = time.perf_counter()
        i = 0
        n_done = 0
        lateness = []
        while n_done < len(events):
            now = time.perf_counter() - t0
            while i < len(events) and events[i][0] <= now:
                t, cid, k, W, H, D = events[i]
                L, R = pools[(W, H, D)][k % len(pools[(W, H, D)])]
                disp = np.empty((H, W), np.uint16)
                rid = i
                pending[rid] = (L, R, disp, cid, k)
                mpv.mpv_server_submit(srv, cid, L, R, disp, rid)
                lateness.append(now - t)
                i += 1
            for c in mpv.mpv_server_poll(srv):
                L, R, disp, cid, k = pending.pop(c.request_id)
                lat.append(c.t_done_ms - c.t_submit_ms)
                waits.append(c.t_start_ms - c.t_submit_ms)
                service.append(c.t_done_ms - c.t_start_ms)
                sizes.append(L.shape[1])
                t_arrive.append(c.t_submit_ms)
                status.append(c.status)
                if keep_outputs:
                    outputs[c.request_id] = (cid, k, disp)
                n_done += 1
            if i < len(events) and events[i][0] > now + 2e-4:
                time.sleep(1e-4)
        wall = time.perf_counter() - t0
        stats = mpv.mpv_server_stats(srv)
    finally:
        mpv.mpv_server_destroy(srv)
    lat = np.array(lat)
    ok = np.array(status) == 0
    waits, service, sizes = np.array(waits), np.array(service), np.array(sizes)

    def pct(a, q):
        return float(np.percentile(a, q)) if a.size else None

    by_size = {}
    for w in sorted(set(sizes.tolist())):
        m = ok & (sizes == w)
        by_size[f"width{w}"] = dict(frames=int(m.sum()), p50_ms=pct(lat[m], 50),
                                    p99_ms=pct(lat[m], 99), service_p50_ms=pct(service[m], 50))
    return dict(
        frames=int(len(events)), ok=int(ok.sum()), wall_s=wall,
        fps=float(ok.sum() / wall),
        p50_ms=float(np.percentile(lat[ok], 50)) if ok.any() else None,
        p99_ms=float(np.percentile(lat[ok], 99)) if ok.any() else None,
        p90_ms=pct(lat[ok], 90), max_ms=float(lat[ok].max()) if ok.any() else None,
        queue_wait_p50_ms=pct(waits[ok], 50), queue_wait_p99_ms=pct(waits[ok], 99),
        service_p50_ms=pct(service[ok], 50), service_p99_ms=pct(service[ok], 99),
        by_size=by_size,
        max_submit_lag_ms=float(1e3 * max(lateness)) if lateness else 0.0,
        submit_lag_p99_ms=float(1e3 * np.percentile(lateness, 99)) if lateness else 0.0,
        evictions=int(stats["evictions"]), peak_inflight=int(stats["peak_inflight"]),
        outputs=outputs,
    )


def main():
    # every kernel loaded at start-up: a lazy load while frames are in flight holds the host
    # (set before CUDA initialises; an explicit setting in the environment wins)
    os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--hz", type=float, default=30.0)
    ap.add_argument("--budget-mb", type=float, default=0.0)
    ap.add_argument("--max-inflight", type=int, default=8)
    ap.add_argument("--pool", type=int, default=8)
    ap.add_argument("--learned", default=None,
                    help="weights of the learned proposal (cameras whose range fits it)")
    args = ap.parse_args()
    mpv.load()
    cams = camera_specs()
    sizes = sorted({(W, H, D) for _, W, H, D in cams})
    pools = frame_pools(sizes, args.pool)
    import torch
    torch.cuda.init()
    res = run(cams, pools, seconds=args.seconds, hz=args.hz,
              budget=int(args.budget_mb * 2**20), max_inflight=args.max_inflight,
              proposal=args.learned)
    res.pop("outputs")
    mode = ("learned proposal where the network fits (1280x720 D128), pyramid elsewhere"
            if args.learned else "plain 3-scale MPV")
    res["workload"] = "8 cameras (2x640x480 D64, 4x1280x720 D128, 2x1920x1080 D192), " \
                      f"Poisson {args.hz:g} Hz each, {mode}, 8 paths, LR"
    print(json.dumps(res))


if __name__ == "__main__":
    main()
