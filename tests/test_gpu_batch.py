"""Batched matching (one CUDA graph per batch signature) and the autotuner.

Every pair of a batch must equal the same pair matched alone and the oracle, bit for bit,
on first submission (capture) and on replay.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402

BASE = dict(num_scales=3, num_paths=8, p1=10, trunc=30)


@pytest.fixture(scope="module")
def mpv():
    from paper_2001_09678_gb300 import build, mpv as m
    build.build()
    m.load()
    return m


def _u16(t):
    return t.cpu().numpy().view(np.uint16)


def _oracle(L, R, D):
    p = ref.params(max_disparity=D, window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1,
                   ssim_window=5, **BASE)
    return ref.match(L, R, p)


def _single(m, L, R, D):
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(max_disparity=D, **BASE))
        l = torch.from_numpy(L).cuda()
        r = torch.from_numpy(R).cuda()
        d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        m.mpv_match(ctx, l, r, d)
        m.mpv_sync(ctx)
        return _u16(d)
    finally:
        m.mpv_destroy(ctx)


def _run_batch(m, ctx, pairs_np, repeats=2):
    tens = []
    for (L, R, D) in pairs_np:
        tens.append(dict(left=torch.from_numpy(L).cuda(), right=torch.from_numpy(R).cuda(),
                         disp=torch.full(L.shape, -2, dtype=torch.int16, device="cuda"),
                         max_disparity=D))
    outs = []
    for _ in range(repeats):
        for t in tens:
            t["disp"].fill_(-2)
        m.mpv_match_batch(ctx, tens)
        m.mpv_sync(ctx)
        outs.append([_u16(t["disp"]) for t in tens])
    return outs


def test_small_mixed_batch_equals_alone_and_oracle(mpv):
    specs = [(160, 96, 32, 1), (200, 120, 48, 2), (96, 64, 16, 3), (160, 96, 32, 4),
             (200, 120, 48, 5), (96, 64, 16, 6)]
    pairs = []
    for W, H, D, seed in specs:
        L, R, _ = synth.slanted_pair(W, H, seed=seed, d_max=D - 4)
        pairs.append((L, R, D))
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=128, **BASE))
        runs = _run_batch(mpv, ctx, pairs, repeats=3)      # capture, then two replays
    finally:
        mpv.mpv_destroy(ctx)
    for i, (L, R, D) in enumerate(pairs):
        want = _oracle(L, R, D)
        alone = _single(mpv, L, R, D)
        assert np.array_equal(alone, want), i
        for run in runs:
            assert np.array_equal(run[i], want), i


def test_autotune_choice_does_not_change_results(mpv):
    L, R, _ = synth.slanted_pair(320, 180, seed=9, d_max=60)
    D = 64
    want = _oracle(L, R, D)
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=D, **BASE))
        l = torch.from_numpy(L).cuda()
        r = torch.from_numpy(R).cuda()
        d = torch.zeros(L.shape, dtype=torch.int16, device="cuda")
        lanes = mpv.mpv_autotune(ctx, dict(left=l, right=r, disp=d))
        assert lanes in (4, 8)
        assert mpv.mpv_autotune(ctx, dict(left=l, right=r, disp=d)) == lanes   # cached
        d.fill_(0)
        mpv.mpv_match(ctx, l, r, d)
        mpv.mpv_sync(ctx)
    finally:
        mpv.mpv_destroy(ctx)
    assert np.array_equal(_u16(d), want)


def _gen(spec):
    seed, W, H, D = spec
    L, R, _ = synth.slanted_pair(W, H, seed=seed, d_max=min(120.0, D - 8.0))
    return L, R


def _gen_and_oracle(spec):
    seed, W, H, D = spec
    L, R = _gen(spec)
    return _oracle(L, R, D)


def test_mixed_batch_of_64(mpv):
    # 16 x 640x480 (D=64), 32 x 1280x720 (D=128), 16 x 1920x1080 (D=192), seeds 1000+i;
    # every pair is checked against the oracle (computed in worker processes, largest
    # pairs first so that the pool drains evenly)
    specs = synth.mixed_batch_specs()
    assert len(specs) == 64
    order = sorted(range(64), key=lambda i: -specs[i][1] * specs[i][2] * specs[i][3])
    ctx_mp = mp.get_context("spawn")
    with ctx_mp.Pool(min(32, os.cpu_count() or 4)) as pool:
        oracle_async = pool.map_async(_gen_and_oracle, [specs[i] for i in order], chunksize=1)
        images = pool.map(_gen, specs)
        want = dict(zip(order, oracle_async.get()))
    pairs = [(L, R, spec[3]) for (L, R), spec in zip(images, specs)]
    runs = {}
    for mode in ("PERSISTENT", "STREAMS"):          # both batch paths
        ctx = mpv.mpv_create(0)
        try:
            mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=128, **BASE))
            mpv.mpv_set_batch_mode(ctx, getattr(mpv, "MPV_BATCH_" + mode))
            runs[mode] = _run_batch(mpv, ctx, pairs, repeats=2)
            assert mpv.mpv_batch_info(ctx)[0] == (mode == "PERSISTENT")
        finally:
            mpv.mpv_destroy(ctx)
    for i in range(64):
        for mode, r in runs.items():
            assert np.array_equal(r[0][i], want[i]), f"pair {i} ({mode}) differs from the oracle"
    runs = runs["PERSISTENT"]
    for i, (L, R, D) in enumerate(pairs):
        assert np.array_equal(runs[0][i], runs[1][i]), f"pair {i}: replay differs"
    for i in (1, 20, 50):
        L, R, D = pairs[i]
        assert np.array_equal(runs[0][i], _single(mpv, L, R, D)), f"pair {i}: batch != alone"


def test_persistent_batch_and_its_bounded_wait(mpv):
    # batches of supported pairs run through the persistent kernel; a stage that can
    # never complete ends the launch by the bounded wait (about 1 ms here) with
    # MPV_ERR_TIMEOUT from mpv_sync, and the context matches correctly afterwards
    specs = [(160, 96, 32, 11), (200, 120, 48, 12), (96, 64, 16, 13), (256, 144, 64, 14)]
    pairs = [(synth.slanted_pair(W, H, seed=s, d_max=D - 4)[:2]) + (D,) for W, H, D, s in specs]
    want = [_oracle(L, R, D) for L, R, D in pairs]
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=128, **BASE))
        mpv.mpv_set_batch_mode(ctx, mpv.MPV_BATCH_PERSISTENT)
        # other content through the same workspace first: every launch must clear what it
        # accumulates into, whatever the memory held before
        _run_batch(mpv, ctx, [(R, L, D) for L, R, D in pairs], repeats=1)
        runs = _run_batch(mpv, ctx, pairs, repeats=2)
        persistent, lanes, queues, cb, pms, sms, occ = mpv.mpv_batch_info(ctx)
        assert persistent == 1 and lanes in (4, 8) and queues in (16, 32) and cb in (2, 8) and occ in (2, 3, 4)
        assert pms > 0 and sms > 0                     # the tuner timed both paths
        for run in runs:
            for got, w in zip(run, want):
                assert np.array_equal(got, w)
        mpv.mpv_debug_batch_stall(ctx, 2_000_000)
        tens = [dict(left=torch.from_numpy(L).cuda(), right=torch.from_numpy(R).cuda(),
                     disp=torch.full(L.shape, -2, dtype=torch.int16, device="cuda"),
                     max_disparity=D) for L, R, D in pairs]
        mpv.mpv_match_batch(ctx, tens)
        with pytest.raises(mpv.MpvError) as e:
            mpv.mpv_sync(ctx)
        assert e.value.status == mpv.MPV_ERR_TIMEOUT
        mpv.mpv_sync(ctx)                              # reported once
        runs = _run_batch(mpv, ctx, pairs, repeats=1)  # still usable, still exact
        for got, w in zip(runs[0], want):
            assert np.array_equal(got, w)
    finally:
        mpv.mpv_destroy(ctx)


def test_stream_path_when_persistent_does_not_apply(mpv):
    # a gradient table is outside the persistent kernel: the batch runs as a graph of
    # streams and still equals the oracle
    pairs = [synth.slanted_pair(160, 96, seed=21 + i, d_max=28)[:2] + (32,) for i in range(3)]
    lut = np.full(256, 10, np.int32)
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=32, **BASE))
        mpv.mpv_set_gradient_penalty(ctx, lut)
        runs = _run_batch(mpv, ctx, pairs, repeats=1)
        assert mpv.mpv_batch_info(ctx)[0] == 0
    finally:
        mpv.mpv_destroy(ctx)
    for (L, R, D), got in zip(pairs, runs[0]):
        assert np.array_equal(got, _oracle(L, R, D))
