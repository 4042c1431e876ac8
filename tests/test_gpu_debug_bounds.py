"""The bounds-checked build of the library (MPV_DEBUG_BOUNDS) on tiny and small pairs.

In that build every risky device index (the passes' prefetch and re-indexing, the
gradient table, the summed-volume reductions, the cost kernel's staged columns, the
seeding's parent pixels) is checked before use; a failed check records its site in a
device error word and skips the access, and mpv_sync returns MPV_ERR_INTERNAL.  Pairs
of 5-16 pixels (scan paths along diagonals of 1-3 pixels at every corner), 64x48 through
three scales, the gradient table and the layered merge, single and batched, must run
without a failed check and equal the oracle.  Runs in a child process that loads
libmpv_debug.so.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
from oracle import ref
from paper_2001_09678_gb300 import mpv, synth
mpv.load()
def lut(p1):
    g = np.arange(256, dtype=np.float64)
    return np.floor(p1 * np.exp(-g / 8.0) + 0.5).astype(np.int32)
cases = [  # (W, H, D, scales, paths, merge, gradient)
    (5, 8, 4, 1, 8, 0, False), (8, 5, 5, 1, 8, 0, False), (5, 5, 5, 1, 4, 0, False),
    (16, 16, 8, 1, 8, 0, False), (16, 16, 8, 2, 8, 0, False), (16, 16, 8, 1, 8, 0, True),
    (64, 48, 32, 3, 8, 0, False), (64, 48, 32, 3, 8, 0, True), (64, 48, 32, 3, 8, 1, False),
    (64, 48, 32, 3, 8, 1, True), (23, 17, 16, 2, 8, 0, False),
]
n = 0
for W, H, D, S, P, merge, grad in cases:
    L, R, _ = synth.slanted_pair(W, H, seed=W * 100 + H + D, d_max=max(1.0, D - 2.0))
    kw = dict(max_disparity=D, num_scales=S, num_paths=P, p1=10, trunc=30, merge_mode=merge)
    t = lut(10) if grad else None
    want = ref.match(L, R, ref.params(window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1,
                                      ssim_window=5, grad_lut=t, **kw))
    ctx = mpv.mpv_create(0)
    mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
    if grad:
        mpv.mpv_set_gradient_penalty(ctx, t)
    l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
    d = torch.full((H, W), -2, dtype=torch.int16, device="cuda")
    mpv.mpv_match(ctx, l, r, d)
    mpv.mpv_sync(ctx)        # raises MpvError(MPV_ERR_INTERNAL) on a failed check
    got = d.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, want), (W, H, D, S, P, merge, grad, int((got != want).sum()))
    mpv.mpv_destroy(ctx)
    n += 1
# a batch of small pairs through both batch paths
pairs = [synth.slanted_pair(W, H, seed=70 + W, d_max=D - 2.0)[:2] + (D,)
         for W, H, D in ((64, 48, 32), (23, 17, 16), (16, 16, 16), (40, 24, 16))]
for mode in (mpv.MPV_BATCH_PERSISTENT, mpv.MPV_BATCH_STREAMS):
    ctx = mpv.mpv_create(0)
    mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=32, num_scales=2))
    mpv.mpv_set_batch_mode(ctx, mode)
    tens = [dict(left=torch.from_numpy(L).cuda(), right=torch.from_numpy(R).cuda(),
                 disp=torch.full(L.shape, -2, dtype=torch.int16, device="cuda"), max_disparity=D)
            for L, R, D in pairs]
    mpv.mpv_match_batch(ctx, tens)
    mpv.mpv_sync(ctx)
    for (L, R, D), t in zip(pairs, tens):
        want = ref.match(L, R, ref.params(max_disparity=D, num_scales=2, num_paths=8, p1=10,
                                          trunc=30, window=0, block=(0, 0, 0, 0), lr_check=1,
                                          lr_tol=1, ssim_window=5))
        assert np.array_equal(t["disp"].cpu().numpy().view(np.uint16), want), (mode, L.shape)
    mpv.mpv_destroy(ctx)
    n += 1
print("bounds-checked runs ok:", n)
'''


def test_bounds_checked_build_on_small_pairs():
    from paper_2001_09678_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, MPV_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "bounds-checked runs ok: 13" in r.stdout
