"""mpv_match_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (a host framework owning a fixed device pool, a real-time loop that must not
allocate once running, a plug-in in a process whose device memory is budgeted elsewhere)
get the whole matcher with its scratch in the library's fixed device array.  Its output
must equal mpv_match's on the same pair, on consecutive calls that reuse the array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def mpv():
    from paper_2001_09678_gb300 import build, mpv as m
    build.build()
    m.load()
    return m


def _u16(t):
    return t.cpu().numpy().view(np.uint16)


def _match_with_context(m, params, left, right):
    ctx = m.mpv_create(torch.cuda.current_device())
    try:
        m.mpv_set_params(ctx, params)
        d = torch.full(left.shape, -3, dtype=torch.int16, device="cuda")
        m.mpv_match(ctx, left, right, d)
        m.mpv_sync(ctx)
        return _u16(d)
    finally:
        m.mpv_destroy(ctx)


def test_noalloc_matches_context_path_on_consecutive_calls(mpv):
    params = mpv.mpv_default_params(max_disparity=64, num_scales=3, num_paths=8)
    ora = ref.params(max_disparity=64, num_scales=3, num_paths=8, p1=params.p1,
                     trunc=params.trunc, window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1,
                     ssim_window=5)
    outs = []
    # two different pairs in a row: the second call reuses the first call's array
    for seed, (W, H) in ((41, (640, 480)), (42, (600, 440))):
        L, R, _ = synth.slanted_pair(W, H, seed=seed, d_max=60)
        left = torch.from_numpy(L).cuda()
        right = torch.from_numpy(R).cuda()
        d = torch.full((H, W), -3, dtype=torch.int16, device="cuda")
        mpv.mpv_match_noalloc(params, left, right, d)
        torch.cuda.synchronize()
        got = _u16(d)
        want = _match_with_context(mpv, params, left, right)
        assert np.array_equal(got, want), f"{(got != want).sum()} pixels differ"
        exact = ref.match(L, R, ora)
        assert np.array_equal(got, exact), f"{(got != exact).sum()} pixels differ from the oracle"
        outs.append(got)
    assert (outs[0] != 0xFFFF).mean() > 0.5


def test_noalloc_rejects_pairs_beyond_its_scratch(mpv):
    params = mpv.mpv_default_params(max_disparity=128, num_scales=3, num_paths=8)
    left = torch.zeros((720, 1280), dtype=torch.uint8, device="cuda")
    d = torch.full((720, 1280), 9, dtype=torch.int16, device="cuda")
    with pytest.raises(mpv.MpvError) as e:
        mpv.mpv_match_noalloc(params, left, left, d)
    assert e.value.status == mpv.MPV_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert (d == 9).all()
