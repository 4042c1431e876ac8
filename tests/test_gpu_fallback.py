"""The learned proposal's exact fallback, and what the trained network gains.

A learned-proposal match decides on the device, after its winner-take-all, whether the
proposed windows missed (more than fallback_edge_bp of every 10000 matched pixels won on
a window edge while the range went on past it) and then re-matches the frame with the
pyramid (Section 3.4) or at full range on one scale, the exact method.  A network that
predicts one constant centre must therefore end with exactly the oracle's pyramid (or
full-range) result.  The gain test runs the committed network on held-out 1280x720 pairs
against full-range single-scale MPV, next to an untrained and a constant-centre network.
"""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2001_09678_gb300", "weights", "proposal_d128_s3.bin")
KW = dict(max_disparity=64, num_scales=3, num_paths=8, p1=10, trunc=30)


@pytest.fixture(scope="module")
def m():
    from paper_2001_09678_gb300 import build, mpv
    build.build()
    mpv.load()
    return mpv


@pytest.fixture(scope="module")
def constant_net():
    # predicts disparity 0.5 * D everywhere: right only where the scene happens to be
    from paper_2001_09678_gb300 import learn
    fd, path = tempfile.mkstemp(suffix=".bin")
    os.close(fd)
    learn.save_weights(path, learn._constant_layers(2 + 16, 0.5), KW["max_disparity"], 4)
    yield path
    os.unlink(path)


def _pair():
    return synth.slanted_pair(320, 192, seed=77, d_max=56)[:2]


def _learned(m, weights, L, R, **kw):
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(proposal=m.MPV_PROPOSAL_LEARNED,
                                                   **dict(KW, **kw)))
        m.mpv_load_proposal_weights(ctx, weights)
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        out = []
        for _ in range(2):      # the second call replays the cached graph
            d.fill_(-2)
            m.mpv_match(ctx, l, r, d)
            m.mpv_sync(ctx)
            out.append(d.cpu().numpy().view(np.uint16))
        assert np.array_equal(out[0], out[1])
        return out[1], m.mpv_proposal_stats(ctx), m.mpv_proposal_fallbacks(ctx)
    finally:
        m.mpv_destroy(ctx)


def _oracle(L, R, **kw):
    p = dict(KW, window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1, ssim_window=5)
    p.update(kw)
    return ref.match(L, R, ref.params(**p))


def test_missed_windows_fall_back_to_the_pyramid(m, constant_net):
    L, R = _pair()
    got, (hits, px), (frames, falls) = _learned(m, constant_net, L, R)
    assert px == 2 * L.size and hits * 10000 > 1500 * px      # the default threshold
    assert (frames, falls) == (2, 2)
    assert np.array_equal(got, _oracle(L, R))


def test_gated_launches_without_graphs(m, constant_net):
    # while profiling the matcher launches directly: the fallback's launches are then
    # always enqueued and return at once unless the decision opened them
    L, R = _pair()
    pyr = _oracle(L, R)
    for bp, expect_fall in ((1500, True), (10000, False)):
        ctx = m.mpv_create(0)
        try:
            m.mpv_set_params(ctx, m.mpv_default_params(proposal=m.MPV_PROPOSAL_LEARNED,
                                                       fallback_edge_bp=bp, **KW))
            m.mpv_load_proposal_weights(ctx, constant_net)
            m.mpv_profile_enable(ctx, True)
            l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
            d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
            m.mpv_match(ctx, l, r, d)
            m.mpv_sync(ctx)
            got = d.cpu().numpy().view(np.uint16)
            assert m.mpv_proposal_fallbacks(ctx) == (1, int(expect_fall))
        finally:
            m.mpv_destroy(ctx)
        assert np.array_equal(got, pyr) == expect_fall


def test_missed_windows_fall_back_to_full_range(m, constant_net):
    L, R = _pair()
    got, _, (frames, falls) = _learned(m, constant_net, L, R, fallback=m.MPV_FALLBACK_FULL)
    assert (frames, falls) == (2, 2)
    assert np.array_equal(got, _oracle(L, R, num_scales=1))


def test_threshold_and_no_fallback(m, constant_net):
    L, R = _pair()
    pyr = _oracle(L, R)
    # never (no pixel count can exceed all of them) and none: the network's own result
    never, (hits, px), (frames, falls) = _learned(m, constant_net, L, R, fallback_edge_bp=10000)
    assert (frames, falls) == (2, 0)
    none, _, (frames, falls) = _learned(m, constant_net, L, R, fallback=m.MPV_FALLBACK_NONE)
    assert (frames, falls) == (0, 0)          # no decision is taken at all
    assert np.array_equal(never, none)
    assert (never != pyr).mean() > 0.05
    # just below / at the frame's own ratio
    bp = hits * 10000 // px
    below, _, (_, falls) = _learned(m, constant_net, L, R, fallback_edge_bp=int(bp) - 1)
    assert falls == 2 and np.array_equal(below, pyr)
    at, _, (_, falls) = _learned(m, constant_net, L, R, fallback_edge_bp=int(bp) + 1)
    assert falls == 0 and np.array_equal(at, none)


def test_invalid_fallback_parameters_are_rejected(m):
    ctx = m.mpv_create(0)
    try:
        for bad in (dict(fallback=3), dict(fallback=-1), dict(fallback_edge_bp=-1),
                    dict(fallback_edge_bp=10001), dict(windows=(8, -1))):
            with pytest.raises(m.MpvError):
                m.mpv_set_params(ctx, m.mpv_default_params(**bad))
    finally:
        m.mpv_destroy(ctx)


def test_trained_network_gain_on_held_out_pairs(m):
    """20 held-out 1280x720 D=128 pairs (seeds 900000+, never trained on), the network's
    own windows (no fallback): the trained proposal stays within 1 % bad pixels (> 1 px)
    of full-range single-scale MPV; untrained and constant-centre networks do not."""
    from paper_2001_09678_gb300 import learn
    res = learn.evaluate(WEIGHTS, npairs=20, log=lambda *_: None)
    trained = res["trained"]["bad_pixel_rate"]
    assert trained <= 0.01, res
    for name in ("untrained", "constant"):
        assert res[name]["bad_pixel_rate"] >= max(0.10, 10 * trained), (name, res)
        assert res[name]["edge_hit_rate"] > res["trained"]["edge_hit_rate"], (name, res)
    # with the default fallback the constant network's frames all fall back and its
    # result becomes the pyramid's
    assert res["constant"]["fallbacks_with_default"] == 20, res
    assert res["trained"]["fallbacks_with_default"] == 0, res
