"""The learned window proposal inside the matcher.

Parity is on the matcher given the same windows: with the windows the network produced
(read back from the device), the oracle's finest level must reproduce the device's
left-right-checked map bit for bit.  The network input is checked against the oracle's
pyramid and cost volume to one BF16 rounding.
"""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cnn_ref, ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402

KW = dict(max_disparity=64, num_scales=3, num_paths=8, p1=10, trunc=30)
# the network's own result, not the exact fallback's (tests/test_gpu_fallback.py covers that)
NOFB = dict(fallback=0)


@pytest.fixture(scope="module")
def m():
    from paper_2001_09678_gb300 import build, mpv
    build.build()
    mpv.load()
    return mpv


def _weights_file(cin0, seed):
    from paper_2001_09678_gb300 import learn
    fd, path = tempfile.mkstemp(suffix=".bin")
    os.close(fd)
    layers = learn.init_weights(cin0, seed=seed)
    learn.save_weights(path, layers, KW["max_disparity"], 4)
    return path, layers


def test_learned_match_equals_oracle_given_windows(m):
    L, R, _ = synth.slanted_pair(256, 160, seed=31, d_max=56)
    path, _ = _weights_file(2 + 16, seed=1)
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(proposal=m.MPV_PROPOSAL_LEARNED, **NOFB, **KW))
        m.mpv_load_proposal_weights(ctx, path)
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        m.mpv_match(ctx, l, r, d)
        m.mpv_sync(ctx)
        hits, pixels = m.mpv_proposal_stats(ctx)
        assert pixels == 2 * 256 * 160 and 0 <= hits <= pixels
        los = []
        for view in (0, 1):
            lo = torch.zeros(L.shape, dtype=torch.int16, device="cuda")
            m.mpv_debug_stage(ctx, l, r, view, 2, lo=lo)
            los.append(lo.cpu().numpy().view(np.uint16).astype(np.int32))
        got = d.cpu().numpy().view(np.uint16)
    finally:
        m.mpv_destroy(ctx)
        os.unlink(path)
    Dw = 17
    assert all((lo >= 0).all() and (lo <= 64 - Dw).all() for lo in los)
    maps = []
    for view, lo in zip((0, 1), los):
        I0, I1 = (L, R) if view == 0 else (np.ascontiguousarray(R[:, ::-1]),
                                           np.ascontiguousarray(L[:, ::-1]))
        Cv = ref.cost_volume(I0, I1, 5, Dw, lo=lo)
        S = ref.aggregate(Cv, 8, 10, 30, lo=lo)
        maps.append(ref.wta(S, lo=lo))
    want = ref.lr_check(maps[0], maps[1][:, ::-1], 1)
    assert np.array_equal(got, want), f"{(got != want).sum()} pixels differ"


def test_features_match_oracle_pyramid_and_cost(m):
    L, R, _ = synth.slanted_pair(200, 120, seed=32, d_max=56)
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(**KW))
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        out = torch.empty((18, 30, 50), dtype=torch.bfloat16, device="cuda")
        m.mpv_proposal_features(ctx, l, r, 0, out)
        torch.cuda.synchronize()
        got = out.float().cpu().numpy().astype(np.float64)
    finally:
        m.mpv_destroy(ctx)
    L0 = ref.downsample2(ref.downsample2(L))
    R0 = ref.downsample2(ref.downsample2(R))
    C0 = ref.cost_volume(L0, R0, 5, 16)
    want = np.concatenate([(L0[None] / 255.0 - 0.5), (R0[None] / 255.0 - 0.5),
                           np.moveaxis(C0, 2, 0) / 255.0])
    # one BF16 rounding of the exact value (relative 2^-8)
    assert np.all(np.abs(got - want) <= np.abs(want) * 2.0**-8 + 1e-7)


def test_learned_requires_weights_and_matching_channels(m):
    L, R, _ = synth.slanted_pair(128, 96, seed=33, d_max=40)
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(proposal=m.MPV_PROPOSAL_LEARNED, **NOFB, **KW))
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        d = torch.zeros(L.shape, dtype=torch.int16, device="cuda")
        with pytest.raises(m.MpvError):          # no network loaded
            m.mpv_match(ctx, l, r, d)
        path, _ = _weights_file(2 + 32, seed=2)   # built for D_top = 32, not 16
        m.mpv_load_proposal_weights(ctx, path)
        os.unlink(path)
        with pytest.raises(m.MpvError):
            m.mpv_match(ctx, l, r, d)
        with pytest.raises(m.MpvError):
            m.mpv_load_proposal_weights(ctx, "/nonexistent/weights.bin")
    finally:
        m.mpv_destroy(ctx)


def test_pipeline_prediction_equals_the_network_kernels(m):
    # the matcher runs the network channels-last; the training kernels run it planar: the
    # same BF16 operands and the same FP32 accumulation order give the same prediction
    from paper_2001_09678_gb300 import learn
    L, R, _ = synth.slanted_pair(200, 120, seed=34, d_max=56)
    path, layers = _weights_file(2 + 16, seed=5)
    ctx = m.mpv_create(0)
    pyr = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(proposal=m.MPV_PROPOSAL_LEARNED, **NOFB, **KW))
        m.mpv_load_proposal_weights(ctx, path)
        m.mpv_set_params(pyr, m.mpv_default_params(**KW))
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        Wq, Hq = m.mpv_level_info(ctx, 200, 120, 0)[:2]
        net = learn.Net(layers)
        for view in (0, 1):
            q = torch.full((Hq, Wq), -1.0, device="cuda")
            m.mpv_proposal_predict(ctx, l, r, view, q)
            feat = torch.empty((18, Hq, Wq), dtype=torch.bfloat16, device="cuda")
            m.mpv_proposal_features(pyr, l, r, view, feat)
            torch.cuda.synchronize()
            pred, _ = net.forward(feat[None])
            assert torch.equal(q, pred[0, 0]), float((q - pred[0, 0]).abs().max())
    finally:
        m.mpv_destroy(ctx)
        m.mpv_destroy(pyr)
        os.unlink(path)


def test_full_size_learned_match_equals_oracle_given_windows(m):
    # the committed network at its own configuration: 1280x720, D = 128, 3 scales, the
    # finest level searching centre +- 8 (17 labels, a padded 32-label stride)
    weights = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "paper_2001_09678_gb300", "weights", "proposal_d128_s3.bin")
    L, R, _ = synth.slanted_pair(1280, 720, seed=900123)
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(proposal=m.MPV_PROPOSAL_LEARNED, **NOFB,
                                                   max_disparity=128, num_scales=3,
                                                   num_paths=8, p1=10, trunc=30))
        m.mpv_load_proposal_weights(ctx, weights)
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        m.mpv_match(ctx, l, r, d)
        m.mpv_sync(ctx)
        los = []
        for view in (0, 1):
            lo = torch.zeros(L.shape, dtype=torch.int16, device="cuda")
            m.mpv_debug_stage(ctx, l, r, view, 2, lo=lo)
            los.append(lo.cpu().numpy().view(np.uint16).astype(np.int32))
        got = d.cpu().numpy().view(np.uint16)
    finally:
        m.mpv_destroy(ctx)
    Dw = 17
    assert all((lo >= 0).all() and (lo <= 128 - Dw).all() for lo in los)
    maps = []
    for view, lo in zip((0, 1), los):
        I0, I1 = (L, R) if view == 0 else (np.ascontiguousarray(R[:, ::-1]),
                                           np.ascontiguousarray(L[:, ::-1]))
        Cv = ref.cost_volume(I0, I1, 5, Dw, lo=lo)
        S = ref.aggregate(Cv, 8, 10, 30, lo=lo)
        maps.append(ref.wta(S, lo=lo))
    want = ref.lr_check(maps[0], maps[1][:, ::-1], 1)
    assert np.array_equal(got, want), f"{(got != want).sum()} pixels differ"
    assert (got != 0xFFFF).mean() > 0.6     # occlusions and the image border fail the check
