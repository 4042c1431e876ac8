"""Continuous-batching server: results in the mix equal results alone, frames of several
cameras overlap on the GPU, the device-memory budget is honoured."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2001_09678_gb300 import serve, synth  # noqa: E402

CAMS = [(0, 160, 96, 32), (1, 160, 96, 32), (2, 256, 144, 64), (3, 256, 144, 64)]


@pytest.fixture(scope="module")
def setup():
    pools = {}
    for (W, H, D) in sorted({(W, H, D) for _, W, H, D in CAMS}):
        pools[(W, H, D)] = [synth.slanted_pair(W, H, seed=700 + 13 * k + W, d_max=D - 8)[:2]
                            for k in range(3)]
    from paper_2001_09678_gb300 import build, mpv
    build.build()
    mpv.load()
    # each pool frame matched alone
    alone = {}
    for (W, H, D), frames in pools.items():
        ctx = mpv.mpv_create(0)
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=D))
        for k, (L, R) in enumerate(frames):
            l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
            d = torch.empty((H, W), dtype=torch.int16, device="cuda")
            mpv.mpv_match(ctx, l, r, d)
            mpv.mpv_sync(ctx)
            alone[(W, H, D, k)] = d.cpu().numpy().view(np.uint16)
        mpv.mpv_destroy(ctx)
    return mpv, pools, alone


def _check_outputs(res, pools, alone):
    cams = {cid: (W, H, D) for cid, W, H, D in CAMS}
    for rid, (cid, k, disp) in res["outputs"].items():
        W, H, D = cams[cid]
        want = alone[(W, H, D, k % len(pools[(W, H, D)]))]
        assert np.array_equal(disp, want), (rid, cid, k)


def test_mixed_stream_equals_alone_and_overlaps(setup):
    mpv, pools, alone = setup
    res = serve.run(CAMS, pools, seconds=1.5, hz=30.0, max_inflight=8, keep_outputs=True)
    assert res["ok"] == res["frames"] > 100
    _check_outputs(res, pools, alone)
    assert res["peak_inflight"] >= 2          # frames of different cameras overlapped
    assert 0 < res["p50_ms"] <= res["p99_ms"]


def test_budget_forces_eviction_and_keeps_results(setup):
    mpv, pools, alone = setup
    ctx = mpv.mpv_create(0)
    mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=64))
    big = mpv.mpv_workspace_bytes(ctx, 256, 144) + 4 * 256 * 144
    mpv.mpv_destroy(ctx)
    # room for one 256x144 camera (plus a little): cameras take turns being resident
    res = serve.run(CAMS, pools, seconds=0.8, hz=30.0, budget=big + 4096, max_inflight=8,
                    keep_outputs=True)
    assert res["ok"] == res["frames"]
    assert res["evictions"] > 0
    _check_outputs(res, pools, alone)


def test_camera_that_cannot_fit_fails_with_oom(setup):
    mpv, pools, alone = setup
    res = serve.run(CAMS[:1], pools, seconds=0.3, hz=30.0, budget=1 << 16, max_inflight=2)
    assert res["ok"] == 0 and res["frames"] > 0


def test_learned_proposal_where_the_network_fits(setup):
    # the committed network takes D = 128 over 3 scales (2 + 32 input channels): the
    # 256x144 D128 cameras match with the learned proposal, the D32 cameras with the pyramid
    mpv, _, _ = setup
    import os
    weights = os.path.join(os.path.dirname(serve.__file__), "weights", "proposal_d128_s3.bin")
    cams = [(0, 160, 96, 32), (1, 256, 144, 128), (2, 256, 144, 128)]
    pools = {(160, 96, 32): [synth.slanted_pair(160, 96, seed=810 + k, d_max=24)[:2]
                             for k in range(2)],
             (256, 144, 128): [synth.slanted_pair(256, 144, seed=820 + k, d_max=100)[:2]
                               for k in range(2)]}
    alone = {}
    for (W, H, D), frames in pools.items():
        ctx = mpv.mpv_create(0)
        learned = D == 128
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(
            max_disparity=D, proposal=mpv.MPV_PROPOSAL_LEARNED if learned else 0))
        if learned:
            mpv.mpv_load_proposal_weights(ctx, weights)
        for k, (L, R) in enumerate(frames):
            l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
            d = torch.empty((H, W), dtype=torch.int16, device="cuda")
            mpv.mpv_match(ctx, l, r, d)
            mpv.mpv_sync(ctx)
            alone[(W, H, D, k)] = d.cpu().numpy().view(np.uint16)
        mpv.mpv_destroy(ctx)
    res = serve.run(cams, pools, seconds=1.0, hz=30.0, max_inflight=4, keep_outputs=True,
                    proposal=weights)
    assert res["ok"] == res["frames"] > 50
    geom = {cid: (W, H, D) for cid, W, H, D in cams}
    for rid, (cid, k, disp) in res["outputs"].items():
        W, H, D = geom[cid]
        assert np.array_equal(disp, alone[(W, H, D, k % 2)]), (rid, cid, k)
