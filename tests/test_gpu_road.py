"""Road detection on the GPU (Section 3.5) against the CPU oracle: v-disparity,
u-disparity, road profile and its sum, element by element.
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


def gpu_road(m, U, D, eta, with_u=True):
    H, W = U.shape
    ctx = m.mpv_create(0)
    try:
        d = torch.from_numpy(U.view(np.int16)).cuda()
        vd = torch.full((H, D), -7, dtype=torch.int32, device="cuda")
        ud = torch.full((W, D), -7, dtype=torch.int32, device="cuda") if with_u else None
        prof = torch.full((D,), -7, dtype=torch.int32, device="cuda")
        en = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        m.mpv_road_detect(ctx, d, D, eta, vd, prof, en, udisp=ud)
        torch.cuda.synchronize()
        return (vd.cpu().numpy().view(np.uint32), ud.cpu().numpy().view(np.uint32) if with_u
                else None, prof.cpu().numpy(), int(en.item()))
    finally:
        m.mpv_destroy(ctx)


CASES = [
    # W, H, D, eta, generator arguments
    (320, 240, 32, 6, dict(horizon=80, rows_per_label=4, n_obstacles=3)),
    (1280, 720, 128, 8, dict(horizon=300, rows_per_label=3, n_obstacles=6)),
    (1920, 1080, 192, 5, dict(horizon=400, rows_per_label=3, n_obstacles=8)),  # global steps
    (203, 117, 40, 2, dict(horizon=30, rows_per_label=2, n_obstacles=2)),
    (64, 20, 32, 3, dict(horizon=5, rows_per_label=1, n_obstacles=0)),         # no path fits
    (33, 300, 17, 256, dict(horizon=100, rows_per_label=9, n_obstacles=1)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_road_bit_exact(mpv, case):
    W, H, D, eta, kw = CASES[case]
    U = synth.road_disparity(W, H, D, seed=60 + case, **kw)
    vd, ud, prof, en = gpu_road(mpv, U, D, eta)
    want_vd, want_ud = ref.vdisparity(U, D), ref.udisparity(U, D)
    want_en, want_prof = ref.road_profile(want_vd, eta)
    assert np.array_equal(vd, want_vd)
    assert np.array_equal(ud, want_ud)
    assert en == want_en and np.array_equal(prof, want_prof)


def test_road_on_the_matcher_output(mpv):
    L, R, _ = synth.slanted_pair(256, 160, seed=61, d_max=56)
    kw = dict(max_disparity=64, num_scales=2, num_paths=8)
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        d = torch.zeros(L.shape, dtype=torch.int16, device="cuda")
        mpv.mpv_match(ctx, l, r, d)
        vd = torch.zeros((160, 64), dtype=torch.int32, device="cuda")
        prof = torch.zeros(64, dtype=torch.int32, device="cuda")
        en = torch.zeros(1, dtype=torch.int64, device="cuda")
        mpv.mpv_road_detect(ctx, d, 64, 4, vd, prof, en)
        torch.cuda.synchronize()
        U = d.cpu().numpy().view(np.uint16)
    finally:
        mpv.mpv_destroy(ctx)
    want_vd = ref.vdisparity(U, 64)
    want_en, want_prof = ref.road_profile(want_vd, 4)
    assert np.array_equal(vd.cpu().numpy().view(np.uint32), want_vd)
    assert int(en.item()) == want_en and np.array_equal(prof.cpu().numpy(), want_prof)


def test_road_argument_checks(mpv):
    ctx = mpv.mpv_create(0)
    try:
        d = torch.zeros((10, 10), dtype=torch.int16, device="cuda")
        vd = torch.zeros((10, 8), dtype=torch.int32, device="cuda")
        prof = torch.zeros(8, dtype=torch.int32, device="cuda")
        en = torch.zeros(1, dtype=torch.int64, device="cuda")
        for D, eta in ((8, 1), (8, 257), (0, 4), (1025, 4)):
            with pytest.raises(mpv.MpvError):
                mpv.mpv_road_detect(ctx, d, D, eta, vd, prof, en)
    finally:
        mpv.mpv_destroy(ctx)
