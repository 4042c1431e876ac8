"""GPU matcher (through the C ABI) against the CPU oracle: bit-exact, element by element.

All costs and energies are integers on both sides, so every comparison is equality.
"""
import hashlib
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ORA_KEYS = ("max_disparity", "num_scales", "num_paths", "p1", "trunc", "ssim_window", "window",
            "block", "lr_check", "lr_tol")


@pytest.fixture(scope="module")
def mpv():
    from paper_2001_09678_gb300 import build, mpv as m
    build.build()
    m.load()
    return m


def _u16(t):
    return t.cpu().numpy().view(np.uint16)


def gpu_match(m, L, R, want_right=False, **kw):
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(**kw))
        l = torch.from_numpy(np.ascontiguousarray(L)).cuda()
        r = torch.from_numpy(np.ascontiguousarray(R)).cuda()
        d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        dr = torch.full(L.shape, -2, dtype=torch.int16, device="cuda") if want_right else None
        m.mpv_match_batch(ctx, [dict(left=l, right=r, disp=d, disp_right=dr)])
        m.mpv_sync(ctx)
        return (_u16(d), _u16(dr)) if want_right else _u16(d)
    finally:
        m.mpv_destroy(ctx)


def ora_params(**kw):
    base = dict(max_disparity=128, num_scales=3, num_paths=8, p1=10, trunc=30, ssim_window=5,
                window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1)
    base.update({k: v for k, v in kw.items() if k in ORA_KEYS})
    return ref.params(**base)


CASES = {
    # config-1 workload: 320x240, D=32, single scale, 4 paths, p1=10, T=30
    "bands_320x240_d32": (lambda: synth.bands_pair(320, 240, seed=0)[:2],
                          dict(max_disparity=32, num_scales=1, num_paths=4)),
    "ragged_203x117_s3": (lambda: synth.bands_pair(203, 117, seed=4)[:2],
                          dict(max_disparity=48, num_scales=3, num_paths=8, window=12)),
    "n3_notrunc_s2": (lambda: synth.bands_pair(150, 70, seed=5)[:2],
                      dict(max_disparity=40, num_scales=2, num_paths=8, ssim_window=3,
                           trunc=ref.NO_TRUNC, p1=3)),
    "wide_range_k8": (lambda: synth.bands_pair(300, 40, seed=6, disparities=(40, 90, 170))[:2],
                      dict(max_disparity=256, num_scales=1, num_paths=4)),
    "window_100_k4": (lambda: synth.bands_pair(260, 50, seed=7, disparities=(30, 80, 150))[:2],
                      dict(max_disparity=200, num_scales=2, num_paths=8, window=100)),
    "tiny_5x5_d1": (lambda: synth.bands_pair(5, 5, seed=8, disparities=(0, 0, 0))[:2],
                    dict(max_disparity=1, num_scales=1, num_paths=8)),
    "s4_40x40": (lambda: synth.bands_pair(40, 40, seed=9, disparities=(2, 6, 9))[:2],
                 dict(max_disparity=16, num_scales=4, num_paths=8, window=4)),
    "zero_penalty": (lambda: synth.bands_pair(96, 64, seed=10)[:2],
                     dict(max_disparity=24, num_scales=1, num_paths=8, p1=0, trunc=0)),
    "lr_tol0_trunc_big": (lambda: synth.bands_pair(128, 64, seed=11)[:2],
                          dict(max_disparity=32, num_scales=2, num_paths=4, lr_tol=0, p1=7,
                               trunc=200)),
    "no_lr": (lambda: synth.bands_pair(100, 60, seed=12)[:2],
              dict(max_disparity=32, num_scales=2, num_paths=8, lr_check=0)),
    "blocks_3_then_lerp": (lambda: synth.bands_pair(160, 96, seed=13)[:2],
                           dict(max_disparity=64, num_scales=3, num_paths=8, block=(3, 1))),
    "lerp_everywhere": (lambda: synth.bands_pair(160, 96, seed=14)[:2],
                        dict(max_disparity=64, num_scales=3, num_paths=8, block=(1, 1))),
    "s4_blocks": (lambda: synth.bands_pair(200, 120, seed=15)[:2],
                  dict(max_disparity=64, num_scales=4, num_paths=8, block=(2, 2, 1), window=12)),
    "slanted_320x240_s3": (lambda: synth.slanted_pair(320, 240, seed=16, d_max=60)[:2],
                           dict(max_disparity=64, num_scales=3, num_paths=8)),
    "odd_window_17": (lambda: synth.slanted_pair(256, 144, seed=17, d_max=100)[:2],
                      dict(max_disparity=128, num_scales=2, num_paths=8, window=17)),
    # 32-label rows of 33 and 35 pixels (one straight-line chunk, then the guarded tail)
    # and heights that leave part of the last warp's four rows outside the image
    "narrow_33x50_d32": (lambda: synth.bands_pair(33, 50, seed=40, disparities=(2, 5, 9))[:2],
                         dict(max_disparity=32, num_scales=1, num_paths=8)),
    "narrow_70x45_win32": (lambda: synth.bands_pair(70, 45, seed=41, disparities=(4, 11, 20))[:2],
                           dict(max_disparity=64, num_scales=2, num_paths=8, window=32)),
    # one view (no left-right check) and 4 paths: the row blocks of a single view
    "narrow_40x29_d32_4p_nolr": (lambda: synth.bands_pair(40, 29, seed=42,
                                                          disparities=(3, 8, 14))[:2],
                                 dict(max_disparity=32, num_scales=1, num_paths=4, lr_check=0)),
    # stencil radius ceil(T/p1) - 1 = 1, 3, 4 (the default p1=10, T=30 gives 2)
    "radius1": (lambda: synth.slanted_pair(192, 96, seed=18, d_max=40)[:2],
                dict(max_disparity=48, num_scales=2, num_paths=8, p1=10, trunc=20)),
    "radius3": (lambda: synth.slanted_pair(192, 96, seed=19, d_max=40)[:2],
                dict(max_disparity=48, num_scales=2, num_paths=8, p1=10, trunc=40)),
    "radius4_t45": (lambda: synth.slanted_pair(192, 96, seed=20, d_max=40)[:2],
                    dict(max_disparity=48, num_scales=3, num_paths=8, p1=10, trunc=45)),
    # packed widths: 48 labels (top level of D=192, 3 scales) and 64 labels
    "dw48_s3": (lambda: synth.slanted_pair(400, 120, seed=22, d_max=180)[:2],
                dict(max_disparity=192, num_scales=3, num_paths=8)),
    "dw64_s1": (lambda: synth.bands_pair(200, 60, seed=23, disparities=(10, 30, 55))[:2],
                dict(max_disparity=64, num_scales=1, num_paths=8)),
    # the largest range the boundary accepts
    "max_range_d1024": (lambda: synth.bands_pair(1040, 24, seed=30,
                                                 disparities=(100, 500, 900))[:2],
                        dict(max_disparity=1024, num_scales=1, num_paths=4)),
    # summed energies just below 2^16: paths * (255 + T) = 65528 and 65532
    "energy_bound_8paths": (lambda: synth.slanted_pair(192, 96, seed=31, d_max=40)[:2],
                            dict(max_disparity=48, num_scales=2, num_paths=8, p1=2000,
                                 trunc=7936)),
    "energy_bound_4paths": (lambda: synth.slanted_pair(192, 96, seed=32, d_max=40)[:2],
                            dict(max_disparity=48, num_scales=2, num_paths=4, p1=4100,
                                 trunc=16128)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_disparity_bit_exact(mpv, name):
    make, kw = CASES[name]
    L, R = make()
    want_l, want_r = ref.match(L, R, ora_params(**kw), want_right=True)
    got_l, got_r = gpu_match(mpv, L, R, want_right=True, **kw)
    assert np.array_equal(got_l, want_l), f"{(got_l != want_l).sum()} pixels differ"
    assert np.array_equal(got_r, want_r), f"{(got_r != want_r).sum()} right pixels differ"


@pytest.mark.parametrize("view", [0, 1])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_stage_volumes_bit_exact(mpv, view, level):
    L, R, _ = synth.bands_pair(123, 77, seed=21)
    kw = dict(max_disparity=48, num_scales=3, num_paths=8, window=12)
    p = ora_params(**kw)
    I0, I1 = (L, R) if view == 0 else (np.ascontiguousarray(R[:, ::-1]),
                                       np.ascontiguousarray(L[:, ::-1]))
    lo, Cv, S, d = ref.view_stage(I0, I1, p, level)
    Hl, Wl, Dw = Cv.shape
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
        assert mpv.mpv_level_info(ctx, 123, 77, level)[0:2] == (Wl, Hl)
        assert mpv.mpv_level_info(ctx, 123, 77, level)[3] == Dw
        l = torch.from_numpy(L).cuda()
        r = torch.from_numpy(R).cuda()
        glo = torch.zeros((Hl, Wl), dtype=torch.int16, device="cuda")
        gc = torch.zeros((Hl, Wl, Dw), dtype=torch.int16, device="cuda")
        gs = torch.zeros((Hl, Wl, Dw), dtype=torch.int32, device="cuda")
        gd = torch.zeros((Hl, Wl), dtype=torch.int16, device="cuda")
        mpv.mpv_debug_stage(ctx, l, r, view, level, glo, gc, gs, gd)
    finally:
        mpv.mpv_destroy(ctx)
    assert np.array_equal(_u16(glo).astype(np.int32), lo)
    assert np.array_equal(_u16(gc).astype(np.int32), Cv)
    assert np.array_equal(gs.cpu().numpy().astype(np.int64), S)
    assert np.array_equal(_u16(gd), d)


def test_golden_outputs(mpv):
    with open(os.path.join(GOLDEN, "oracle_disparity.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for name, W, H, seed, kv, digest in rows:
        kw = {k: int(v) for k, v in (s.split("=") for s in kv.split(","))}
        L, R, _ = synth.bands_pair(int(W), int(H), seed=int(seed))
        got = gpu_match(mpv, L, R, **kw)
        assert hashlib.sha256(got.astype("<u2").tobytes()).hexdigest() == digest, name


def test_host_entry_point(mpv):
    L, R, _ = synth.bands_pair(96, 64, seed=30)
    kw = dict(max_disparity=32, num_scales=2, num_paths=8)
    want = ref.match(L, R, ora_params(**kw))
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
        out = np.zeros(L.shape, np.uint16)
        mpv.mpv_match_host(ctx, L, R, out)
    finally:
        mpv.mpv_destroy(ctx)
    assert np.array_equal(out, want)


def test_padded_pitches(mpv):
    L, R, _ = synth.bands_pair(90, 50, seed=31)
    kw = dict(max_disparity=24, num_scales=2, num_paths=4)
    want = ref.match(L, R, ora_params(**kw))
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
        lp = torch.zeros((50, 128), dtype=torch.uint8, device="cuda")
        rp = torch.zeros((50, 128), dtype=torch.uint8, device="cuda")
        lp[:, :90] = torch.from_numpy(L).cuda()
        rp[:, :90] = torch.from_numpy(R).cuda()
        d = torch.full((50, 100), -2, dtype=torch.int16, device="cuda")
        mpv.mpv_match(ctx, lp[:, :90], rp[:, :90], d[:, :90])
        mpv.mpv_sync(ctx)
    finally:
        mpv.mpv_destroy(ctx)
    out = _u16(d)
    assert np.array_equal(out[:, :90], want)
    assert (out[:, 90:] == 0xFFFE).all()          # untouched padding


def test_invalid_arguments_leave_outputs_untouched(mpv):
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=64, num_scales=3))
        l = torch.zeros((40, 60), dtype=torch.uint8, device="cuda")
        d = torch.full((40, 60), 7, dtype=torch.int16, device="cuda")
        with pytest.raises(mpv.MpvError) as e:      # D = 64 > width 60
            mpv.mpv_match(ctx, l, l, d)
        assert e.value.status == mpv.MPV_ERR_INVALID_ARG
        bad = mpv.mpv_default_params(num_paths=6)
        with pytest.raises(mpv.MpvError):
            mpv.mpv_set_params(ctx, bad)
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=16, num_scales=4))
        l2 = torch.zeros((32, 60), dtype=torch.uint8, device="cuda")
        d2 = torch.full((32, 60), 7, dtype=torch.int16, device="cuda")
        with pytest.raises(mpv.MpvError):           # top level 8 x 4 is below 5 x 5
            mpv.mpv_match(ctx, l2, l2, d2)
        assert (d2 == 7).all()
        torch.cuda.synchronize()
        assert (d == 7).all()
    finally:
        mpv.mpv_destroy(ctx)


def test_workspace_limit_reports_oom(mpv):
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=32, num_scales=1))
        mpv.mpv_set_workspace_limit(ctx, 1 << 16)
        l = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
        d = torch.zeros((64, 64), dtype=torch.int16, device="cuda")
        with pytest.raises(mpv.MpvError) as e:
            mpv.mpv_match(ctx, l, l, d)
        assert e.value.status == mpv.MPV_ERR_OOM
    finally:
        mpv.mpv_destroy(ctx)


def test_full_size_config_bit_exact(mpv):
    # the benchmark's workload: 1280x720, D=128, 3 scales, 8 paths, left-right check
    L, R, _ = synth.slanted_pair(1280, 720, seed=0)
    kw = dict(max_disparity=128, num_scales=3, num_paths=8, p1=10, trunc=30)
    want = ref.match(L, R, ora_params(**kw))
    got = gpu_match(mpv, L, R, **kw)
    assert np.array_equal(got, want), f"{(got != want).sum()} pixels differ"
