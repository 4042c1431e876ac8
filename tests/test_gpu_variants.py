"""The paper's layered merge (Section 3.2), the gradient-weighted TV penalty (Eq. EU) and the
top level split into independent tiles (Section 3.4) on the GPU, against the CPU oracle:
bit-exact disparities, right-view maps and stage volumes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402

ORA_KEYS = ("max_disparity", "num_scales", "num_paths", "p1", "trunc", "ssim_window", "window",
            "block", "lr_check", "lr_tol", "merge_mode", "top_block", "windows")


@pytest.fixture(scope="module")
def mpv():
    from paper_2001_09678_gb300 import build, mpv as m
    build.build()
    m.load()
    return m


def _u16(t):
    return t.cpu().numpy().view(np.uint16)


def exp_table(p1, sigma):
    """round(p1 e^{-g / sigma}) for g = 0..255: the weighting e^{-|G|} with a scale."""
    g = np.arange(256, dtype=np.float64)
    return np.floor(p1 * np.exp(-g / sigma) + 0.5).astype(np.int32)


def ora_params(lut=None, **kw):
    base = dict(max_disparity=128, num_scales=3, num_paths=8, p1=10, trunc=30, ssim_window=5,
                window=0, block=(0, 0, 0, 0), lr_check=1, lr_tol=1, merge_mode=0)
    base.update({k: v for k, v in kw.items() if k in ORA_KEYS})
    return ref.params(grad_lut=lut, **base)


def gpu_match(m, L, R, lut=None, **kw):
    ctx = m.mpv_create(0)
    try:
        m.mpv_set_params(ctx, m.mpv_default_params(**kw))
        if lut is not None:
            m.mpv_set_gradient_penalty(ctx, lut)
        l = torch.from_numpy(np.ascontiguousarray(L)).cuda()
        r = torch.from_numpy(np.ascontiguousarray(R)).cuda()
        d = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        dr = torch.full(L.shape, -2, dtype=torch.int16, device="cuda")
        m.mpv_match_batch(ctx, [dict(left=l, right=r, disp=d, disp_right=dr)])
        m.mpv_sync(ctx)
        return _u16(d), _u16(dr)
    finally:
        m.mpv_destroy(ctx)


PAPER = 1
CASES = {
    # layered merge
    "paper_bands_320x240_d32_p4": (lambda: synth.bands_pair(320, 240, seed=0)[:2],
                                   dict(max_disparity=32, num_scales=1, num_paths=4,
                                        merge_mode=PAPER), None),
    "paper_slanted_s3": (lambda: synth.slanted_pair(256, 144, seed=40, d_max=60)[:2],
                         dict(max_disparity=64, num_scales=3, num_paths=8, merge_mode=PAPER),
                         None),
    "paper_d64_s1_k2": (lambda: synth.bands_pair(200, 60, seed=41, disparities=(10, 30, 55))[:2],
                        dict(max_disparity=64, num_scales=1, num_paths=8, merge_mode=PAPER),
                        None),
    "paper_n3_notrunc": (lambda: synth.bands_pair(150, 70, seed=42)[:2],
                         dict(max_disparity=40, num_scales=2, num_paths=8, ssim_window=3,
                              trunc=ref.NO_TRUNC, p1=3, merge_mode=PAPER), None),
    "paper_ragged_s3": (lambda: synth.bands_pair(203, 117, seed=43)[:2],
                        dict(max_disparity=48, num_scales=3, num_paths=8, window=12,
                             merge_mode=PAPER), None),
    "paper_wide_k8": (lambda: synth.bands_pair(300, 40, seed=44, disparities=(40, 90, 170))[:2],
                      dict(max_disparity=256, num_scales=1, num_paths=4, merge_mode=PAPER), None),
    # gradient-weighted penalty, summed merge
    "grad_slanted_s3": (lambda: synth.slanted_pair(256, 144, seed=45, d_max=60)[:2],
                        dict(max_disparity=64, num_scales=3, num_paths=8), exp_table(10, 16)),
    "grad_bands_d32_p4": (lambda: synth.bands_pair(160, 120, seed=46)[:2],
                          dict(max_disparity=32, num_scales=1, num_paths=4), exp_table(10, 4)),
    "grad_window_100_k4": (lambda: synth.bands_pair(260, 50, seed=47,
                                                    disparities=(30, 80, 150))[:2],
                           dict(max_disparity=200, num_scales=2, num_paths=8, window=100),
                           exp_table(10, 30)),
    "grad_zero_slopes": (lambda: synth.slanted_pair(128, 96, seed=48, d_max=40)[:2],
                         dict(max_disparity=48, num_scales=2, num_paths=8, p1=12, trunc=40),
                         np.where(np.arange(256) % 3 == 0, 0, 12).astype(np.int32)),
    "grad_d128_s3_w32": (lambda: synth.slanted_pair(288, 160, seed=78, d_max=110)[:2],
                         dict(max_disparity=128, num_scales=3, num_paths=8), exp_table(10, 16)),
    "grad_tiles_s2_b16": (lambda: synth.slanted_pair(256, 160, seed=79, d_max=60)[:2],
                          dict(max_disparity=64, num_scales=2, num_paths=8, top_block=16),
                          exp_table(10, 8)),
    "grad_energy_bound": (lambda: synth.slanted_pair(192, 96, seed=80, d_max=40)[:2],
                          dict(max_disparity=48, num_scales=2, num_paths=8, p1=2000,
                               trunc=7936), exp_table(2000, 16)),
    # layered merge at its packed bound (255 + 10 T below the sentinel)
    "paper_trunc_1612": (lambda: synth.slanted_pair(192, 96, seed=81, d_max=40)[:2],
                         dict(max_disparity=48, num_scales=2, num_paths=8, p1=500, trunc=1612,
                              merge_mode=PAPER), None),
    "paper_grad_trunc_1612": (lambda: synth.slanted_pair(192, 96, seed=82, d_max=40)[:2],
                              dict(max_disparity=48, num_scales=2, num_paths=8, p1=500,
                                   trunc=1612, merge_mode=PAPER), exp_table(500, 16)),
    # both
    "paper_grad_s3": (lambda: synth.slanted_pair(224, 128, seed=49, d_max=56)[:2],
                      dict(max_disparity=64, num_scales=3, num_paths=8, merge_mode=PAPER),
                      exp_table(10, 16)),
    "paper_radius4_s2": (lambda: synth.slanted_pair(192, 112, seed=75, d_max=40)[:2],
                         dict(max_disparity=48, num_scales=2, num_paths=8, p1=10, trunc=45,
                              window=12, merge_mode=PAPER), None),
    "paper_d128_s3_w32": (lambda: synth.slanted_pair(288, 160, seed=77, d_max=110)[:2],
                          dict(max_disparity=128, num_scales=3, num_paths=8, merge_mode=PAPER),
                          None),
    "paper_tiles_s3": (lambda: synth.slanted_pair(224, 128, seed=76, d_max=56)[:2],
                       dict(max_disparity=64, num_scales=3, num_paths=8, merge_mode=PAPER,
                            top_block=9), None),
    # the top level split into independent tiles (Section 3.4 read literally)
    "tiles_s3_b16": (lambda: synth.slanted_pair(256, 160, seed=70, d_max=60)[:2],
                     dict(max_disparity=64, num_scales=3, num_paths=8, top_block=16), None),
    "tiles_s1_b24_p4": (lambda: synth.bands_pair(320, 240, seed=71)[:2],
                        dict(max_disparity=32, num_scales=1, num_paths=4, top_block=24), None),
    "tiles_radius4_b7": (lambda: synth.slanted_pair(192, 96, seed=72, d_max=40)[:2],
                         dict(max_disparity=48, num_scales=2, num_paths=8, p1=10, trunc=45,
                              top_block=7), None),
    "tiles_general_notrunc": (lambda: synth.bands_pair(150, 70, seed=73)[:2],
                              dict(max_disparity=40, num_scales=1, num_paths=8, p1=3,
                                   trunc=ref.NO_TRUNC, top_block=20), None),
    "tiles_paper_grad": (lambda: synth.slanted_pair(224, 128, seed=74, d_max=56)[:2],
                         dict(max_disparity=64, num_scales=3, num_paths=8, merge_mode=PAPER,
                              top_block=12), exp_table(10, 16)),
    # a window width per finer level (Section 3.4, the variable form of Eqs. Ot1/Ot2):
    # strides of 48 and 16 labels, padded strides, the layered merge and the gradient table
    "windows_48_16_d128": (lambda: synth.slanted_pair(288, 160, seed=83, d_max=110)[:2],
                           dict(max_disparity=128, num_scales=3, num_paths=8,
                                windows=(48, 16)), None),
    "windows_20_8_ragged": (lambda: synth.bands_pair(203, 117, seed=84)[:2],
                            dict(max_disparity=48, num_scales=3, num_paths=8, windows=(20, 8)),
                            None),
    "windows_s4_paper_grad": (lambda: synth.slanted_pair(256, 160, seed=85, d_max=100)[:2],
                              dict(max_disparity=128, num_scales=4, num_paths=8,
                                   windows=(0, 24, 12), merge_mode=PAPER), exp_table(10, 16)),
    "full_windows_48_16_1280x720": (lambda: synth.slanted_pair(1280, 720, seed=0)[:2],
                                    dict(max_disparity=128, num_scales=3, num_paths=8,
                                         windows=(48, 16)), None),
    # the benchmarked variants at their full size: 1280x720, D = 128, 3 scales (the
    # 1280-step horizontal chains, the prefetch rings' wrap, every window shift)
    "full_paper_1280x720_d128": (lambda: synth.slanted_pair(1280, 720, seed=0)[:2],
                                 dict(max_disparity=128, num_scales=3, num_paths=8,
                                      merge_mode=PAPER), None),
    "full_grad_1280x720_d128": (lambda: synth.slanted_pair(1280, 720, seed=0)[:2],
                                dict(max_disparity=128, num_scales=3, num_paths=8),
                                exp_table(10, 16)),
    "full_paper_grad_1280x720_d128": (lambda: synth.slanted_pair(1280, 720, seed=0)[:2],
                                      dict(max_disparity=128, num_scales=3, num_paths=8,
                                           merge_mode=PAPER), exp_table(10, 16)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_variant_disparity_bit_exact(mpv, name):
    make, kw, lut = CASES[name]
    L, R = make()
    want_l, want_r = ref.match(L, R, ora_params(lut, **kw), want_right=True)
    got_l, got_r = gpu_match(mpv, L, R, lut, **kw)
    assert np.array_equal(got_l, want_l), f"{(got_l != want_l).sum()} pixels differ"
    assert np.array_equal(got_r, want_r), f"{(got_r != want_r).sum()} right pixels differ"


@pytest.mark.parametrize("view", [0, 1])
@pytest.mark.parametrize("level", [0, 2])
@pytest.mark.parametrize("variant", ["paper", "grad", "paper_grad", "tiles"])
def test_variant_stage_volumes_bit_exact(mpv, view, level, variant):
    L, R, _ = synth.bands_pair(123, 77, seed=50)
    kw = dict(max_disparity=48, num_scales=3, num_paths=8, window=12,
              merge_mode=PAPER if variant.startswith("paper") else 0,
              top_block=5 if variant == "tiles" else 0)
    lut = exp_table(10, 8) if variant.endswith("grad") else None
    p = ora_params(lut, **kw)
    I0, I1 = (L, R) if view == 0 else (np.ascontiguousarray(R[:, ::-1]),
                                       np.ascontiguousarray(L[:, ::-1]))
    lo, Cv, S, d = ref.view_stage(I0, I1, p, level)
    Hl, Wl, Dw = Cv.shape
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
        if lut is not None:
            mpv.mpv_set_gradient_penalty(ctx, lut)
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
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


def test_variant_batch_matches_oracle(mpv):
    # a mixed batch under a CUDA graph, with the table switched on after a first batch
    pairs = [synth.slanted_pair(160, 96, seed=51 + i, d_max=40)[:2] for i in range(3)]
    kw = dict(max_disparity=48, num_scales=2, num_paths=8, merge_mode=PAPER)
    lut = exp_table(10, 12)
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(**kw))
        tens = [(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(),
                 torch.zeros(L.shape, dtype=torch.int16, device="cuda")) for L, R in pairs]
        batch = [dict(left=l, right=r, disp=d) for l, r, d in tens]
        for table in (None, lut, None):
            mpv.mpv_set_gradient_penalty(ctx, table)
            for _ in range(2):                       # the second run replays the graph
                for _, _, d in tens:
                    d.fill_(-2)
                mpv.mpv_match_batch(ctx, batch)
                mpv.mpv_sync(ctx)
                for (L, R), (_, _, d) in zip(pairs, tens):
                    want = ref.match(L, R, ora_params(table, **kw))
                    assert np.array_equal(_u16(d), want)
    finally:
        mpv.mpv_destroy(ctx)


def test_gradient_table_validation(mpv):
    L, R, _ = synth.bands_pair(64, 48, seed=52)
    ctx = mpv.mpv_create(0)
    try:
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=16, num_scales=1, p1=10))
        with pytest.raises(mpv.MpvError):
            mpv.mpv_set_gradient_penalty(ctx, np.full(256, -1, np.int32))
        with pytest.raises(ValueError):
            mpv.mpv_set_gradient_penalty(ctx, np.zeros(10, np.int32))
        mpv.mpv_set_gradient_penalty(ctx, np.full(256, 11, np.int32))   # above p1 = 10
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        d = torch.zeros(L.shape, dtype=torch.int16, device="cuda")
        with pytest.raises(mpv.MpvError):
            mpv.mpv_match(ctx, l, r, d)
        # raising p1 makes the same table valid; a constant table p1 is the plain matcher
        mpv.mpv_set_params(ctx, mpv.mpv_default_params(max_disparity=16, num_scales=1, p1=11))
        mpv.mpv_match(ctx, l, r, d)
        mpv.mpv_sync(ctx)
        want = ref.match(L, R, ora_params(None, max_disparity=16, num_scales=1, p1=11))
        assert np.array_equal(_u16(d), want)
    finally:
        mpv.mpv_destroy(ctx)
