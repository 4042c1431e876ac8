"""Pins of the oracle's variable window width per pyramid level (Section 3.4).

Eqs. Ot1 and Ot2 count the work of a finer level as its pixels times a window of d/4
labels; the variable form gives each finer level its own width Dw_l (clamped to the
level's range).  Pinned by the node count written out for two settings, by the special
case of equal widths (the single-width matcher), by the window each level reports, by
validation, and by exact recovery of a noise-free plane through three scales with
narrow and wide windows.
"""
import numpy as np
import pytest

from oracle import ref
from paper_2001_09678_gb300 import synth


def test_level_windows():
    p = ref.params(max_disparity=128, num_scales=3, windows=(48, 16))
    assert [ref.level_window(p, l) for l in range(3)] == [32, 48, 16]
    # a width above the level's range is clamped to it (level 1 of D = 128 has 64 labels);
    # an unset level takes `window`
    p = ref.params(max_disparity=128, num_scales=3, window=20, windows=(100, 0))
    assert [ref.level_window(p, l) for l in range(3)] == [32, 64, 20]
    # four scales of D = 128: ranges 16, 32, 64, 128; level 1 unset takes D/4 = 32
    p = ref.params(max_disparity=128, num_scales=4, windows=(0, 40, 8))
    assert [ref.level_window(p, l) for l in range(4)] == [16, 32, 40, 8]


def test_node_count_with_per_level_windows():
    # 1280 x 720, D = 128, three scales: 320x180 x 32 (full top range) + 640x360 x 48 +
    # 1280x720 x 16 = 1,843,200 + 11,059,200 + 14,745,600
    p = ref.params(max_disparity=128, num_scales=3, windows=(48, 16))
    assert ref.node_count(1280, 720, p) == 27_648_000
    # 640 x 480, D = 64, windows (8, 24): 160x120 x 16 + 320x240 x 8 + 640x480 x 24
    p = ref.params(max_disparity=64, num_scales=3, windows=(8, 24))
    assert ref.node_count(640, 480, p) == 307_200 + 614_400 + 7_372_800


def test_equal_widths_are_the_single_width_matcher():
    L, R, _ = synth.slanted_pair(160, 96, seed=60, d_max=40)
    a = ref.match(L, R, ref.params(max_disparity=48, num_scales=3, num_paths=8, window=14))
    b = ref.match(L, R, ref.params(max_disparity=48, num_scales=3, num_paths=8,
                                   windows=(14, 14)))
    assert np.array_equal(a, b)
    # and different widths change the result somewhere (the parameter is used)
    c = ref.match(L, R, ref.params(max_disparity=48, num_scales=3, num_paths=8,
                                   windows=(4, 24)))
    assert not np.array_equal(a, c)


@pytest.mark.parametrize("windows", [(12, 4), (40, 2), (6, 30)])
def test_plane_recovery_with_per_level_windows(windows):
    # d = 20 is a multiple of 4: every level sees an exact integer shift, the top level
    # finds 5, its doubled seed 10 is exact at level 1 and 20 at level 2, so every window
    # (even 2 labels wide) contains the true disparity
    W, H, d = 192, 96, 20
    L0, L1 = synth.plane_pair(W, H, d, seed=12)
    p = ref.params(max_disparity=64, num_scales=3, num_paths=8, lr_check=0, windows=windows)
    out = ref.match_view(L0, L1, p)
    m = 4 * (2 + 4)
    assert (out[m:H - m, d + m:W - m] == d).all()


def test_negative_width_is_rejected():
    # ora_check_params: 0 accepts, -1 rejects
    p = ref.params(max_disparity=64, num_scales=3, windows=(8, -1))
    assert ref.check_params(96, 64, p) == -1
    ok = ref.params(max_disparity=64, num_scales=3, windows=(8, 1))
    assert ref.check_params(96, 64, ok) == 0
