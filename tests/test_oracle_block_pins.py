"""Pins of the top level split into independent tiles (Section 3.4, read literally: the
top level is cut into blocks and MPV runs on every block)."""
import numpy as np
import pytest

from oracle import ref
from paper_2001_09678_gb300 import synth


@pytest.mark.parametrize("merge", [ref.MERGE_SUM, ref.MERGE_PAPER])
@pytest.mark.parametrize("gradient", [False, True])
def test_tiles_are_independent_problems(merge, gradient):
    rng = np.random.default_rng(3 + merge + 2 * gradient)
    B, tw, th, Dw = 4, 3, 2, 5
    W, H = B * tw, B * th
    Cv = rng.integers(0, 200, (H, W, Dw)).astype(np.int32)
    img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    lut = (np.arange(256) % 7) if gradient else None
    S = ref.aggregate_blocks(Cv, 8, 6, 20, B, merge, grad_lut=lut, I0=img)
    one = ref.aggregate_paper if merge == ref.MERGE_PAPER else ref.aggregate_grad
    for by in range(th):
        for bx in range(tw):
            ys, xs = slice(by * B, (by + 1) * B), slice(bx * B, (bx + 1) * B)
            want = one(np.ascontiguousarray(Cv[ys, xs]), 8, 6, 20, grad_lut=lut,
                       I0=np.ascontiguousarray(img[ys, xs]))
            assert (S[ys, xs] == want).all()


def test_ragged_tiles_and_windows():
    # tiles that do not divide the image: the last row/column of tiles is smaller
    rng = np.random.default_rng(9)
    W, H, Dw, B = 11, 7, 4, 3
    Cv = rng.integers(0, 100, (H, W, Dw)).astype(np.int32)
    lo = rng.integers(0, 5, (H, W)).astype(np.int32)
    S = ref.aggregate_blocks(Cv, 4, 5, 15, B, lo=lo)
    for y0 in range(0, H, B):
        for x0 in range(0, W, B):
            ys, xs = slice(y0, min(H, y0 + B)), slice(x0, min(W, x0 + B))
            want = ref.aggregate(np.ascontiguousarray(Cv[ys, xs]), 4, 5, 15,
                                 lo=np.ascontiguousarray(lo[ys, xs]))
            assert (S[ys, xs] == want).all()


def test_one_tile_is_the_whole_image():
    rng = np.random.default_rng(4)
    Cv = rng.integers(0, 200, (6, 9, 7)).astype(np.int32)
    assert (ref.aggregate_blocks(Cv, 8, 10, 30, 9) == ref.aggregate(Cv, 8, 10, 30)).all()
    assert (ref.aggregate_blocks(Cv, 8, 10, 30, 64, ref.MERGE_PAPER) ==
            ref.aggregate_paper(Cv, 8, 10, 30)).all()


def test_tiled_top_level_matcher_recovers_a_plane():
    W, H, d = 192, 96, 20
    L0, L1 = synth.plane_pair(W, H, d, seed=12)
    p = ref.params(max_disparity=64, num_scales=3, num_paths=8, lr_check=0, top_block=16)
    out = ref.match_view(L0, L1, p)
    m = 4 * (2 + 4)
    assert (out[m:H - m, d + m:W - m] == d).all()
    assert ref.check_params(W, H, ref.params(top_block=-1)) != 0
