"""Pins of the oracle's road detection on disparity maps (Section 3.5: v-disparity,
u-disparity, and the road Viterbi e(i,j) = Hx(i,j) + max_{0 < j - j' < eta} e(i-1,j')).
"""
import itertools

import numpy as np
import pytest

from oracle import ref
from paper_2001_09678_gb300 import synth


def test_histograms_closed_forms():
    rng = np.random.default_rng(0)
    D = 7
    U = rng.integers(0, D, (9, 11)).astype(np.uint16)
    U[2, 3] = 0xFFFF                      # rejected pixel
    U[4, 5] = D + 3                       # out of the histogram's range
    Hx, Hy = ref.vdisparity(U, D), ref.udisparity(U, D)
    for j in range(9):
        for i in range(D):
            assert Hx[j, i] == np.count_nonzero(U[j] == i)
    for j in range(11):
        for i in range(D):
            assert Hy[j, i] == np.count_nonzero(U[:, j] == i)
    valid = np.count_nonzero(U < D)
    assert Hx.sum() == Hy.sum() == valid == 9 * 11 - 2
    # a constant map puts every pixel of a row (column) in one bin
    C = np.full((5, 6), 3, np.uint16)
    assert (ref.vdisparity(C, 4)[:, 3] == 6).all() and (ref.udisparity(C, 4)[:, 3] == 5).all()


def _brute_road(Hx, eta):
    H, D = Hx.shape
    best, best_key, best_path = -1, None, None
    for start in range(H):
        for steps in itertools.product(range(1, eta), repeat=D - 1):
            path = [start]
            for s in steps:
                path.append(path[-1] + s)
            if path[-1] >= H:
                continue
            total = int(sum(Hx[path[i], i] for i in range(D)))
            # ties: the smallest final row, then the smallest row at each earlier step
            key = (-total, tuple(reversed(path)))
            if best_key is None or key < best_key:
                best_key, best, best_path = key, total, path
    return best, best_path


@pytest.mark.parametrize("seed", range(12))
def test_road_profile_brute_force(seed):
    rng = np.random.default_rng(seed)
    H, D = int(rng.integers(3, 8)), int(rng.integers(1, 5))
    eta = int(rng.integers(2, 5))
    Hx = rng.integers(0, 4 if seed % 2 else 50, (H, D)).astype(np.uint32)
    best, P = ref.road_profile(Hx, eta)
    want, path = _brute_road(Hx, eta)
    assert best == want
    if path is None:
        assert (P == -1).all()
    else:
        assert P.tolist() == path


def test_road_profile_needs_room():
    # D = 4 disparities need at least 4 rows with eta = 2 (steps of exactly one row)
    Hx = np.ones((3, 4), np.uint32)
    best, P = ref.road_profile(Hx, 2)
    assert best == -1 and (P == -1).all()
    best, P = ref.road_profile(np.ones((4, 4), np.uint32), 2)
    assert best == 4 and P.tolist() == [0, 1, 2, 3]


def test_flat_road_is_recovered():
    # a flat road: disparity i on rows horizon + 3i .. horizon + 3i + 2, every pixel valid,
    # no obstacles or outliers: the path takes the first row of every band
    W, H, D, hz = 64, 120, 24, 40
    U = synth.road_disparity(W, H, D, seed=2, horizon=hz, rows_per_label=3, n_obstacles=0,
                             outliers=0.0, invalid=0.0)
    best, P = ref.road_profile(ref.vdisparity(U, D), eta=4)
    # d = 0 also covers the rows above the horizon; from d = 1 on the path is on the road
    assert P[1:].tolist() == [hz + 3 * i for i in range(1, D)]
    assert best == D * W


def test_road_with_obstacles_and_noise_stays_on_the_road():
    W, H, D, hz = 320, 240, 32, 80
    U = synth.road_disparity(W, H, D, seed=3, horizon=hz, rows_per_label=4, n_obstacles=4,
                             outliers=0.03, invalid=0.05)
    best, P = ref.road_profile(ref.vdisparity(U, D), eta=6)
    band = [(hz + 4 * i, hz + 4 * i + 3) for i in range(D)]
    on_road = sum(lo <= P[i] <= hi for i, (lo, hi) in enumerate(band))
    assert on_road >= D - 2          # the first disparities share rows with the background
