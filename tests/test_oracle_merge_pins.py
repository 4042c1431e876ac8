"""Pins of the oracle's penalty-general passes and the paper's layered merge.

The paper's own merge (Section 3.2, Fig. merging, Table alg) runs the scan directions in
layers - left/right, up/down, then the two diagonal pairs - merging the two passes of a
layer by the minimum (horizontal) or the mean (the others), the left-to-right pass charging
jumps to a larger disparity twice; Eq. EU weights the TV term by the image gradient.  These
tests hold the oracle's restatement to brute force over all labelings of every scan chain,
to hand-computed cases and to closed forms.
"""
import itertools

import numpy as np
import pytest

from oracle import ref
from paper_2001_09678_gb300 import synth

NT = ref.NO_TRUNC
DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (-1, 1), (1, -1)]


def _eps(u, v, slope, T, double_up):
    """Jump penalty from predecessor label v to label u."""
    if u == v:
        return 0
    up = u > v
    s = 2 * slope if (double_up and up) else slope
    cap = (2 * T if (double_up and up) else T) if T != NT else None
    e = s * abs(u - v)
    return e if cap is None else min(e, cap)


def _chains(W, H, dx, dy):
    """Every scan chain of direction (dx,dy), in scan order."""
    out = []
    for y in range(H):
        for x in range(W):
            px, py = x - dx, y - dy
            if 0 <= px < W and 0 <= py < H:
                continue                       # not a chain start
            ch = []
            cx, cy = x, y
            while 0 <= cx < W and 0 <= cy < H:
                ch.append((cx, cy))
                cx += dx
                cy += dy
            out.append(ch)
    return out


def _slope(img, lut, p1, a, b):
    if lut is None:
        return p1
    return int(lut[abs(int(img[a[1], a[0]]) - int(img[b[1], b[0]]))])


def _brute_pass(Q, lo, dx, dy, p1, T, lut=None, img=None, double_up=False):
    """F(p,u): minimum over all labelings of the chain prefix ending at p with label u of
    the data terms plus the jump penalties (no recursion, no envelope)."""
    H, W, Dw = Q.shape
    F = np.zeros(Q.shape, np.int64)
    for ch in _chains(W, H, dx, dy):
        for i in range(len(ch)):
            pre = ch[:i + 1]
            best = {}
            for lab in itertools.product(range(Dw), repeat=len(pre)):
                e = 0
                for j, (x, y) in enumerate(pre):
                    e += int(Q[y, x, lab[j]])
                    if j:
                        (qx, qy) = pre[j - 1]
                        u = int(lo[y, x]) + lab[j]
                        v = int(lo[qy, qx]) + lab[j - 1]
                        e += _eps(u, v, _slope(img, lut, p1, (x, y), (qx, qy)), T, double_up)
                k = lab[-1]
                best[k] = min(best.get(k, e), e)
            x, y = pre[-1]
            for k in range(Dw):
                F[y, x, k] = best[k]
    return F


def _brute_paper(Cv, lo, npaths, p1, T, lut=None, img=None):
    Q = Cv.astype(np.int64)
    for layer in range(npaths // 2):
        (fx, fy), (bx, by) = DIRS[2 * layer], DIRS[2 * layer + 1]
        F = _brute_pass(Q, lo, fx, fy, p1, T, lut, img, double_up=(fx, fy) == (1, 0))
        B = _brute_pass(Q, lo, bx, by, p1, T, lut, img)
        F = F - F.min(axis=2, keepdims=True)
        B = B - B.min(axis=2, keepdims=True)
        Q = np.minimum(F, B) if layer == 0 else (F + B) // 2
    return Q


def _case(seed, W, H, Dw, D, windowed):
    rng = np.random.default_rng(seed)
    Cv = rng.integers(0, 120, (H, W, Dw)).astype(np.int32)
    lo = (rng.integers(0, D - Dw + 1, (H, W)) if windowed else np.zeros((H, W))).astype(np.int32)
    img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    return Cv, lo, img


# ------------------------------------------------------------------------------------
# envelopes with separate upward / downward penalties
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_general_envelope_fast_equals_full_connectivity(seed):
    rng = np.random.default_rng(seed)
    Dw = int(rng.integers(1, 12))
    A = rng.integers(0, 200, Dw)
    if seed % 3 == 0:
        A[rng.integers(0, Dw)] = 1 << 40                  # an absent label
    lo_prev, lo = (int(v) for v in rng.integers(0, 6, 2))
    p_up, p_dn = (int(v) for v in rng.choice([0, 1, 3, 8, 25], 2))
    T_up, T_dn = (int(v) for v in rng.choice([0, 4, 17, 60, NT], 2))
    fast = ref.envelope_pen(A, lo_prev, lo, p_up, p_dn, T_up, T_dn)
    naive = ref.envelope_pen(A, lo_prev, lo, p_up, p_dn, T_up, T_dn, naive=True)
    def pen(u, v):
        if u > v:
            return p_up * (u - v) if T_up == NT else min(p_up * (u - v), T_up)
        return p_dn * (v - u) if T_dn == NT else min(p_dn * (v - u), T_dn)

    want = [min(int(A[j]) + pen(lo + k, lo_prev + j) for j in range(Dw)) for k in range(Dw)]
    assert fast.tolist() == naive.tolist() == want


def test_symmetric_general_envelope_is_the_plain_envelope():
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = rng.integers(0, 300, 9)
        p1, T = int(rng.integers(0, 30)), int(rng.choice([7, 40, NT]))
        assert (ref.envelope_pen(A, 2, 4, p1, p1, T, T) == ref.envelope(A, 2, 4, p1, T)).all()


# ------------------------------------------------------------------------------------
# passes with per-step penalties: brute force over the chains
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("dx,dy", DIRS)
@pytest.mark.parametrize("double_up", [False, True])
def test_pass_with_gradient_penalty_brute_force(dx, dy, double_up):
    Cv, lo, img = _case(20 + dx + 3 * dy, 4, 3, 3, 5, windowed=True)
    lut = np.maximum(0, 12 - np.arange(256) // 8)          # slopes 12 .. 0, all <= p1
    p1, T = 12, 30
    F = _brute_pass(Cv, lo, dx, dy, p1, T, lut, img, double_up)
    Lhat, st = ref.path_pen(Cv, dx, dy, p1, T, lo=lo, grad_lut=lut, I0=img,
                            double_up=double_up, normalize_out=True, check=True)
    assert st == 0
    assert (Lhat == F - F.min(axis=2, keepdims=True)).all()
    # the bounded form is the literal energy minus the predecessor's minimum
    L, _ = ref.path_pen(Cv, dx, dy, p1, T, lo=lo, grad_lut=lut, I0=img, double_up=double_up)
    H, W, _ = Cv.shape
    for y in range(H):
        for x in range(W):
            px, py = x - dx, y - dy
            base = F[py, px].min() if (0 <= px < W and 0 <= py < H) else 0
            assert (L[y, x] == F[y, x] - base).all()


def test_gradient_sum_with_constant_table_is_the_plain_sum():
    L0, L1, _ = synth.bands_pair(40, 24, seed=8)
    Cv = ref.cost_volume(L0, L1, 5, 12)
    lut = np.full(256, 10)
    for npaths in (4, 8):
        assert (ref.aggregate_grad(Cv, npaths, 10, 30, grad_lut=lut, I0=L0) ==
                ref.aggregate(Cv, npaths, 10, 30)).all()


def test_gradient_table_frees_jumps_across_an_edge():
    # 1x3 scanline, intensities 10, 10, 200: the step into x=2 crosses a 190-level edge
    # whose slope is 0, so the jump there is free; the step into x=1 costs p1 per label
    img = np.array([[10, 10, 200]], np.uint8)
    lut = np.full(256, 10)
    lut[190] = 0
    Cv = np.array([[[0, 50], [0, 50], [50, 0]]], np.int32)
    L, _ = ref.path_pen(Cv, 1, 0, 10, NT, grad_lut=lut, I0=img)
    # x=1: A = [0, 50] -> M' = [0, 10]; L = [0, 60] - 0
    assert L[0, 1].tolist() == [0, 60]
    # x=2: A = [0, 60], slope 0 -> M' = [0, 0]; L = [50, 0]
    assert L[0, 2].tolist() == [50, 0]
    Lp, _ = ref.path_pen(Cv, 1, 0, 10, NT)          # no table: the jump costs 10
    assert Lp[0, 2].tolist() == [50, 10]


# ------------------------------------------------------------------------------------
# the layered merge
# ------------------------------------------------------------------------------------

def test_double_penalty_hand_case():
    # two pixels of one row, labels {0,1}.  Left-to-right: jumping up 0 -> 1 costs 2*p1,
    # jumping down 1 -> 0 costs p1 (p1 = 10, no truncation)
    Cv = np.array([[[0, 100], [100, 0]]], np.int32)
    F, _ = ref.path_pen(Cv, 1, 0, 10, NT, double_up=True)
    assert F[0, 1].tolist() == [100, 20]
    F, _ = ref.path_pen(Cv, 1, 0, 10, NT, double_up=False)
    assert F[0, 1].tolist() == [100, 10]
    Cv = np.array([[[100, 0], [0, 100]]], np.int32)
    F, _ = ref.path_pen(Cv, 1, 0, 10, NT, double_up=True)
    assert F[0, 1].tolist() == [10, 100]              # downward jump: single penalty
    # with truncation T = 15 the doubled upward jump is capped at 2T = 30
    Cv = np.array([[[0, 100, 100, 100], [100, 100, 100, 0]]], np.int32)
    F, _ = ref.path_pen(Cv, 1, 0, 10, 15, double_up=True)
    assert F[0, 1, 3] == 30


@pytest.mark.parametrize("npaths", [4, 8])
@pytest.mark.parametrize("windowed", [False, True])
@pytest.mark.parametrize("gradient", [False, True])
def test_paper_merge_brute_force(npaths, windowed, gradient):
    Cv, lo, img = _case(40 + npaths + 2 * windowed + gradient, 4, 3, 3, 6, windowed)
    lut = (np.arange(256) * 7 % 9) if gradient else None
    T = 25 if npaths == 8 else NT
    want = _brute_paper(Cv, lo, npaths, 9, T, lut, img if gradient else None)
    got = ref.aggregate_paper(Cv, npaths, 9, T, lo=lo, grad_lut=lut,
                              I0=img if gradient else None)
    assert (got == want).all()


def test_paper_merge_on_a_row_is_min_of_the_two_horizontal_passes():
    # on a 1-pixel-high image the vertical and diagonal chains are single pixels, whose
    # normalised passes are the normalised data term: the result is the horizontal layer
    rng = np.random.default_rng(5)
    Cv = rng.integers(0, 200, (1, 7, 4)).astype(np.int32)
    F = _brute_pass(Cv, np.zeros((1, 7), np.int32), 1, 0, 6, 20, double_up=True)
    B = _brute_pass(Cv, np.zeros((1, 7), np.int32), -1, 0, 6, 20)
    want = np.minimum(F - F.min(axis=2, keepdims=True), B - B.min(axis=2, keepdims=True))
    for npaths in (4, 8):
        assert (ref.aggregate_paper(Cv, npaths, 6, 20) == want).all()


def test_paper_merge_zero_penalty_is_per_pixel_argmin():
    L0, L1, _ = synth.bands_pair(64, 40, seed=2)
    p = ref.params(max_disparity=24, num_scales=1, num_paths=8, p1=0, trunc=0, lr_check=0,
                   merge_mode=ref.MERGE_PAPER)
    d = ref.match_view(L0, L1, p)
    Cv = ref.cost_volume(L0, L1, 5, 24)
    assert (d == np.argmin(Cv, axis=2)).all()


@pytest.mark.parametrize("npaths", [4, 8])
def test_paper_merge_exact_recovery_single_plane(npaths):
    W, H, d = 96, 48, 7
    L0, L1 = synth.plane_pair(W, H, d, seed=11)
    p = ref.params(max_disparity=16, num_scales=1, num_paths=npaths, lr_check=0,
                   merge_mode=ref.MERGE_PAPER)
    out = ref.match_view(L0, L1, p)
    m = 2 + 4
    assert (out[m:H - m, d + m:W - m] == d).all()


def test_paper_merge_energies_stay_within_sixteen_bits():
    L0, L1, _ = synth.bands_pair(48, 32, seed=6)
    Cv = ref.cost_volume(L0, L1, 5, 16)
    S = ref.aggregate_paper(Cv, 8, 10, 30)
    # each layer adds at most one (doubled for left-to-right) truncated jump
    assert S.min() >= 0 and S.max() <= 255 + 5 * 30
    assert (S.min(axis=2) >= 0).all()


def test_merge_and_table_validation():
    assert ref.check_params(64, 48, ref.params(merge_mode=2)) != 0
    bad = np.zeros(256, np.int32)
    bad[3] = 11                                    # above p1 = 10
    assert ref.check_params(64, 48, ref.params(p1=10, grad_lut=bad)) != 0
    assert ref.check_params(64, 48, ref.params(p1=10, grad_lut=np.full(256, 10))) == 0
