"""The two reformulations of the Section 3.3 envelope that the packed GPU passes evaluate,
restated plainly and checked against the oracle's two-sweep envelope with separate upward
and downward slopes and caps:

* the doubled left-to-right pass of the layered merge (upward jumps cost 2 min(P d, T)) as
  a radius-R stencil plus two caps, min_v A(v) + 2T and min_{v>=u} A(v) + T, exact when
  every jump beyond R labels is truncated;
* the untruncated sweeps F(u) = min_{v<=u} A(v) + Pu (u-v), G(u) = min_{v>=u} A(v) +
  Pd (v-u) capped by min_v A(v) + T (any slope, Eq. EU's per-step weights), formed over the
  predecessor's window and continued linearly from its edge labels for current labels
  beyond it.

Labels are absolute: the predecessor's window starts at lo_prev, the current one at lo.
"""
import numpy as np
import pytest

from oracle import ref

BIG = 1 << 40


def _pred(A, q):
    """Predecessor energy at predecessor index q (absent outside its window)."""
    return int(A[q]) if 0 <= q < len(A) else BIG


def doubled_stencil(A, lo_prev, lo, P, T, R):
    """min(A(u), A(u-d) + 2 min(P d, T), A(u+d) + min(P d, T) for d <= R,
           min_v A(v) + 2T, min_{v>=u} A(v) + T)  for each current label u."""
    Dw = len(A)
    m = int(A.min())
    s = lo - lo_prev
    out = np.zeros(Dw, np.int64)
    for j in range(Dw):
        q = j + s                                       # predecessor index of label lo + j
        suffix = m if q < 0 else (int(A[q:].min()) if q < Dw else BIG)
        best = min(_pred(A, q), m + 2 * T, suffix + T)
        for d in range(1, R + 1):
            best = min(best, _pred(A, q - d) + 2 * min(P * d, T), _pred(A, q + d) + min(P * d, T))
        out[j] = best
    return out


def capped_sweeps(A, lo_prev, lo, Pu, Pd, Tu, Td):
    """Untruncated sweeps over the predecessor's window, linear continuation beyond it, then
    the caps (min A + Tu, and for unequal caps the suffix minimum + Td)."""
    Dw = len(A)
    m = int(A.min())
    F = [min(int(A[v]) + Pu * (q - v) for v in range(q + 1)) for q in range(Dw)]
    G = [min(int(A[v]) + Pd * (v - q) for v in range(q, Dw)) for q in range(Dw)]
    s = lo - lo_prev
    out = np.zeros(Dw, np.int64)
    for j in range(Dw):
        q = j + s
        if q >= Dw:       # above every predecessor label: upward jumps only
            out[j] = min(F[Dw - 1] + Pu * (q - Dw + 1), m + Tu)
        elif q < 0:       # below every predecessor label: downward jumps only
            out[j] = min(G[0] + Pd * (-q), m + Td)
        else:
            v = min(F[q], G[q], m + Tu)
            if Tu != Td:
                v = min(v, int(A[q:].min()) + Td)
            out[j] = v
    return out


@pytest.mark.parametrize("seed", range(6))
def test_doubled_pass_stencil_form_equals_the_envelope(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(60):
        Dw = int(rng.integers(1, 33))
        R = int(rng.choice([2, 4]))
        P = int(rng.integers(1, 60))
        T = int(rng.integers(P, (R + 1) * P + 1))      # every jump beyond R labels costs T
        A = rng.integers(0, 400, Dw).astype(np.int64)
        lo_prev = int(rng.integers(0, 60))
        lo = max(0, lo_prev + int(rng.integers(-45, 46)) if rng.random() < 0.7 else lo_prev)
        want = ref.envelope_pen(A, lo_prev, lo, 2 * P, P, 2 * T, T)
        assert np.array_equal(doubled_stencil(A, lo_prev, lo, P, T, R), want)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("doubled", [False, True])
def test_capped_sweeps_equal_the_envelope(seed, doubled):
    rng = np.random.default_rng(200 + seed + 50 * doubled)
    for _ in range(60):
        Dw = int(rng.integers(1, 33))
        T = int(rng.integers(0, 200))
        P = int(rng.integers(0, T + 2))                # zero slopes and slopes above T
        A = rng.integers(0, 400, Dw).astype(np.int64)
        lo_prev = int(rng.integers(0, 60))
        lo = max(0, lo_prev + int(rng.integers(-45, 46)) if rng.random() < 0.7 else lo_prev)
        up = 2 if doubled else 1
        # a slope above T acts as T: the truncated cost min(P d, T) is then T for every d
        Pe = min(P, T)
        want = ref.envelope_pen(A, lo_prev, lo, up * P, P, up * T, T)
        got = capped_sweeps(A, lo_prev, lo, up * Pe, Pe, up * T, T)
        assert np.array_equal(got, want)


def test_minimum_outside_the_window_reaches_a_byte_plus_t():
    # With windows the predecessor's best label can lie outside the current window: every
    # current label then pays a jump, and the energies' minimum L = C + M' - min A reaches
    # C + T (here the cost is 255 everywhere).  The packed kernels' sentinel has to stay
    # above the cap min A + T formed from such minima (255 + 2T).
    P, T, Dw = 10, 30, 8
    A = np.array([0] + [500] * (Dw - 1), np.int64)      # best label at the bottom
    M = ref.envelope_pen(A, 0, 10, P, P, T, T)          # the window moved up by 10 labels
    L = 255 + M - A.min()
    assert L.min() == 255 + T
