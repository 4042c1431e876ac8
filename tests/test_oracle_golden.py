"""Stored values: the paper's printed complexity ratios, and oracle outputs written by
tests/golden/make_golden.py (a regression fixture for the GPU parity tests)."""
import hashlib
import os

import numpy as np

from oracle import ref
from paper_2001_09678_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_printed_complexity_ratios():
    # Section 3.4, Eqs. Ot0-O: per-level node counts over m*n*d, rounded as printed
    m, n, d = 1280, 720, 128
    p = ref.params(max_disparity=d, num_scales=3, num_paths=8)
    levels = []
    for l in range(3):
        Wl, Hl = ref.level_dims(m, n, 3, l)
        levels.append(Wl * Hl * ref.level_window(p, l))
    for key, printed in _rows("complexity_ratios.txt"):
        count = sum(levels) if key == "total" else levels[int(key)]
        assert round(count / (m * n * d), 4) == float(printed), key


def _kw(s):
    return {k: int(v) for k, v in (item.split("=") for item in s.split(","))}


def test_oracle_matches_stored_outputs():
    for name, W, H, seed, kv, digest in _rows("oracle_disparity.txt"):
        L, R, _ = synth.bands_pair(int(W), int(H), seed=int(seed))
        d = ref.match(L, R, ref.params(**_kw(kv)))
        assert hashlib.sha256(d.astype("<u2").tobytes()).hexdigest() == digest, name
