"""Writes the stored oracle outputs under tests/golden/ (calls only the oracle).

Run from the repository root:  python tests/golden/make_golden.py
The inputs come from the integer-only scene recipe (uniform bytes, 3x3 box, bands),
which is bit-identical on every machine.
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ref  # noqa: E402
from paper_2001_09678_gb300 import synth  # noqa: E402

CASES = [
    # name, W, H, seed, params
    ("bands_64x48_d16_s1_p4", 64, 48, 0, dict(max_disparity=16, num_scales=1, num_paths=4)),
    ("bands_96x64_d32_s2_p8", 96, 64, 1, dict(max_disparity=32, num_scales=2, num_paths=8)),
]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_disparity.txt")
    lines = ["# name W H seed params sha256(uint16 little-endian disparity, LR-checked)"]
    for name, W, H, seed, kw in CASES:
        L, R, _ = synth.bands_pair(W, H, seed=seed)
        d = ref.match(L, R, ref.params(**kw))
        h = hashlib.sha256(d.astype("<u2").tobytes()).hexdigest()
        kv = ",".join(f"{k}={v}" for k, v in kw.items())
        lines.append(f"{name} {W} {H} {seed} {kv} {h}")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
