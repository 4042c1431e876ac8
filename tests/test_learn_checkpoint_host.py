"""Training checkpoints of the learned proposal (host side, no GPU): round trip, and
every kind of damage detected (CRC, truncation, version, magic)."""
import os
import struct

import numpy as np
import pytest

from paper_2001_09678_gb300 import learn


def _state(seed=0):
    rng = np.random.default_rng(seed)
    layers = learn.init_weights(34, seed=seed)
    adam = [tuple(rng.normal(size=a.shape).astype(np.float32) for a in (w, w, b, b))
            for w, b, _ in layers]
    return dict(layers=layers, adam=adam, step=1234, pairs=56, samples=112,
                next_seed=10056, rng=bytes(rng.integers(0, 256, 5056, dtype=np.uint8)),
                D=128, factor=4)


def test_round_trip(tmp_path):
    p = tmp_path / "c.ckpt"
    st = _state()
    learn.save_checkpoint(str(p), st)
    got = learn.load_checkpoint(str(p))
    for k in ("step", "pairs", "samples", "next_seed", "rng", "D", "factor"):
        assert got[k] == st[k], k
    for (w, b, r), (w2, b2, r2) in zip(st["layers"], got["layers"]):
        assert np.array_equal(w, w2) and np.array_equal(b, b2) and r == r2
    for m, m2 in zip(st["adam"], got["adam"]):
        assert all(np.array_equal(a, a2) for a, a2 in zip(m, m2))
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]   # written atomically


def test_damage_is_detected(tmp_path):
    p = tmp_path / "c.ckpt"
    learn.save_checkpoint(str(p), _state(1))
    good = p.read_bytes()
    for pos in (10, 100, len(good) // 2, len(good) - 5):     # any flipped byte
        bad = bytearray(good)
        bad[pos] ^= 0x40
        p.write_bytes(bytes(bad))
        with pytest.raises(ValueError):
            learn.load_checkpoint(str(p))
    p.write_bytes(good[:-100])                                 # truncated
    with pytest.raises(ValueError):
        learn.load_checkpoint(str(p))
    p.write_bytes(b"MPVP" + good[4:])                          # a weight file's magic
    with pytest.raises(ValueError):
        learn.load_checkpoint(str(p))
    # a future version with a valid CRC is refused by the version check
    import zlib
    body = bytearray(good[:-4])
    body[4:8] = struct.pack("<i", 2)
    p.write_bytes(bytes(body) + struct.pack("<I", zlib.crc32(bytes(body)) & 0xFFFFFFFF))
    with pytest.raises(ValueError, match="version"):
        learn.load_checkpoint(str(p))
