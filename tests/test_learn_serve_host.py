"""Host-side pieces of the learned proposal and the serving driver (no GPU)."""
import os
import tempfile

import numpy as np

from paper_2001_09678_gb300 import learn, serve


def test_weight_file_round_trip_is_bit_identical():
    layers = learn.init_weights(34, seed=3)
    fd, path = tempfile.mkstemp(suffix=".bin")
    os.close(fd)
    try:
        learn.save_weights(path, layers, 128, 4)
        back, D, f = learn.load_weights(path)
        assert (D, f) == (128, 4)
        for (w, b, r), (w2, b2, r2) in zip(layers, back):
            assert w.tobytes() == w2.tobytes() and b.tobytes() == b2.tobytes() and r == r2
        learn.save_weights(path + "2", back, D, f)
        assert open(path, "rb").read() == open(path + "2", "rb").read()
    finally:
        for p in (path, path + "2"):
            if os.path.exists(p):
                os.unlink(p)


def test_layer_shapes():
    shapes = learn.layer_shapes(34)
    assert shapes[0] == (34, 32, True) and shapes[-1] == (32, 1, False) and len(shapes) == 6


def test_camera_arrivals_are_poisson_at_the_rate():
    t = serve.arrivals(camera=3, hz=30.0, seconds=200.0)
    assert np.all(np.diff(t) > 0) and t[-1] < 200.0
    assert abs(len(t) / 200.0 - 30.0) < 1.5          # mean rate
    gaps = np.diff(t)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential gaps: CV = 1
    # seeded per camera: reproducible, and different cameras differ
    assert np.array_equal(t, serve.arrivals(camera=3, hz=30.0, seconds=200.0))
    assert not np.array_equal(t[:10], serve.arrivals(camera=4, hz=30.0, seconds=200.0)[:10])


def test_eight_camera_layout():
    cams = serve.camera_specs()
    assert len(cams) == 8
    assert sorted({(W, H, D) for _, W, H, D in cams}) == [(640, 480, 64), (1280, 720, 128),
                                                          (1920, 1080, 192)]
