"""Pins of the CNN oracle (oracle/cnn_ref.py): finite differences and closed forms."""
import numpy as np
import pytest

from oracle import cnn_ref


def test_bf16_rounding_ties_to_even():
    one = np.float32(1.0)
    vals = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, -2.5, 3.0e-3], np.float32)
    want = [1.0, 1.0, 1 + 2**-6, -2.5]
    got = cnn_ref.bf16(vals)
    assert list(got[:4]) == want
    torch = pytest.importorskip("torch")
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, ref)
    assert one == 1.0


def test_conv_identity_and_shift_kernels():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 5, 6))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0
    assert np.allclose(cnn_ref.conv3x3(x, w), x)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 1, 2] = 1.0            # out(y,x) = in(y, x+1), zero beyond the border
    y = cnn_ref.conv3x3(x[:, :1], w)
    assert np.allclose(y[:, 0, :, :-1], x[:, 0, :, 1:]) and np.allclose(y[:, 0, :, -1], 0)


def _numgrad(f, a, eps=1e-6):
    g = np.zeros_like(a)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = a[i]
        a[i] = old + eps
        fp = f()
        a[i] = old - eps
        fm = f()
        a[i] = old
        g[i] = (fp - fm) / (2 * eps)
    return g


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 4, 5))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    g = rng.normal(size=(2, 2, 4, 5))
    f = lambda: float((cnn_ref.conv3x3(x, w, b) * g).sum())
    dx, dw, db = cnn_ref.conv3x3_backward(x, w, g)
    assert np.allclose(dx, _numgrad(f, x), atol=1e-6)
    assert np.allclose(dw, _numgrad(f, w), atol=1e-6)
    assert np.allclose(db, _numgrad(f, b), atol=1e-6)


def test_network_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 4, 5, 4))
    layers = [(rng.normal(size=(3, 4, 3, 3)) * 0.5, rng.normal(size=3) * 0.1, True),
              (rng.normal(size=(3, 3, 3, 3)) * 0.5, rng.normal(size=3) * 0.1, True),
              (rng.normal(size=(1, 3, 3, 3)) * 0.5, rng.normal(size=1) * 0.1, False)]
    t = rng.normal(size=(1, 1, 5, 4))

    def loss():
        p, _ = cnn_ref.forward(x, layers, round_bf16=False)
        return cnn_ref.huber(p, t, 0.3)[0]

    p, acts = cnn_ref.forward(x, layers, round_bf16=False)
    _, gout = cnn_ref.huber(p, t, 0.3)
    grads = cnn_ref.backward(acts, layers, gout, round_bf16=False)
    for (w, b, _), (dw, db) in zip(layers, grads):
        assert np.allclose(dw, _numgrad(loss, w), atol=1e-5)
        assert np.allclose(db, _numgrad(loss, b), atol=1e-5)


def test_huber_closed_form():
    p = np.array([0.0, 0.1, 2.0, -3.0])
    t = np.zeros(4)
    loss, g = cnn_ref.huber(p, t, 0.5)
    assert np.isclose(loss, (0 + 0.5 * 0.01 / 0.5 + (2 - 0.25) + (3 - 0.25)) / 4)
    assert np.allclose(g, np.array([0, 0.2, 1, -1]) / 4)
