"""The learned proposal's BF16/FP32 network kernels against the float64 CNN oracle.

The oracle is fed the same BF16-rounded inputs and weights the device holds, so the
remaining differences come from FP32 accumulation (and, through the network, from BF16
rounding of activations that sit near a rounding boundary): the tolerances below are
stated relative to the magnitude of the summed terms.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cnn_ref  # noqa: E402


@pytest.fixture(scope="module")
def m():
    from paper_2001_09678_gb300 import build, mpv
    build.build()
    mpv.load()
    return mpv


def _bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)


def test_conv_forward_matches_oracle(m):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 34, 37, 45)).astype(np.float32)
    w = (rng.normal(size=(32, 34, 3, 3)) * 0.1).astype(np.float32)
    b = rng.normal(size=32).astype(np.float32)
    out = torch.empty((2, 32, 37, 45), dtype=torch.float32, device="cuda")
    m.mpv_cnn_conv3x3(_bf(x), _bf(w), torch.from_numpy(b).cuda(), 32, True, out_f32=out)
    xq, wq = cnn_ref.bf16(x), cnn_ref.bf16(w)
    want = np.maximum(cnn_ref.conv3x3(xq, wq, b), 0)
    scale = cnn_ref.conv3x3(np.abs(xq), np.abs(wq)) + np.abs(b)[None, :, None, None]
    assert np.all(np.abs(out.cpu().numpy() - want) <= 1e-5 * scale + 1e-6)


@pytest.mark.parametrize("n,cin,cout,h,w,relu", [
    (1, 5, 32, 17, 9, True),       # one k-step, most channels padding
    (3, 32, 1, 45, 61, False),     # the output layer's width (one channel of 16)
    (2, 33, 32, 30, 70, True),     # a ragged last k-step, ragged tiles in x and y
    (1, 208, 32, 19, 21, True),    # the widest input the shared-memory operands hold
    (2, 34, 32, 180, 320, True),   # the network's first layer at its size: more tiles
])                                 # than blocks, so blocks loop over tiles
def test_conv_tensor_core_shapes(m, n, cin, cout, h, w, relu):
    # BF16 input with 32 or 1 output channels runs on the tcgen05 kernel; the BF16 output
    # is the FP32 one rounded to nearest even
    rng = np.random.default_rng(cin * 7 + cout)
    x = rng.normal(size=(n, cin, h, w)).astype(np.float32)
    wt = (rng.normal(size=(cout, cin, 3, 3)) * 0.1).astype(np.float32)
    b = rng.normal(size=cout).astype(np.float32)
    out = torch.full((n, cout, h, w), float("nan"), dtype=torch.float32, device="cuda")
    outb = torch.empty((n, cout, h, w), dtype=torch.bfloat16, device="cuda")
    m.mpv_cnn_conv3x3(_bf(x), _bf(wt), torch.from_numpy(b).cuda(), cout, relu, out_bf16=outb,
                      out_f32=out)
    xq, wq = cnn_ref.bf16(x), cnn_ref.bf16(wt)
    want = cnn_ref.conv3x3(xq, wq, b)
    if relu:
        want = np.maximum(want, 0)
    scale = cnn_ref.conv3x3(np.abs(xq), np.abs(wq)) + np.abs(b)[None, :, None, None]
    got = out.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-5 * scale + 1e-6)
    assert torch.equal(outb, out.to(torch.bfloat16))


def test_conv_fp32_input_one_channel_out(m):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 32, 20, 17)).astype(np.float32)
    w = (rng.normal(size=(1, 32, 3, 3)) * 0.1).astype(np.float32)
    out = torch.empty((1, 1, 20, 17), dtype=torch.float32, device="cuda")
    m.mpv_cnn_conv3x3(torch.from_numpy(x).cuda(), _bf(w), None, 1, False, out_f32=out)
    wq = cnn_ref.bf16(w)
    want = cnn_ref.conv3x3(x.astype(np.float64), wq)
    scale = cnn_ref.conv3x3(np.abs(x.astype(np.float64)), np.abs(wq))
    assert np.all(np.abs(out.cpu().numpy() - want) <= 1e-5 * scale + 1e-6)


def test_weight_gradient_matches_oracle(m):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 32, 40, 36)).astype(np.float32)
    g = rng.normal(size=(2, 32, 40, 36)).astype(np.float32)
    dw = torch.zeros((32, 32, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.zeros(32, dtype=torch.float32, device="cuda")
    m.mpv_cnn_conv3x3_wgrad(_bf(x), torch.from_numpy(g).cuda(), dw, db)
    xq = cnn_ref.bf16(x)
    _, want_w, want_b = cnn_ref.conv3x3_backward(xq, np.zeros((32, 32, 3, 3)), g.astype(np.float64))
    _, scale_w, scale_b = cnn_ref.conv3x3_backward(np.abs(xq), np.zeros((32, 32, 3, 3)),
                                                   np.abs(g).astype(np.float64))
    assert np.all(np.abs(dw.cpu().numpy() - want_w) <= 1e-5 * scale_w + 1e-6)
    assert np.all(np.abs(db.cpu().numpy() - want_b) <= 1e-5 * scale_b + 1e-6)


def test_network_gradients_match_oracle(m):
    from paper_2001_09678_gb300 import learn
    rng = np.random.default_rng(3)
    layers = learn.init_weights(34, seed=4)
    net = learn.Net(layers)
    x = rng.uniform(-0.5, 0.5, size=(2, 34, 24, 20)).astype(np.float32)
    t = rng.uniform(0, 1, size=(2, 1, 24, 20)).astype(np.float32)
    xb = _bf(x)
    pred, acts = net.forward(xb)
    grad = torch.empty_like(pred)
    loss = torch.zeros(1, device="cuda")
    m.mpv_cnn_huber(pred, torch.from_numpy(t).cuda(), 1.0 / 128, grad, loss)
    grads = net.backward(acts, grad)
    # forward: the device stores every hidden activation in BF16; a value whose FP32 and
    # float64 sums straddle a BF16 rounding boundary rounds one BF16 ulp (2^-8 relative)
    # differently, and that propagates: agreement to 1e-3 of the output scale
    p_ref, _ = cnn_ref.forward(x, layers, round_bf16=True)
    assert np.allclose(pred.cpu().numpy(), p_ref, rtol=1e-3, atol=1e-3)
    # backward: fed the device's own stored activations (same ReLU masks), the float64
    # chain rule must agree with the FP32 kernels to FP32 accumulation error
    acts_dev = [a.float().cpu().numpy().astype(np.float64) for a in acts]
    _, g_ref = cnn_ref.huber(pred.cpu().numpy().astype(np.float64), t, 1.0 / 128)
    grads_ref = cnn_ref.backward(acts_dev, layers, g_ref, round_bf16=True)
    # element by element, against the magnitude of the summed terms: the same chain run on
    # |activations|, |weights| and |output gradient| (the ReLU masks are unchanged, the
    # stored activations past a ReLU being >= 0).  FP32 accumulation of at most
    # N*H*W = 960 terms per weight-gradient element and 288 per data-gradient element,
    # compounded over the six layers, stays below 2e-4 of that magnitude.
    layers_abs = [(np.abs(w), np.abs(b), relu) for (w, b, relu) in layers]
    scales = cnn_ref.backward([np.abs(a) for a in acts_dev], layers_abs, np.abs(g_ref),
                              round_bf16=True)
    for i, ((dw, db), (rw, rb), (sw, sb)) in enumerate(zip(grads, grads_ref, scales)):
        dw, db = dw.cpu().numpy(), db.cpu().numpy()
        bad_w = np.abs(dw - rw) > 2e-4 * sw + 1e-12
        bad_b = np.abs(db - rb) > 2e-4 * sb + 1e-12
        assert not bad_w.any(), f"layer {i}: {bad_w.sum()} weight-gradient elements off"
        assert not bad_b.any(), f"layer {i}: {bad_b.sum()} bias-gradient elements off"
        # where the terms cancel (deep layers) that bound is loose; the whole gradient must
        # then also agree to 1e-4 relative in norm
        assert np.linalg.norm(dw - rw) <= 1e-4 * np.linalg.norm(rw), i
        assert np.linalg.norm(db - rb) <= 1e-4 * (np.linalg.norm(rb) + 1e-30), i


def test_huber_and_adam(m):
    p = torch.tensor([0.0, 0.1, 2.0, -3.0], device="cuda")
    t = torch.zeros(4, device="cuda")
    g = torch.empty(4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    m.mpv_cnn_huber(p, t, 0.5, g, loss)
    assert np.allclose(g.cpu().numpy(), np.array([0, 0.2, 1, -1]) / 4)
    assert np.isclose(loss.item(), (0.01 + 1.75 + 2.75) / 4)
    w = torch.tensor([1.0, -2.0], device="cuda")
    gr = torch.tensor([0.5, -0.25], device="cuda")
    mm, vv = torch.zeros(2, device="cuda"), torch.zeros(2, device="cuda")
    m.mpv_cnn_adam(w, gr, mm, vv, 0.1, 1)
    # first bias-corrected Adam step moves each weight by lr * sign(g) (up to eps)
    assert np.allclose(w.cpu().numpy(), [0.9, -1.9], atol=1e-6)


def test_training_reduces_loss(m):
    from paper_2001_09678_gb300 import learn
    rng = np.random.default_rng(5)
    net = learn.Net(learn.init_weights(34, seed=6))
    xn = rng.uniform(-0.5, 0.5, size=(4, 34, 32, 32)).astype(np.float32)
    x = _bf(xn)
    # a target the network can fit: an affine function of the first input channel
    t = torch.from_numpy((0.5 + 0.5 * xn[:, :1]).astype(np.float32)).cuda()
    losses = [net.train_step(x, t, 3e-3, 1.0 / 128).item() for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]


def test_resumed_training_equals_uninterrupted(m, tmp_path):
    # one 16x16 sample: the weight gradient is one block's sums (no atomic reordering), so
    # training is bitwise reproducible and a resumed run must equal an uninterrupted one
    from paper_2001_09678_gb300 import learn
    rng = np.random.default_rng(9)
    xn = rng.uniform(-0.5, 0.5, size=(1, 34, 16, 16)).astype(np.float32)
    x = _bf(xn)
    t = torch.from_numpy((0.5 + 0.5 * xn[:, :1]).astype(np.float32)).cuda()
    a = learn.Net(learn.init_weights(34, seed=10))
    for _ in range(5):
        a.train_step(x, t, 2e-3, 1.0 / 128)
    path = str(tmp_path / "mid.ckpt")
    learn.save_checkpoint(path, dict(layers=a.numpy_layers(), adam=a.adam_state(), step=a.step,
                                     pairs=0, samples=0, next_seed=0, rng=b"", D=128, factor=4))
    for _ in range(5):
        a.train_step(x, t, 2e-3, 1.0 / 128)
    b = learn.Net.from_checkpoint(learn.load_checkpoint(path))
    assert b.step == 5
    for _ in range(5):
        b.train_step(x, t, 2e-3, 1.0 / 128)
    torch.cuda.synchronize()
    assert a.step == b.step == 10
    for La, Lb in zip(a.layers, b.layers):
        for k in ("w", "b", "wb", "mw", "vw", "mb", "vb"):
            assert torch.equal(La[k], Lb[k]), k
