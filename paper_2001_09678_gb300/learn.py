"""Learned disparity-window proposal: network, training loop and weight files.

The network (six 3x3 convolutions, 2 + D_top -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU
between them) reads the top pyramid level of a pair -- its left and right images and
its full-range cost slice -- and predicts, per top-level pixel, the full-resolution
disparity divided by D.  The matcher turns the prediction into a window of Dw labels
per full-resolution pixel (centre +- Dw/2) in place of the pyramid's seeding.

Every arithmetic step runs in the library's kernels (mpv_cnn_*): forward convolutions,
ReLU and convolution backward passes, the Huber loss and the Adam update.  torch only
holds the device buffers.  Training labels are the plain pyramid matcher's own maps.

Weight file (little endian): b"MPVP", version=1, layers, D, factor, then per layer
(cin, cout, relu) as int32, then per layer the fp32 weights [cout][cin][3][3] and the
fp32 biases [cout].
"""
from __future__ import annotations

import struct

import numpy as np

from . import mpv

HIDDEN = 32
LAYERS = 6


def layer_shapes(cin0: int):
    shapes = []
    cin = cin0
    for i in range(LAYERS):
        cout = 1 if i == LAYERS - 1 else HIDDEN
        shapes.append((cin, cout, i < LAYERS - 1))
        cin = cout
    return shapes


def init_weights(cin0: int, seed: int = 0):
    """He-scaled uniform initial weights (numpy fp32) and zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout, relu in layer_shapes(cin0):
        bound = np.sqrt(6.0 / (cin * 9)) * (1.0 if relu else 0.1)
        w = rng.uniform(-bound, bound, (cout, cin, 3, 3)).astype(np.float32)
        b = np.zeros(cout, np.float32)
        if not relu:
            b[:] = 0.3
        out.append((w, b, relu))
    return out


def save_weights(path, layers, D, factor):
    with open(path, "wb") as f:
        f.write(b"MPVP" + struct.pack("<4i", 1, len(layers), D, factor))
        for w, b, relu in layers:
            f.write(struct.pack("<3i", w.shape[1], w.shape[0], int(relu)))
        for w, b, relu in layers:
            f.write(np.ascontiguousarray(w, np.float32).tobytes())
            f.write(np.ascontiguousarray(b, np.float32).tobytes())


def load_weights(path):
    with open(path, "rb") as f:
        data = f.read()
    assert data[:4] == b"MPVP", "not a proposal weight file"
    ver, n, D, factor = struct.unpack_from("<4i", data, 4)
    assert ver == 1
    off = 20
    shapes = []
    for _ in range(n):
        shapes.append(struct.unpack_from("<3i", data, off))
        off += 12
    layers = []
    for cin, cout, relu in shapes:
        w = np.frombuffer(data, np.float32, cout * cin * 9, off).reshape(cout, cin, 3, 3).copy()
        off += 4 * w.size
        b = np.frombuffer(data, np.float32, cout, off).copy()
        off += 4 * cout
        layers.append((w, b, bool(relu)))
    return layers, D, factor


class Net:
    """Device copies of the weights (fp32 master, bf16 working copy) and Adam state."""

    def __init__(self, layers, device="cuda"):
        import torch
        self.torch = torch
        self.device = device
        self.layers = []
        for w, b, relu in layers:
            wf = torch.from_numpy(np.ascontiguousarray(w)).to(device)
            bf = torch.from_numpy(np.ascontiguousarray(b)).to(device)
            wb = torch.empty(wf.shape, dtype=torch.bfloat16, device=device)
            mpv.mpv_cnn_to_bf16(wf, wb)
            self.layers.append(dict(w=wf, b=bf, wb=wb, relu=relu,
                                    mw=torch.zeros_like(wf), vw=torch.zeros_like(wf),
                                    mb=torch.zeros_like(bf), vb=torch.zeros_like(bf)))
        self.step = 0

    def numpy_layers(self):
        return [(L["w"].cpu().numpy(), L["b"].cpu().numpy(), L["relu"]) for L in self.layers]

    def forward(self, x_bf16):
        """x: [N, Cin, H, W] bf16 -> (prediction fp32 [N,1,H,W], stored activations)."""
        torch = self.torch
        N, _, H, W = x_bf16.shape
        acts = [x_bf16]
        h = x_bf16
        out = None
        for i, L in enumerate(self.layers):
            cout = L["w"].shape[0]
            if i + 1 < len(self.layers):
                nxt = torch.empty((N, cout, H, W), dtype=torch.bfloat16, device=self.device)
                mpv.mpv_cnn_conv3x3(h, L["wb"], L["b"], cout, L["relu"], out_bf16=nxt)
                acts.append(nxt)
                h = nxt
            else:
                out = torch.empty((N, cout, H, W), dtype=torch.float32, device=self.device)
                mpv.mpv_cnn_conv3x3(h, L["wb"], L["b"], cout, L["relu"], out_f32=out)
        return out, acts

    def backward(self, acts, gout):
        """Weight and bias gradients (fp32) for output gradient gout [N,1,H,W]."""
        torch = self.torch
        grads = [None] * len(self.layers)
        g = gout
        for i in range(len(self.layers) - 1, -1, -1):
            L = self.layers[i]
            if L["relu"]:
                gm = torch.empty_like(g)
                mpv.mpv_cnn_relu_backward(g, acts[i + 1], gm)
                g = gm
            dw = torch.zeros_like(L["w"])
            db = torch.zeros_like(L["b"])
            mpv.mpv_cnn_conv3x3_wgrad(acts[i], g, dw, db)
            grads[i] = (dw, db)
            if i > 0:
                cin = L["w"].shape[1]
                wt = torch.empty((cin, L["w"].shape[0], 3, 3), dtype=torch.bfloat16,
                                 device=self.device)
                mpv.mpv_cnn_flip_transpose(L["wb"], wt)
                dx = torch.empty((g.shape[0], cin, g.shape[2], g.shape[3]), dtype=torch.float32,
                                 device=self.device)
                mpv.mpv_cnn_conv3x3(g, wt, None, cin, False, out_f32=dx)
                g = dx
        return grads

    def adam(self, grads, lr):
        self.step += 1
        for L, (dw, db) in zip(self.layers, grads):
            mpv.mpv_cnn_adam(L["w"], dw, L["mw"], L["vw"], lr, self.step, weight_bf16=L["wb"])
            mpv.mpv_cnn_adam(L["b"], db, L["mb"], L["vb"], lr, self.step)

    def train_step(self, x_bf16, target, lr, delta):
        torch = self.torch
        pred, acts = self.forward(x_bf16)
        grad = torch.empty_like(pred)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        mpv.mpv_cnn_huber(pred, target, delta, grad, loss)
        grads = self.backward(acts, grad)
        self.adam(grads, lr)
        return loss
