"""CPU oracle of the learned-proposal network and its gradients (numpy, float64).

TEST INFRASTRUCTURE ONLY: used by the test suite to check the library's BF16/FP32 CNN
kernels; the matcher never imports it.  Written from the definitions: a 3x3
convolution with zero padding is a sum of nine shifted, channel-mixed copies of the
input; its gradients follow by the chain rule (backward data = the same sum with the
transposed, flipped kernel; backward weight = the correlation of the output gradient
with the shifted input).  `bf16` rounds to bfloat16 (round to nearest, ties to even)
so that the oracle can be fed exactly the values the device holds.
"""
import numpy as np


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b=None):
    """x [N,Cin,H,W], w [Cout,Cin,3,3] -> [N,Cout,H,W], zero padding."""
    N, Cin, H, W = x.shape
    xp = np.zeros((N, Cin, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((N, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + W])
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv3x3_backward(x, w, g):
    """Gradients of sum(g * conv3x3(x, w, b)) w.r.t. x, w and b."""
    N, Cin, H, W = x.shape
    xp = np.zeros((N, Cin, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dw = np.zeros_like(w, dtype=np.float64)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", g, xp[:, :, ky:ky + H, kx:kx + W])
            dxp[:, :, ky:ky + H, kx:kx + W] += np.einsum("oc,nohw->nchw", w[:, :, ky, kx], g)
    return dxp[:, :, 1:-1, 1:-1], dw, g.sum(axis=(0, 2, 3))


def huber(p, t, delta):
    r = p - t
    a = np.abs(r)
    n = r.size
    loss = np.where(a < delta, 0.5 * r * r / delta, a - 0.5 * delta).sum() / n
    grad = np.where(a < delta, r / delta, np.sign(r)) / n
    return loss, grad


def forward(x, layers, round_bf16=True):
    """layers: list of (w, b, relu).  Returns the output and the list of layer inputs
    (post-activation values as stored on the device: BF16 when round_bf16)."""
    acts = [bf16(x) if round_bf16 else np.asarray(x, np.float64)]
    h = acts[0]
    for i, (w, b, relu) in enumerate(layers):
        wq = bf16(w) if round_bf16 else w
        z = conv3x3(h, wq, b)
        if relu:
            z = np.maximum(z, 0.0)
        if i + 1 < len(layers):
            h = bf16(z) if round_bf16 else z
            acts.append(h)
        else:
            h = z
    return h, acts


def backward(acts, layers, gout, round_bf16=True):
    """Weight and bias gradients of every layer for output gradient gout."""
    grads = [None] * len(layers)
    g = gout
    for i in range(len(layers) - 1, -1, -1):
        w, b, relu = layers[i]
        wq = bf16(w) if round_bf16 else w
        if relu:
            # the device masks by the stored (post-ReLU) activation of this layer's output
            out_act = acts[i + 1] if i + 1 < len(acts) else None
            if out_act is not None:
                g = g * (out_act > 0)
        dx, dw, db = conv3x3_backward(acts[i], wq, g)
        grads[i] = (dw, db)
        g = dx
    return grads
