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

Training checkpoint (little endian): b"MPVC", version=1, layers, D, factor as int32, then
the Adam step, the generated pairs consumed, the samples seen and the next data seed as
int64, the sampler's RNG state (int64 length, then bytes), per layer (cin, cout, relu) as
int32, then per layer the fp32 weights, biases, and the Adam first and second moments of
both; last, the CRC-32 (zlib) of every preceding byte as uint32.  A training run resumed
from it continues the same data stream and optimizer; its replay buffer starts empty and
refills from the next pairs.
"""
from __future__ import annotations

import os
import struct
import zlib

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


CKPT_MAGIC, CKPT_VERSION = b"MPVC", 1


def save_checkpoint(path, state):
    """state: dict(layers=[(w, b, relu)], adam=[(mw, vw, mb, vb)], step, pairs, samples,
    next_seed, rng (bytes), D, factor).  Written to a temporary file and renamed, so a
    crash mid-write leaves the previous checkpoint intact."""
    parts = [CKPT_MAGIC, struct.pack("<4i", CKPT_VERSION, len(state["layers"]), state["D"],
                                     state["factor"]),
             struct.pack("<4q", state["step"], state["pairs"], state["samples"],
                         state["next_seed"]),
             struct.pack("<q", len(state["rng"])), bytes(state["rng"])]
    for w, b, relu in state["layers"]:
        parts.append(struct.pack("<3i", w.shape[1], w.shape[0], int(relu)))
    for (w, b, _), (mw, vw, mb, vb) in zip(state["layers"], state["adam"]):
        for a in (w, b, mw, vw, mb, vb):
            parts.append(np.ascontiguousarray(a, np.float32).tobytes())
    body = b"".join(parts)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))
    os.replace(tmp, path)


def load_checkpoint(path):
    """The state save_checkpoint wrote; ValueError on a wrong magic, version, size or CRC."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < 4 + 16 + 32 + 8 + 4 or data[:4] != CKPT_MAGIC:
        raise ValueError("not a proposal training checkpoint")
    body, (crc,) = data[:-4], struct.unpack("<I", data[-4:])
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError("checkpoint CRC mismatch (corrupt or truncated file)")
    ver, n, D, factor = struct.unpack_from("<4i", body, 4)
    if ver != CKPT_VERSION:
        raise ValueError(f"checkpoint version {ver}, expected {CKPT_VERSION}")
    step, pairs, samples, next_seed = struct.unpack_from("<4q", body, 20)
    (nrng,) = struct.unpack_from("<q", body, 52)
    off = 60
    rng = body[off:off + nrng]
    off += nrng
    shapes = []
    for _ in range(n):
        shapes.append(struct.unpack_from("<3i", body, off))
        off += 12
    layers, adam = [], []
    for cin, cout, relu in shapes:
        arrs = []
        for size, shape in ((cout * cin * 9, (cout, cin, 3, 3)), (cout, (cout,)),
                            (cout * cin * 9, (cout, cin, 3, 3)), (cout * cin * 9, (cout, cin, 3, 3)),
                            (cout, (cout,)), (cout, (cout,))):
            arrs.append(np.frombuffer(body, np.float32, size, off).reshape(shape).copy())
            off += 4 * size
        w, b, mw, vw, mb, vb = arrs
        layers.append((w, b, bool(relu)))
        adam.append((mw, vw, mb, vb))
    if off != len(body):
        raise ValueError("checkpoint size does not match its header")
    return dict(layers=layers, adam=adam, step=step, pairs=pairs, samples=samples,
                next_seed=next_seed, rng=rng, D=D, factor=factor)


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

    def adam_state(self):
        return [tuple(L[k].cpu().numpy() for k in ("mw", "vw", "mb", "vb")) for L in self.layers]

    @classmethod
    def from_checkpoint(cls, state, device="cuda"):
        """A network with the checkpoint's weights, Adam moments and step."""
        net = cls(state["layers"], device)
        torch = net.torch
        for L, moments in zip(net.layers, state["adam"]):
            for k, a in zip(("mw", "vw", "mb", "vb"), moments):
                L[k].copy_(torch.from_numpy(np.ascontiguousarray(a)))
        net.step = int(state["step"])
        return net

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


# ---------------------------------------------------------------------------------------
# Training and evaluation
# ---------------------------------------------------------------------------------------

W_TRAIN, H_TRAIN, D_TRAIN, S_TRAIN = 1280, 720, 128, 3
BASE = dict(max_disparity=D_TRAIN, num_scales=S_TRAIN, num_paths=8, p1=10, trunc=30)


def _gen_pair(seed):
    from . import synth
    L, R, _ = synth.slanted_pair(W_TRAIN, H_TRAIN, seed=seed)
    return seed, L, R


def _constant_layers(cin0, value):
    layers = init_weights(cin0, seed=0)
    out = []
    for i, (w, b, relu) in enumerate(layers):
        w = np.zeros_like(w)
        b = np.zeros_like(b)
        if i == len(layers) - 1:
            b[:] = value
        out.append((w, b, relu))
    return out


class _Samples:
    """Features and targets of both views of each pair, produced by the library."""

    def __init__(self, torch):
        self.torch = torch
        f = 1 << (S_TRAIN - 1)
        self.Wq, self.Hq = (W_TRAIN + f - 1) // f, (H_TRAIN + f - 1) // f
        self.cin = 2 + (D_TRAIN + f - 1) // f
        self.ctx = mpv.mpv_create(0)
        mpv.mpv_set_params(self.ctx, mpv.mpv_default_params(lr_check=0, **BASE))
        self.disp = torch.empty((H_TRAIN, W_TRAIN), dtype=torch.int16, device="cuda")
        self.disp_r = torch.empty((H_TRAIN, W_TRAIN), dtype=torch.int16, device="cuda")

    def make(self, L, R, feats_out, targets_out):
        """Writes 2 samples (left view, mirrored right view) into the given slots."""
        torch = self.torch
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        mpv.mpv_proposal_features(self.ctx, l, r, 0, feats_out[0])
        mpv.mpv_proposal_features(self.ctx, l, r, 1, feats_out[1])
        mpv.mpv_match_batch(self.ctx, [dict(left=l, right=r, disp=self.disp,
                                            disp_right=self.disp_r)])
        f = 1 << (S_TRAIN - 1)
        mpv.mpv_cnn_target(self.disp, f, D_TRAIN, targets_out[0])
        # the right view's map in the mirrored problem's coordinates
        mirrored = torch.flip(self.disp_r, dims=[1]).contiguous()
        mpv.mpv_cnn_target(mirrored, f, D_TRAIN, targets_out[1])

    def close(self):
        mpv.mpv_destroy(self.ctx)


def train(seconds=600.0, out="proposal.bin", capacity=4096, batch=8, steps_per_pair=4,
          lr=1e-3, delta=1.0 / 128, seed0=10000, log=print, checkpoint=None,
          checkpoint_every=300.0, resume=None):
    """Trains on generated pairs for `seconds`.  checkpoint: a path written every
    checkpoint_every seconds and at the end; resume: a checkpoint to continue from (its
    optimizer state, step, data position and sampler; the learning-rate schedule
    continues from the elapsed fraction it implies)."""
    import multiprocessing as mp
    import os
    import time

    import torch
    mpv.load()
    smp = _Samples(torch)
    feats = torch.empty((capacity, smp.cin, smp.Hq, smp.Wq), dtype=torch.bfloat16, device="cuda")
    targets = torch.empty((capacity, 1, smp.Hq, smp.Wq), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cpu").manual_seed(0)
    n = 0
    pairs = 0
    seed_next = seed0
    if resume:
        st = load_checkpoint(resume)
        net = Net.from_checkpoint(st)
        n, pairs, seed_next = int(st["samples"]), int(st["pairs"]), int(st["next_seed"])
        gen.set_state(torch.frombuffer(bytearray(st["rng"]), dtype=torch.uint8))
        log(f"resumed at step {net.step}, {pairs} pairs, next seed {seed_next}")
    else:
        net = Net(init_weights(smp.cin, seed=1))
    t0 = time.perf_counter()
    t_ckpt = t0

    def write_ckpt():
        save_checkpoint(checkpoint, dict(layers=net.numpy_layers(), adam=net.adam_state(),
                                         step=net.step, pairs=pairs, samples=n,
                                         next_seed=seed_next, rng=gen.get_state().numpy().tobytes(),
                                         D=D_TRAIN, factor=1 << (S_TRAIN - 1)))
    losses = []
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        for _seed, L, R in pool.imap(_gen_pair, range(seed_next, seed_next + 10**6), 4):
            seed_next = _seed + 1
            slot = n % capacity
            s2 = (slot + 1) % capacity
            smp.make(L, R, (feats[slot], feats[s2]), (targets[slot], targets[s2]))
            n += 2
            pairs += 1
            have = min(n, capacity)
            for _ in range(steps_per_pair):
                idx = torch.randint(0, have, (batch,), generator=gen).cuda()
                frac = min(1.0, (time.perf_counter() - t0) / seconds)
                step_lr = lr * (0.1 ** frac)
                loss = net.train_step(feats[idx].contiguous(), targets[idx].contiguous(),
                                      step_lr, delta)
            if pairs % 50 == 0:
                losses.append(float(loss.item()))
                log(f"pairs {pairs} samples {n} loss {losses[-1]:.5f} "
                    f"t {time.perf_counter() - t0:.0f}s")
            if checkpoint and time.perf_counter() - t_ckpt > checkpoint_every:
                write_ckpt()
                t_ckpt = time.perf_counter()
            if time.perf_counter() - t0 > seconds:
                pool.terminate()
                break
    smp.close()
    if checkpoint:
        write_ckpt()
    save_weights(out, net.numpy_layers(), D_TRAIN, 1 << (S_TRAIN - 1))
    return dict(pairs=pairs, samples=n, steps=net.step, losses=losses,
                seconds=time.perf_counter() - t0)


def evaluate(weights, npairs=40, seed0=900000, log=print):
    """Bad-pixel rate (> 1 px) against full-range single-scale MPV of: the pyramid, the
    trained proposal, an untrained network and a constant-centre network, each network on
    its own windows (no fallback); edge-hit rate and frame time of each, and how many
    frames each network's matcher re-matches under the default fallback."""
    import multiprocessing as mp
    import os
    import tempfile
    import time

    import torch
    mpv.load()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        data = pool.map(_gen_pair, range(seed0, seed0 + npairs))
    f = 1 << (S_TRAIN - 1)
    cin = 2 + (D_TRAIN + f - 1) // f
    tmp = tempfile.mkdtemp()
    variants = {"trained": weights}
    for name, layers in (("untrained", init_weights(cin, seed=7)),
                         ("constant", _constant_layers(cin, 0.5))):
        p = os.path.join(tmp, name + ".bin")
        save_weights(p, layers, D_TRAIN, f)
        variants[name] = p

    def ctx_for(**kw):
        c = mpv.mpv_create(0)
        prm = dict(BASE)
        prm.update(kw)
        mpv.mpv_set_params(c, mpv.mpv_default_params(**prm))
        return c

    full = ctx_for(num_scales=1)
    pyr = ctx_for()
    learned = {}
    defaults = {}      # the same networks with the matcher's default fallback
    for name, p in variants.items():
        c = ctx_for(proposal=mpv.MPV_PROPOSAL_LEARNED, fallback=mpv.MPV_FALLBACK_NONE)
        mpv.mpv_load_proposal_weights(c, p)
        learned[name] = c
        c = ctx_for(proposal=mpv.MPV_PROPOSAL_LEARNED)
        mpv.mpv_load_proposal_weights(c, p)
        defaults[name] = c
    stats = {k: dict(bad=0, both=0, edge=0, px=0, ms=0.0, fallback=0)
             for k in ["pyramid"] + list(variants)}
    d_ref = torch.empty((H_TRAIN, W_TRAIN), dtype=torch.int16, device="cuda")
    d = torch.empty_like(d_ref)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _seed, L, R in data:
        l, r = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
        mpv.mpv_match(full, l, r, d_ref)
        ref_np = d_ref.cpu().numpy().view(np.uint16)
        for name, c in [("pyramid", pyr)] + list(learned.items()):
            for _ in range(2):           # the second run is timed (warm workspace)
                ev0.record()
                mpv.mpv_match(c, l, r, d)
                ev1.record()
            torch.cuda.synchronize()
            st = stats[name]
            st["ms"] += ev0.elapsed_time(ev1)
            got = d.cpu().numpy().view(np.uint16)
            both = (got != 0xFFFF) & (ref_np != 0xFFFF)
            st["both"] += int(both.sum())
            st["bad"] += int((np.abs(got.astype(int) - ref_np.astype(int)) > 1)[both].sum())
            if name != "pyramid":
                hits, px = mpv.mpv_proposal_stats(c)
                st["edge"] += hits
                st["px"] += px
        for c in defaults.values():
            mpv.mpv_match(c, l, r, d)
        torch.cuda.synchronize()
    falls = {}
    for name, c in defaults.items():
        mpv.mpv_sync(c)
        falls[name] = mpv.mpv_proposal_fallbacks(c)[1]
    for c in [full, pyr] + list(learned.values()) + list(defaults.values()):
        mpv.mpv_destroy(c)
    out = {}
    for k, st in stats.items():
        out[k] = dict(bad_pixel_rate=st["bad"] / max(1, st["both"]),
                      edge_hit_rate=(st["edge"] / st["px"]) if st["px"] else None,
                      ms_per_frame=st["ms"] / npairs)
        if k in falls:
            out[k]["fallbacks_with_default"] = falls[k]
        log(f"{k:10s} bad>1px {out[k]['bad_pixel_rate']:.4f}  edge {out[k]['edge_hit_rate']}  "
            f"{out[k]['ms_per_frame']:.3f} ms")
    return out


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=600.0)
    ap.add_argument("--out", default="proposal.bin")
    ap.add_argument("--eval-pairs", type=int, default=40)
    ap.add_argument("--eval-only", action="store_true")
    ap.add_argument("--report", default=None)
    ap.add_argument("--checkpoint", default=None, help="write a training checkpoint here")
    ap.add_argument("--resume", default=None, help="continue from this checkpoint")
    args = ap.parse_args()
    res = {}
    if not args.eval_only:
        res["train"] = train(seconds=args.seconds, out=args.out, checkpoint=args.checkpoint,
                             resume=args.resume)
    res["eval"] = evaluate(args.out, npairs=args.eval_pairs)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(res, f, indent=1)
    print(json.dumps(res["eval"]))


if __name__ == "__main__":
    main()
