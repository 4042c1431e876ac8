"""Seeded synthetic stereo pairs shaped like driving scenes.

This module generates inputs only: it holds none of the matcher's arithmetic and is
shared by the tests, the benchmark and the training-data pipeline.  The paper's own
data (KITTI 2012 and its 640x480 driving sequences) is not available, so these scenes
stand in for it: piecewise-planar surfaces (the paper's TV prior models planes,
Section 3.2) over a textured left image, with the right image produced by warping with
the ground-truth disparity.

Random numbers come from a counter-based splitmix64 generator (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", 2014) so that every value is a pure
function of (seed, stream, index) on any machine.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def raw64(seed: int, stream: int, n: int) -> np.ndarray:
    """n raw 64-bit outputs of stream `stream` of generator `seed`."""
    key = _mix(np.array([(seed * 0x10001 + stream * 0x9E37 + 1) & 0xFFFFFFFFFFFFFFFF],
                        dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        ctr = np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN + key
    return _mix(ctr)


def uniform_bytes(seed, stream, shape):
    n = int(np.prod(shape))
    return (raw64(seed, stream, n) >> np.uint64(56)).astype(np.uint8).reshape(shape)


def uniform01(seed, stream, shape):
    n = int(np.prod(shape))
    return ((raw64(seed, stream, n) >> np.uint64(11)).astype(np.float64)
            * (1.0 / 9007199254740992.0)).reshape(shape)


def uniform_int(seed, stream, shape, lo, hi):
    """Integers in [lo, hi] by multiply-shift of the top 32 bits."""
    n = int(np.prod(shape))
    top = (raw64(seed, stream, n) >> np.uint64(32)).astype(np.uint64)
    span = np.uint64(hi - lo + 1)
    with np.errstate(over="ignore"):
        v = (top * span) >> np.uint64(32)
    return (v.astype(np.int64) + lo).reshape(shape)


def gaussian(seed, stream, shape):
    """Standard normal samples by the Box-Muller transform."""
    n = int(np.prod(shape))
    m = (n + 1) // 2
    u1 = uniform01(seed, stream, (m,))
    u2 = uniform01(seed, stream + 1000003, (m,))
    r = np.sqrt(-2.0 * np.log(1.0 - u1))
    z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
    return z[:n].reshape(shape)


def box3(img: np.ndarray) -> np.ndarray:
    """3x3 box smoothing with replicated border, (sum + 4) // 9 (texture recipe)."""
    p = np.pad(img.astype(np.int32), 1, mode="edge")
    H, W = img.shape
    s = sum(p[dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3))
    return ((s + 4) // 9).astype(np.uint8)


# ------------------------------------------------------------------------------------
# Gradient noise (Perlin's improved noise: quintic fade, hashed gradients, 2-D form)
# ------------------------------------------------------------------------------------

def _perm_table(seed, stream):
    p = np.arange(256, dtype=np.int64)
    r = uniform_int(seed, stream, (256,), 0, 1 << 30)
    for i in range(255, 0, -1):  # Fisher-Yates
        j = int(r[i] % (i + 1))
        p[i], p[j] = p[j], p[i]
    return np.concatenate([p, p])


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def gradient_noise(W, H, period, seed, stream):
    """One octave of 2-D gradient noise sampled at pixel centres, values about [-1, 1]."""
    perm = _perm_table(seed, stream)
    ang = 2.0 * math.pi * np.arange(16) / 16.0
    gx_t, gy_t = np.cos(ang), np.sin(ang)
    ys, xs = np.meshgrid((np.arange(H) + 0.5) / period, (np.arange(W) + 0.5) / period,
                         indexing="ij")
    xi, yi = np.floor(xs).astype(np.int64), np.floor(ys).astype(np.int64)
    xf, yf = xs - xi, ys - yi
    xi &= 255
    yi &= 255

    def grad(ix, iy, dx, dy):
        h = perm[perm[ix] + iy] & 15
        return gx_t[h] * dx + gy_t[h] * dy

    n00 = grad(xi, yi, xf, yf)
    n10 = grad(xi + 1, yi, xf - 1, yf)
    n01 = grad(xi, yi + 1, xf, yf - 1)
    n11 = grad(xi + 1, yi + 1, xf - 1, yf - 1)
    u, v = _fade(xf), _fade(yf)
    a = n00 + u * (n10 - n00)
    b = n01 + u * (n11 - n01)
    return (a + v * (b - a)) * 1.41421356


def perlin_texture(W, H, seed, stream, octaves=4, base_period=64.0, contrast=110.0):
    acc = np.zeros((H, W))
    amp_sum = 0.0
    for o in range(octaves):
        amp = 0.5 ** o
        acc += amp * gradient_noise(W, H, base_period / (2 ** o), seed, stream * 16 + o)
        amp_sum += amp
    return np.clip(np.rint(128.0 + contrast * acc / amp_sum * 2.0), 0, 255).astype(np.uint8)


# ------------------------------------------------------------------------------------
# Scenes
# ------------------------------------------------------------------------------------

def bands_pair(W=320, H=240, seed=0, disparities=(5, 12, 20), noise=2):
    """Three fronto-parallel planes in vertical bands.

    Left: uniform bytes smoothed by a 3x3 box.  Ground truth: band k (width W//3, the
    last takes the remainder) at disparity disparities[k].  Right pixel x' shows the
    nearest band (largest disparity) whose surface lands on it, i.e. x' + d_k inside
    band k; where none does, a fresh uniform byte.  Then uniform integer noise in
    [-noise, noise], clamped.  Returns (left, right, gt) as uint8, uint8, int32.
    """
    left = box3(uniform_bytes(seed, 0, (H, W)))
    bw = W // 3
    edges = [0, bw, 2 * bw, W]
    gt = np.zeros((H, W), np.int32)
    for k in range(3):
        gt[:, edges[k]:edges[k + 1]] = disparities[k]
    fresh = uniform_bytes(seed, 1, (H, W))
    right = fresh.copy()
    best = np.full(W, -1, np.int64)
    xs = np.arange(W)
    for k in range(3):
        d = disparities[k]
        src = xs + d
        ok = (src >= edges[k]) & (src < edges[k + 1]) & (d > best)
        best[ok] = d
    for xp in range(W):
        if best[xp] >= 0:
            right[:, xp] = left[:, xp + best[xp]]
    if noise:
        n = uniform_int(seed, 2, (H, W), -noise, noise)
        right = np.clip(right.astype(np.int64) + n, 0, 255).astype(np.uint8)
    return left, right, gt


def plane_pair(W, H, d, seed=0, smooth=False):
    """A single noise-free fronto-parallel plane at integer disparity d.

    Both images are cut from one uniform-byte texture of width W + d: left(x) = T(x),
    right(x') = T(x' + d), so that right(x - d) = left(x) exactly.
    """
    T = uniform_bytes(seed, 7, (H, W + d))
    if smooth:
        T = box3(T)
    return np.ascontiguousarray(T[:, :W]), np.ascontiguousarray(T[:, d:d + W])


def slanted_pair(W=1280, H=720, seed=0, n_planes=40, d_max=120.0, max_slope=0.2,
                 sigma=2.0):
    """Slanted planes on Voronoi regions over a gradient-noise texture.

    Left: 4-octave gradient noise, base period 64 px.  n_planes Voronoi seeds uniform in
    the image; region k carries the plane d = d0 + gx (x - sx) + gy (y - sy) with
    d0 ~ U[0, d_max] and |(gx, gy)| <= max_slope, clamped to [0, d_max].  Right pixel x'
    shows the front-most surface (largest disparity) whose point x with x - d(x) = x'
    lies in its own region; its intensity is the left image interpolated at x.  Pixels
    no surface reaches take an independent noise texture.  Then Gaussian noise of
    standard deviation sigma, rounded and clamped.
    Returns (left uint8, right uint8, gt float64 disparity).
    """
    left = perlin_texture(W, H, seed, 1)
    holes = perlin_texture(W, H, seed, 2)
    sxy = uniform01(seed, 3, (n_planes, 2)) * np.array([W, H])
    d0 = uniform01(seed, 4, (n_planes,)) * d_max
    ang = uniform01(seed, 5, (n_planes,)) * 2 * math.pi
    mag = uniform01(seed, 6, (n_planes,)) * max_slope
    gx, gy = mag * np.cos(ang), mag * np.sin(ang)

    ys, xs = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    # Voronoi labels (ties to the lower index)
    best = np.full((H, W), np.inf)
    label = np.zeros((H, W), np.int64)
    for k in range(n_planes):
        dist = (xs - sxy[k, 0]) ** 2 + (ys - sxy[k, 1]) ** 2
        m = dist < best
        best[m] = dist[m]
        label[m] = k

    def plane(k, x, y):
        return np.clip(d0[k] + gx[k] * (x - sxy[k, 0]) + gy[k] * (y - sxy[k, 1]), 0.0, d_max)

    gt = np.zeros((H, W))
    for k in range(n_planes):
        m = label == k
        gt[m] = plane(k, xs[m], ys[m])

    # z-buffered forward mapping, solved per plane in closed form inside the bounding
    # box of the plane's region (shifted left by up to d_max)
    zbest = np.full((H, W), -1.0)
    xsrc = np.zeros((H, W))
    for k in range(n_planes):
        yy, xx = np.nonzero(label == k)
        if yy.size == 0:
            continue
        y0, y1 = yy.min(), yy.max() + 1
        c0, c1 = max(0, int(xx.min() - d_max) - 2), min(W, int(xx.max()) + 2)
        ysb, xsb = ys[y0:y1, c0:c1], xs[y0:y1, c0:c1]
        rows = np.arange(y0, y1)[:, None].repeat(c1 - c0, 1)
        zb, xb = zbest[y0:y1, c0:c1], xsrc[y0:y1, c0:c1]
        a = 1.0 - gx[k]
        xk = (xsb + d0[k] - gx[k] * sxy[k, 0] + gy[k] * (ysb - sxy[k, 1])) / a
        for xc in (xk, xsb.copy(), xsb + d_max):   # the plane, and its two clamped parts
            inside = (xc >= 0) & (xc <= W - 1)
            xi = np.clip(np.rint(xc).astype(np.int64), 0, W - 1)
            dk = plane(k, xc, ysb)
            ok = inside & (label[rows, xi] == k) & (np.abs(xc - dk - xsb) < 1e-6) & (dk > zb)
            zb[ok] = dk[ok]
            xb[ok] = xc[ok]
    rows = np.arange(H)[:, None].repeat(W, 1)
    x0 = np.clip(np.floor(xsrc).astype(np.int64), 0, W - 1)
    x1 = np.clip(x0 + 1, 0, W - 1)
    f = xsrc - np.floor(xsrc)
    lf = left.astype(np.float64)
    warped = lf[rows, x0] * (1 - f) + lf[rows, x1] * f
    right = np.where(zbest >= 0, warped, holes.astype(np.float64))
    right = right + sigma * gaussian(seed, 8, (H, W))
    right = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return left, right, gt


MIXED_BATCH = ((16, 640, 480, 64), (32, 1280, 720, 128), (16, 1920, 1080, 192))


def mixed_batch_specs(counts=MIXED_BATCH, seed0=1000):
    """(seed, W, H, D) of the 64-pair mixed-resolution batch, in order."""
    out = []
    i = 0
    for n, W, H, D in counts:
        for _ in range(n):
            out.append((seed0 + i, W, H, D))
            i += 1
    return out


def road_disparity(W=1280, H=720, D=128, seed=0, horizon=300, rows_per_label=3,
                   n_obstacles=6, outliers=0.02, invalid=0.05):
    """A disparity map of a flat road seen by a level camera: rows below the horizon
    carry the disparity floor((y - horizon) / rows_per_label) (clipped to D - 1), rows
    above it a far background (0); n_obstacles fronto-parallel boxes standing on the road
    (constant disparity, the road's at their bottom row); a share of outliers (uniform
    disparities) and of rejected pixels (0xFFFF).  Returns uint16 [H][W]."""
    ys = np.arange(H)[:, None].repeat(W, 1)
    road = np.clip((ys - horizon) // rows_per_label, 0, D - 1)
    U = np.where(ys >= horizon, road, 0).astype(np.int64)
    box = uniform01(seed, 1, (n_obstacles, 4))
    for k in range(n_obstacles):
        bottom = int(horizon + 20 + box[k, 0] * (H - horizon - 21))
        d = int(min(D - 1, (bottom - horizon) // rows_per_label))
        h = int(10 + box[k, 1] * 3 * (d + 5))
        w = int(10 + box[k, 2] * 4 * (d + 5))
        x0 = int(box[k, 3] * max(1, W - w))
        U[max(0, bottom - h):bottom, x0:x0 + w] = d
    r = uniform01(seed, 2, (H, W))
    noise = uniform_int(seed, 3, (H, W), 0, D)
    U = np.where(r < outliers, noise, U)
    U = np.where((r >= outliers) & (r < outliers + invalid), 0xFFFF, U)
    return U.astype(np.uint16)
