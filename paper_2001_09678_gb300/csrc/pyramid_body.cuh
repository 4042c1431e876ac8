// pyramid_body.cuh -- pyramid, window seeding, winner-take-all and left-right check (see
// pyramid.cu) as device functions of (block or pixel index, thread index), shared by the
// stand-alone kernels and the batch scheduler's persistent kernel.
#pragma once
#include "mpv_internal.cuh"

namespace mpv {

namespace {

__device__ __forceinline__ void mirror_body(const ImageJob &j, int W, int H, int x, int y)
{
    if (x >= W || y >= H) return;
    j.dst[(int64_t)y * j.dst_pitch + x] = j.src[(int64_t)y * j.src_pitch + (W - 1 - x)];
}

// 2x2 box mean, round half up; the last row/column is replicated when odd.
__device__ __forceinline__ void down2_body(const ImageJob &j, int W, int H, int x, int y)
{
    const int W2 = (W + 1) >> 1, H2 = (H + 1) >> 1;
    if (x >= W2 || y >= H2) return;
    const int x0 = 2 * x, x1 = min(2 * x + 1, W - 1);
    const int y0 = 2 * y, y1 = min(2 * y + 1, H - 1);
    const uint8_t *r0 = j.src + (int64_t)y0 * j.src_pitch;
    const uint8_t *r1 = j.src + (int64_t)y1 * j.src_pitch;
    const int s = r0[x0] + r0[x1] + r1[x0] + r1[x1];
    j.dst[(int64_t)y * j.dst_pitch + x] = (uint8_t)((s + 2) >> 2);
}

// The next two pyramid levels of up to four images in one launch, the first from the
// source (read mirrored for the right view's pair, whose full-resolution copy is written
// on the way), the second from the first through shared memory.  Same arithmetic as two
// down2 passes: 2x2 box mean, round half up, last row/column replicated when odd
// at each level.  A block makes 64 x 2 pixels of the first level and 32 x 1 of the second.
constexpr int kPyrCols = 64;

// One block of pyramid2_kernel (block (bx, by) of image j); threads at or beyond
// 2 * kPyrCols only join the block barrier.
__device__ __forceinline__ void pyramid2_body(const PyrJob &j, int W, int H, int bx, int by, int tid,
                                              uint8_t (*t1)[kPyrCols])
{
    const int W1 = (W + 1) >> 1, H1 = (H + 1) >> 1;
    const int tx = tid % kPyrCols, ty = tid / kPyrCols;
    const int x = bx * kPyrCols + tx, y = by * 2 + ty;
    if (tid < 2 * kPyrCols && x < W1 && y < H1) {
        const int x0 = 2 * x, x1 = min(2 * x + 1, W - 1);
        const int y0 = 2 * y, y1 = min(2 * y + 1, H - 1);
        const int c0 = j.mirror ? W - 1 - x0 : x0, c1 = j.mirror ? W - 1 - x1 : x1;
        const uint8_t *r0 = j.src + (int64_t)y0 * j.src_pitch;
        const uint8_t *r1 = j.src + (int64_t)y1 * j.src_pitch;
        const int a = r0[c0], b = r0[c1], c = r1[c0], d = r1[c1];
        const uint8_t v = (uint8_t)((a + b + c + d + 2) >> 2);
        j.d1[(int64_t)y * j.p1 + x] = v;
        t1[ty][tx] = v;
        if (j.full) {   // each full-resolution pixel of the mirrored copy once
            uint8_t *f0 = j.full + (int64_t)y0 * j.full_pitch;
            f0[x0] = (uint8_t)a;
            if (2 * x + 1 < W) f0[x0 + 1] = (uint8_t)b;
            if (2 * y + 1 < H) {
                uint8_t *f1 = f0 + j.full_pitch;
                f1[x0] = (uint8_t)c;
                if (2 * x + 1 < W) f1[x0 + 1] = (uint8_t)d;
            }
        }
    }
    if (!j.d2) return;   // the same for the whole block (one image per block)
    __syncthreads();
    if (tid < kPyrCols / 2) {
        const int W2 = (W1 + 1) >> 1, H2 = (H1 + 1) >> 1;
        const int X = bx * (kPyrCols / 2) + tid, Y = by;
        if (X < W2 && Y < H2) {
            // first-level pixels 2X, min(2X+1, W1-1) and rows 2Y, min(2Y+1, H1-1): all in
            // this block's tile
            const int u0 = 2 * tid;
            const int u1 = min(2 * X + 1, W1 - 1) - bx * kPyrCols;
            const int v1 = min(2 * Y + 1, H1 - 1) - 2 * Y;
            const int sum = t1[0][u0] + t1[0][u1] + t1[v1][u0] + t1[v1][u1];
            j.d2[(int64_t)Y * j.p2 + X] = (uint8_t)((sum + 2) >> 2);
        }
    }
}

// Window start of pixel (x, y) of `view` (seed_kernel).
__device__ __forceinline__ void seed_body(const SeedArgs &a, int x, int y, int view)
{
    if (x >= a.W || y >= a.H) return;
    const uint16_t *dp = a.dprev[view];
    if (!MPV_IN(a.err, (x >> 1) < a.Wp && (y >> 1) < a.Hp, 11)) return;
    int c;
    if (a.block == 2) {
        // the same rule on the block's (up to) four values, each loaded once
        const int qx0 = (x >> 1) & ~1, qy0 = (y >> 1) & ~1;
        const bool hx = qx0 + 1 < a.Wp, hy = qy0 + 1 < a.Hp;
        const uint16_t *r0 = dp + (int64_t)qy0 * a.Wp + qx0;
        int v[4], ok[4];
        v[0] = r0[0];
        ok[0] = 1;
        v[1] = hx ? r0[1] : 0;
        ok[1] = hx;
        v[2] = hy ? r0[a.Wp] : 0;
        ok[2] = hy;
        v[3] = (hx && hy) ? r0[a.Wp + 1] : 0;
        ok[3] = hx && hy;
        int best = 0x7FFFFFFF, best_n = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            int m = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) m += ok[q] && v[q] == v[p];
            if (ok[p] && (m > best_n || (m == best_n && v[p] < best))) {
                best = v[p];
                best_n = m;
            }
        }
        c = 2 * best;
    } else if (a.block >= 2) {
        // mode of the doubled coarse disparities of the block, ties to the smaller value
        const int b = a.block;
        const int qx0 = ((x >> 1) / b) * b, qy0 = ((y >> 1) / b) * b;
        const int qx1 = min(qx0 + b, a.Wp), qy1 = min(qy0 + b, a.Hp);
        int best = 0x7FFFFFFF, best_n = 0;
        for (int qy = qy0; qy < qy1; ++qy)
            for (int qx = qx0; qx < qx1; ++qx) {
                const int v = dp[(int64_t)qy * a.Wp + qx];
                int m = 0;
                for (int ry = qy0; ry < qy1; ++ry)
                    for (int rx = qx0; rx < qx1; ++rx) m += (dp[(int64_t)ry * a.Wp + rx] == v);
                if (m > best_n || (m == best_n && v < best)) {
                    best = v;
                    best_n = m;
                }
            }
        c = 2 * best;
    } else {
        // each pixel its own block: even positions copy, odd ones take the rounded
        // mean of their 2 or 4 doubled neighbours (index clamped at the border)
        const int xa = x >> 1, xb = (x & 1) ? min((x + 1) >> 1, a.Wp - 1) : xa;
        const int ya = y >> 1, yb = (y & 1) ? min((y + 1) >> 1, a.Hp - 1) : ya;
        const int nx = (x & 1) ? 2 : 1, ny = (y & 1) ? 2 : 1;
        int sum = dp[(int64_t)ya * a.Wp + xa];
        if (nx == 2) sum += dp[(int64_t)ya * a.Wp + xb];
        if (ny == 2) {
            sum += dp[(int64_t)yb * a.Wp + xa];
            if (nx == 2) sum += dp[(int64_t)yb * a.Wp + xb];
        }
        const int k = nx * ny;
        c = (2 * sum + (k >> 1)) / k;
    }
    const int lo = min(max(c - (a.Dw >> 1), 0), a.D - a.Dw);
    a.lo[view][(int64_t)y * a.W + x] = (uint16_t)lo;
}


// Winner-take-all over each pixel's window, ties to the smallest disparity.  Four lanes
// per pixel; the key (S << 16 | k) orders by energy, then by label.

// LPP lanes per pixel: 4, or 2 for 16-label strides (two 8-label chunks)
// Thread g (of LPP per pixel) of wta_kernel for `view`; every lane of the warp calls it.
template <int LPP>
__device__ __forceinline__ void wta_body(const LevelArgs &a, int64_t g, int view)
{
    const int64_t i = g / LPP;
    const int sub = (int)(g % LPP);
    const int64_t npx = (int64_t)a.W * a.H;
    const bool in = i < npx;
    const ViewLevel &v = a.v[view];
    uint32_t best = 0xFFFFFFFFu;
    if (in) {
        // rows of Dws = 16k labels are 32k-byte aligned: each lane reads 8 labels at a
        // time, the pixel's 4 lanes consecutive 16-byte chunks
        const uint4 *row = (const uint4 *)(v.S + i * a.Dws);
        const uint4 *row2 = v.S2 ? (const uint4 *)(v.S2 + i * a.Dws) : nullptr;
        for (int c = sub; c < a.Dws / 8; c += LPP) {
            uint4 q = row[c];
            if (row2) {   // layered merge: the last layer's two passes, floor of the mean
                const uint4 q2 = row2[c];
                q.x = avg_u16x2(q.x, q2.x);
                q.y = avg_u16x2(q.y, q2.y);
                q.z = avg_u16x2(q.z, q2.z);
                q.w = avg_u16x2(q.w, q2.w);
            }
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = c * 8 + e;
                const uint32_t val = (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xFFFFu);
                if (k < a.Dw) best = min(best, (val << 16) | (uint32_t)k);
            }
        }
    }
#pragma unroll
    for (int o = 1; o < LPP; o <<= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    const int lo = (in && v.lo) ? (int)v.lo[i] : 0;
    if (in && sub == 0) v.d[i] = (uint16_t)(lo + (best & 0xFFFFu));
}

// Left-right check.  dRm is the right view's map in mirrored coordinates.
__device__ __forceinline__ void lr_body(const uint16_t *__restrict__ dL,
                                        const uint16_t *__restrict__ dRm, int W, int H, int tol,
                                        int check, uint16_t *out, int out_pitch,
                                        uint16_t *out_right, int right_pitch, int x, int y)
{
    if (x >= W || y >= H) return;
    const int64_t row = (int64_t)y * W;
    const int d = dL[row + x];
    uint16_t v = (uint16_t)d;
    if (check) {
        v = 0xFFFFu;
        if (x - d >= 0) {
            const int dr = dRm[row + (W - 1 - (x - d))];
            if (abs(d - dr) <= tol) v = (uint16_t)d;
        }
    }
    out[(int64_t)y * out_pitch + x] = v;
    if (out_right) out_right[(int64_t)y * right_pitch + x] = dRm[row + (W - 1 - x)];
}

}  // namespace

}  // namespace mpv
