// cost_body.cuh -- the integer SSIM cost volume (see cost.cu), as a device function of
// (block index, thread index) shared by the stand-alone kernel and the batch
// scheduler's persistent kernel.
#pragma once
#include "mpv_internal.cuh"

namespace mpv {

namespace {

constexpr int kSegPix = 256;          // pixels per block (one row segment)
constexpr int kCostThreads = 256;
constexpr int kCostWarps = kCostThreads / 32;

// Floor of 255 (den - num) / (2 den) for |num| <= den, den > 0, exactly, where
// num = A1 A2 and den = B1 B2.  fA1, fB1, fB2 are float evaluations of A1, B1, B2 (each
// from at most three correctly rounded operations on exact integers below 2^27: relative
// error <= 3 * 2^-24), fA2 = (float)A2; the products and the fast division add 4 * 2^-24,
// so |num/den| <= 1 is known to 10 * 2^-24 and t = 127.5 (1 - num/den) to better than
// 127.5 * 10 * 2^-24 + 2 ulp(255) < 1.1e-4.  A fractional part of t in [1e-3, 1 - 1e-3]
// therefore already has the exact floor; otherwise the integers decide.
__device__ __forceinline__ int ssim_quotient(float fA1, float fA2, float fB1, float fB2,
                                             int A2, int sx, int vx, int sy, int vy, int c1,
                                             int c2)
{
    const float t = fmaf(-127.5f, __fdividef(fA1 * fA2, fB1 * fB2), 127.5f);
    const float fl = floorf(t);
    const float fr = t - fl;
    int q = (int)fl;
    if (fr < 1e-3f || fr > 1.0f - 1e-3f) {
        const long long A1 = 2LL * sx * sy + c1;
        const long long B1 = (long long)sx * sx + (long long)sy * sy + c1;
        const long long B2 = (long long)vx + vy + c2;
        const long long dd = B1 * B2;
        const long long nn = A1 * A2;
        const long long X = 255LL * (dd - nn);
        const long long Y = 2LL * dd;
        q = min(max(q, 0), 255);
        long long R = X - (long long)q * Y;
        while (R < 0) {
            --q;
            R += Y;
        }
        while (R >= Y) {
            ++q;
            R -= Y;
        }
    }
    return q;
}

// Shared-memory layout of one block.
struct CostSmem {
    int ncol0, ncol1;     // staged columns of I0 and I1
    int nc1;              // I1 centres with statistics
    size_t off_col0, off_col1, off_cs, off_st0, off_st1, bytes;
};

__host__ __device__ inline CostSmem cost_smem_layout(int R, int uspan_max)
{
    CostSmem L;
    L.ncol0 = kSegPix + 2 * R + 2;
    L.ncol1 = kSegPix + 2 * R + 1 + uspan_max;
    L.nc1 = kSegPix + uspan_max;
    size_t o = 0;
    L.off_col0 = o;
    o += sizeof(uint2) * L.ncol0;
    L.off_col1 = o;
    o += sizeof(uint2) * L.ncol1;
    L.off_cs = o;                          // column sums and sums of squares (int2)
    o += sizeof(int2) * (L.ncol1 > L.ncol0 ? L.ncol1 : L.ncol0);
    o = (o + 15) & ~(size_t)15;
    L.off_st0 = o;                         // I0 statistics of the segment's pixels
    o += sizeof(int4) * kSegPix;
    L.off_st1 = o;                         // I1 statistics of the reachable centres
    o += sizeof(int4) * L.nc1;
    L.bytes = o;
    return L;
}

template <int N>
__device__ __forceinline__ int colprod(uint2 a, uint2 b)
{
    return (int)__dp4a(a.x, b.x, N == 5 ? __dp4a(a.y, b.y, 0u) : 0u);
}

// Packs column xc (clamped) of rows y-R..y+R (clamped) and returns (sum, sum of squares).
template <int N>
__device__ __forceinline__ uint2 pack_column(const uint8_t *img, int pitch, int W, int H, int y,
                                             int xc, int2 &ss)
{
    constexpr int R = N / 2;
    const int xa = min(max(xc, 0), W - 1);
    uint32_t w0 = 0, w1 = 0;
#pragma unroll
    for (int r = 0; r < N; ++r) {
        const int yy = min(max(y - R + r, 0), H - 1);
        const uint32_t v = img[(int64_t)yy * pitch + xa];
        if (r < 4)
            w0 |= v << (8 * r);
        else
            w1 = v;
    }
    ss.x = (int)__dp4a(w0, 0x01010101u, w1);
    ss.y = (int)__dp4a(w0, w0, w1 * w1);
    return make_uint2(w0, w1);
}

// One block of the cost kernel: row segment bx, row by, view bz; smem: the block's
// dynamic shared memory (cost_smem_layout bytes).
template <int N>
__device__ __forceinline__ void cost_body(const LevelArgs &a, int uspan_max, int bx, int by,
                                          int bz, int tid, unsigned char *smem)
{
    constexpr int R = N / 2;
    constexpr int n = N * N;
    constexpr int NR = 2 * R + 1;          // ring of column products
    const int view = bz;
    const ViewLevel &V = a.v[view];
    const int W = a.W, H = a.H, Dw = a.Dw, Dws = a.Dws;
    const int y = by;
    // the row's ceil(W / kSegPix) segments of equal width, a multiple of 32 pixels (whole
    // pixels for every warp and sub-stream): the widest block sets a launch's time
    const int nseg = (W + kSegPix - 1) / kSegPix;
    const int seg = min(kSegPix, ((W + nseg - 1) / nseg + 31) & ~31);
    const int x0 = bx * seg;
    const int npx = min(seg, W - x0);
    if (npx <= 0) return;   // (whole block; only for rows far wider than 8192 pixels)
    const int c1 = a.c1, c2 = a.c2;

    __shared__ int lo_s[kSegPix];
    __shared__ int red[2];
    const CostSmem L = cost_smem_layout(R, uspan_max);
    uint2 *col0 = (uint2 *)(smem + L.off_col0);
    uint2 *col1 = (uint2 *)(smem + L.off_col1);
    int2 *cs = (int2 *)(smem + L.off_cs);
    int4 *st0 = (int4 *)(smem + L.off_st0);
    int4 *st1 = (int4 *)(smem + L.off_st1);

    if (a.zero_s) {   // this segment's summed energies start at zero (16-byte stores)
        uint4 *sz = (uint4 *)(V.S + ((int64_t)y * W + x0) * Dws);
        const int n16 = npx * Dws / 8;     // Dws is a multiple of 16
        for (int i = tid; i < n16; i += kCostThreads) sz[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        red[0] = 0x7FFFFFFF;
        red[1] = 0;
    }
    __syncthreads();
    for (int i = tid; i < npx; i += kCostThreads) {
        const int l = V.lo ? (int)V.lo[(int64_t)y * W + x0 + i] : 0;
        lo_s[i] = l;
        atomicMin(&red[0], l);
        atomicMax(&red[1], l);
    }
    __syncthreads();
    const int umin = red[0], umax = red[1] + Dw - 1;
    const int uspan = umax - umin;
    const int b0 = x0 - R - 1 - umax;       // first staged I1 column
    const int a0 = x0 - R - 1;              // first staged I0 column
    const int nb = npx + 2 * R + 1 + uspan; // staged I1 columns
    const int na = npx + 2 * R + 2;
    const int ncen = npx + uspan;           // I1 centres x0 - umax .. x0 + npx - 1 - umin

    // I0: packed columns, column sums, then patch statistics of the segment's pixels
    for (int i = tid; i < na; i += kCostThreads) {
        int2 ss;
        col0[i] = pack_column<N>(V.I0, V.pitch0, W, H, y, a0 + i, ss);
        cs[i] = ss;
    }
    __syncthreads();
    for (int i = tid; i < npx; i += kCostThreads) {
        int s = 0, q = 0;
#pragma unroll
        for (int d = 0; d < NR; ++d) {   // centre x0+i is staged column i + R + 1
            const int2 t = cs[i + 1 + d];
            s += t.x;
            q += t.y;
        }
        const int v = n * q - s * s;
        st0[i] = make_int4(s, v, __float_as_int((float)s), __float_as_int((float)v));
    }
    __syncthreads();
    // I1: packed columns, column sums, statistics of every reachable centre
    for (int i = tid; i < nb; i += kCostThreads) {
        int2 ss;
        col1[i] = pack_column<N>(V.I1, V.pitch1, W, H, y, b0 + i, ss);
        cs[i] = ss;
    }
    __syncthreads();
    for (int i = tid; i < ncen; i += kCostThreads) {
        // centre x' = x0 - umax + i is staged column i + R + 1
        int s = 0, q = 0;
#pragma unroll
        for (int d = 0; d < NR; ++d) {
            const int2 t = cs[i + 1 + d];
            s += t.x;
            q += t.y;
        }
        const int v = n * q - s * s;
        st1[i] = make_int4(s, v, __float_as_int((float)s), __float_as_int((float)v));
    }
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const int LP = Dws < 32 ? Dws : 32;     // lanes per pixel stream
    const int nsub = 32 / LP;
    const int sub = lane / LP, kl = lane - sub * LP;
    const int per_warp = seg / kCostWarps;
    const int sub_len = per_warp / nsub;
    const int xs = warp * per_warp + sub * sub_len;      // segment-relative
    const int xe = min(xs + sub_len, npx);
    const float c1f = (float)c1, c2f = (float)c2;
    uint8_t *out = V.C + ((int64_t)y * W + x0) * Dws;

    for (int k = kl; k < Dws; k += LP) {
        if (k >= Dw) {           // padding labels: never read as costs
            for (int x = xs; x < xe; ++x) out[(int64_t)x * Dws + k] = 255;
            continue;
        }
        int ring[NR];
        int sxy = 0;
        int prev_lo = -1;
        for (int xb = xs; xb < xe; xb += NR) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const int x = xb + j;            // segment-relative pixel
                if (x < xe) {
                    const int lo = lo_s[x];
                    const int u = lo + k;
                    // I0 column of virtual column x0+x+d is staged at x + 1 + R + d;
                    // I1 column of x0+x+d-u at x + 1 + R + d + umax - u
                    const int ib = x + 1 + R + umax - u;
                    if (!MPV_IN(a.err, ib - R >= 0 && ib + R < nb && x + 1 + 2 * R < na &&
                                           x + umax - u >= 0 && x + umax - u < ncen, 10)) {
                        prev_lo = -1;   // (bounds-checked builds) skip this node
                        continue;
                    }
                    if (lo != prev_lo) {
                        sxy = 0;
#pragma unroll
                        for (int d = -R; d <= R; ++d) {
                            const int p = colprod<N>(col0[x + 1 + R + d], col1[ib + d]);
                            ring[(j + d + NR) % NR] = p;
                            sxy += p;
                        }
                        prev_lo = lo;
                    } else {
                        const int p = colprod<N>(col0[x + 1 + 2 * R], col1[ib + R]);
                        sxy += p - ring[(j + R) % NR];
                        ring[(j + R) % NR] = p;
                    }
                    const int xp = x0 + x - u;
                    int q = 255;
                    if (xp >= 0) {
                        const int4 s0 = st0[x];
                        const int4 s1 = st1[x + umax - u];
                        const int A2 = 2 * (n * sxy - s0.x * s1.x) + c2;
                        const float fsx = __int_as_float(s0.z), fsy = __int_as_float(s1.z);
                        const float fA1 = fmaf(2.0f * fsx, fsy, c1f);
                        const float fB1 = fmaf(fsx, fsx, fmaf(fsy, fsy, c1f));
                        const float fB2 = __int_as_float(s0.w) + (__int_as_float(s1.w) + c2f);
                        q = ssim_quotient(fA1, (float)A2, fB1, fB2, A2, s0.x, s0.y, s1.x, s1.y,
                                          c1, c2);
                    }
                    out[(int64_t)x * Dws + k] = (uint8_t)q;
                }
            }
        }
    }
}

}  // namespace

}  // namespace mpv
