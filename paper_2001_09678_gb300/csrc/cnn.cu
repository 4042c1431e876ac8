// cnn.cu -- the learned disparity-window proposal: a small 3x3 CNN and its training
// kernels (forward, backward, loss, optimizer), plus its input features and its output
// windows.  BF16 activations and weights, FP32 accumulation and FP32 gradients.
//
// Network (trained by paper_2001_09678_gb300/learn.py): six 3x3 convolutions with zero
// padding, 2 + D_top input channels (the top pyramid level's left and right images and
// its full-range cost slice), 32 hidden channels with ReLU, 1 output channel: the
// disparity at full resolution divided by D, at the top level's resolution.
#include <cuda_bf16.h>

#include "mpv_internal.cuh"

namespace mpv {

namespace {

constexpr int kTile = 16;          // output tile side of the convolution kernels

// out[n][co][y][x] = b[co] + sum_{ci,ky,kx} w[co][ci][ky][kx] in[n][ci][y+ky-1][x+kx-1]
// (zero padding), optional ReLU; one thread per output pixel and all output channels.
__device__ __forceinline__ float ld_act(const __nv_bfloat16 *p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ld_act(const float *p, int64_t i) { return p[i]; }

template <int COUT, class TIn>
__global__ void __launch_bounds__(kTile *kTile) conv3x3_kernel(
    const TIn *__restrict__ in, int Cin, int H, int W,
    const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b, int relu,
    __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f)
{
    extern __shared__ float smem[];
    float *ws = smem;                                   // [Cin*9][COUT]
    float *tile = smem + Cin * 9 * COUT;                // [18][18] of one input channel
    const int n = blockIdx.z;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int x = x0 + tx, y = y0 + ty;
    for (int i = threadIdx.x; i < Cin * 9 * COUT; i += kTile * kTile) {
        const int co = i % COUT, r = i / COUT;         // r = ci*9 + k
        ws[i] = __bfloat162float(w[(int64_t)co * Cin * 9 + r]);
    }
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = b ? b[co] : 0.f;
    const int64_t plane = (int64_t)H * W;
    const TIn *src = in + (int64_t)n * Cin * plane;
    for (int ci = 0; ci < Cin; ++ci) {
        __syncthreads();
        for (int i = threadIdx.x; i < 18 * 18; i += kTile * kTile) {
            const int yy = y0 - 1 + i / 18, xx = x0 - 1 + i % 18;
            tile[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W)
                          ? ld_act(src, ci * plane + (int64_t)yy * W + xx)
                          : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = tile[(ty + k / 3) * 18 + tx + k % 3];
            const float *wr = ws + (ci * 9 + k) * COUT;
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wr[co], v, acc[co]);
        }
    }
    if (x >= W || y >= H) return;
    const int64_t o = (int64_t)n * COUT * plane + (int64_t)y * W + x;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        float v = acc[co];
        if (relu) v = fmaxf(v, 0.f);
        if (out_f) out_f[o + co * plane] = v;
        if (out_bf) out_bf[o + co * plane] = __float2bfloat16(v);
    }
}

// dW[co][ci][k] += sum over a tile of g[n][co][y][x] in[n][ci][y+ky-1][x+kx-1];
// db[co] += sum g.  One block per (tile, sample); partial sums added atomically.
__global__ void __launch_bounds__(kTile *kTile) conv3x3_wgrad_kernel(
    const __nv_bfloat16 *__restrict__ in, int Cin, const float *__restrict__ g, int Cout,
    int H, int W, float *__restrict__ dw, float *__restrict__ db)
{
    extern __shared__ float smem[];
    float *gt = smem;                         // [Cout][16*16]
    float *it = smem + Cout * kTile * kTile;  // [Cin][18*18]
    const int n = blockIdx.z;
    const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
    const int64_t plane = (int64_t)H * W;
    for (int i = threadIdx.x; i < Cout * kTile * kTile; i += kTile * kTile) {
        const int co = i / (kTile * kTile), p = i % (kTile * kTile);
        const int yy = y0 + p / kTile, xx = x0 + p % kTile;
        gt[i] = (yy < H && xx < W) ? g[((int64_t)n * Cout + co) * plane + (int64_t)yy * W + xx]
                                   : 0.f;
    }
    for (int i = threadIdx.x; i < Cin * 18 * 18; i += kTile * kTile) {
        const int ci = i / (18 * 18), p = i % (18 * 18);
        const int yy = y0 - 1 + p / 18, xx = x0 - 1 + p % 18;
        it[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W)
                    ? __bfloat162float(in[((int64_t)n * Cin + ci) * plane + (int64_t)yy * W + xx])
                    : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Cout * Cin * 9; e += kTile * kTile) {
        const int co = e / (Cin * 9), r = e % (Cin * 9), ci = r / 9, k = r % 9;
        const float *gp = gt + co * kTile * kTile;
        const float *ip = it + ci * 18 * 18 + (k / 3) * 18 + (k % 3);
        float s = 0.f;
        for (int py = 0; py < kTile; ++py)
#pragma unroll 4
            for (int px = 0; px < kTile; ++px) s = fmaf(gp[py * kTile + px], ip[py * 18 + px], s);
        atomicAdd(dw + e, s);
    }
    if (db)
        for (int co = threadIdx.x; co < Cout; co += kTile * kTile) {
            float s = 0.f;
            for (int p = 0; p < kTile * kTile; ++p) s += gt[co * kTile * kTile + p];
            atomicAdd(db + co, s);
        }
}

// g_pre = g * (act > 0) (ReLU backward), bf16 activations
__global__ void relu_mask_kernel(const float *__restrict__ g, const __nv_bfloat16 *__restrict__ act,
                                 float *__restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat162float(act[i]) > 0.f ? g[i] : 0.f;
}

// wt[ci][co][2-ky][2-kx] = w[co][ci][ky][kx]: backward-data weights
__global__ void flip_transpose_kernel(const __nv_bfloat16 *__restrict__ w, int Cout, int Cin,
                                      __nv_bfloat16 *__restrict__ wt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Cout * Cin * 9) return;
    const int co = e / (Cin * 9), r = e % (Cin * 9), ci = r / 9, k = r % 9;
    wt[((int64_t)ci * Cout + co) * 9 + (8 - k)] = w[e];
}

// Huber loss (delta) of prediction p against target t, mean over n; grad = dL/dp.
__global__ void huber_kernel(const float *__restrict__ p, const float *__restrict__ t,
                             float delta, int64_t n, float *__restrict__ grad,
                             float *__restrict__ loss)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < n) {
        const float r = p[i] - t[i];
        const float a = fabsf(r);
        l = a < delta ? 0.5f * r * r / delta : a - 0.5f * delta;
        grad[i] = (a < delta ? r / delta : copysignf(1.f, r)) / (float)n;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l / (float)n);
}

// Adam on fp32 master weights; also refreshes their bf16 copy.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *__restrict__ wbf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wbf) wbf[i] = __float2bfloat16(wi);
}

__global__ void to_bf16_kernel(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b,
                               int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Network input at the top level: (I0/255 - 1/2, I1/255 - 1/2, C(k)/255 for k < Dw).
__global__ void features_kernel(const uint8_t *__restrict__ I0, int p0, const uint8_t *__restrict__ I1,
                                int p1, const uint8_t *__restrict__ C, int Dws, int Dw, int W,
                                int H, __nv_bfloat16 *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const int64_t plane = (int64_t)H * W, px = (int64_t)y * W + x;
    out[px] = __float2bfloat16(I0[(int64_t)y * p0 + x] * (1.f / 255.f) - 0.5f);
    out[plane + px] = __float2bfloat16(I1[(int64_t)y * p1 + x] * (1.f / 255.f) - 0.5f);
    const uint8_t *c = C + px * Dws;
    for (int k = 0; k < Dw; ++k) out[(2 + k) * plane + px] = __float2bfloat16(c[k] * (1.f / 255.f));
}

// The same features channels-last, cstr channels per pixel (zero beyond 2 + Dw), written
// in 16-byte pieces: [view][y][x][cstr].
__global__ void features_nhwc_kernel(const uint8_t *__restrict__ I0, int p0,
                                     const uint8_t *__restrict__ I1, int p1,
                                     const uint8_t *__restrict__ C, int Dws, int Dw, int W, int H,
                                     int cstr, __nv_bfloat16 *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const int64_t px = (int64_t)y * W + x;
    const uint8_t *c = C + px * Dws;
    for (int q = 0; q < cstr / 8; ++q) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int ch = 8 * q + e;
            float f = 0.f;
            if (ch == 0) f = I0[(int64_t)y * p0 + x] * (1.f / 255.f) - 0.5f;
            else if (ch == 1) f = I1[(int64_t)y * p1 + x] * (1.f / 255.f) - 0.5f;
            else if (ch - 2 < Dw) f = c[ch - 2] * (1.f / 255.f);
            v[e] = __float2bfloat16(f);
        }
        *(uint4 *)(out + px * cstr + 8 * q) = *(const uint4 *)v;
    }
}

// Training target at the top level's resolution: mean of the f x f block of the
// full-resolution disparity map (blocks clipped at the border), divided by D.
__global__ void target_kernel(const uint16_t *__restrict__ d, int pitch, int W, int H, int f,
                              int Wq, int Hq, float inv_D, float *__restrict__ t)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= Wq) return;
    float s = 0.f;
    int c = 0;
    for (int yy = y * f; yy < min(y * f + f, H); ++yy)
        for (int xx = x * f; xx < min(x * f + f, W); ++xx) {
            s += d[(int64_t)yy * pitch + xx];
            ++c;
        }
    t[(int64_t)y * Wq + x] = c ? s / c * inv_D : 0.f;
}

// Window starts of the finest level from the prediction q (top level, units of D):
// bilinear upsampling by f with pixel centres aligned, c = D q, lo = clamp(rint(c) - Dw/2).
__global__ void proposal_windows_kernel(const float *__restrict__ q, int Wq, int Hq, int f,
                                        int W, int H, int D, int Dw, uint16_t *__restrict__ lo)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const float u = fminf(fmaxf((x + 0.5f) / f - 0.5f, 0.f), (float)(Wq - 1));
    const float v = fminf(fmaxf((y + 0.5f) / f - 0.5f, 0.f), (float)(Hq - 1));
    const int x0 = (int)u, y0 = (int)v;
    const int x1 = min(x0 + 1, Wq - 1), y1 = min(y0 + 1, Hq - 1);
    const float ax = u - x0, ay = v - y0;
    const float top = q[y0 * Wq + x0] * (1.f - ax) + q[y0 * Wq + x1] * ax;
    const float bot = q[y1 * Wq + x0] * (1.f - ax) + q[y1 * Wq + x1] * ax;
    const float c = (top * (1.f - ay) + bot * ay) * D;
    const int l = (int)rintf(c) - Dw / 2;
    lo[(int64_t)y * W + x] = (uint16_t)min(max(l, 0), D - Dw);
}


// Tensor-core form of conv3x3_kernel<32, bf16> (inference and training forward): an
// implicit GEMM  out[p][co] = sum_k A[p][k] B[k][co]  with p = pixel, k = (tap, ci).
// The block stages the weights once as [co][tap][ci] and, for each of its row tiles, the
// input tile channels-last in shared memory (channel stride CP, padded so that ldmatrix
// rows fall in distinct banks); every warp multiplies 32 pixels x 32 channels with
// mma.sync m16n8k16 (BF16 in, FP32 accumulate).  Row tile: 8 rows x 16 columns of
// pixels, 4 warps of 2 rows each; kMmaRowTiles tiles per block share the staged weights.
constexpr int kMmaRows = 8, kMmaCols = 16, kMmaRowTiles = 2;

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                        const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(unsigned &r0, unsigned &r1, const void *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// NT: n-tiles of 8 output channels (4: the 32-channel layers; 1: the output layer, its
// one channel padded to 8 with zero weights)
// NHWC: activations channels-last, [n][y][x][cstr] with the first Cin channels valid and
// cstr a multiple of 8 (the pipeline's own buffers: 16-byte copies of whole pixels);
// otherwise [n][c][y][x] (the public entry points).
template <int NT, bool NHWC>
__global__ void __launch_bounds__(128) conv3x3_mma_kernel(
    const __nv_bfloat16 *__restrict__ in, int Cin, int cstr, int CP, int H, int W,
    const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b, int Cout, int relu,
    __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f)
{
    constexpr int NC = 8 * NT;                           // output channels of the tile
    extern __shared__ __align__(16) __nv_bfloat16 sm[];
    constexpr int TR = kMmaRows + 2, TC = kMmaCols + 2;
    __nv_bfloat16 *xs = sm;                              // [TR][TC][CP]
    __nv_bfloat16 *ws = sm + TR * TC * CP;               // [NC][9][CP]
    const int n = blockIdx.z;
    const int x0 = blockIdx.x * kMmaCols;
    const int64_t plane = (int64_t)H * W;
    const __nv_bfloat16 *src = in + (int64_t)n * (NHWC ? cstr : Cin) * plane;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    const int K16 = (Cin + 15) / 16 * 16;                // channels the k-steps cover
    if (NHWC) {
        // weights already in this layout (zero padding included): 16-byte copies
        const uint4 *wsrc = (const uint4 *)w;
        uint4 *wdst = (uint4 *)ws;
        const int nvec = NC * 9 * CP / 8;
        for (int i = threadIdx.x; i < nvec; i += 128) wdst[i] = wsrc[i];
    } else
    // weights: one (co, ci) pair per step, its 9 taps contiguous in global memory;
    // output channels Cout .. NC-1 have zero weights
    for (int i0 = threadIdx.x; i0 < NC * Cin; i0 += 256) {   // two pairs per round
        __nv_bfloat16 v[2][9];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + h * 128;
            const int co = i / Cin;
            const __nv_bfloat16 *wr = w + (int64_t)i * 9;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap)
                v[h][tap] = (i < NC * Cin && co < Cout) ? wr[tap] : zero;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = i0 + h * 128;
            if (i >= NC * Cin) break;
            const int co = i / Cin, c = i - co * Cin;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) ws[(co * 9 + tap) * CP + c] = v[h][tap];
        }
    }
    // channels Cin .. K16-1 are zero in both operands (never rewritten below)
    const int npad = K16 - Cin;
    if (!NHWC)
        for (int i = threadIdx.x; i < NC * 9 * npad; i += 128)
            ws[(i / npad) * CP + Cin + i % npad] = zero;
    for (int i = threadIdx.x; i < TR * TC * npad; i += 128)
        xs[(i / npad) * CP + Cin + i % npad] = zero;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ldmatrix row addresses: A rows = pixels of row (2*warp + mt), B rows = channels
    const int arow = lane & 15, acol = (lane >> 4) * 8;
    const int brow = lane & 7, bcol = ((lane >> 3) & 1) * 8;
    const int g = lane >> 2, t = lane & 3;
    for (int rt = 0; rt < kMmaRowTiles; ++rt) {
        const int y0 = (blockIdx.y * kMmaRowTiles + rt) * kMmaRows;
        if (y0 >= H) break;                              // uniform over the block
        __syncthreads();                                 // the previous tile is consumed
        if (NHWC) {
            // whole pixels in 16-byte pieces (cstr / 8 per pixel), consecutive threads on
            // consecutive pieces, a batch of loads before the stores
            constexpr int kBatch = 8;
            const int per = cstr / 8, npieces = TR * TC * per;
            for (int i0 = threadIdx.x; i0 < npieces; i0 += 128 * kBatch) {
                uint4 v[kBatch];
#pragma unroll
                for (int b2 = 0; b2 < kBatch; ++b2) {
                    const int i = i0 + b2 * 128;
                    const int pp = i / per, q = i - pp * per;
                    const int py = pp / TC, px = pp - py * TC;
                    const int yy = y0 - 1 + py, xx = x0 - 1 + px;
                    v[b2] = make_uint4(0u, 0u, 0u, 0u);
                    if (i < npieces && yy >= 0 && yy < H && xx >= 0 && xx < W)
                        v[b2] = *(const uint4 *)(src + ((int64_t)yy * W + xx) * cstr + 8 * q);
                }
#pragma unroll
                for (int b2 = 0; b2 < kBatch; ++b2) {
                    const int i = i0 + b2 * 128;
                    if (i >= npieces) break;
                    const int pp = i / per, q = i - pp * per;
                    *(uint4 *)(xs + pp * CP + 8 * q) = v[b2];
                }
            }
        } else {
        // input tile, consecutive threads on consecutive pixels of a row; each thread
        // issues kStageBatch loads before its stores, so that their latencies overlap
        constexpr int kStageBatch = 8;
        const int ntile = TR * TC * Cin;
        for (int i0 = threadIdx.x; i0 < ntile; i0 += 128 * kStageBatch) {
            __nv_bfloat16 v[kStageBatch];
            int dst[kStageBatch];
#pragma unroll
            for (int b = 0; b < kStageBatch; ++b) {
                const int i = i0 + b * 128;
                const int px = i % TC, q = i / TC, py = q % TR, c = q / TR;
                const int yy = y0 - 1 + py, xx = x0 - 1 + px;
                const bool in_img = i < ntile && yy >= 0 && yy < H && xx >= 0 && xx < W;
                v[b] = in_img ? src[c * plane + (int64_t)yy * W + xx] : zero;
                dst[b] = i < ntile ? (py * TC + px) * CP + c : -1;
            }
#pragma unroll
            for (int b = 0; b < kStageBatch; ++b)
                if (dst[b] >= 0) xs[dst[b]] = v[b];
        }
        }
        __syncthreads();
        float acc[2][NT][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
            for (int c0 = 0; c0 < K16; c0 += 16) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int py = 2 * warp + mt + ky, px = arow + kx;
                    ldsm_x4(a[mt][0], a[mt][1], a[mt][2], a[mt][3],
                            xs + (py * TC + px) * CP + c0 + acol);
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    unsigned b0, b1;
                    ldsm_x2(b0, b1, ws + ((nt * 8 + brow) * 9 + tap) * CP + c0 + bcol);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
                        mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                }
            }
        }
        // accumulator layout: d0,d1 at (row g, cols 2t, 2t+1), d2,d3 at (row g+8, same cols)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int y = y0 + 2 * warp + mt;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int x = x0 + g + (e >= 2 ? 8 : 0);
                    const int co = nt * 8 + 2 * t + (e & 1);
                    if (x >= W || y >= H || co >= Cout) continue;
                    float v = acc[mt][nt][e] + (b ? b[co] : 0.f);
                    if (relu) v = fmaxf(v, 0.f);
                    const int64_t o = NHWC ? ((int64_t)n * plane + (int64_t)y * W + x) * Cout + co
                                           : ((int64_t)n * Cout + co) * plane + (int64_t)y * W + x;
                    if (out_f) out_f[o] = v;
                    if (out_bf) out_bf[o] = __float2bfloat16(v);
                }
        }
    }
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t conv_smem_bytes(int Cin, int Cout) { return sizeof(float) * ((size_t)Cin * 9 * Cout + 18 * 18); }

template <class TIn>
void launch_conv3x3_t(const TIn *in, int N, int Cin, int H, int W, const __nv_bfloat16 *w,
                      const float *b, int Cout, int relu, __nv_bfloat16 *out_bf, float *out_f,
                      cudaStream_t s)
{
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, N);
    const size_t smem = conv_smem_bytes(Cin, Cout);
    if (Cout == 32) {
        cudaFuncSetAttribute(conv3x3_kernel<32, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_kernel<32, TIn><<<grid, kTile * kTile, smem, s>>>(in, Cin, H, W, w, b, relu, out_bf, out_f);
    } else {
        cudaFuncSetAttribute(conv3x3_kernel<1, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_kernel<1, TIn><<<grid, kTile * kTile, smem, s>>>(in, Cin, H, W, w, b, relu, out_bf, out_f);
    }
}

template <bool NHWC>
void launch_mma(const __nv_bfloat16 *in, int N, int Cin, int cstr, int H, int W,
                const __nv_bfloat16 *w, const float *b, int Cout, int relu, __nv_bfloat16 *out_bf,
                float *out_f, cudaStream_t s)
{
    // channel stride: Cin rounded up to 16 (whole k-steps) plus 8 (bank spread)
    const int CP = mma_channel_stride(Cin);
    const int NC = Cout == 32 ? 32 : 8;
    const size_t smem =
        sizeof(__nv_bfloat16) * (size_t)CP * ((kMmaRows + 2) * (kMmaCols + 2) + NC * 9);
    const int rows = kMmaRows * kMmaRowTiles;
    dim3 grid((W + kMmaCols - 1) / kMmaCols, (H + rows - 1) / rows, N);
    if (Cout == 32) {
        cudaFuncSetAttribute(conv3x3_mma_kernel<4, NHWC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_mma_kernel<4, NHWC><<<grid, 128, smem, s>>>(in, Cin, cstr, CP, H, W, w, b, Cout,
                                                            relu, out_bf, out_f);
    } else {
        cudaFuncSetAttribute(conv3x3_mma_kernel<1, NHWC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_mma_kernel<1, NHWC><<<grid, 128, smem, s>>>(in, Cin, cstr, CP, H, W, w, b, Cout,
                                                            relu, out_bf, out_f);
    }
}

void launch_conv3x3_nhwc(const __nv_bfloat16 *in, int N, int Cin, int cstr, int H, int W,
                         const __nv_bfloat16 *w, const float *b, int Cout, int relu,
                         __nv_bfloat16 *out_bf, float *out_f, cudaStream_t s)
{
    launch_mma<true>(in, N, Cin, cstr, H, W, w, b, Cout, relu, out_bf, out_f, s);
}

void launch_conv3x3(const __nv_bfloat16 *in, int N, int Cin, int H, int W, const __nv_bfloat16 *w,
                    const float *b, int Cout, int relu, __nv_bfloat16 *out_bf, float *out_f,
                    cudaStream_t s)
{
    if (Cout != 32 && Cout != 1) {
        launch_conv3x3_t(in, N, Cin, H, W, w, b, Cout, relu, out_bf, out_f, s);
        return;
    }
    launch_mma<false>(in, N, Cin, Cin, H, W, w, b, Cout, relu, out_bf, out_f, s);
}

void launch_conv3x3_wgrad(const __nv_bfloat16 *in, int N, int Cin, const float *g, int Cout, int H,
                          int W, float *dw, float *db, cudaStream_t s)
{
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, N);
    const size_t smem = sizeof(float) * ((size_t)Cout * kTile * kTile + (size_t)Cin * 18 * 18);
    cudaFuncSetAttribute(conv3x3_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    conv3x3_wgrad_kernel<<<grid, kTile * kTile, smem, s>>>(in, Cin, g, Cout, H, W, dw, db);
}

void launch_features(const uint8_t *I0, int p0, const uint8_t *I1, int p1, const uint8_t *C,
                     int Dws, int Dw, int W, int H, __nv_bfloat16 *out, cudaStream_t s)
{
    features_kernel<<<dim3(blocks(W, 128), H), 128, 0, s>>>(I0, p0, I1, p1, C, Dws, Dw, W, H, out);
}

void launch_features_nhwc(const uint8_t *I0, int p0, const uint8_t *I1, int p1, const uint8_t *C,
                          int Dws, int Dw, int W, int H, int cstr, __nv_bfloat16 *out,
                          cudaStream_t s)
{
    features_nhwc_kernel<<<dim3(blocks(W, 128), H), 128, 0, s>>>(I0, p0, I1, p1, C, Dws, Dw, W,
                                                                 H, cstr, out);
}

void launch_proposal_windows(const float *q, int Wq, int Hq, int f, int W, int H, int D, int Dw,
                             uint16_t *lo, cudaStream_t s)
{
    proposal_windows_kernel<<<dim3(blocks(W, 128), H), 128, 0, s>>>(q, Wq, Hq, f, W, H, D, Dw, lo);
}

}  // namespace mpv

using namespace mpv;

extern "C" {

mpv_status mpv_cnn_conv3x3(const void *in, int32_t in_f32, int32_t n, int32_t cin, int32_t h,
                           int32_t w, const void *weight, const float *bias, int32_t cout,
                           int32_t relu, void *out_bf16, float *out_f32, void *cuda_stream)
{
    if (!in || !weight || n < 1 || cin < 1 || h < 1 || w < 1 || (cout != 32 && cout != 1) ||
        (!out_bf16 && !out_f32) || conv_smem_bytes(cin, cout) > 200 * 1024)
        return MPV_ERR_INVALID_ARG;
    if (in_f32)
        launch_conv3x3_t((const float *)in, n, cin, h, w, (const __nv_bfloat16 *)weight, bias,
                         cout, relu, (__nv_bfloat16 *)out_bf16, out_f32, (cudaStream_t)cuda_stream);
    else
        launch_conv3x3((const __nv_bfloat16 *)in, n, cin, h, w, (const __nv_bfloat16 *)weight, bias,
                       cout, relu, (__nv_bfloat16 *)out_bf16, out_f32, (cudaStream_t)cuda_stream);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_conv3x3_wgrad(const void *in, int32_t n, int32_t cin, const float *grad,
                                 int32_t cout, int32_t h, int32_t w, float *dweight, float *dbias,
                                 void *cuda_stream)
{
    if (!in || !grad || !dweight || n < 1 || cin < 1 || cout < 1 || h < 1 || w < 1 ||
        sizeof(float) * ((size_t)cout * 256 + (size_t)cin * 324) > 200 * 1024)
        return MPV_ERR_INVALID_ARG;
    launch_conv3x3_wgrad((const __nv_bfloat16 *)in, n, cin, grad, cout, h, w, dweight, dbias,
                         (cudaStream_t)cuda_stream);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_flip_transpose(const void *weight, int32_t cout, int32_t cin, void *out,
                                  void *cuda_stream)
{
    if (!weight || !out || cout < 1 || cin < 1) return MPV_ERR_INVALID_ARG;
    const int e = cout * cin * 9;
    flip_transpose_kernel<<<blocks(e, 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        (const __nv_bfloat16 *)weight, cout, cin, (__nv_bfloat16 *)out);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_relu_backward(const float *grad, const void *act, float *out, int64_t count,
                                 void *cuda_stream)
{
    if (!grad || !act || !out || count < 0) return MPV_ERR_INVALID_ARG;
    relu_mask_kernel<<<blocks(count, 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        grad, (const __nv_bfloat16 *)act, out, count);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_huber(const float *pred, const float *target, float delta, int64_t count,
                         float *grad, float *loss, void *cuda_stream)
{
    if (!pred || !target || !grad || count < 1 || !(delta > 0.f)) return MPV_ERR_INVALID_ARG;
    huber_kernel<<<blocks(count, 256), 256, 0, (cudaStream_t)cuda_stream>>>(pred, target, delta,
                                                                           count, grad, loss);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_adam(float *weight, const float *grad, float *m, float *v, int64_t count,
                        float lr, float beta1, float beta2, float eps, int32_t step,
                        void *weight_bf16, void *cuda_stream)
{
    if (!weight || !grad || !m || !v || count < 1 || step < 1) return MPV_ERR_INVALID_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<blocks(count, 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        weight, grad, m, v, count, lr, beta1, beta2, eps, c1, c2, (__nv_bfloat16 *)weight_bf16);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_to_bf16(const float *in, void *out, int64_t count, void *cuda_stream)
{
    if (!in || !out || count < 0) return MPV_ERR_INVALID_ARG;
    to_bf16_kernel<<<blocks(count, 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        in, (__nv_bfloat16 *)out, count);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status mpv_cnn_target(const uint16_t *disp, int32_t disp_pitch, int32_t width, int32_t height,
                          int32_t factor, int32_t max_disparity, float *target, void *cuda_stream)
{
    if (!disp || !target || factor < 1 || width < 1 || height < 1 || max_disparity < 1)
        return MPV_ERR_INVALID_ARG;
    const int Wq = (width + factor - 1) / factor, Hq = (height + factor - 1) / factor;
    target_kernel<<<dim3(blocks(Wq, 128), Hq), 128, 0, (cudaStream_t)cuda_stream>>>(
        disp, disp_pitch, width, height, factor, Wq, Hq, 1.f / max_disparity, target);
    return cudaGetLastError() == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

}  // extern "C"
