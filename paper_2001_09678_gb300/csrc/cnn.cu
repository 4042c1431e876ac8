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


// Tensor-core form of conv3x3_kernel<32 or 1, bf16> (inference and training forward) on
// the fifth-generation tensor cores: an implicit GEMM
//     D[m][co] = sum_{tap, ci} A[m][(tap, ci)] B[co][(tap, ci)]
// with m one of the 128 pixels of an output tile of 16 rows x 8 columns (M = 128), N = 32
// output channels (16 for the one-channel output layer, its other rows zero weights) and
// K = 9 taps x the input channels rounded up to 16, in k-steps of 16 (kind::f16, BF16
// operands, FP32 accumulation in tensor memory).
//
// Shared memory holds both operands K-major without swizzling, as 8-row x 16-byte core
// matrices.  The input tile with its one-pixel halo (18 x 10 pixels) is stored as planes of
// 8 channels: plane c8 holds channels 8 c8 .. 8 c8 + 7 of every staged pixel, 16 bytes per
// pixel, pixels row-major.  Eight consecutive output pixels of one row then form a core
// matrix for every tap: the A operand of tap (ky, kx) starts at staged pixel ky * 10 + kx,
// its core matrices follow each other along M at one staged row (160 bytes) and along K at
// one plane.  The weights are stored [tap][c8][co][8], so that B's core matrices follow
// each other along N at 8 channels (128 bytes) and along K at one plane of NC x 16 bytes.
// One thread issues the 9 x (K/16) MMAs of a tile and commits them to an mbarrier; the
// four warps read their 32 rows of the accumulator back (tcgen05.ld) for the epilogue.
constexpr int kTcRows = 16, kTcCols = 8;                 // output tile (M = 128 pixels)
constexpr int kTcTR = kTcRows + 2, kTcTC = kTcCols + 2;  // staged input tile, 18 x 10
constexpr int kTcPix = kTcTR * kTcTC;
// bytes of one plane of 8 channels; the extra 16 bytes spread one pixel's planes over banks
constexpr int kTcPlane = kTcPix * 16 + 16;
constexpr int kTcBlocksPerSm = 4;                        // resident blocks the grid aims for
constexpr long long kTcWaitCycles = 2000000000LL;        // about a second

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand without swizzling: start address,
// byte distance between core matrices adjacent along K (lbo) and along M or N (sbo), each
// in 16-byte units, and the descriptor version of this architecture (bit 46).
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), BF16 A and B (bits
// 7-9, 10-12), both K-major (bits 15, 16 clear), N / 8 (bits 17-22), M / 16 (bits 24-28).
template <int M, int N>
__host__ __device__ constexpr uint32_t umma_instr_desc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ bool mbar_phase_done(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// 32 lanes x X columns of 32 bits from tensor memory: thread t of the warp gets lane
// (warp's first lane + t), columns col .. col + X - 1
template <int X>
struct TmemRow;
template <>
struct TmemRow<32> {
    __device__ __forceinline__ static void ld(uint32_t taddr, uint32_t (&r)[32])
    {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
            "%26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
              "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    }
};
template <>
struct TmemRow<16> {
    __device__ __forceinline__ static void ld(uint32_t taddr, uint32_t (&r)[16])
    {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
};

size_t tc_smem_bytes(int Cin, int Cout)
{
    const int ncg = tc_planes(Cin), nc = tc_width(Cout);
    return (size_t)ncg * kTcPlane + (size_t)9 * ncg * nc * 16 + 16;
}

// NC: the MMA width N (32, or 16 for the one-channel output layer).
// NHWC: activations [n][y][x][cstr] (cstr a multiple of 8, channels Cin .. cstr - 1 zero)
// and weights pre-arranged [9][tc_planes(Cin)][NC][8] with zero padding (the matcher's own
// buffers); otherwise activations [n][c][y][x] and weights [Cout][Cin][3][3] (the public
// entry points).  err (optional): set to 1 when the wait for the tensor cores ran out; the
// outputs of the block's unfinished tiles are then NaN.
template <int NC, bool NHWC>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(
    const __nv_bfloat16 *__restrict__ in, int Cin, int cstr, int H, int W, int nimg,
    const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b, int Cout, int relu,
    __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f, int *err)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    const int ncg = tc_planes(Cin), ks = ncg / 2;
    unsigned char *As = tsm;                                   // ncg planes
    unsigned char *Bs = tsm + (size_t)ncg * kTcPlane;          // [9][ncg][NC][8]
    uint64_t *mbar = (uint64_t *)(Bs + (size_t)9 * ncg * NC * 16);
    uint32_t *tslot = (uint32_t *)(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the planes start zero: channels the staging never writes (Cin or cstr up to the
    // k-steps' multiple of 16) stay zero in every tile
    for (int i = tid; i < ncg * kTcPlane / 16; i += 128)
        ((uint4 *)As)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (NHWC) {
        const int nvec = 9 * ncg * NC;
        for (int i = tid; i < nvec; i += 128) ((uint4 *)Bs)[i] = ((const uint4 *)w)[i];
    } else {
        // element (tap, ci, co) at ((tap * ncg + ci / 8) * NC + co) * 8 + ci % 8, zero for
        // absent channels
        __nv_bfloat16 *bw = (__nv_bfloat16 *)Bs;
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        const int ntot = 9 * ncg * 8 * NC;
        for (int i = tid; i < ntot; i += 128) {
            const int co = i % NC, r = i / NC, ci = r % (ncg * 8), tap = r / (ncg * 8);
            bw[((tap * ncg + ci / 8) * NC + co) * 8 + ci % 8] =
                (co < Cout && ci < Cin) ? w[((int64_t)co * Cin + ci) * 9 + tap] : zero;
        }
    }
    if (warp == 0) {   // 32 columns of tensor memory: the 128 x NC FP32 accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
                         smem_addr(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int tx = (W + kTcCols - 1) / kTcCols, ty = (H + kTcRows - 1) / kTcRows;
    const int ntiles = tx * ty * nimg;
    const int64_t plane = (int64_t)H * W;
    constexpr uint32_t idesc = umma_instr_desc<128, NC>();
    const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs), mb = smem_addr(mbar);
    uint32_t phase = 0;
    int tile = blockIdx.x;
    bool failed = false;

    for (; tile < ntiles; tile += gridDim.x) {
        const int n = tile / (tx * ty), r = tile - n * (tx * ty);
        const int y0 = (r / tx) * kTcRows, x0 = (r % tx) * kTcCols;
        // the input tile with its one-pixel halo, zero outside the image, in 16-byte pieces
        // (8 channels of one pixel); consecutive threads on consecutive pieces, a batch of
        // loads before the stores
        constexpr int kBatch = 8;
        if (NHWC) {
            const __nv_bfloat16 *src = in + (int64_t)n * cstr * plane;
            // 16-byte pieces per pixel, never more than the planes the operand holds
            // (channels Cin .. cstr - 1 are zero, so those beyond the planes are not needed)
            const int per = min(cstr / 8, ncg), npieces = kTcPix * per;
            for (int i0 = tid; i0 < npieces; i0 += 128 * kBatch) {
                uint4 v[kBatch];
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = i0 + q * 128;
                    const int pp = i / per, c8 = i - pp * per;
                    const int py = pp / kTcTC, px = pp - py * kTcTC;
                    const int yy = y0 - 1 + py, xx = x0 - 1 + px;
                    v[q] = make_uint4(0u, 0u, 0u, 0u);
                    if (i < npieces && yy >= 0 && yy < H && xx >= 0 && xx < W)
                        v[q] = *(const uint4 *)(src + ((int64_t)yy * W + xx) * cstr + 8 * c8);
                }
#pragma unroll
                for (int q = 0; q < kBatch; ++q) {
                    const int i = i0 + q * 128;
                    if (i >= npieces) break;
                    const int pp = i / per, c8 = i - pp * per;
                    *(uint4 *)(As + c8 * kTcPlane + pp * 16) = v[q];
                }
            }
        } else {
            // piece (plane c8, pixel pp): consecutive threads on consecutive pixels, each
            // gathering its 8 channels from 8 channel planes of the image
            const __nv_bfloat16 *src = in + (int64_t)n * Cin * plane;
            const int cgi = (Cin + 7) / 8, npieces = kTcPix * cgi;
            for (int i = tid; i < npieces; i += 128) {
                const int c8 = i / kTcPix, pp = i - c8 * kTcPix;
                const int py = pp / kTcTC, px = pp - py * kTcTC;
                const int yy = y0 - 1 + py, xx = x0 - 1 + px;
                uint32_t pk[4] = {0u, 0u, 0u, 0u};
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                    const __nv_bfloat16 *s0 = src + (int64_t)(8 * c8) * plane + (int64_t)yy * W + xx;
                    unsigned short h[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        h[e] = 8 * c8 + e < Cin ? __bfloat16_as_ushort(s0[(int64_t)e * plane]) : 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) pk[e] = (uint32_t)h[2 * e] | ((uint32_t)h[2 * e + 1] << 16);
                }
                *(uint4 *)(As + c8 * kTcPlane + pp * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        // the staged tile, written through the generic proxy, before the tensor cores read it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int tap = 0; tap < 9; ++tap) {
                const uint32_t aoff = (uint32_t)(((tap / 3) * kTcTC + tap % 3) * 16);
                for (int s = 0; s < ks; ++s) {
                    const uint64_t ad =
                        umma_smem_desc(a0 + 2 * s * kTcPlane + aoff, kTcPlane, kTcTC * 16);
                    const uint64_t bd = umma_smem_desc(
                        b0 + (uint32_t)((tap * ncg + 2 * s) * NC * 16), NC * 16, 128);
                    umma_bf16(tmem, ad, bd, idesc, (tap | s) != 0);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    mb)
                : "memory");
        }
        // the products (bounded wait; the block agrees on the outcome)
        bool ok = mbar_phase_done(mb, phase);
        if (!ok) {
            const long long t0 = clock64();
            while (!(ok = mbar_phase_done(mb, phase)) && clock64() - t0 < kTcWaitCycles) {
            }
        }
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t acc[NC];
        TmemRow<NC>::ld(tmem + ((uint32_t)(warp * 32) << 16), acc);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // accumulator row m = 32 warp + lane: output pixel (y0 + m / 8, x0 + m % 8)
        const int m = warp * 32 + lane;
        const int oy = y0 + m / kTcCols, ox = x0 + m % kTcCols;
        if (oy < H && ox < W) {
            const int64_t pix = (int64_t)oy * W + ox;
            bool done = false;
            if constexpr (NC == 32 && NHWC) {
                if (Cout == 32 && out_bf && !out_f) {   // the matcher's hidden layers
                    uint4 *dst = (uint4 *)(out_bf + ((int64_t)n * plane + pix) * 32);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int co = 8 * q + 2 * e;
                            float v0 = __uint_as_float(acc[co]) + (b ? b[co] : 0.f);
                            float v1 = __uint_as_float(acc[co + 1]) + (b ? b[co + 1] : 0.f);
                            if (relu) {
                                v0 = fmaxf(v0, 0.f);
                                v1 = fmaxf(v1, 0.f);
                            }
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                            pk[e] = *(const uint32_t *)&h2;
                        }
                        dst[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int co = 0; co < NC; ++co) {
                    if (co >= Cout) break;
                    float v = __uint_as_float(acc[co]) + (b ? b[co] : 0.f);
                    if (relu) v = fmaxf(v, 0.f);
                    const int64_t o = NHWC ? ((int64_t)n * plane + pix) * Cout + co
                                           : ((int64_t)n * Cout + co) * plane + pix;
                    if (out_f) out_f[o] = v;
                    if (out_bf) out_bf[o] = __float2bfloat16(v);
                }
            }
        }
        // every warp's reads of the accumulator and of the staged tile are complete before
        // the next tile overwrites them
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed) {
        // the wait ran out: record it, and mark the block's unfinished tiles as NaN
        if (tid == 0 && err) atomicCAS(err, 0, 1);
        for (; tile < ntiles; tile += gridDim.x) {
            const int n = tile / (tx * ty), r = tile - n * (tx * ty);
            const int oy = (r / tx) * kTcRows + tid / kTcCols, ox = (r % tx) * kTcCols + tid % kTcCols;
            if (oy >= H || ox >= W) continue;
            const int64_t pix = (int64_t)oy * W + ox;
            for (int co = 0; co < Cout && co < NC; ++co) {
                const int64_t o = NHWC ? ((int64_t)n * plane + pix) * Cout + co
                                       : ((int64_t)n * Cout + co) * plane + pix;
                if (out_f) out_f[o] = __int_as_float(0x7FC00000);
                if (out_bf) out_bf[o] = __ushort_as_bfloat16((unsigned short)0x7FC0);
            }
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
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

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

template <bool NHWC>
void launch_tc(const __nv_bfloat16 *in, int N, int Cin, int cstr, int H, int W,
               const __nv_bfloat16 *w, const float *b, int Cout, int relu, __nv_bfloat16 *out_bf,
               float *out_f, int *err, cudaStream_t s)
{
    const int64_t tiles = (int64_t)((W + kTcCols - 1) / kTcCols) * ((H + kTcRows - 1) / kTcRows) * N;
    const int64_t cap = (int64_t)kTcBlocksPerSm * sm_count();
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    const size_t smem = tc_smem_bytes(Cin, Cout);
    if (Cout == 32) {
        cudaFuncSetAttribute(conv3x3_tc_kernel<32, NHWC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_tc_kernel<32, NHWC><<<grid, 128, smem, s>>>(in, Cin, cstr, H, W, N, w, b, Cout,
                                                            relu, out_bf, out_f, err);
    } else {
        cudaFuncSetAttribute(conv3x3_tc_kernel<16, NHWC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_tc_kernel<16, NHWC><<<grid, 128, smem, s>>>(in, Cin, cstr, H, W, N, w, b, Cout,
                                                            relu, out_bf, out_f, err);
    }
}

void launch_conv3x3_nhwc(const __nv_bfloat16 *in, int N, int Cin, int cstr, int H, int W,
                         const __nv_bfloat16 *w, const float *b, int Cout, int relu,
                         __nv_bfloat16 *out_bf, float *out_f, int *err, cudaStream_t s)
{
    launch_tc<true>(in, N, Cin, cstr, H, W, w, b, Cout, relu, out_bf, out_f, err, s);
}

bool conv3x3_tc_ok(int Cin, int Cout)
{
    return (Cout == 32 || Cout == 1) && tc_smem_bytes(Cin, Cout) <= kTcMaxSmem;
}

void launch_conv3x3(const __nv_bfloat16 *in, int N, int Cin, int H, int W, const __nv_bfloat16 *w,
                    const float *b, int Cout, int relu, __nv_bfloat16 *out_bf, float *out_f,
                    cudaStream_t s)
{
    // widths the tensor-core tile covers (the network's 32 and 1 channels) with operands
    // that fit in shared memory; any other shape on the CUDA cores
    if (!conv3x3_tc_ok(Cin, Cout)) {
        launch_conv3x3_t(in, N, Cin, H, W, w, b, Cout, relu, out_bf, out_f, s);
        return;
    }
    launch_tc<false>(in, N, Cin, Cin, H, W, w, b, Cout, relu, out_bf, out_f, nullptr, s);
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
        (!out_bf16 && !out_f32) ||
        ((in_f32 || !conv3x3_tc_ok(cin, cout)) && conv_smem_bytes(cin, cout) > 200 * 1024))
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
