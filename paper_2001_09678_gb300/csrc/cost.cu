// cost.cu -- integer SSIM matching-cost volume (Section 3.2, Eq. components, Eq. ssim).
//
// For pixel (x,y) of I0 and disparity u the cost compares the N x N patch of I0
// centred at (x,y) with the patch of I1 centred at (x-u,y), coordinates clamped to the
// image.  With alpha = beta = gamma = 1 and C3 = C2/2, SSIM = A1*A2 / (B1*B2) where, for
// the patch sums Sx, Sy, Sxx, Syy, Sxy and n = N*N,
//     A1 = 2 Sx Sy + c1,              B1 = Sx^2 + Sy^2 + c1,
//     A2 = 2 (n Sxy - Sx Sy) + c2,    B2 = n (Sxx + Syy) - Sx^2 - Sy^2 + c2,
// (c1, c2 = C1, C2 scaled by n^2 and rounded) and the cost is
//     floor(255 (B1 B2 - A1 A2) / (2 B1 B2))  in [0, 255];  255 when x - u < 0.
//
// GPU design: one block per (row, 32-pixel tile, view).  The block stages the N rows
// of I0 and the span of I1 the tile can reach in shared memory, forms per-pixel patch
// statistics of both images once, and the per-(column, disparity) vertical products
// Sum_dy I0*I1 once per tile; each node then sums N of those products.  The quotient
// is estimated in fp32 and made exact with an int64 check only when the estimate
// lies within 1e-3 of an integer (the fp32 error is below 2e-4; see below).
#include "mpv_internal.cuh"

namespace mpv {

namespace {

constexpr int TX = 32;       // pixels per tile
constexpr int UCAP = 256;    // widest disparity span handled with shared column products
constexpr int kThreads = 256;

// Floor of 255 (den - num) / (2 den) for |num| <= den, den > 0, exactly.
// fp32 estimate: A1, A2, B1, B2 are integers below 2^27 in magnitude, so each
// conversion and product carries relative error <= 2^-24, the quotient <= 2 ulp; the
// estimate t = 127.5 (1 - num/den) is off by less than 127.5 * 8 * 2^-24 + 3 ulp(255)
// < 2e-4.  A fractional part in [1e-3, 1 - 1e-3] therefore already has the right floor.
__device__ __forceinline__ int ssim_quotient(int A1, int A2, int B1, int B2)
{
    const float num = (float)A1 * (float)A2;
    const float den = (float)B1 * (float)B2;
    const float t = 127.5f - 127.5f * __fdividef(num, den);
    const float fl = floorf(t);
    const float fr = t - fl;
    int q = (int)fl;
    if (fr < 1e-3f || fr > 1.0f - 1e-3f) {
        const long long dd = (long long)B1 * (long long)B2;
        const long long nn = (long long)A1 * (long long)A2;
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

template <int N>
__global__ void __launch_bounds__(kThreads) cost_kernel(LevelArgs a)
{
    constexpr int R = N / 2;
    constexpr int n = N * N;
    const int view = blockIdx.z;
    const ViewLevel &V = a.v[view];
    const int W = a.W, H = a.H, Dw = a.Dw;
    const int y = blockIdx.y;
    const int x0 = blockIdx.x * TX;
    const int nx = min(TX, W - x0);
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int lo_s[TX];
    __shared__ int sx_s[TX], sxq_s[TX], vx_s[TX];
    __shared__ int red[2];
    __shared__ uint8_t i0_s[N][TX + 2 * R];

    if (tid == 0) {
        red[0] = 0x7FFFFFFF;
        red[1] = 0;
    }
    __syncthreads();
    if (tid < nx) {
        const int l = V.lo ? (int)V.lo[(int64_t)y * W + x0 + tid] : 0;
        lo_s[tid] = l;
        atomicMin(&red[0], l);
        atomicMax(&red[1], l);
    }
    __syncthreads();
    const int minlo = red[0], maxlo = red[1];
    const int U = maxlo - minlo + Dw;                  // disparity span of the tile
    const int bmin = x0 - R - (maxlo + Dw - 1);         // first I1 column reached
    const int WB = nx + 2 * R + U - 1;                  // I1 columns staged
    const int NC = WB - 2 * R;                          // I1 patch centres
    const bool use_cp = U <= UCAP;
    const int CPW = TX + 2 * R + 1;                     // odd row stride: no bank conflicts

    uint8_t *i1_s = smem_raw;                                     // [N][WB]
    int *sy_s = (int *)(smem_raw + ((N * WB + 15) & ~15));        // [NC]
    int *syq_s = sy_s + NC;                                       // [NC]
    int *vy_s = syq_s + NC;                                       // [NC]
    int *cp_s = vy_s + NC;                                        // [U][CPW]

    // stage rows y-R..y+R of I0 (tile + halo) and of I1 (reachable span), clamped
    for (int i = tid; i < N * (TX + 2 * R); i += kThreads) {
        const int dy = i / (TX + 2 * R), c = i % (TX + 2 * R);
        const int yy = min(max(y + dy - R, 0), H - 1);
        const int xx = min(max(x0 - R + c, 0), W - 1);
        i0_s[dy][c] = V.I0[(int64_t)yy * V.pitch0 + xx];
    }
    for (int i = tid; i < N * WB; i += kThreads) {
        const int dy = i / WB, c = i % WB;
        const int yy = min(max(y + dy - R, 0), H - 1);
        const int xx = min(max(bmin + c, 0), W - 1);
        i1_s[i] = V.I1[(int64_t)yy * V.pitch1 + xx];
    }
    __syncthreads();

    // patch statistics: I0 for the tile's pixels, I1 for every reachable centre
    if (tid < nx) {
        int s = 0, q = 0;
#pragma unroll
        for (int dy = 0; dy < N; ++dy)
#pragma unroll
            for (int dx = 0; dx < N; ++dx) {
                const int v = i0_s[dy][tid + dx];
                s += v;
                q += v * v;
            }
        sx_s[tid] = s;
        sxq_s[tid] = s * s;
        vx_s[tid] = n * q - s * s;
    }
    for (int c = tid; c < NC; c += kThreads) {
        int s = 0, q = 0;
#pragma unroll
        for (int dy = 0; dy < N; ++dy)
#pragma unroll
            for (int dx = 0; dx < N; ++dx) {
                const int v = i1_s[dy * WB + c + dx];
                s += v;
                q += v * v;
            }
        sy_s[c] = s;
        syq_s[c] = s * s;
        vy_s[c] = n * q - s * s;
    }
    // vertical products P(a, uu) = sum_dy I0(y+dy, a) * I1(y+dy, a - minlo - uu)
    if (use_cp) {
        const int na = nx + 2 * R;
        for (int i = tid; i < U * na; i += kThreads) {
            const int uu = i / na, col = i % na;
            const int b = col + (U - 1) - uu;           // I1 staged column of a - u
            int acc = 0;
#pragma unroll
            for (int dy = 0; dy < N; ++dy) acc += (int)i0_s[dy][col] * (int)i1_s[dy * WB + b];
            cp_s[uu * CPW + col] = acc;
        }
    }
    __syncthreads();

    const int c1 = a.c1, c2 = a.c2;
    const int Dws = a.Dws;
    const int lane = tid & 31, warp = tid >> 5;
    // one warp per pixel, lanes over labels: the pixel's Dws cost bytes are contiguous
    for (int i = warp; i < nx; i += kThreads / 32) {
        uint8_t *out = V.C + ((int64_t)y * W + x0 + i) * Dws;
        const int lo = lo_s[i];
        const int sx = sx_s[i], sxq = sxq_s[i], vx = vx_s[i];
        for (int k = lane; k < Dws; k += 32) {
            const int u = lo + k;
            const int xp = x0 + i - u;
            int q = 255;
            if (k < Dw && xp >= 0) {
                int sxy = 0;
                if (use_cp) {
                    const int *row = cp_s + (lo - minlo + k) * CPW + i;
#pragma unroll
                    for (int dx = 0; dx < N; ++dx) sxy += row[dx];
                } else {
                    const int b0 = xp - R - bmin;
#pragma unroll
                    for (int dy = 0; dy < N; ++dy)
#pragma unroll
                        for (int dx = 0; dx < N; ++dx)
                            sxy += (int)i0_s[dy][i + dx] * (int)i1_s[dy * WB + b0 + dx];
                }
                const int cc = xp - R - bmin;           // I1 centre index
                const int sy = sy_s[cc];
                const int sxsy = sx * sy;
                const int A1 = 2 * sxsy + c1;
                const int B1 = sxq + syq_s[cc] + c1;
                const int A2 = 2 * (n * sxy - sxsy) + c2;
                const int B2 = vx + vy_s[cc] + c2;
                q = ssim_quotient(A1, A2, B1, B2);
            }
            out[k] = (uint8_t)q;
        }
    }
}

size_t cost_smem_bytes(int N, int Dmax, int Dw)
{
    const int R = N / 2;
    const int U = Dmax;   // upper bound of the span (maxlo - minlo + Dw <= D)
    const int WB = TX + 2 * R + U - 1;
    const int NC = WB - 2 * R;
    size_t b = (size_t)((N * WB + 15) & ~15) + 3 * sizeof(int) * (size_t)NC;
    const int ucp = U < UCAP ? U : UCAP;
    b += sizeof(int) * (size_t)ucp * (TX + 2 * R + 1);
    (void)Dw;
    return b;
}

}  // namespace

void launch_cost(const LevelArgs &a, cudaStream_t s)
{
    dim3 grid((a.W + TX - 1) / TX, a.H, a.nviews);
    const size_t smem = cost_smem_bytes(a.N, a.D, a.Dw);
    if (a.N == 5) {
        cudaFuncSetAttribute(cost_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cost_kernel<5><<<grid, kThreads, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(cost_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cost_kernel<3><<<grid, kThreads, smem, s>>>(a);
    }
}

}  // namespace mpv
