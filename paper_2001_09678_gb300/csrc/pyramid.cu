// pyramid.cu -- image pyramid, window seeding, winner-take-all and left-right check.
//
// Section 3.4 of the paper: the pair is down-sampled by 2 per level; only the top
// level searches the full range; each finer level searches a per-pixel window whose
// centre comes from the coarser level's disparities, doubled (the sampling rate), as a
// block mode at intermediate levels and by linear interpolation at the finest level.
#include "mpv_internal.cuh"

namespace mpv {

namespace {

__global__ void mirror_kernel(const int *gate, ImageJob j0, ImageJob j1, int W, int H)
{
    if (gate && *gate == 0) return;
    const ImageJob j = blockIdx.z == 0 ? j0 : j1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    j.dst[(int64_t)y * j.dst_pitch + x] = j.src[(int64_t)y * j.src_pitch + (W - 1 - x)];
}

struct Jobs4 {
    ImageJob j[4];
};

struct PyrJobs4 {
    PyrJob j[4];
};

// 2x2 box mean, round half up; the last row/column is replicated when odd.
__global__ void down2_kernel(Jobs4 jobs, int W, int H, const int *gate)
{
    if (gate && *gate == 0) return;
    const ImageJob j = jobs.j[blockIdx.z];
    const int W2 = (W + 1) >> 1, H2 = (H + 1) >> 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
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
// down2_kernel passes: 2x2 box mean, round half up, last row/column replicated when odd
// at each level.  A block makes 64 x 2 pixels of the first level and 32 x 1 of the second.
constexpr int kPyrCols = 64;

__global__ void __launch_bounds__(2 * kPyrCols) pyramid2_kernel(PyrJobs4 jobs, int W, int H,
                                                                 const int *gate)
{
    if (gate && *gate == 0) return;
    const PyrJob j = jobs.j[blockIdx.z];
    const int W1 = (W + 1) >> 1, H1 = (H + 1) >> 1;
    const int tx = threadIdx.x % kPyrCols, ty = threadIdx.x / kPyrCols;
    const int x = blockIdx.x * kPyrCols + tx, y = blockIdx.y * 2 + ty;
    __shared__ uint8_t t1[2][kPyrCols];
    if (x < W1 && y < H1) {
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
    if (!j.d2) return;   // the same for the whole block (one image per blockIdx.z)
    __syncthreads();
    if (threadIdx.x < kPyrCols / 2) {
        const int W2 = (W1 + 1) >> 1, H2 = (H1 + 1) >> 1;
        const int X = blockIdx.x * (kPyrCols / 2) + threadIdx.x, Y = blockIdx.y;
        if (X < W2 && Y < H2) {
            // first-level pixels 2X, min(2X+1, W1-1) and rows 2Y, min(2Y+1, H1-1): all in
            // this block's tile
            const int u0 = 2 * threadIdx.x;
            const int u1 = min(2 * X + 1, W1 - 1) - blockIdx.x * kPyrCols;
            const int v1 = min(2 * Y + 1, H1 - 1) - 2 * Y;
            const int sum = t1[0][u0] + t1[0][u1] + t1[v1][u0] + t1[v1][u1];
            j.d2[(int64_t)Y * j.p2 + X] = (uint8_t)((sum + 2) >> 2);
        }
    }
}

__global__ void seed_kernel(SeedArgs a)
{
    if (a.gate && *a.gate == 0) return;
    const int view = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.W || y >= a.H) return;
    const uint16_t *dp = a.dprev[view];
    int c;
    if (a.block >= 2) {
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

// floor((a + b) / 2) of each 16-bit half: a & b + ((a ^ b) >> 1), the shift masked so
// that no bit crosses from the high half into the low half
__device__ __forceinline__ uint32_t avg_u16x2(uint32_t a, uint32_t b)
{
    return (a & b) + (((a ^ b) >> 1) & 0x7FFF7FFFu);
}

// Winner-take-all over each pixel's window, ties to the smallest disparity.  Four lanes
// per pixel; the key (S << 16 | k) orders by energy, then by label.

// LPP lanes per pixel: 4, or 2 for 16-label strides (two 8-label chunks)
template <int LPP>
__global__ void wta_kernel(LevelArgs a)
{
    if (a.gate && *a.gate == 0) return;
    const int view = blockIdx.z;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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

// Window-edge hits of the learned proposal: pixels whose minimum sits on an edge of
// their window while the range continues beyond it (k = d - lo is 0 with lo > 0, or
// Dw - 1 with lo + Dw < D).  A fixed grid strides over the pixels and every block adds
// its two counts with one pair of atomics.
constexpr int kEdgeBlocks = 304, kEdgeThreads = 256;

__global__ void __launch_bounds__(kEdgeThreads) edge_kernel(LevelArgs a)
{
    const ViewLevel &v = a.v[blockIdx.z];
    const int64_t npx = (int64_t)a.W * a.H;
    unsigned hits = 0, px = 0;
    for (int64_t i = (int64_t)blockIdx.x * kEdgeThreads + threadIdx.x; i < npx;
         i += (int64_t)kEdgeBlocks * kEdgeThreads) {
        const int lo = v.lo ? (int)v.lo[i] : 0;
        const int k = (int)v.d[i] - lo;
        hits += (k == 0 && lo > 0) || (k == a.Dw - 1 && lo + a.Dw < a.D);
        ++px;
    }
    for (int o = 16; o > 0; o >>= 1) {
        hits += __shfl_xor_sync(0xFFFFFFFFu, hits, o);
        px += __shfl_xor_sync(0xFFFFFFFFu, px, o);
    }
    __shared__ unsigned part[2][kEdgeThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = hits;
        part[1][threadIdx.x >> 5] = px;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long h = 0, p = 0;
        for (int w = 0; w < kEdgeThreads / 32; ++w) {
            h += part[0][w];
            p += part[1][w];
        }
        if (p) {
            atomicAdd(a.edge, h);
            atomicAdd(a.edge + 1, p);
        }
    }
}

// Stage dump: C and S in the documented [H][W][Dw] layout (u16 and u32).
__global__ void unpack_kernel(LevelArgs a, int view, uint16_t *cost, uint32_t *sum)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)a.W * a.H * a.Dw;
    if (e >= n) return;
    const int64_t pix = e / a.Dw;
    const int k = (int)(e - pix * a.Dw);
    const ViewLevel &v = a.v[view];
    if (cost) cost[e] = v.C[pix * a.Dws + k];
    if (sum) {
        const int64_t j = pix * a.Dws + k;
        sum[e] = v.S2 ? ((uint32_t)v.S[j] + (uint32_t)v.S2[j]) >> 1 : v.S[j];
    }
}

// Left-right check.  dRm is the right view's map in mirrored coordinates.
__global__ void lr_kernel(const uint16_t *__restrict__ dL, const uint16_t *__restrict__ dRm,
                          int W, int H, int tol, int check, uint16_t *out, int out_pitch,
                          uint16_t *out_right, int right_pitch, const int *gate)
{
    if (gate && *gate == 0) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
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

void launch_mirror(const ImageJob *jobs, int njobs, int W, int H, cudaStream_t s,
                   const int *gate)
{
    dim3 grid((W + 127) / 128, H, njobs);
    mirror_kernel<<<grid, 128, 0, s>>>(gate, jobs[0], njobs > 1 ? jobs[1] : jobs[0], W, H);
}

void launch_down2(const ImageJob *jobs, int njobs, int W, int H, cudaStream_t s,
                  const int *gate)
{
    Jobs4 j4;
    for (int i = 0; i < 4; ++i) j4.j[i] = jobs[i < njobs ? i : 0];
    const int W2 = (W + 1) / 2, H2 = (H + 1) / 2;
    dim3 grid((W2 + 127) / 128, H2, njobs);
    down2_kernel<<<grid, 128, 0, s>>>(j4, W, H, gate);
}

void launch_pyramid2(const PyrJob *jobs, int njobs, int W, int H, cudaStream_t s,
                     const int *gate)
{
    PyrJobs4 j4;
    for (int i = 0; i < 4; ++i) j4.j[i] = jobs[i < njobs ? i : 0];
    const int W1 = (W + 1) / 2, H1 = (H + 1) / 2;
    dim3 grid((W1 + kPyrCols - 1) / kPyrCols, (H1 + 1) / 2, njobs);
    pyramid2_kernel<<<grid, 2 * kPyrCols, 0, s>>>(j4, W, H, gate);
}

void launch_seed(const SeedArgs &a, cudaStream_t s)
{
    dim3 grid((a.W + 127) / 128, a.H, a.nviews);
    seed_kernel<<<grid, 128, 0, s>>>(a);
}

void launch_wta(const LevelArgs &a, cudaStream_t s)
{
    const int lpp = a.Dws >= 32 ? 4 : 2;
    const int64_t nthreads = lpp * (int64_t)a.W * a.H;
    dim3 grid((unsigned)((nthreads + 255) / 256), 1, a.nviews);
    if (lpp == 4)
        wta_kernel<4><<<grid, 256, 0, s>>>(a);
    else
        wta_kernel<2><<<grid, 256, 0, s>>>(a);
    if (a.edge) edge_kernel<<<dim3(kEdgeBlocks, 1, a.nviews), kEdgeThreads, 0, s>>>(a);
}

void launch_unpack(const LevelArgs &a, int view, uint16_t *cost, uint32_t *sum, cudaStream_t s)
{
    const int64_t n = (int64_t)a.W * a.H * a.Dw;
    unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, view, cost, sum);
}

void launch_lr(const uint16_t *dL, const uint16_t *dRm, int W, int H, int tol, int check,
               uint16_t *out, int out_pitch, uint16_t *out_right, int right_pitch,
               cudaStream_t s, const int *gate)
{
    dim3 grid((W + 127) / 128, H, 1);
    lr_kernel<<<grid, 128, 0, s>>>(dL, dRm, W, H, tol, check, out, out_pitch, out_right,
                                    right_pitch, gate);
}

namespace {

// The fallback decision of a learned-proposal frame: re-match when more than edge_bp of
// every 10000 matched pixels won on a window edge (one thread).
__global__ void fallback_gate_kernel(const unsigned long long *edge, int edge_bp,
                                     FallbackGate *gate, unsigned long long *counters,
                                     cudaGraphConditionalHandle cond, int has_cond)
{
    const unsigned long long hits = edge[0], px = edge[1];
    const int open = hits * 10000ull > (unsigned long long)edge_bp * px ? 1 : 0;
    gate->hits = hits;
    gate->px = px;
    gate->open = open;
    if (counters) {
        atomicAdd(counters, 1ull);
        if (open) atomicAdd(counters + 1, 1ull);
    }
    if (has_cond) cudaGraphSetConditional(cond, (unsigned)open);
}

}  // namespace

void launch_fallback_gate(const unsigned long long *edge, int edge_bp, FallbackGate *gate,
                          unsigned long long *counters, cudaStream_t s,
                          const cudaGraphConditionalHandle *cond)
{
    fallback_gate_kernel<<<1, 1, 0, s>>>(edge, edge_bp, gate, counters,
                                         cond ? *cond : cudaGraphConditionalHandle{}, cond != nullptr);
}

}  // namespace mpv
