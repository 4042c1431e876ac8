// pyramid.cu -- image pyramid, window seeding, winner-take-all and left-right check.
//
// Section 3.4 of the paper: the pair is down-sampled by 2 per level; only the top
// level searches the full range; each finer level searches a per-pixel window whose
// centre comes from the coarser level's disparities, doubled (the sampling rate), as a
// block mode at intermediate levels and by linear interpolation at the finest level.
#include "pyramid_body.cuh"

namespace mpv {

namespace {

__global__ void mirror_kernel(const int *gate, ImageJob j0, ImageJob j1, int W, int H)
{
    if (gate && *gate == 0) return;
    mirror_body(blockIdx.z == 0 ? j0 : j1, W, H, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

struct Jobs4 {
    ImageJob j[4];
};

struct PyrJobs4 {
    PyrJob j[4];
};

__global__ void down2_kernel(Jobs4 jobs, int W, int H, const int *gate)
{
    if (gate && *gate == 0) return;
    down2_body(jobs.j[blockIdx.z], W, H, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(2 * kPyrCols) pyramid2_kernel(PyrJobs4 jobs, int W, int H,
                                                                 const int *gate)
{
    if (gate && *gate == 0) return;
    __shared__ uint8_t t1[2][kPyrCols];
    pyramid2_body(jobs.j[blockIdx.z], W, H, blockIdx.x, blockIdx.y, threadIdx.x, t1);
}

// One block per row (blockIdx.x) and view (blockIdx.y); the threads stride over the row.
__global__ void __launch_bounds__(256) seed_kernel(SeedArgs a)
{
    if (a.gate && *a.gate == 0) return;
#pragma unroll 4
    for (int x = threadIdx.x; x < a.W; x += blockDim.x) seed_body(a, x, blockIdx.x, blockIdx.y);
}

template <int LPP>
__global__ void wta_kernel(LevelArgs a)
{
    if (a.gate && *a.gate == 0) return;
    wta_body<LPP>(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.z);
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
    lr_body(dL, dRm, W, H, tol, check, out, out_pitch, out_right, right_pitch,
            blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
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
    seed_kernel<<<dim3(a.H, a.nviews, 1), 256, 0, s>>>(a);
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
