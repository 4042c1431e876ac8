// aggregate.cu -- directional Viterbi passes summed over 4 or 8 scan directions.
//
// Section 3.2 / Eq. e(p,u): along each scan direction r the energy of node (p,u) is
// its cost plus the cheapest predecessor node (p-r, v) plus the jump penalty
// eps(u,v) = min(p1 |u-v|, T), with every node of the predecessor connected (full
// connectivity).  Section 3.3 evaluates that minimum in O(2m) by one upward and one
// downward sweep over the labels.  Here the two sweeps are written as prefix minima:
//     min_{v<=u} A(v) + p1 (u - v) = p1 u + min_{v<=u} (A(v) - p1 v)
//     min_{v>=u} A(v) + p1 (v - u) = -p1 u + min_{v>=u} (A(v) + p1 v)
// so a warp evaluates them as two shuffle scans over its lanes.  Labels are absolute
// disparities: a predecessor with a different window start connects through the
// penalty, and labels outside its window are virtual nodes (absent).  Energies are
// kept in the bounded form L = C + M' - min_v A(v) (a per-pixel constant shift that
// leaves every argmin unchanged), and each pass adds L into the summed volume S.
//
// v1 layout: one warp per scan path, K = ceil(Dw/32) consecutive labels per lane.
#include "mpv_internal.cuh"

namespace mpv {

namespace {

constexpr int kWarps = 8;

__constant__ int c_dirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                 {1, 1}, {-1, -1}, {-1, 1}, {1, -1}};

__device__ __forceinline__ int warp_min(int v)
{
    return __reduce_min_sync(0xFFFFFFFFu, v);
}

// Start pixel and number of paths of direction (dx,dy) on a W x H level.
__device__ __forceinline__ int num_paths_dir(int dx, int dy, int W, int H)
{
    if (dy == 0) return H;
    if (dx == 0) return W;
    return W + H - 1;
}

__device__ __forceinline__ void path_start(int dx, int dy, int W, int H, int i, int &x, int &y)
{
    if (dy == 0) {
        x = dx > 0 ? 0 : W - 1;
        y = i;
    } else if (dx == 0) {
        x = i;
        y = dy > 0 ? 0 : H - 1;
    } else if (i < W) {
        x = i;
        y = dy > 0 ? 0 : H - 1;
    } else {
        x = dx > 0 ? 0 : W - 1;
        y = dy > 0 ? (i - W + 1) : (H - 2 - (i - W));
    }
}

template <int K>
__global__ void __launch_bounds__(kWarps * 32) aggregate_kernel(LevelArgs a)
{
    const int view = blockIdx.z;
    const int dir = blockIdx.y;
    const int dx = c_dirs[dir][0], dy = c_dirs[dir][1];
    const int W = a.W, H = a.H, Dw = a.Dw;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int path = blockIdx.x * kWarps + warp;
    if (path >= num_paths_dir(dx, dy, W, H)) return;
    const ViewLevel &V = a.v[view];
    const int P1 = a.p1, T = a.trunc;

    extern __shared__ int sh[];
    int *pB = sh + warp * 2 * (32 * K + 2);   // [32K+1]: index j+1 holds prefix min up to j
    int *sC = pB + (32 * K + 1);              // [32K+1]: index j holds suffix min from j

    int x, y;
    path_start(dx, dy, W, H, path, x, y);
    int A[K];
    int prev_lo = 0;
    bool first = true;
    while (x >= 0 && x < W && y >= 0 && y < H) {
        const int64_t pix = (int64_t)y * W + x;
        const int cur_lo = V.lo ? (int)V.lo[pix] : 0;
        const uint16_t *cp = V.C + pix * Dw;
        uint32_t *sp = V.S + pix * Dw;
        int c[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int k = lane * K + t;
            c[t] = k < Dw ? (int)cp[k] : kInf;
        }
        int L[K];
        if (first) {
#pragma unroll
            for (int t = 0; t < K; ++t) L[t] = c[t];
            first = false;
        } else {
            // minimum of the predecessor and the two scans
            int m = A[0];
#pragma unroll
            for (int t = 1; t < K; ++t) m = min(m, A[t]);
            const int amin = warp_min(m);
            int pb[K], sc[K];
            int run = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t) {
                run = min(run, A[t] - P1 * (lane * K + t));
                pb[t] = run;
            }
            int incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl = min(incl, v);
            }
            int excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
            if (lane == 0) excl = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t) pb[t] = min(pb[t], excl);
            run = kInf;
#pragma unroll
            for (int t = K - 1; t >= 0; --t) {
                run = min(run, A[t] + P1 * (lane * K + t));
                sc[t] = run;
            }
            incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_down_sync(0xFFFFFFFFu, incl, o);
                if (lane + o < 32) incl = min(incl, v);
            }
            excl = __shfl_down_sync(0xFFFFFFFFu, incl, 1);
            if (lane == 31) excl = kInf;
#pragma unroll
            for (int t = 0; t < K; ++t) sc[t] = min(sc[t], excl);

            const int s = cur_lo - prev_lo;      // uniform across the warp
            const int cap = amin + T;
            if (s == 0) {
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const int j = lane * K + t;
                    const int M = min(min(P1 * j + pb[t], sc[t] - P1 * j), cap);
                    L[t] = c[t] + M - amin;
                }
            } else {
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    pB[lane * K + t + 1] = pb[t];
                    sC[lane * K + t] = sc[t];
                }
                if (lane == 0) {
                    pB[0] = kInf;
                    sC[32 * K] = kInf;
                }
                __syncwarp();
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const int jj = s + lane * K + t;  // label index in the predecessor window
                    const int pi = min(max(jj, -1), 32 * K - 1) + 1;
                    const int si = min(max(jj, 0), 32 * K);
                    const int M = min(min(P1 * jj + pB[pi], sC[si] - P1 * jj), cap);
                    L[t] = c[t] + M - amin;
                }
                __syncwarp();
            }
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (lane * K + t >= Dw) L[t] = kInf;
        }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int k = lane * K + t;
            if (k < Dw) atomicAdd(sp + k, (uint32_t)L[t]);
            A[t] = L[t];
        }
        prev_lo = cur_lo;
        x += dx;
        y += dy;
    }
}

template <int K>
void launch_k(const LevelArgs &a, cudaStream_t s)
{
    const int maxp = a.W + a.H - 1;
    dim3 grid((maxp + kWarps - 1) / kWarps, a.npaths, a.nviews);
    const size_t smem = sizeof(int) * kWarps * 2 * (32 * K + 2);
    cudaFuncSetAttribute(aggregate_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    aggregate_kernel<K><<<grid, kWarps * 32, smem, s>>>(a);
}

}  // namespace

void launch_aggregate(const LevelArgs &a, cudaStream_t s)
{
    const int K = (a.Dw + 31) / 32;
    if (K <= 1) launch_k<1>(a, s);
    else if (K <= 2) launch_k<2>(a, s);
    else if (K <= 4) launch_k<4>(a, s);
    else if (K <= 8) launch_k<8>(a, s);
    else if (K <= 16) launch_k<16>(a, s);
    else launch_k<32>(a, s);
}

}  // namespace mpv
