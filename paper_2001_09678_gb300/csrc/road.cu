// road.cu -- road detection on the disparity map (Section 3.5).
//
// v-disparity Hx[j][i]: the number of pixels of image row j with disparity i (Eq.
// disp_map); u-disparity Hy[j][i]: the same per image column (Eq. hy, read with the
// disparity index); the road profile: the row path j = P(i) over all disparities that
// maximises sum_i Hx[P(i)][i] under 0 < P(i) - P(i-1) < eta (Eqs. e and P_hat), ties to
// the smaller row at the end and at every predecessor.  Pixels whose value is not below
// D (0xFFFF: rejected by the left-right check) are not counted.
#include "mpv_internal.cuh"

namespace mpv {

namespace {

constexpr int kHistThreads = 256;
constexpr int kUCols = 32;               // columns per block of the u-disparity
constexpr int kRoadThreads = 1024;

// One block per image row: a shared histogram of D bins.
__global__ void __launch_bounds__(kHistThreads) vdisp_kernel(const uint16_t *__restrict__ U,
                                                             int W, int pitch, int D,
                                                             uint32_t *__restrict__ Hx)
{
    extern __shared__ uint32_t hist[];
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < D; i += kHistThreads) hist[i] = 0;
    __syncthreads();
    const uint16_t *row = U + (int64_t)j * pitch;
    for (int x = threadIdx.x; x < W; x += kHistThreads) {
        const int u = row[x];
        if (u < D) atomicAdd(&hist[u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < D; i += kHistThreads) Hx[(int64_t)j * D + i] = hist[i];
}

// One block per 32 columns: lane = column, warps stride over the rows.
__global__ void __launch_bounds__(kHistThreads) udisp_kernel(const uint16_t *__restrict__ U,
                                                             int W, int H, int pitch, int D,
                                                             uint32_t *__restrict__ Hy)
{
    extern __shared__ uint32_t hist[];          // [kUCols][D]
    const int x0 = blockIdx.x * kUCols;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kUCols * D; i += kHistThreads) hist[i] = 0;
    __syncthreads();
    const int x = x0 + lane;
    constexpr int kRows = kHistThreads / 32, kBatch = 8;
    if (x < W)
        for (int y0 = warp; y0 < H; y0 += kRows * kBatch) {
            int u[kBatch];   // the batch's loads are issued before its shared atomics
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int y = y0 + b * kRows;
                u[b] = y < H ? U[(int64_t)y * pitch + x] : D;
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b)
                if (u[b] < D) atomicAdd(&hist[lane * D + u[b]], 1u);
        }
    __syncthreads();
    const int ncols = min(kUCols, W - x0);
    for (int i = threadIdx.x; i < ncols * D; i += kHistThreads) Hy[(int64_t)x0 * D + i] = hist[i];
}

// The road Viterbi in one block: threads own rows, the disparities are the sequential
// steps.  e holds the best prefix sum ending at (i, j), -1 when unreachable; the step
// back from (i, j) is stored as the row difference j - j' (1 .. eta-1, 0 = none), in
// shared memory when it fits (SMEM_BACK) or in the global scratch otherwise.  The
// histogram is staged kRoadChunk disparities at a time, transposed, so that each step
// reads shared memory only.
constexpr int kRoadChunk = 32;          // at most; fewer when the rows are many

template <bool SMEM_BACK>
__global__ void __launch_bounds__(kRoadThreads) road_kernel(const uint32_t *__restrict__ Hx,
                                                            int H, int D, int eta, int chunk_n,
                                                            uint8_t *__restrict__ back_g,
                                                            int32_t *__restrict__ P,
                                                            int64_t *__restrict__ energy)
{
    extern __shared__ __align__(16) unsigned char sm[];
    int32_t *e0 = (int32_t *)sm;
    int32_t *e1 = e0 + H;
    uint32_t *chunk = (uint32_t *)(e1 + H);            // [chunk_n][H]
    uint8_t *back = SMEM_BACK ? (uint8_t *)(chunk + chunk_n * H) : back_g;
    __shared__ unsigned long long red[kRoadThreads / 32];
    int32_t *prev = e0, *cur = e1;
    for (int i0 = 0; i0 < D; i0 += chunk_n) {
        const int nc = min(chunk_n, D - i0);
        __syncthreads();                                // the previous chunk is consumed
        // a thread's loads of a row are issued together, then stored transposed
        for (int j = threadIdx.x; j < H; j += kRoadThreads) {
            uint32_t v[kRoadChunk];
#pragma unroll
            for (int c = 0; c < kRoadChunk; ++c)
                if (c < nc) v[c] = Hx[(int64_t)j * D + i0 + c];
#pragma unroll
            for (int c = 0; c < kRoadChunk; ++c)
                if (c < nc) chunk[c * H + j] = v[c];
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            const int i = i0 + c;
            if (i == 0) {
                for (int j = threadIdx.x; j < H; j += kRoadThreads) prev[j] = (int32_t)chunk[j];
            } else {
                for (int j = threadIdx.x; j < H; j += kRoadThreads) {
                    int32_t best = -1;
                    int arg = 0;
                    // predecessors in chunks of 8 loaded together, each chunk reduced as a
                    // tree; the earlier (smaller) row wins ties inside a chunk and between
                    // chunks (strict comparison against the running best)
                    for (int j0 = max(0, j - eta + 1); j0 < j; j0 += 8) {
                        int32_t v[8];
                        int ix[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            ix[e] = j0 + e;
                            v[e] = j0 + e < j ? prev[j0 + e] : -2;
                        }
#pragma unroll
                        for (int w = 1; w < 8; w <<= 1)
#pragma unroll
                            for (int e = 0; e < 8; e += 2 * w)
                                if (v[e + w] > v[e]) {
                                    v[e] = v[e + w];
                                    ix[e] = ix[e + w];
                                }
                        if (v[0] > best) {
                            best = v[0];
                            arg = ix[0];
                        }
                    }
                    cur[j] = best < 0 ? -1 : best + (int32_t)chunk[c * H + j];
                    back[(int64_t)i * H + j] = (uint8_t)(best < 0 ? 0 : j - arg);
                }
                int32_t *t = prev;
                prev = cur;
                cur = t;
            }
            __syncthreads();
        }
    }
    // best final row: key = (e + 1) << 32 | ~j, maximal for the largest e, then smallest j
    unsigned long long key = 0;
    for (int j = threadIdx.x; j < H; j += kRoadThreads) {
        const unsigned long long k =
            ((unsigned long long)(uint32_t)(prev[j] + 1) << 32) | (0xFFFFFFFFu - (uint32_t)j);
        key = k > key ? k : key;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xFFFFFFFFu, key, o);
        key = v > key ? v : key;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = 0;
        for (int w = 0; w < kRoadThreads / 32; ++w) k = red[w] > k ? red[w] : k;
        const int64_t best = (int64_t)(k >> 32) - 1;
        int j = best < 0 ? -1 : (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
        for (int i = D - 1; i >= 0; --i) {
            P[i] = j;
            if (j >= 0 && i > 0) j -= back[(int64_t)i * H + j];
        }
        *energy = best;
    }
}

}  // namespace

size_t road_scratch_bytes(int H, int D) { return (size_t)H * D; }

// shared memory of the road kernel: e (two rows of H), the staged chunk of disparities
// (as many as fit in 96 KB, up to 32), and the steps back when they fit
int road_chunk(int H)
{
    int c = kRoadChunk;
    while (c > 1 && (size_t)4 * c * H > 96 * 1024) c >>= 1;
    return c;
}
size_t road_smem_base(int H) { return (8 + 4 * (size_t)road_chunk(H)) * (size_t)H; }
bool road_back_in_smem(int H, int D) { return road_smem_base(H) + (size_t)H * D <= 200 * 1024; }

void launch_road(const uint16_t *U, int W, int H, int pitch, int D, int eta, uint32_t *Hx,
                 uint32_t *Hy, int32_t *P, int64_t *energy, uint8_t *scratch, cudaStream_t s)
{
    vdisp_kernel<<<H, kHistThreads, sizeof(uint32_t) * D, s>>>(U, W, pitch, D, Hx);
    if (Hy) {
        const size_t smem = sizeof(uint32_t) * kUCols * D;
        cudaFuncSetAttribute(udisp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        udisp_kernel<<<(W + kUCols - 1) / kUCols, kHistThreads, smem, s>>>(U, W, H, pitch, D, Hy);
    }
    if (road_back_in_smem(H, D)) {
        const size_t smem = road_smem_base(H) + (size_t)H * D;
        cudaFuncSetAttribute(road_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        road_kernel<true><<<1, kRoadThreads, smem, s>>>(Hx, H, D, eta, road_chunk(H), nullptr, P,
                                                         energy);
    } else {
        const size_t smem = road_smem_base(H);
        cudaFuncSetAttribute(road_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        road_kernel<false><<<1, kRoadThreads, smem, s>>>(Hx, H, D, eta, road_chunk(H), scratch, P,
                                                          energy);
    }
}

}  // namespace mpv
