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
// GPU design ("fast SSIM", Fig. fast_ssim, read as running box sums).  One block per
// 256-pixel row segment and view:
//  * the block stages, in shared memory, every image column its pixels can reach as the
//    N patch-row bytes packed in a 64-bit word, and the patch statistics of every centre
//    (sum S, V = n * sum of squares - S^2, and both as floats);
//  * each lane owns one label and slides along the row: the cross sum Sxy of pixel x
//    follows from pixel x-1 by adding the entering column product (two dp4a) and
//    subtracting the leaving one, kept in a register ring of the last N products; where
//    the window start changes between neighbours the lane re-sums the N products;
//  * the quotient is estimated in fp32 from A2 (exact int) and the float statistics and
//    made exact with an int64 check only when the estimate lies within 1e-3 of an
//    integer (the estimate's error is below 2e-4; see ssim_quotient).
#include "cost_body.cuh"

namespace mpv {

namespace {

template <int N>
__global__ void __launch_bounds__(kCostThreads) cost_kernel(LevelArgs a, int uspan_max)
{
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    cost_body<N>(a, uspan_max, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, smem);
}

}  // namespace

void launch_cost(const LevelArgs &a, cudaStream_t s)
{
    // widest disparity span of a segment: window starts lie in [0, D - Dw]
    const int uspan_max = a.D - 1;
    const int R = a.N / 2;
    const CostSmem L = cost_smem_layout(R, uspan_max);
    dim3 grid((a.W + kSegPix - 1) / kSegPix, a.H, a.nviews);
    if (a.N == 5) {
        cudaFuncSetAttribute(cost_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L.bytes);
        cost_kernel<5><<<grid, kCostThreads, L.bytes, s>>>(a, uspan_max);
    } else {
        cudaFuncSetAttribute(cost_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L.bytes);
        cost_kernel<3><<<grid, kCostThreads, L.bytes, s>>>(a, uspan_max);
    }
}

}  // namespace mpv
