// mpv_internal.cuh -- shared declarations of the CUDA matcher (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpv {

constexpr int kMaxScales = 4;
constexpr int kMaxViews = 2;
// Large value for absent (virtual) nodes; sums of it with penalties stay below 2^30.
constexpr int kInf = 1 << 28;

// Buffers of one view at one pyramid level.  View 0 is the left view (I0 = left,
// I1 = right); view 1 is the matcher run on the mirrored, swapped pair.
struct ViewLevel {
    const uint8_t *I0;
    const uint8_t *I1;
    int pitch0, pitch1;      // bytes
    const uint16_t *lo;      // window starts [H][W]; nullptr = 0 (full range)
    uint16_t *C;             // cost volume [H][W][Dw], u fastest
    uint32_t *S;             // summed path energies [H][W][Dw]
    uint16_t *d;             // pre-check WTA map [H][W]
};

struct LevelArgs {
    int W, H;        // level size
    int D;           // full label range of the level
    int Dw;          // labels evaluated per pixel
    int nviews;
    ViewLevel v[kMaxViews];
    // cost
    int N;           // SSIM window side
    int c1, c2;      // SSIM constants scaled by n^2
    // aggregation
    int p1;          // effective jump penalty per label (min(p1, T))
    int trunc;       // effective truncation (kInf when none)
    int npaths;
};

struct SeedArgs {
    int W, H, Wp, Hp;
    int block, Dw, D;
    int nviews;
    const uint16_t *dprev[kMaxViews];
    uint16_t *lo[kMaxViews];
};

struct ImageJob {       // one 2x2 down-sampling or mirror job
    const uint8_t *src;
    int src_pitch;
    uint8_t *dst;
    int dst_pitch;
};

void launch_mirror(const ImageJob *jobs, int njobs, int W, int H, cudaStream_t s);
void launch_down2(const ImageJob *jobs, int njobs, int W, int H, cudaStream_t s);
void launch_seed(const SeedArgs &a, cudaStream_t s);
void launch_cost(const LevelArgs &a, cudaStream_t s);
void launch_aggregate(const LevelArgs &a, cudaStream_t s);
void launch_wta(const LevelArgs &a, cudaStream_t s);
void launch_lr(const uint16_t *dL, const uint16_t *dRm, int W, int H, int tol, int check,
               uint16_t *out, int out_pitch, uint16_t *out_right, int right_pitch,
               cudaStream_t s);

}  // namespace mpv
