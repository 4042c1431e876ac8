// mpv_internal.cuh -- shared declarations of the CUDA matcher (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mpv.h"

namespace mpv {

constexpr int kMaxScales = 4;
constexpr int kMaxViews = 2;
// Large value for absent (virtual) nodes in 32-bit arithmetic.
constexpr int kInf = 1 << 28;
// Absent nodes in the packed 16-bit arithmetic: above every valid energy (< 8192) and
// still below 2^16 after adding any penalty term (< 16384).
constexpr uint32_t kInf16 = 0x4000u;

// Buffers of one view at one pyramid level.  View 0 is the left view (I0 = left,
// I1 = right); view 1 is the matcher run on the mirrored, swapped pair.
struct ViewLevel {
    const uint8_t *I0;
    const uint8_t *I1;
    int pitch0, pitch1;      // bytes
    const uint16_t *lo;      // window starts [H][W]; nullptr = 0 (full range)
    uint8_t *C;              // cost volume [H][W][Dws], u fastest (costs are <= 255)
    uint16_t *S;             // summed path energies [H][W][Dws]
    uint16_t *d;             // pre-check WTA map [H][W]
};

struct LevelArgs {
    int W, H;        // level size
    int D;           // full label range of the level
    int Dw;          // labels evaluated per pixel
    int Dws;         // per-pixel stride of C and S: Dw rounded up to 16
    int nviews;
    ViewLevel v[kMaxViews];
    // cost
    int N;           // SSIM window side
    int c1, c2;      // SSIM constants scaled by n^2
    // aggregation
    int p1;          // effective jump penalty per label
    int trunc;       // effective truncation: min(T, p1 * (D - 1))
    int radius;      // labels beyond which the truncation dominates: ceil(T/p1) - 1
    int npaths;
    int lanes;       // lanes per scan path for 32/64-label strides (4 or 8; autotuned)
};

// Launch shapes chosen per image shape by the autotuner.
struct Tuning {
    int lanes = 8;   // aggregation: lanes per scan path (4 or 8)
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
// stage dumps: C (u8, stride Dws) -> u16 [.][Dw]; S (u16, stride Dws) -> u32 [.][Dw]
void launch_unpack(const LevelArgs &a, int view, uint16_t *cost, uint32_t *sum, cudaStream_t s);

// ---- the pipeline shared by every entry point ----------------------------------------

struct Geometry {
    int S;
    int W[kMaxScales], H[kMaxScales], D[kMaxScales], Dw[kMaxScales], Dws[kMaxScales];
    int block[kMaxScales], pitch[kMaxScales];
};

struct Layout {
    size_t total = 0;
    size_t img0[kMaxViews][kMaxScales], img1[kMaxViews][kMaxScales];
    size_t lo[kMaxViews][kMaxScales], d[kMaxViews][kMaxScales];
    size_t C[kMaxViews], S[kMaxViews];
};

struct PairJob {
    const uint8_t *left, *right;
    int W, H, pitch, D;
    uint16_t *disp;
    int disp_pitch;
    uint16_t *disp_right;
};

// Optional per-stage hook (profiling); called around each stage's launches.
struct StageHook {
    void (*begin)(void *user, int stage, int nkernels, cudaStream_t s);
    void (*end)(void *user, int stage, cudaStream_t s);
    void *user;
};

// Optional stage dump of one view and level (device outputs, each may be null).
struct StageSink {
    int view = -1, level = -1;
    uint16_t *lo = nullptr, *cost = nullptr, *disp = nullptr;
    uint32_t *sum = nullptr;
};

bool params_valid(const mpv_params &p);
mpv_status validate_pair(const mpv_params &p, int W, int H, int pitch, int disp_pitch, int D);
void make_geometry(const mpv_params &p, int W, int H, int D, Geometry &g);
Layout make_layout(const Geometry &g, int nviews);
int views_needed(const mpv_params &p, const PairJob &job, const StageSink *dbg);

// Enqueues the whole matcher for one pair on stream s, with its scratch at `workspace`
// (at least make_layout(...).total bytes).
mpv_status enqueue_pair(const mpv_params &p, const PairJob &job, uint8_t *workspace,
                        cudaStream_t s, const StageHook *hook, const StageSink *dbg,
                        const Tuning &tune = Tuning());

}  // namespace mpv
