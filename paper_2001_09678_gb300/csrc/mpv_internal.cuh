// mpv_internal.cuh -- shared declarations of the CUDA matcher (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "../../include/mpv.h"

namespace mpv {

constexpr int kMaxScales = 4;
constexpr int kMaxViews = 2;
// Large value for absent (virtual) nodes in 32-bit arithmetic.
constexpr int kInf = 1 << 28;
// Absent nodes in the packed 16-bit arithmetic: above every valid energy (< 8192) and
// still below 2^16 after adding any penalty term (< 16384).
constexpr uint32_t kInf16 = 0x4000u;

// Bounds-checked builds (compiled with MPV_DEBUG_BOUNDS): MPV_IN(err, ok, site) is false
// when an index check fails, after recording the first failing site in the device error
// word err (the caller then skips the access); mpv_sync reports MPV_ERR_INTERNAL.  In
// the normal build it is the constant true and the checks vanish.
#ifdef MPV_DEBUG_BOUNDS
__device__ __forceinline__ bool mpv_in(int *err, bool ok, int site)
{
    if (!ok && err) atomicCAS(err, 0, site);
    return ok;
}
#define MPV_IN(err, ok, site) mpv_in((err), (ok), (site))
#else
#define MPV_IN(err, ok, site) true
#endif

// floor((a + b) / 2) of each 16-bit half: a & b + ((a ^ b) >> 1), the shift masked so
// that no bit crosses from the high half into the low half
__device__ __forceinline__ uint32_t avg_u16x2(uint32_t a, uint32_t b)
{
    return (a & b) + (((a ^ b) >> 1) & 0x7FFF7FFFu);
}

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
    const uint16_t *S2;      // layered merge: the final layer's second pass (WTA and the
                             // stage dump read floor((S + S2) / 2)); nullptr otherwise
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
    unsigned long long *edge;  // optional [2]: WTA at a window edge inside the range, pixels
    int block_cut;   // > 0: independent block_cut x block_cut tiles (scan paths restart)
    int zero_s;      // the cost kernel also clears S (the summed merge accumulates into it)
    const int *gate; // optional device word: 0 = every kernel of this level returns at once
    int *err;        // bounds-checked builds: the device error word (see MPV_IN)
};

// Launch shapes chosen per image shape by the autotuner.
struct Tuning {
    int lanes = 8;   // aggregation: lanes per scan path (4 or 8)
    int *err = nullptr;   // bounds-checked builds: the context's device error word
};

struct SeedArgs {
    int W, H, Wp, Hp;
    int block, Dw, D;
    int nviews;
    const uint16_t *dprev[kMaxViews];
    uint16_t *lo[kMaxViews];
    const int *gate;   // as LevelArgs::gate
    int *err;          // as LevelArgs::err
};

struct ImageJob {       // one 2x2 down-sampling or mirror job
    const uint8_t *src;
    int src_pitch;
    uint8_t *dst;
    int dst_pitch;
};

// gate (optional device word): 0 = the launch does nothing
void launch_mirror(const ImageJob *jobs, int njobs, int W, int H, cudaStream_t s,
                   const int *gate = nullptr);
void launch_down2(const ImageJob *jobs, int njobs, int W, int H, cudaStream_t s,
                  const int *gate = nullptr);

struct PyrJob {         // the next two pyramid levels of one image (pyramid2_kernel)
    const uint8_t *src;  // source level, W x H
    int src_pitch;
    int mirror;          // read the source mirrored (x -> W-1-x)
    uint8_t *full;       // optional: the mirrored source written out
    int full_pitch;
    uint8_t *d1;         // the level below the source
    int p1;
    uint8_t *d2;         // optional: the level below that
    int p2;
};
void launch_pyramid2(const PyrJob *jobs, int njobs, int W, int H, cudaStream_t s,
                     const int *gate = nullptr);
void launch_seed(const SeedArgs &a, cudaStream_t s);
void launch_cost(const LevelArgs &a, cudaStream_t s);
void launch_aggregate(const LevelArgs &a, cudaStream_t s);

// General passes (any radius and width, per-step penalties, layered merge).
struct MergeArgs {
    int in_mode;            // data term: 0 cost bytes C, 1 min(qa, qb), 2 floor((qa + qb) / 2)
    int out_mode;           // 0 add the bounded energies into S, 1 store the per-pixel
                            //   min-normalised energies into out[view][direction parity]
    int dir0, ndirs;        // scan directions dir0 .. dir0 + ndirs - 1
    int double_up_dir;      // direction whose upward jumps cost twice, -1 for none
    const int *lut;         // 256 slopes indexed by |I0(p) - I0(p-r)|, or nullptr (p1)
    const uint16_t *qa[kMaxViews], *qb[kMaxViews];
    uint16_t *out[kMaxViews][2];
};
void launch_aggregate_general(const LevelArgs &a, const MergeArgs &m, cudaStream_t s);
// one layer of the layered merge (out_mode 1); returns the number of launches
int launch_layer(const LevelArgs &a, const MergeArgs &m, cudaStream_t s);
void launch_wta(const LevelArgs &a, cudaStream_t s);
void launch_lr(const uint16_t *dL, const uint16_t *dRm, int W, int H, int tol, int check,
               uint16_t *out, int out_pitch, uint16_t *out_right, int right_pitch,
               cudaStream_t s, const int *gate = nullptr);
// stage dumps: C (u8, stride Dws) -> u16 [.][Dw]; S (u16, stride Dws) -> u32 [.][Dw]
void launch_unpack(const LevelArgs &a, int view, uint16_t *cost, uint32_t *sum, cudaStream_t s);

// ---- road detection on the disparity map ------------------------------------------------

// Hx [H][D] (required), Hy [W][D] (optional), profile P [D], best sum; scratch of
// road_scratch_bytes(H, D) when !road_back_in_smem(H, D).
void launch_road(const uint16_t *U, int W, int H, int pitch, int D, int eta, uint32_t *Hx,
                 uint32_t *Hy, int32_t *P, int64_t *energy, uint8_t *scratch, cudaStream_t s);
size_t road_scratch_bytes(int H, int D);
bool road_back_in_smem(int H, int D);
constexpr int kRoadMaxRows = 4096;

// ---- learned proposal ---------------------------------------------------------------------

constexpr int kProposalLayers = 6;

// Device copy of the proposal network (BF16 weights, FP32 biases).
struct ProposalNet {
    int layers = 0;
    int cin[kProposalLayers], cout[kProposalLayers], relu[kProposalLayers];
    const void *w[kProposalLayers];     // __nv_bfloat16 [cout][cin][3][3]
    const float *b[kProposalLayers];
    const void *wt[kProposalLayers];    // the same in the tensor-core kernel's layout
    int train_D = 0, factor = 0;
};

void launch_conv3x3(const __nv_bfloat16 *in, int N, int Cin, int H, int W, const __nv_bfloat16 *w,
                    const float *b, int Cout, int relu, __nv_bfloat16 *out_bf, float *out_f,
                    cudaStream_t s);
void launch_features(const uint8_t *I0, int p0, const uint8_t *I1, int p1, const uint8_t *C,
                     int Dws, int Dw, int W, int H, __nv_bfloat16 *out, cudaStream_t s);
// channels-last forms used by the matcher's own proposal network (cstr: multiple of 8)
void launch_features_nhwc(const uint8_t *I0, int p0, const uint8_t *I1, int p1, const uint8_t *C,
                          int Dws, int Dw, int W, int H, int cstr, __nv_bfloat16 *out,
                          cudaStream_t s);
// Tensor-core convolution (tcgen05): 8-channel planes of the input channels rounded up to
// whole k-steps of 16, and the MMA width for Cout output channels (32, or 16 for Cout = 1).
__host__ __device__ inline int tc_planes(int Cin) { return (Cin + 15) / 16 * 2; }
__host__ __device__ inline int tc_width(int Cout) { return Cout == 32 ? 32 : 16; }
// elements of the weights in the kernel's layout [9][tc_planes(Cin)][tc_width(Cout)][8]
// (element (tap, ci, co) at ((tap * planes + ci / 8) * width + co) * 8 + ci % 8, zero for
// absent input or output channels)
inline size_t tc_weight_elems(int Cin, int Cout)
{
    return (size_t)9 * tc_planes(Cin) * tc_width(Cout) * 8;
}
constexpr size_t kTcMaxSmem = 200 * 1024;   // shared memory the convolution may request
bool conv3x3_tc_ok(int Cin, int Cout);
// wt: the weights in the tensor-core layout above; err (optional): set to 1 when the wait
// for the tensor cores ran out
void launch_conv3x3_nhwc(const __nv_bfloat16 *in, int N, int Cin, int cstr, int H, int W,
                         const __nv_bfloat16 *wt, const float *b, int Cout, int relu,
                         __nv_bfloat16 *out_bf, float *out_f, int *err, cudaStream_t s);
// channels per pixel of the network input in the matcher's buffers
inline int feature_stride(int Dw_top) { return (2 + Dw_top + 7) / 8 * 8; }
void launch_proposal_windows(const float *q, int Wq, int Hq, int f, int W, int H, int D, int Dw,
                             uint16_t *lo, cudaStream_t s);

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
    // cost and summed volumes used at each level: C[v] and S[v] for every level, or with
    // level_volumes one pair per level (no address reused within a launch)
    size_t Cl[kMaxViews][kMaxScales] = {}, Sl[kMaxViews][kMaxScales] = {};
    size_t X[kMaxViews][3] = {};                  // layered merge: three more volumes per view
    size_t feat = 0, act0 = 0, act1 = 0, q = 0;   // learned proposal (both views)
    size_t edge = 0;                              // edge-hit counters
    size_t gate = 0;   // learned proposal with a fallback: FallbackGate, past both layouts
};

// The learned proposal's fallback decision of one frame (device memory).
struct FallbackGate {
    int open;                       // 1: the fallback's launches run
    int pad;
    unsigned long long hits, px;    // the learned frame's window-edge counters
};
// cond (optional): the IF node of a captured graph whose body holds the fallback; the
// decision also sets that node's condition
void launch_fallback_gate(const unsigned long long *edge, int edge_bp, FallbackGate *gate,
                          unsigned long long *counters, cudaStream_t s,
                          const cudaGraphConditionalHandle *cond = nullptr);
// Parameters of the fallback matcher of a learned-proposal configuration.
mpv_params fallback_params(const mpv_params &p);

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
    float *proposal = nullptr;   // learned proposal: the network's top-level prediction
};

bool params_valid(const mpv_params &p);
mpv_status validate_pair(const mpv_params &p, int W, int H, int pitch, int disp_pitch, int D);
void make_geometry(const mpv_params &p, int W, int H, int D, Geometry &g);
Layout make_layout(const Geometry &g, int nviews, const mpv_params &p, bool level_volumes = false);
// Window width of the finest level under the learned proposal (centre +- 8 by default).
int learned_window(const mpv_params &p, int D);
int views_needed(const mpv_params &p, const PairJob &job, const StageSink *dbg);

// Buffers and pyramid jobs of one pair in its workspace, shared by the launch sequence
// (enqueue_pair) and the batch scheduler.
struct PairPlan {
    Geometry g;
    Layout L;
    int nviews = 1;
    const uint8_t *I0[kMaxViews][kMaxScales] = {}, *I1[kMaxViews][kMaxScales] = {};
    int P0[kMaxViews][kMaxScales] = {}, P1[kMaxViews][kMaxScales] = {};
    ImageJob mirror[2];      // one scale with the right view: its mirrored full-size pair
    int nmirror = 0;
    PyrJob pyr[4];           // the two levels below the input, all images
    int npyr = 0;
    ImageJob down[kMaxScales][4];   // level l from level l+1, for l <= top - 3
    int ndown[kMaxScales] = {};
};
void plan_pair(const mpv_params &p, const PairJob &job, uint8_t *base, int nviews,
               bool level_volumes, PairPlan &pp);
// Arguments of level l (both views) and of its window seeding (l > 0).
LevelArgs level_args(const mpv_params &p, const PairPlan &pp, uint8_t *base, int l,
                     const Tuning &tune, const int *gate);
SeedArgs seed_args(const PairPlan &pp, uint8_t *base, int l, const int *gate,
                   int *err = nullptr);

// Enqueues the whole matcher for one pair on stream s, with its scratch at `workspace`
// (at least make_layout(...).total bytes).
// counters (optional, device): learned frames and fallbacks, added to by the decision.
// gate (optional, device): the whole pair's launches return at once while *gate == 0.
// aux (optional): with s capturing a CUDA graph, the learned proposal's fallback goes into
// the body of a conditional node (captured on aux) instead of gated launches.
mpv_status enqueue_pair(const mpv_params &p, const PairJob &job, uint8_t *workspace,
                        cudaStream_t s, const StageHook *hook, const StageSink *dbg,
                        const Tuning &tune = Tuning(), const ProposalNet *net = nullptr,
                        const int *grad_lut = nullptr, unsigned long long *counters = nullptr,
                        const int *gate = nullptr, cudaStream_t aux = nullptr);
// The context's loaded proposal network fits a range of D labels.
bool proposal_fits(const mpv_ctx *ctx, int D);

// ---- batches through one persistent kernel (batch.cu) -------------------------------

// Launch shapes of a persistent batch, chosen by the batch autotuner.
struct BatchTune {
    int lanes = 8;         // lanes per scan path of the 32-label passes (8 or 4)
    int queues = 16;       // work queues (groups of pairs, like streams)
    int cost_blocks = 4;   // cost-kernel blocks per work item
    int occupancy = 2;     // resident blocks per SM the persistent kernel is built for
                           // (2, 3 or 4: fewer registers a thread, more warps)
    bool stall = false;    // test hook: one stage never completes (bounded-wait test)
    int *err = nullptr;    // bounds-checked builds: the device error word
    // the tuner's verdict: the persistent kernel was faster than the stream graph, with
    // the times it measured (ms per batch)
    bool persistent = true;
    float ms = 0.f, streams_ms = 0.f;
};

// Device addresses of an uploaded plan.
struct BatchDevice {
    void *pairs = nullptr, *items = nullptr, *queues = nullptr, *totals = nullptr;
    void *state = nullptr;   // cleared before every launch: status, abort, heads, counters
    size_t state_bytes = 0, smem = 0;
    int nqueues = 0, nitems = 0;
    int occupancy = 2;   // BatchTune::occupancy of the launch
};

class BatchPlan {
public:
    BatchPlan();
    ~BatchPlan();
    BatchPlan(const BatchPlan &) = delete;
    BatchPlan &operator=(const BatchPlan &) = delete;
    struct Impl;
    Impl *impl;
};

// The persistent path handles the summed merge with pyramid windows, radius <= 2 and
// label strides of 16, 32, 48 or 64 (else the batch runs as a graph of streams).
bool batch_supported(const mpv_params &p, int W, int H, int D);
// Workspace of one pair on the persistent path (a volume pair per level).
size_t batch_pair_bytes(const mpv_params &p, const PairJob &job);
mpv_status plan_batch(const mpv_params &p, const PairJob *jobs, int n, uint8_t *base,
                      const size_t *offsets, const BatchTune &tune, BatchPlan &plan);
size_t batch_device_bytes(const BatchPlan &plan);
mpv_status upload_batch(const BatchPlan &plan, void *dev, BatchDevice &out);
// Clears the state, runs the persistent kernel, copies the status word to status_host.
mpv_status launch_batch(const BatchDevice &bd, long long wait_cycles, int *status_host,
                        cudaStream_t s);

// Network input of the top level of `view` (2 + D_top channels, BF16) into out.
mpv_status enqueue_features(const mpv_params &p, const PairJob &job, uint8_t *workspace,
                            cudaStream_t s, int view, __nv_bfloat16 *out);

}  // namespace mpv
