// batch.cu -- a batch of stereo pairs through one persistent kernel over a device work list.
//
// Every stage of every pair (pyramid, window seeding, cost, directional passes,
// winner-take-all per level and view, left-right check) becomes a list of work items,
// each a few blocks' worth of the stand-alone kernel's work, run by the same device
// functions.  The items of a group of pairs form one queue, in the order the stages
// depend on each other; a batch has several queues (the pairs dealt to them largest
// first, like streams).  A fixed grid of CTAs claims items: a CTA scans the queues'
// heads and claims a head item only once every item of the stage it depends on has
// completed (per-stage completion counters in device memory), so no CTA ever waits
// while holding an item and every claim makes progress.  Stages of different pairs
// overlap freely: a CTA that finds the head of one queue blocked takes work from another.
//
// The one wait -- for some claimable item -- is bounded: after `wait_cycles` of clock64()
// without a claim the CTA records MPV_ERR_TIMEOUT in the batch's status word, raises the
// abort flag that makes every other CTA leave at its next claim, and returns.  The host
// reads the status after the launch (mpv_sync).
//
// Within one launch no address of the workspace is written after it has been read (each
// pair has its own region, each level its own cost and summed volumes), so the
// non-coherent loads of the passes never meet a stale line.
#include <algorithm>
#include <cstring>
#include <vector>

#include "agg_stencil.cuh"
#include "cost_body.cuh"
#include "pyramid_body.cuh"

namespace mpv {

namespace {

constexpr int kBT = 256;          // threads of the persistent kernel
constexpr int kBW = kBT / 32;     // its warps: the passes run 8 warps per stencil block

enum : uint8_t { kPyr2, kDown2, kMirror, kSeed, kCost, kAgg, kWta, kLr };

// the passes' launch shapes (lanes per path, packed words per lane, shared-memory minimum)
enum : uint8_t { kS16x8, kS32x8m, kS32x8, kS32x4, kS48x4, kS64x8, kNumShapes };

struct BLevel {
    LevelArgs a;      // both views
    SeedArgs seed;    // level > 0
    int shape;        // one of the kS* shapes
    int lpp;          // winner-take-all lanes per pixel
};

struct BPair {
    BLevel lv[kMaxScales];
    PyrJob pyr[4];
    ImageJob down[4];           // four scales: the top level from level 1
    ImageJob mirror[2];
    int S, W, H, npyr, ndown, nmirror;
    const uint16_t *dL, *dRm;
    uint16_t *out, *out_right;
    int out_pitch, right_pitch, lr_tol, lr_check;
};

struct BItem {
    uint8_t kind, level, view, dir;
    uint16_t pair, count;   // count: blocks (or rows) of the stand-alone kernel in the item
    int b0, b1;             // first block / row
    int dep, dep2;          // stage counters that must be complete (-1: none)
    int own;                // the stage counter this item completes into
};

struct BQueue {
    int begin, end;
};

// Device state of one launch (cleared before it): queue heads, stage counters, status.
struct BState {
    int status;
    int abort;
    int heads[1];           // [nqueues], then the stage counters
};

// stage counters of one pair
constexpr int kStPyrA = 0, kStPyrB = 1;
constexpr int stage_of(int l, int v, int k) { return 2 + (l * 2 + v) * 4 + k; }   // k: seed, cost, agg, wta
constexpr int kStLr = 2 + kMaxScales * 2 * 4;
constexpr int kStagesPerPair = kStLr + 1;

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool stage_done(const int *counters, const int *totals, int st)
{
    return st < 0 || ld_acquire(counters + st) >= totals[st];
}

template <int G, int KW, bool XM>
__device__ __noinline__ void run_pass(const LevelArgs &a, int pb, int dir, int view, int tid,
                                      unsigned char *sm, bool win)
{
    MergeArgs mg{};
    mg.dir0 = dir;
    mg.double_up_dir = -1;
    if (win)
        agg_stencil_body<G, KW, 2, true, false, false, false, XM, kBW>(a, mg, pb, 0, view, tid, sm);
    else
        agg_stencil_body<G, KW, 2, false, false, false, false, XM, kBW>(a, mg, pb, 0, view, tid,
                                                                        sm);
}

__device__ __noinline__ void run_cost(const LevelArgs &a, int b0, int count, int view, int tid,
                                      unsigned char *sm)
{
    const int nseg = (a.W + kSegPix - 1) / kSegPix;
    for (int b = b0; b < b0 + count; ++b) {
        if (a.N == 5)
            cost_body<5>(a, a.D - 1, b % nseg, b / nseg, view, tid, sm);
        else
            cost_body<3>(a, a.D - 1, b % nseg, b / nseg, view, tid, sm);
        __syncthreads();   // the staging is reused by the next block
    }
}

__device__ __noinline__ void run_wta(const LevelArgs &a, int lpp, int b0, int count, int view,
                                     int tid)
{
    for (int b = b0; b < b0 + count; ++b) {
        const int64_t g = (int64_t)b * kBT + tid;
        if (lpp == 4) wta_body<4>(a, g, view);
        else wta_body<2>(a, g, view);
    }
}

__device__ void run_item(const BPair &P, const BItem &it, int tid, unsigned char *sm,
                         uint8_t (*t1)[kPyrCols], unsigned char *la_smem)
{
    switch (it.kind) {
    case kPyr2: {
        const PyrJob &j = P.pyr[it.view];
        for (int b = 0; b < it.count; ++b) {
            pyramid2_body(j, P.W, P.H, it.b0 + b, it.b1, tid, t1);
            __syncthreads();   // t1 is reused by the next block
        }
        break;
    }
    case kDown2: {
        const ImageJob &j = P.down[it.view];
        const int W1 = P.lv[1].a.W, H1 = P.lv[1].a.H;
        const int W0 = (W1 + 1) >> 1;
        for (int y = it.b1; y < it.b1 + it.count; ++y)
            for (int x = tid; x < W0; x += kBT) down2_body(j, W1, H1, x, y);
        break;
    }
    case kMirror: {
        const ImageJob &j = P.mirror[it.view];
        for (int y = it.b1; y < it.b1 + it.count; ++y)
            for (int x = tid; x < P.W; x += kBT) mirror_body(j, P.W, P.H, x, y);
        break;
    }
    case kSeed: {
        const SeedArgs &s = P.lv[it.level].seed;
        for (int y = it.b1; y < it.b1 + it.count; ++y)
            for (int x = tid; x < s.W; x += kBT) seed_body(s, x, y, it.view);
        break;
    }
    case kCost:
        run_cost(P.lv[it.level].a, it.b0, it.count, it.view, tid, sm);
        break;
    case kAgg: {
        // the level's arguments in shared memory (read-only during the pass)
        const BLevel &L = P.lv[it.level];
        LevelArgs *la = (LevelArgs *)la_smem;
        for (int i = tid; i < (int)(sizeof(LevelArgs) / 4); i += kBT)
            ((int *)la)[i] = ((const int *)&L.a)[i];
        __syncthreads();
        const bool win = L.a.v[0].lo != nullptr;
        switch (L.shape) {
        case kS16x8: run_pass<8, 1, false>(*la, it.b0, it.dir, it.view, tid, sm, win); break;
        case kS32x8m: run_pass<8, 2, true>(*la, it.b0, it.dir, it.view, tid, sm, win); break;
        case kS32x8: run_pass<8, 2, false>(*la, it.b0, it.dir, it.view, tid, sm, win); break;
        case kS32x4: run_pass<4, 4, false>(*la, it.b0, it.dir, it.view, tid, sm, win); break;
        case kS48x4: run_pass<4, 6, false>(*la, it.b0, it.dir, it.view, tid, sm, win); break;
        default: run_pass<8, 4, false>(*la, it.b0, it.dir, it.view, tid, sm, win); break;
        }
        break;
    }
    case kWta:
        run_wta(P.lv[it.level].a, P.lv[it.level].lpp, it.b0, it.count, it.view, tid);
        break;
    default: {   // kLr
        for (int y = it.b1; y < it.b1 + it.count; ++y)
            for (int x = tid; x < P.W; x += kBT)
                lr_body(P.dL, P.dRm, P.W, P.H, P.lr_tol, P.lr_check, P.out, P.out_pitch,
                        P.out_right, P.right_pitch, x, y);
        break;
    }
    }
}

// Claims the next item (its index) or returns -1 when every queue is drained, the batch
// was aborted, or no item became claimable within wait_cycles (status: timeout).
__device__ int claim(const BItem *items, const BQueue *queues, int nq, const int *totals,
                     BState *st, int *counters, long long wait_cycles)
{
    const long long t0 = clock64();
    int *heads = st->heads;
    unsigned sleep = 32;
    for (;;) {
        if (*(volatile int *)&st->abort) return -1;
        bool left = false;
        for (int k = 0; k < nq; ++k) {
            const int q = (blockIdx.x + k) % nq;
            const int h = *(volatile int *)&heads[q];
            const int i = queues[q].begin + h;
            if (i >= queues[q].end) continue;
            left = true;
            const BItem &it = items[i];
            if (!stage_done(counters, totals, it.dep) || !stage_done(counters, totals, it.dep2))
                continue;
            if (atomicCAS(&heads[q], h, h + 1) == h) {
                __threadfence();
                return i;
            }
            left = true;
            k = -1;   // the head moved: rescan from this queue onwards
            continue;
        }
        if (!left) return -1;
        if (clock64() - t0 > wait_cycles) {
            atomicCAS(&st->status, 0, (int)MPV_ERR_TIMEOUT);
            atomicExch(&st->abort, 1);
            return -1;
        }
        __nanosleep(sleep);
        sleep = min(sleep * 2, 1024u);
    }
}

// MINB: resident blocks per SM the kernel is compiled for.  One kernel holds every item
// kind, so the register budget of its largest item (a stencil pass) caps them all: 2
// gives the passes their registers, 3 and 4 trade spills in the passes for more warps
// in every other item; the batch autotuner times each.
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB)
batch_kernel(const BPair *pairs, const BItem *items, const BQueue *queues, int nq,
             const int *totals, BState *st, long long wait_cycles)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint8_t t1[2][kPyrCols];
    __shared__ __align__(16) unsigned char la[sizeof(LevelArgs)];
    __shared__ int s_item;
    int *counters = st->heads + nq;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = claim(items, queues, nq, totals, st, counters, wait_cycles);
        __syncthreads();
        const int i = s_item;
        if (i < 0) return;
        const BItem &it = items[i];
        run_item(pairs[it.pair], it, tid, sm, t1, la);
        __syncthreads();   // the item's writes are done; s_item may be overwritten
        if (tid == 0) {
            __threadfence();
            atomicAdd(counters + it.own, 1);
        }
    }
}

int pass_shape(const LevelArgs &a, int lanes)
{
    switch (a.Dws) {
    case 16: return kS16x8;
    case 32: return lanes == 4 ? kS32x4 : (a.Dw == a.Dws ? kS32x8m : kS32x8);
    case 48: return kS48x4;
    default: return kS64x8;
    }
}

size_t pass_smem(int shape, bool win)
{
    switch (shape) {
    case kS16x8: return win ? StencilSmem<8, 1, 2, true, false, false, kBW>::bytes
                            : StencilSmem<8, 1, 2, false, false, false, kBW>::bytes;
    case kS32x8m:
    case kS32x8: return win ? StencilSmem<8, 2, 2, true, false, false, kBW>::bytes
                            : StencilSmem<8, 2, 2, false, false, false, kBW>::bytes;
    case kS32x4: return win ? StencilSmem<4, 4, 2, true, false, false, kBW>::bytes
                            : StencilSmem<4, 4, 2, false, false, false, kBW>::bytes;
    case kS48x4: return win ? StencilSmem<4, 6, 2, true, false, false, kBW>::bytes
                            : StencilSmem<4, 6, 2, false, false, false, kBW>::bytes;
    default: return win ? StencilSmem<8, 4, 2, true, false, false, kBW>::bytes
                        : StencilSmem<8, 4, 2, false, false, false, kBW>::bytes;
    }
}

int paths_of_dir(int dir, int W, int H)
{
    if (dir < 2) return H;
    if (dir < 4) return W;
    return W + H - 1;
}

}  // namespace

bool batch_supported(const mpv_params &p, int W, int H, int D)
{
    if (p.merge_mode != MPV_MERGE_SUM || p.proposal != MPV_PROPOSAL_PYRAMID || p.top_block > 0)
        return false;
    Geometry g;
    make_geometry(p, W, H, D, g);
    for (int l = 0; l < g.S; ++l) {
        const int Dws = g.Dws[l];
        if (Dws != 16 && Dws != 32 && Dws != 48 && Dws != 64) return false;
        const int64_t span = (int64_t)p.p1 * (g.D[l] - 1);
        const int64_t Teff = (int64_t)p.trunc < span ? p.trunc : span;
        const int64_t p1 = p.p1 < Teff ? p.p1 : Teff;
        const int64_t radius = p1 > 0 ? (Teff + p1 - 1) / p1 - 1 : 0;
        if (radius > 2) return false;
        // the packed sentinel must exceed the windowed caps (see aggregate.cu)
        if (l > 0 && 255 + 2 * Teff >= (int64_t)kInf16) return false;
    }
    return true;
}

// The plan of one batch on the host: descriptors, items, queues, stage totals.
struct BatchPlan::Impl {
    std::vector<BPair> pairs;
    std::vector<BItem> items;
    std::vector<BQueue> queues;
    std::vector<int> totals;
    size_t smem = 0;
};

BatchPlan::BatchPlan() : impl(new Impl) {}
BatchPlan::~BatchPlan() { delete impl; }

size_t batch_pair_bytes(const mpv_params &p, const PairJob &job)
{
    Geometry g;
    make_geometry(p, job.W, job.H, job.D, g);
    return make_layout(g, views_needed(p, job, nullptr), p, true).total;
}

mpv_status plan_batch(const mpv_params &p, const PairJob *jobs, int n, uint8_t *base,
                      const size_t *offsets, const BatchTune &tune, BatchPlan &plan)
{
    BatchPlan::Impl &B = *plan.impl;
    B.pairs.assign(n, BPair{});
    B.items.clear();
    B.totals.assign((size_t)n * kStagesPerPair, 0);
    const int nq = std::max(1, std::min(tune.queues, n));
    std::vector<std::vector<BItem>> q(nq);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)jobs[a].W * jobs[a].H * jobs[a].D > (int64_t)jobs[b].W * jobs[b].H * jobs[b].D;
    });
    size_t smem = 0;
    Tuning lt;
    lt.lanes = tune.lanes;
    lt.err = tune.err;
    for (int r = 0; r < n; ++r) {
        const int pi = order[r];
        const PairJob &job = jobs[pi];
        if (!batch_supported(p, job.W, job.H, job.D)) return MPV_ERR_UNSUPPORTED;
        uint8_t *pb = base + offsets[pi];
        const int nviews = views_needed(p, job, nullptr);
        PairPlan pp;
        plan_pair(p, job, pb, nviews, true, pp);
        BPair &P = B.pairs[pi];
        const int S = pp.g.S, top = S - 1;
        P.S = S;
        P.W = job.W;
        P.H = job.H;
        P.npyr = pp.npyr;
        for (int k = 0; k < pp.npyr; ++k) P.pyr[k] = pp.pyr[k];
        P.nmirror = pp.nmirror;
        for (int k = 0; k < pp.nmirror; ++k) P.mirror[k] = pp.mirror[k];
        P.ndown = top >= 3 ? pp.ndown[0] : 0;
        for (int k = 0; k < P.ndown; ++k) P.down[k] = pp.down[0][k];
        for (int l = 0; l < S; ++l) {
            BLevel &Lv = P.lv[l];
            Lv.a = level_args(p, pp, pb, l, lt, nullptr);
            Lv.a.zero_s = 1;   // the cost blocks clear the summed volume (summed merge)
            if (l > 0) Lv.seed = seed_args(pp, pb, l, nullptr, tune.err);
            Lv.shape = pass_shape(Lv.a, tune.lanes);
            Lv.lpp = Lv.a.Dws >= 32 ? 4 : 2;
            smem = std::max(smem, pass_smem(Lv.shape, l > 0));
        }
        P.dL = (const uint16_t *)(pb + pp.L.d[0][top]);
        P.dRm = nviews == 2 ? (const uint16_t *)(pb + pp.L.d[1][top]) : P.dL;
        P.out = job.disp;
        P.out_pitch = job.disp_pitch;
        P.out_right = nviews == 2 ? job.disp_right : nullptr;
        P.right_pitch = job.disp_pitch;
        P.lr_tol = p.lr_tol;
        P.lr_check = p.lr_check;
        // cost staging of the widest level range
        const int R = p.ssim_window / 2;
        smem = std::max(smem, cost_smem_layout(R, pp.g.D[top] - 1).bytes);

        // this pair's items, in dependency order
        std::vector<BItem> &Q = q[r % nq];
        const int base_st = pi * kStagesPerPair;
        auto add = [&](uint8_t kind, int level, int view, int dir, int count, int b0, int b1,
                       int dep, int dep2, int own) {
            BItem it{};
            it.kind = kind;
            it.level = (uint8_t)level;
            it.view = (uint8_t)view;
            it.dir = (uint8_t)dir;
            it.pair = (uint16_t)pi;
            it.count = (uint16_t)count;
            it.b0 = b0;
            it.b1 = b1;
            it.dep = dep >= 0 ? base_st + dep : -1;
            it.dep2 = dep2 >= 0 ? base_st + dep2 : -1;
            it.own = base_st + own;
            B.totals[it.own] += 1;
            Q.push_back(it);
        };
        int images_done = -1;
        if (pp.npyr) {
            const int W1 = (job.W + 1) / 2, H1 = (job.H + 1) / 2;
            const int nbx = (W1 + kPyrCols - 1) / kPyrCols, nby = (H1 + 1) / 2;
            for (int j = 0; j < pp.npyr; ++j)
                for (int by = 0; by < nby; by += 4)
                    for (int by2 = by; by2 < std::min(by + 4, nby); ++by2)
                        add(kPyr2, 0, j, 0, nbx, 0, by2, -1, -1, kStPyrA);
            images_done = kStPyrA;
        }
        if (pp.nmirror) {
            for (int j = 0; j < pp.nmirror; ++j)
                for (int y = 0; y < job.H; y += 16)
                    add(kMirror, 0, j, 0, std::min(16, job.H - y), 0, y, -1, -1, kStPyrA);
            images_done = kStPyrA;
        }
        if (P.ndown) {
            const int H0 = pp.g.H[0];
            for (int j = 0; j < P.ndown; ++j)
                for (int y = 0; y < H0; y += 8)
                    add(kDown2, 0, j, 0, std::min(8, H0 - y), 0, y, kStPyrA, -1, kStPyrB);
            images_done = kStPyrB;
        }
        for (int l = 0; l < S; ++l) {
            const LevelArgs &a = P.lv[l].a;
            if (l > 0)
                for (int v = 0; v < nviews; ++v)
                    for (int y = 0; y < a.H; y += 16)
                        add(kSeed, l, v, 0, std::min(16, a.H - y), 0, y,
                            stage_of(l - 1, v, 3), -1, stage_of(l, v, 0));
            const int nseg = (a.W + kSegPix - 1) / kSegPix;
            const int nblk = nseg * a.H;
            const int cb = std::max(1, tune.cost_blocks);
            for (int v = 0; v < nviews; ++v)
                for (int b = 0; b < nblk; b += cb)
                    add(kCost, l, v, 0, std::min(cb, nblk - b), b, 0,
                        l > 0 ? stage_of(l, v, 0) : images_done, -1, stage_of(l, v, 1));
            const int G = (P.lv[l].shape == kS32x4 || P.lv[l].shape == kS48x4) ? 4 : 8;
            const int per_blk = kBW * (32 / G);
            for (int v = 0; v < nviews; ++v)
                for (int d = 0; d < p.num_paths; ++d) {
                    const int np = paths_of_dir(d, a.W, a.H);
                    for (int b = 0; b * per_blk < np; ++b)
                        add(kAgg, l, v, d, 1, b, 0, stage_of(l, v, 1), -1, stage_of(l, v, 2));
                }
            const int64_t wthreads = (int64_t)P.lv[l].lpp * a.W * a.H;
            const int wblk = (int)((wthreads + kBT - 1) / kBT);
            for (int v = 0; v < nviews; ++v)
                for (int b = 0; b < wblk; b += 32)
                    add(kWta, l, v, 0, std::min(32, wblk - b), b, 0, stage_of(l, v, 2), -1,
                        stage_of(l, v, 3));
        }
        for (int y = 0; y < job.H; y += 16)
            add(kLr, top, 0, 0, std::min(16, job.H - y), 0, y, stage_of(top, 0, 3),
                nviews == 2 ? stage_of(top, 1, 3) : -1, kStLr);
    }
    B.queues.clear();
    for (int k = 0; k < nq; ++k) {
        BQueue qq{(int)B.items.size(), 0};
        B.items.insert(B.items.end(), q[k].begin(), q[k].end());
        qq.end = (int)B.items.size();
        B.queues.push_back(qq);
    }
    if (tune.stall) {
        // test hook: the finest level's winner-take-all of the largest pair's left view
        // waits for one item more than exists, so that pair's left-right check never
        // becomes claimable and the launch ends by its bounded wait
        const int pi = order[0];
        B.totals[(size_t)pi * kStagesPerPair + stage_of(B.pairs[pi].S - 1, 0, 3)] += 1;
    }
    B.smem = (smem + 15) / 16 * 16;
    return MPV_OK;
}

size_t batch_device_bytes(const BatchPlan &plan)
{
    const BatchPlan::Impl &B = *plan.impl;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(sizeof(BPair) * B.pairs.size()) + al(sizeof(BItem) * B.items.size()) +
           al(sizeof(BQueue) * B.queues.size()) + al(sizeof(int) * B.totals.size()) +
           al(sizeof(int) * (2 + B.queues.size() + B.totals.size()));
}

mpv_status upload_batch(const BatchPlan &plan, void *dev, BatchDevice &out)
{
    const BatchPlan::Impl &B = *plan.impl;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    uint8_t *d = (uint8_t *)dev;
    std::vector<uint8_t> host(batch_device_bytes(plan), 0);
    size_t o = 0;
    auto put = [&](const void *src, size_t bytes) {
        const size_t at = o;
        if (bytes) std::memcpy(host.data() + at, src, bytes);
        o += al(bytes);
        return d + at;
    };
    out.pairs = put(B.pairs.data(), sizeof(BPair) * B.pairs.size());
    out.items = put(B.items.data(), sizeof(BItem) * B.items.size());
    out.queues = put(B.queues.data(), sizeof(BQueue) * B.queues.size());
    out.totals = put(B.totals.data(), sizeof(int) * B.totals.size());
    out.state = d + o;
    out.state_bytes = sizeof(int) * (2 + B.queues.size() + B.totals.size());
    out.nqueues = (int)B.queues.size();
    out.nitems = (int)B.items.size();
    out.smem = B.smem;
    if (cudaMemcpy(dev, host.data(), o, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    return MPV_OK;
}

template <int MINB>
mpv_status launch_batch_t(const BatchDevice &bd, long long wait_cycles, int *status_host,
                          cudaStream_t s)
{
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (bd.smem > 48 * 1024 &&
        cudaFuncSetAttribute(batch_kernel<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bd.smem) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_UNSUPPORTED;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<MINB>, kBT,
                                                      bd.smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return MPV_ERR_UNSUPPORTED;
    }
    const int grid = std::max(1, std::min(nsm * per_sm, bd.nitems));
    cudaMemsetAsync(bd.state, 0, bd.state_bytes, s);
    batch_kernel<MINB><<<grid, kBT, bd.smem, s>>>(
        (const BPair *)bd.pairs, (const BItem *)bd.items, (const BQueue *)bd.queues, bd.nqueues,
        (const int *)bd.totals, (BState *)bd.state, wait_cycles);
    if (status_host)
        cudaMemcpyAsync(status_host, bd.state, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

mpv_status launch_batch(const BatchDevice &bd, long long wait_cycles, int *status_host,
                        cudaStream_t s)
{
    switch (bd.occupancy) {
    case 2: return launch_batch_t<2>(bd, wait_cycles, status_host, s);
    case 3: return launch_batch_t<3>(bd, wait_cycles, status_host, s);
    case 4: return launch_batch_t<4>(bd, wait_cycles, status_host, s);
    default: return MPV_ERR_INVALID_ARG;
    }
}

}  // namespace mpv
