// pipeline.cu -- validation, pyramid geometry, workspace layout and the launch sequence
// of one stereo pair, shared by every entry point of the C ABI.
#include <nvtx3/nvToolsExt.h>
#include "mpv_internal.cuh"

namespace mpv {

namespace {

int ssim_c1(int N)
{
    const int64_t n = (int64_t)N * N;
    return (int)((65025 * n * n + 5000) / 10000);   // (0.01*255)^2 * n^2, rounded
}

int ssim_c2(int N)
{
    const int64_t n = (int64_t)N * N;
    return (int)((585225 * n * n + 5000) / 10000);  // (0.03*255)^2 * n^2, rounded
}

size_t take(size_t &off, size_t bytes)
{
    const size_t at = off;
    off += (bytes + 255) & ~(size_t)255;
    return at;
}

// Names of the stages as NVTX ranges (host side: the span in which a stage's launches
// are enqueued or captured; no-ops unless a tool such as ncu --nvtx is attached).
const char *const kStageRange[] = {"mpv:pyramid", "mpv:seed", "mpv:cost", "mpv:aggregate",
                                   "mpv:wta", "mpv:lr"};

struct HookScope {
    const StageHook *h;
    int stage;
    cudaStream_t s;
    HookScope(const StageHook *h_, int stage_, int nk, cudaStream_t s_) : h(h_), stage(stage_), s(s_)
    {
        nvtxRangePushA(stage >= 0 && stage < 6 ? kStageRange[stage] : "mpv:stage");
        if (h && h->begin) h->begin(h->user, stage, nk, s);
    }
    ~HookScope()
    {
        if (h && h->end) h->end(h->user, stage, s);
        nvtxRangePop();
    }
};

}  // namespace

bool params_valid(const mpv_params &p)
{
    if (p.struct_size != sizeof(mpv_params)) return false;
    if (p.ssim_window != 3 && p.ssim_window != 5) return false;
    if (p.num_scales < 1 || p.num_scales > kMaxScales) return false;
    if (p.num_paths != 4 && p.num_paths != 8) return false;
    if (p.max_disparity < 1 || p.max_disparity > 1024) return false;
    if (p.p1 < 0 || p.trunc < 0 || p.window < 0 || p.lr_tol < 0) return false;
    if (p.lr_check != 0 && p.lr_check != 1) return false;
    if (p.merge_mode != MPV_MERGE_SUM && p.merge_mode != MPV_MERGE_PAPER) return false;
    if (p.proposal != MPV_PROPOSAL_PYRAMID && p.proposal != MPV_PROPOSAL_LEARNED) return false;
    if (p.top_block < 0) return false;
    for (int i = 0; i < 4; ++i)
        if (p.block[i] < 0 || p.block[i] > 8 || p.windows[i] < 0) return false;
    if (p.fallback != MPV_FALLBACK_NONE && p.fallback != MPV_FALLBACK_PYRAMID &&
        p.fallback != MPV_FALLBACK_FULL)
        return false;
    if (p.fallback_edge_bp < 0 || p.fallback_edge_bp > 10000) return false;
    return true;
}

mpv_params fallback_params(const mpv_params &p)
{
    mpv_params q = p;
    q.proposal = MPV_PROPOSAL_PYRAMID;
    q.fallback = MPV_FALLBACK_NONE;
    if (p.fallback == MPV_FALLBACK_FULL) q.num_scales = 1;   // exact MPV over the full range
    return q;
}

// Level sizes, ranges and windows (Section 3.4): level S-1 is the input, each level
// above halves the size (rounding up) and the range; the top level searches its whole
// range, level l > 0 a window of windows[l-1] labels, else `window`, else D/4.
void make_geometry(const mpv_params &p, int W, int H, int D, Geometry &g)
{
    g.S = p.num_scales;
    int w = W, h = H;
    for (int l = g.S - 1; l >= 0; --l) {
        g.W[l] = w;
        g.H[l] = h;
        const int sh = g.S - 1 - l;
        g.D[l] = (D + (1 << sh) - 1) >> sh;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    int Dw = p.window > 0 ? p.window : D / 4;
    if (Dw < 1) Dw = 1;
    for (int l = 0; l < g.S; ++l) {
        const int w = l > 0 && p.windows[l - 1] > 0 ? p.windows[l - 1] : Dw;
        g.Dw[l] = l == 0 ? g.D[0] : (w < g.D[l] ? w : g.D[l]);
        if (p.proposal == MPV_PROPOSAL_LEARNED && l == g.S - 1 && l > 0)
            g.Dw[l] = learned_window(p, D);
        g.Dws[l] = (g.Dw[l] + 15) / 16 * 16;
        const int b = l > 0 ? p.block[l - 1] : 0;
        g.block[l] = b > 0 ? b : (l == g.S - 1 ? 1 : 2);
        g.pitch[l] = (g.W[l] + 15) / 16 * 16;
    }
}

mpv_status validate_pair(const mpv_params &p, int W, int H, int pitch, int disp_pitch, int D)
{
    const int N = p.ssim_window;
    if (W < N || H < N) return MPV_ERR_INVALID_ARG;
    if (D < 1 || D > W || D > 1024) return MPV_ERR_INVALID_ARG;
    if (pitch < W || disp_pitch < W) return MPV_ERR_INVALID_ARG;
    Geometry g;
    make_geometry(p, W, H, D, g);
    if (g.W[0] < N || g.H[0] < N) return MPV_ERR_INVALID_ARG;
    const int64_t jump = (int64_t)p.p1 * (D - 1);
    const int64_t pen = p.trunc < jump ? p.trunc : jump;
    if ((int64_t)p.num_paths * (255 + pen) >= 65535) return MPV_ERR_INVALID_ARG;
    if ((int64_t)W * H > (int64_t)1 << 27) return MPV_ERR_UNSUPPORTED;
    if (p.proposal == MPV_PROPOSAL_LEARNED && p.num_scales < 2) return MPV_ERR_INVALID_ARG;
    return MPV_OK;
}

int learned_window(const mpv_params &p, int D)
{
    const int w = p.window > 0 ? p.window : 17;
    return w < D ? w : D;
}

Layout make_layout(const Geometry &g, int nviews, const mpv_params &p, bool level_volumes)
{
    const bool learned = p.proposal == MPV_PROPOSAL_LEARNED;
    const bool layered = p.merge_mode == MPV_MERGE_PAPER;
    Layout L;
    size_t off = 0;
    int64_t maxvol = 0;
    for (int l = 0; l < g.S; ++l) {
        const int64_t v = (int64_t)g.W[l] * g.H[l] * g.Dws[l];
        if (v > maxvol) maxvol = v;
    }
    for (int v = 0; v < nviews; ++v) {
        for (int l = 0; l < g.S; ++l) {
            const size_t img = (size_t)g.pitch[l] * g.H[l];
            const bool caller = (v == 0 && l == g.S - 1);
            L.img0[v][l] = caller ? 0 : take(off, img);
            L.img1[v][l] = caller ? 0 : take(off, img);
            L.lo[v][l] = take(off, sizeof(uint16_t) * (size_t)g.W[l] * g.H[l]);
            L.d[v][l] = take(off, sizeof(uint16_t) * (size_t)g.W[l] * g.H[l]);
        }
        L.C[v] = take(off, sizeof(uint8_t) * (size_t)maxvol);
        L.S[v] = take(off, sizeof(uint16_t) * (size_t)maxvol);
        for (int l = 0; l < g.S; ++l) {
            L.Cl[v][l] = L.C[v];
            L.Sl[v][l] = L.S[v];
        }
        if (level_volumes) {   // one level keeps C[v], S[v]; every other has its own pair
            int big = 0;
            for (int l = 0; l < g.S; ++l)
                if ((int64_t)g.W[l] * g.H[l] * g.Dws[l] == maxvol) big = l;
            for (int l = 0; l < g.S; ++l) {
                if (l == big) continue;
                const size_t vol = (size_t)g.W[l] * g.H[l] * g.Dws[l];
                L.Cl[v][l] = take(off, sizeof(uint8_t) * vol);
                L.Sl[v][l] = take(off, sizeof(uint16_t) * vol);
            }
        }
        if (layered)
            for (int i = 0; i < 3; ++i) L.X[v][i] = take(off, sizeof(uint16_t) * (size_t)maxvol);
    }
    if (learned) {
        const size_t px0 = (size_t)g.W[0] * g.H[0];
        L.feat = take(off, 2 * sizeof(__nv_bfloat16) * (size_t)feature_stride(g.Dw[0]) * px0);
        L.act0 = take(off, 2 * sizeof(__nv_bfloat16) * 32 * px0);
        L.act1 = take(off, 2 * sizeof(__nv_bfloat16) * 32 * px0);
        L.q = take(off, 2 * sizeof(float) * px0);
    }
    L.edge = take(off, 2 * sizeof(unsigned long long));
    if (learned && p.fallback != MPV_FALLBACK_NONE) {
        // the fallback matcher reuses the workspace after the learned frame; the decision
        // lies past both layouts
        const mpv_params q = fallback_params(p);
        const int top = g.S - 1;
        Geometry gq;
        make_geometry(q, g.W[top], g.H[top], g.D[top], gq);
        const Layout Lq = make_layout(gq, nviews, q);
        if (Lq.total > off) off = Lq.total;
        L.gate = take(off, sizeof(FallbackGate));
    }
    L.total = off;
    return L;
}

mpv_status enqueue_features(const mpv_params &p, const PairJob &job, uint8_t *base,
                            cudaStream_t s, int view, __nv_bfloat16 *out)
{
    mpv_params q = p;
    q.proposal = MPV_PROPOSAL_PYRAMID;
    q.lr_check = view == 1 ? 1 : 0;
    Geometry g;
    make_geometry(q, job.W, job.H, job.D, g);
    const int nviews = view == 1 ? 2 : 1;
    const Layout L = make_layout(g, nviews, q);
    // run the top level's cost (a debug stage of level 0), then build the features
    StageSink dbg;
    dbg.view = view;
    dbg.level = 0;
    const mpv_status st = enqueue_pair(q, job, base, s, nullptr, &dbg);
    if (st != MPV_OK) return st;
    const int top = g.S - 1;
    const uint8_t *I0 = (view == 0 && top == 0) ? job.left : base + L.img0[view][0];
    const uint8_t *I1 = (view == 0 && top == 0) ? job.right : base + L.img1[view][0];
    const int pitch = (view == 0 && top == 0) ? job.pitch : g.pitch[0];
    launch_features(I0, pitch, I1, pitch, base + L.Cl[view][0], g.Dws[0], g.Dw[0], g.W[0], g.H[0],
                    out, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

int views_needed(const mpv_params &p, const PairJob &job, const StageSink *dbg)
{
    return (p.lr_check || job.disp_right || (dbg && dbg->view == 1)) ? 2 : 1;
}

void plan_pair(const mpv_params &p, const PairJob &job, uint8_t *base, int nviews,
               bool level_volumes, PairPlan &pp)
{
    make_geometry(p, job.W, job.H, job.D, pp.g);
    pp.L = make_layout(pp.g, nviews, p, level_volumes);
    pp.nviews = nviews;
    const Geometry &g = pp.g;
    const Layout &L = pp.L;
    const int top = g.S - 1;
    for (int v = 0; v < nviews; ++v)
        for (int l = 0; l < g.S; ++l) {
            pp.I0[v][l] = base + L.img0[v][l];
            pp.I1[v][l] = base + L.img1[v][l];
            pp.P0[v][l] = pp.P1[v][l] = g.pitch[l];
        }
    pp.I0[0][top] = job.left;
    pp.I1[0][top] = job.right;
    pp.P0[0][top] = pp.P1[0][top] = job.pitch;
    // right view: the mirrored, swapped pair.  The first two levels below the input come
    // from one launch that also writes the mirrored inputs; further levels one by one.
    pp.nmirror = 0;
    if (top == 0 && nviews == 2) {
        pp.mirror[0] = {job.right, job.pitch, base + L.img0[1][top], g.pitch[top]};
        pp.mirror[1] = {job.left, job.pitch, base + L.img1[1][top], g.pitch[top]};
        pp.nmirror = 2;
    }
    pp.npyr = 0;
    if (top >= 1) {
        const int l1 = top - 1, l2 = top - 2;
        for (int v = 0; v < nviews; ++v)
            for (int k = 0; k < 2; ++k) {
                // view 0: (left, right); view 1: (mirrored right, mirrored left)
                const uint8_t *src = (v == 0) == (k == 0) ? job.left : job.right;
                const size_t *dimg = k == 0 ? L.img0[v] : L.img1[v];
                PyrJob &j = pp.pyr[pp.npyr++];
                j.src = src;
                j.src_pitch = job.pitch;
                j.mirror = v;
                j.full = v ? base + dimg[top] : nullptr;
                j.full_pitch = g.pitch[top];
                j.d1 = base + dimg[l1];
                j.p1 = g.pitch[l1];
                j.d2 = l2 >= 0 ? base + dimg[l2] : nullptr;
                j.p2 = l2 >= 0 ? g.pitch[l2] : 0;
            }
    }
    for (int l = 0; l < kMaxScales; ++l) pp.ndown[l] = 0;
    for (int l = top - 3; l >= 0; --l) {
        int n = 0;
        for (int v = 0; v < nviews; ++v) {
            pp.down[l][n++] = {pp.I0[v][l + 1], pp.P0[v][l + 1], base + L.img0[v][l], g.pitch[l]};
            pp.down[l][n++] = {pp.I1[v][l + 1], pp.P1[v][l + 1], base + L.img1[v][l], g.pitch[l]};
        }
        pp.ndown[l] = n;
    }
}

LevelArgs level_args(const mpv_params &p, const PairPlan &pp, uint8_t *base, int l,
                     const Tuning &tune, const int *gate)
{
    const Geometry &g = pp.g;
    const Layout &L = pp.L;
    LevelArgs a{};
    a.W = g.W[l];
    a.H = g.H[l];
    a.D = g.D[l];
    a.Dw = g.Dw[l];
    a.Dws = g.Dws[l];
    a.nviews = pp.nviews;
    a.N = p.ssim_window;
    a.c1 = ssim_c1(a.N);
    a.c2 = ssim_c2(a.N);
    // penalty min(p1 |du|, T) over labels of one level: |du| <= D_l - 1, so a
    // truncation above p1 (D_l - 1) never acts and p1 above T acts as T
    const int64_t span = (int64_t)p.p1 * (g.D[l] - 1);
    const int64_t Teff = (int64_t)p.trunc < span ? p.trunc : span;
    a.trunc = (int)Teff;
    a.p1 = (int)(p.p1 < Teff ? p.p1 : Teff);
    a.radius = a.p1 > 0 ? (int)((Teff + a.p1 - 1) / a.p1) - 1 : 0;
    a.npaths = p.num_paths;
    a.lanes = tune.lanes;
    a.block_cut = l == 0 ? p.top_block : 0;
    a.gate = gate;
    a.err = tune.err;
    for (int v = 0; v < pp.nviews; ++v) {
        ViewLevel &vl = a.v[v];
        vl.I0 = pp.I0[v][l];
        vl.I1 = pp.I1[v][l];
        vl.pitch0 = pp.P0[v][l];
        vl.pitch1 = pp.P1[v][l];
        vl.lo = l == 0 ? nullptr : (const uint16_t *)(base + L.lo[v][l]);
        vl.C = base + L.Cl[v][l];
        vl.S = (uint16_t *)(base + L.Sl[v][l]);
        vl.d = (uint16_t *)(base + L.d[v][l]);
        vl.S2 = nullptr;
    }
    return a;
}

SeedArgs seed_args(const PairPlan &pp, uint8_t *base, int l, const int *gate, int *err)
{
    const Geometry &g = pp.g;
    SeedArgs sa{};
    sa.W = g.W[l];
    sa.H = g.H[l];
    sa.Wp = g.W[l - 1];
    sa.Hp = g.H[l - 1];
    sa.block = g.block[l];
    sa.Dw = g.Dw[l];
    sa.D = g.D[l];
    sa.nviews = pp.nviews;
    sa.gate = gate;
    sa.err = err;
    for (int v = 0; v < pp.nviews; ++v) {
        sa.dprev[v] = (const uint16_t *)(base + pp.L.d[v][l - 1]);
        sa.lo[v] = (uint16_t *)(base + pp.L.lo[v][l]);
    }
    return sa;
}

namespace {

// The fallback of a learned-proposal frame inside the CUDA graph being captured on s: the
// decision kernel sets the condition of an IF node whose body (captured on aux) is the
// fallback matcher, so an untaken fallback costs nothing.
mpv_status enqueue_fallback_node(const mpv_params &q, const PairJob &job, uint8_t *base,
                                 cudaStream_t s, cudaStream_t aux, const Tuning &tune,
                                 const int *grad_lut, const unsigned long long *edge, int edge_bp,
                                 FallbackGate *fg, unsigned long long *counters)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &graph) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive || !graph)
        return MPV_ERR_CUDA;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault) !=
        cudaSuccess)
        return MPV_ERR_CUDA;
    launch_fallback_gate(edge, edge_bp, fg, counters, s, &cond);
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &graph, &deps, nullptr, &ndeps) != cudaSuccess)
        return MPV_ERR_CUDA;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp) != cudaSuccess)
        return MPV_ERR_CUDA;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess)
        return MPV_ERR_CUDA;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return MPV_ERR_CUDA;
    const mpv_status r = enqueue_pair(q, job, base, aux, nullptr, nullptr, tune, nullptr,
                                      grad_lut);
    cudaGraph_t got = nullptr;
    const cudaError_t e = cudaStreamEndCapture(aux, &got);
    if (r != MPV_OK) return r;
    return e == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}

}  // namespace

mpv_status enqueue_pair(const mpv_params &p, const PairJob &job, uint8_t *base, cudaStream_t s,
                        const StageHook *hook, const StageSink *dbg, const Tuning &tune,
                        const ProposalNet *net, const int *grad_lut,
                        unsigned long long *counters, const int *gate, cudaStream_t aux)
{
    Geometry g;
    make_geometry(p, job.W, job.H, job.D, g);
    const int nviews = views_needed(p, job, dbg);
    const bool learned = p.proposal == MPV_PROPOSAL_LEARNED;
    if (learned) {
        if (!net || net->layers != kProposalLayers || net->cin[0] != 2 + g.Dw[0] || g.S < 2)
            return MPV_ERR_INVALID_ARG;
        if (dbg && dbg->level != 0 && dbg->level != g.S - 1) return MPV_ERR_INVALID_ARG;
    }
    PairPlan pp;
    plan_pair(p, job, base, nviews, false, pp);
    const Layout &L = pp.L;
    const bool layered = p.merge_mode == MPV_MERGE_PAPER;
    unsigned long long *edge = (unsigned long long *)(base + L.edge);
    const int S = g.S;
    const int top = S - 1;
    if (pp.nmirror) {
        HookScope hs(hook, MPV_STAGE_PYRAMID, 1, s);
        launch_mirror(pp.mirror, pp.nmirror, job.W, job.H, s, gate);
    }
    if (pp.npyr) {
        HookScope hs(hook, MPV_STAGE_PYRAMID, 1, s);
        launch_pyramid2(pp.pyr, pp.npyr, job.W, job.H, s, gate);
    }
    for (int l = top - 3; l >= 0; --l) {
        HookScope hs(hook, MPV_STAGE_PYRAMID, 1, s);
        launch_down2(pp.down[l], pp.ndown[l], g.W[l + 1], g.H[l + 1], s, gate);
    }

    const int last = dbg ? dbg->level : top;
    if (!dbg && learned) cudaMemsetAsync(edge, 0, 2 * sizeof(unsigned long long), s);
    for (int l = 0; l <= last; ++l) {
        if (learned && l > 0 && l < top) continue;
        LevelArgs a = level_args(p, pp, base, l, tune, gate);
        a.edge = (learned && l == top) ? edge : nullptr;
        if (learned && l == top) {
            // windows of the finest level from the network's prediction at the top level
            HookScope hs(hook, MPV_STAGE_SEED, nviews, s);
            const float *q = (const float *)(base + L.q);
            const size_t px0 = (size_t)g.W[0] * g.H[0];
            for (int v = 0; v < nviews; ++v)
                launch_proposal_windows(q + v * px0, g.W[0], g.H[0], 1 << (g.S - 1), a.W, a.H,
                                        a.D, a.Dw, (uint16_t *)(base + L.lo[v][l]), s);
        } else if (l > 0) {
            HookScope hs(hook, MPV_STAGE_SEED, 1, s);
            const SeedArgs sa = seed_args(pp, base, l, gate, tune.err);
            launch_seed(sa, s);
        }
        {
            HookScope hs(hook, MPV_STAGE_COST, 1, s);
            a.zero_s = !layered;   // the summed merge: instead of a memset of S
            launch_cost(a, s);
        }
        if (learned && l == 0) {
            HookScope hs(hook, MPV_STAGE_SEED, 2 + net->layers, s);
            // channels-last activations: the network input padded to a multiple of 8
            // channels, the hidden layers 32 channels per pixel
            const size_t px0 = (size_t)a.W * a.H;
            const int cstr0 = feature_stride(a.Dw);
            __nv_bfloat16 *feat = (__nv_bfloat16 *)(base + L.feat);
            for (int v = 0; v < nviews; ++v)
                launch_features_nhwc(a.v[v].I0, a.v[v].pitch0, a.v[v].I1, a.v[v].pitch1,
                                     a.v[v].C, a.Dws, a.Dw, a.W, a.H, cstr0,
                                     feat + v * cstr0 * px0, s);
            const __nv_bfloat16 *in = feat;
            int cstr = cstr0;
            __nv_bfloat16 *bufs[2] = {(__nv_bfloat16 *)(base + L.act0),
                                      (__nv_bfloat16 *)(base + L.act1)};
            for (int k = 0; k < net->layers; ++k) {
                const bool lastk = k + 1 == net->layers;
                launch_conv3x3_nhwc(in, nviews, net->cin[k], cstr, a.H, a.W,
                                    (const __nv_bfloat16 *)net->wt[k], net->b[k], net->cout[k],
                                    net->relu[k], lastk ? nullptr : bufs[k & 1],
                                    lastk ? (float *)(base + L.q) : nullptr,
                                    counters ? (int *)(counters + 2) : nullptr, s);
                in = bufs[k & 1];
                cstr = net->cout[k];
            }
            if (dbg && dbg->proposal)
                cudaMemcpyAsync(dbg->proposal, (const float *)(base + L.q) + dbg->view * px0,
                                px0 * sizeof(float), cudaMemcpyDeviceToDevice, s);
            if (!(dbg && dbg->level == 0)) continue;
        }
        if (layered) {
            // Section 3.2: layers of two opposite passes over the previous layer's merged
            // energies; volumes B0..B3 per view, layer k writes (B0,B1) for even k and
            // (B2,B3) for odd k, so the last layer's pair is always (B2,B3)
            const int layers = p.num_paths / 2;
            HookScope hs(hook, MPV_STAGE_AGGREGATE, layers, s);
            uint16_t *B[kMaxViews][4];
            for (int v = 0; v < nviews; ++v) {
                B[v][0] = a.v[v].S;
                for (int i = 0; i < 3; ++i) B[v][i + 1] = (uint16_t *)(base + L.X[v][i]);
            }
            for (int k = 0; k < layers; ++k) {
                MergeArgs m{};
                m.in_mode = k == 0 ? 0 : (k == 1 ? 1 : 2);   // min after the horizontal layer
                m.out_mode = 1;
                m.dir0 = 2 * k;
                m.ndirs = 2;
                m.double_up_dir = 0;                       // left to right
                m.lut = grad_lut;
                const int in = (k & 1) ? 0 : 2, out = (k & 1) ? 2 : 0;
                for (int v = 0; v < nviews; ++v) {
                    m.qa[v] = B[v][in];
                    m.qb[v] = B[v][in + 1];
                    m.out[v][0] = B[v][out];
                    m.out[v][1] = B[v][out + 1];
                }
                launch_layer(a, m, s);
            }
            for (int v = 0; v < nviews; ++v) {
                a.v[v].S = B[v][2];
                a.v[v].S2 = B[v][3];
            }
        } else {
            HookScope hs(hook, MPV_STAGE_AGGREGATE, 1, s);
            // S was cleared by the cost kernel
            if (grad_lut) {
                MergeArgs m{};
                m.in_mode = 0;
                m.out_mode = 0;
                m.dir0 = 0;
                m.ndirs = a.npaths;
                m.double_up_dir = -1;
                m.lut = grad_lut;
                launch_aggregate_general(a, m, s);
            } else {
                launch_aggregate(a, s);
            }
        }
        {
            HookScope hs(hook, MPV_STAGE_WTA, a.edge ? 2 : 1, s);
            launch_wta(a, s);
        }
        if (dbg && l == dbg->level) {
            const ViewLevel &vl = a.v[dbg->view];
            const size_t npx = (size_t)a.W * a.H;
            if (dbg->lo) {
                if (vl.lo)
                    cudaMemcpyAsync(dbg->lo, vl.lo, npx * 2, cudaMemcpyDeviceToDevice, s);
                else
                    cudaMemsetAsync(dbg->lo, 0, npx * 2, s);
            }
            if (dbg->cost || dbg->sum) launch_unpack(a, dbg->view, dbg->cost, dbg->sum, s);
            if (dbg->disp) cudaMemcpyAsync(dbg->disp, vl.d, npx * 2, cudaMemcpyDeviceToDevice, s);
        }
    }
    if (!dbg) {
        HookScope hs(hook, MPV_STAGE_LR, 1, s);
        const uint16_t *dL = (const uint16_t *)(base + L.d[0][top]);
        const uint16_t *dRm = nviews == 2 ? (const uint16_t *)(base + L.d[1][top]) : dL;
        launch_lr(dL, dRm, job.W, job.H, p.lr_tol, p.lr_check, job.disp, job.disp_pitch,
                  nviews == 2 ? job.disp_right : nullptr, job.disp_pitch, s, gate);
        if (learned && p.fallback != MPV_FALLBACK_NONE) {
            // the exact method as fallback and judge: decided on the device from the
            // window-edge hits, its launches always enqueued and gated by the decision
            FallbackGate *fg = (FallbackGate *)(base + L.gate);
            const mpv_params q = fallback_params(p);
            const mpv_status v = validate_pair(q, job.W, job.H, job.pitch, job.disp_pitch, job.D);
            if (v != MPV_OK) return v;
            if (aux) {
                const mpv_status r = enqueue_fallback_node(q, job, base, s, aux, tune, grad_lut,
                                                           edge, p.fallback_edge_bp, fg,
                                                           counters);
                if (r != MPV_OK) return r;
            } else {
                launch_fallback_gate(edge, p.fallback_edge_bp, fg, counters, s);
                const mpv_status r = enqueue_pair(q, job, base, s, hook, nullptr, tune, nullptr,
                                                  grad_lut, nullptr, &fg->open);
                if (r != MPV_OK) return r;
            }
        }
    }
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return MPV_OK;
    return e == cudaErrorMemoryAllocation ? MPV_ERR_OOM : MPV_ERR_CUDA;
}

}  // namespace mpv
