// mpv_api.cu -- C ABI of the matcher: contexts, validation, workspace, launch sequence.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mpv.h"
#include "mpv_internal.cuh"

using namespace mpv;

struct mpv_ctx {
    int device = 0;
    mpv_params p{};
    void *ws = nullptr;
    size_t ws_bytes = 0;
    size_t ws_limit = 0;
    int latched = MPV_OK;
    cudaStream_t last_stream = nullptr;
    void *stage = nullptr;       // device staging of mpv_match_host
    size_t stage_bytes = 0;
    // profiler
    bool profiling = false;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t launches[MPV_NUM_STAGES] = {};
};

namespace {

struct Geometry {
    int S;
    int W[kMaxScales], H[kMaxScales], D[kMaxScales], Dw[kMaxScales], block[kMaxScales];
    int pitch[kMaxScales];  // workspace image pitch per level
};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

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

bool params_valid(const mpv_params &p)
{
    if (p.struct_size != sizeof(mpv_params)) return false;
    if (p.ssim_window != 3 && p.ssim_window != 5) return false;
    if (p.num_scales < 1 || p.num_scales > kMaxScales) return false;
    if (p.num_paths != 4 && p.num_paths != 8) return false;
    if (p.max_disparity < 1 || p.max_disparity > 1024) return false;
    if (p.p1 < 0 || p.trunc < 0 || p.window < 0 || p.lr_tol < 0) return false;
    if (p.lr_check != 0 && p.lr_check != 1) return false;
    if (p.merge_mode != MPV_MERGE_SUM) return false;
    if (p.proposal != MPV_PROPOSAL_PYRAMID && p.proposal != MPV_PROPOSAL_LEARNED) return false;
    for (int i = 0; i < 4; ++i)
        if (p.block[i] < 0 || p.block[i] > 8) return false;
    return true;
}

// Level sizes, ranges and windows (Section 3.4): level S-1 is the input, each level
// above halves the size (rounding up) and the range; the top level searches its
// whole range, the others a window of Dw labels (D/4 by default).
bool geometry(const mpv_params &p, int W, int H, int D, Geometry &g)
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
        g.Dw[l] = l == 0 ? g.D[0] : (Dw < g.D[l] ? Dw : g.D[l]);
        const int b = l > 0 ? p.block[l - 1] : 0;
        g.block[l] = b > 0 ? b : (l == g.S - 1 ? 1 : 2);
        g.pitch[l] = (int)ceil_div(g.W[l], 16) * 16;
    }
    return true;
}

mpv_status validate_pair(const mpv_params &p, int W, int H, int pitch, int disp_pitch, int D)
{
    const int N = p.ssim_window;
    if (W < N || H < N) return MPV_ERR_INVALID_ARG;
    if (D < 1 || D > W || D > 1024) return MPV_ERR_INVALID_ARG;
    if (pitch < W || disp_pitch < W) return MPV_ERR_INVALID_ARG;
    Geometry g;
    geometry(p, W, H, D, g);
    if (g.W[0] < N || g.H[0] < N) return MPV_ERR_INVALID_ARG;
    const int64_t jump = (int64_t)p.p1 * (D - 1);
    const int64_t pen = p.trunc < jump ? p.trunc : jump;
    if ((int64_t)p.num_paths * (255 + pen) >= 65535) return MPV_ERR_INVALID_ARG;
    if ((int64_t)W * H > (int64_t)1 << 27) return MPV_ERR_UNSUPPORTED;
    if (p.proposal == MPV_PROPOSAL_LEARNED) return MPV_ERR_UNSUPPORTED;
    return MPV_OK;
}

// Workspace layout of one pair.
struct Layout {
    size_t total = 0;
    size_t img0[kMaxViews][kMaxScales], img1[kMaxViews][kMaxScales];
    size_t lo[kMaxViews][kMaxScales], d[kMaxViews][kMaxScales];
    size_t C[kMaxViews], S[kMaxViews];
};

size_t take(size_t &off, size_t bytes)
{
    const size_t at = off;
    off += (bytes + 255) & ~(size_t)255;
    return at;
}

Layout layout(const Geometry &g, int nviews)
{
    Layout L;
    size_t off = 0;
    int64_t maxvol = 0;
    for (int l = 0; l < g.S; ++l) {
        const int64_t v = (int64_t)g.W[l] * g.H[l] * g.Dw[l];
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
        L.C[v] = take(off, sizeof(uint16_t) * (size_t)maxvol);
        L.S[v] = take(off, sizeof(uint32_t) * (size_t)maxvol);
    }
    L.total = off;
    return L;
}

mpv_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return MPV_OK;
    if (e == cudaErrorMemoryAllocation) return MPV_ERR_OOM;
    return MPV_ERR_CUDA;
}

mpv_status ensure_workspace(mpv_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return MPV_OK;
    if (ctx->ws_limit && bytes > ctx->ws_limit) return MPV_ERR_OOM;
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    ctx->ws = p;
    ctx->ws_bytes = bytes;
    return MPV_OK;
}

struct Job {
    const uint8_t *left, *right;
    int W, H, pitch, D;
    uint16_t *disp;
    int disp_pitch;
    uint16_t *disp_right;
};

// Stage sink for mpv_debug_stage.
struct StageOut {
    int view = -1, level = -1;
    uint16_t *lo = nullptr, *cost = nullptr, *disp = nullptr;
    uint32_t *sum = nullptr;
};

cudaEvent_t pool_event(mpv_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs `launch` (which enqueues `nkernels` kernels on s) under the profiler.
template <class F>
void stage(mpv_ctx *ctx, int which, int nkernels, cudaStream_t s, F &&launch)
{
    ctx->launches[which] += nkernels;
    if (!ctx->profiling) {
        launch();
        return;
    }
    mpv_ctx::Rec r{which, pool_event(ctx), pool_event(ctx)};
    cudaEventRecord(r.a, s);
    launch();
    cudaEventRecord(r.b, s);
    ctx->recs.push_back(r);
}

// Enqueues the whole matcher for one pair on stream s.
mpv_status enqueue_pair(mpv_ctx *ctx, const Job &job, cudaStream_t s, const StageOut *dbg)
{
    const mpv_params &p = ctx->p;
    Geometry g;
    geometry(p, job.W, job.H, job.D, g);
    const bool need_right = p.lr_check || job.disp_right || (dbg && dbg->view == 1);
    const int nviews = need_right ? 2 : 1;
    const Layout L = layout(g, nviews);
    mpv_status st = ensure_workspace(ctx, L.total);
    if (st != MPV_OK) return st;
    uint8_t *base = (uint8_t *)ctx->ws;
    const int S = g.S;
    const int top = S - 1;

    auto img0 = [&](int v, int l) -> uint8_t * { return base + L.img0[v][l]; };
    auto img1 = [&](int v, int l) -> uint8_t * { return base + L.img1[v][l]; };

    const uint8_t *I0[kMaxViews][kMaxScales];
    const uint8_t *I1[kMaxViews][kMaxScales];
    int P0[kMaxViews][kMaxScales], P1[kMaxViews][kMaxScales];
    for (int v = 0; v < nviews; ++v)
        for (int l = 0; l < S; ++l) {
            I0[v][l] = img0(v, l);
            I1[v][l] = img1(v, l);
            P0[v][l] = P1[v][l] = g.pitch[l];
        }
    I0[0][top] = job.left;
    I1[0][top] = job.right;
    P0[0][top] = P1[0][top] = job.pitch;

    // right view: the mirrored, swapped pair
    if (nviews == 2) {
        ImageJob m[2] = {{job.right, job.pitch, img0(1, top), g.pitch[top]},
                         {job.left, job.pitch, img1(1, top), g.pitch[top]}};
        stage(ctx, MPV_STAGE_PYRAMID, 1, s, [&] { launch_mirror(m, 2, job.W, job.H, s); });
    }
    // pyramid
    for (int l = top - 1; l >= 0; --l) {
        ImageJob jobs[4];
        int n = 0;
        for (int v = 0; v < nviews; ++v) {
            jobs[n++] = {I0[v][l + 1], P0[v][l + 1], img0(v, l), g.pitch[l]};
            jobs[n++] = {I1[v][l + 1], P1[v][l + 1], img1(v, l), g.pitch[l]};
        }
        stage(ctx, MPV_STAGE_PYRAMID, 1, s,
              [&] { launch_down2(jobs, n, g.W[l + 1], g.H[l + 1], s); });
    }

    const int Teff = p.trunc >= MPV_NO_TRUNC ? kInf : p.trunc;
    const int P1eff = p.trunc >= MPV_NO_TRUNC ? p.p1 : (p.p1 < p.trunc ? p.p1 : p.trunc);
    const int last = dbg ? dbg->level : top;
    for (int l = 0; l <= last; ++l) {
        LevelArgs a{};
        a.W = g.W[l];
        a.H = g.H[l];
        a.D = g.D[l];
        a.Dw = g.Dw[l];
        a.nviews = nviews;
        a.N = p.ssim_window;
        a.c1 = ssim_c1(a.N);
        a.c2 = ssim_c2(a.N);
        a.p1 = P1eff;
        a.trunc = Teff;
        a.npaths = p.num_paths;
        for (int v = 0; v < nviews; ++v) {
            ViewLevel &vl = a.v[v];
            vl.I0 = I0[v][l];
            vl.I1 = I1[v][l];
            vl.pitch0 = P0[v][l];
            vl.pitch1 = P1[v][l];
            vl.lo = l == 0 ? nullptr : (const uint16_t *)(base + L.lo[v][l]);
            vl.C = (uint16_t *)(base + L.C[v]);
            vl.S = (uint32_t *)(base + L.S[v]);
            vl.d = (uint16_t *)(base + L.d[v][l]);
        }
        if (l > 0) {
            SeedArgs sa{};
            sa.W = g.W[l];
            sa.H = g.H[l];
            sa.Wp = g.W[l - 1];
            sa.Hp = g.H[l - 1];
            sa.block = g.block[l];
            sa.Dw = g.Dw[l];
            sa.D = g.D[l];
            sa.nviews = nviews;
            for (int v = 0; v < nviews; ++v) {
                sa.dprev[v] = (const uint16_t *)(base + L.d[v][l - 1]);
                sa.lo[v] = (uint16_t *)(base + L.lo[v][l]);
            }
            stage(ctx, MPV_STAGE_SEED, 1, s, [&] { launch_seed(sa, s); });
        }
        stage(ctx, MPV_STAGE_COST, 1, s, [&] { launch_cost(a, s); });
        const size_t vol = (size_t)a.W * a.H * a.Dw;
        stage(ctx, MPV_STAGE_AGGREGATE, 1, s, [&] {
            for (int v = 0; v < nviews; ++v)
                cudaMemsetAsync(a.v[v].S, 0, vol * sizeof(uint32_t), s);
            launch_aggregate(a, s);
        });
        stage(ctx, MPV_STAGE_WTA, 1, s, [&] { launch_wta(a, s); });
        if (dbg && l == dbg->level) {
            const ViewLevel &vl = a.v[dbg->view];
            const size_t npx = (size_t)a.W * a.H;
            if (dbg->lo) {
                if (vl.lo)
                    cudaMemcpyAsync(dbg->lo, vl.lo, npx * 2, cudaMemcpyDeviceToDevice, s);
                else
                    cudaMemsetAsync(dbg->lo, 0, npx * 2, s);
            }
            if (dbg->cost) cudaMemcpyAsync(dbg->cost, vl.C, vol * 2, cudaMemcpyDeviceToDevice, s);
            if (dbg->sum) cudaMemcpyAsync(dbg->sum, vl.S, vol * 4, cudaMemcpyDeviceToDevice, s);
            if (dbg->disp) cudaMemcpyAsync(dbg->disp, vl.d, npx * 2, cudaMemcpyDeviceToDevice, s);
        }
    }
    if (!dbg) {
        const uint16_t *dL = (const uint16_t *)(base + L.d[0][top]);
        const uint16_t *dRm = nviews == 2 ? (const uint16_t *)(base + L.d[1][top]) : dL;
        stage(ctx, MPV_STAGE_LR, 1, s, [&] {
            launch_lr(dL, dRm, job.W, job.H, p.lr_tol, p.lr_check, job.disp, job.disp_pitch,
                      nviews == 2 ? job.disp_right : nullptr, job.disp_pitch, s);
        });
    }
    return cuda_status(cudaGetLastError());
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

mpv_status mpv_default_params(mpv_params *p)
{
    if (!p) return MPV_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(mpv_params);
    p->max_disparity = 128;
    p->num_scales = 3;
    p->num_paths = 8;
    p->p1 = 10;
    p->trunc = 30;
    p->ssim_window = 5;
    p->window = 0;
    p->lr_check = 1;
    p->lr_tol = 1;
    p->merge_mode = MPV_MERGE_SUM;
    p->proposal = MPV_PROPOSAL_PYRAMID;
    return MPV_OK;
}

mpv_status mpv_create(int device, mpv_ctx **out)
{
    if (!out) return MPV_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    if (device < 0 || device >= n) return MPV_ERR_INVALID_ARG;
    mpv_ctx *c = new (std::nothrow) mpv_ctx();
    if (!c) return MPV_ERR_OOM;
    c->device = device;
    mpv_default_params(&c->p);
    *out = c;
    return MPV_OK;
}

mpv_status mpv_set_params(mpv_ctx *ctx, const mpv_params *p)
{
    if (!ctx || !p) return MPV_ERR_INVALID_ARG;
    if (!params_valid(*p)) return MPV_ERR_INVALID_ARG;
    ctx->p = *p;
    return MPV_OK;
}

mpv_status mpv_get_params(const mpv_ctx *ctx, mpv_params *p)
{
    if (!ctx || !p) return MPV_ERR_INVALID_ARG;
    *p = ctx->p;
    return MPV_OK;
}

mpv_status mpv_match(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right, int32_t width,
                     int32_t height, int32_t pitch, uint16_t *disp, int32_t disp_pitch,
                     void *cuda_stream)
{
    mpv_pair pr{};
    pr.left = left;
    pr.right = right;
    pr.width = width;
    pr.height = height;
    pr.pitch = pitch;
    pr.max_disparity = 0;
    pr.disp = disp;
    pr.disp_pitch = disp_pitch;
    pr.disp_right = nullptr;
    return mpv_match_batch(ctx, &pr, 1, cuda_stream);
}

mpv_status mpv_match_batch(mpv_ctx *ctx, const mpv_pair *pairs, int32_t n, void *cuda_stream)
{
    if (!ctx || (n > 0 && !pairs) || n < 0) return MPV_ERR_INVALID_ARG;
    if (ctx->latched != MPV_OK) {
        const mpv_status st = (mpv_status)ctx->latched;
        ctx->latched = MPV_OK;
        return st;
    }
    for (int i = 0; i < n; ++i) {
        const mpv_pair &q = pairs[i];
        if (!q.left || !q.right || !q.disp) return MPV_ERR_INVALID_ARG;
        const int D = q.max_disparity > 0 ? q.max_disparity : ctx->p.max_disparity;
        const mpv_status st = validate_pair(ctx->p, q.width, q.height, q.pitch, q.disp_pitch, D);
        if (st != MPV_OK) return st;
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ctx->last_stream = s;
    for (int i = 0; i < n; ++i) {
        const mpv_pair &q = pairs[i];
        Job j{q.left, q.right, q.width, q.height, q.pitch,
              q.max_disparity > 0 ? q.max_disparity : ctx->p.max_disparity,
              q.disp, q.disp_pitch, q.disp_right};
        const mpv_status st = enqueue_pair(ctx, j, s, nullptr);
        if (st != MPV_OK) return st;
    }
    return MPV_OK;
}

mpv_status mpv_match_host(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                          int32_t width, int32_t height, int32_t pitch, uint16_t *disp,
                          int32_t disp_pitch, void *cuda_stream)
{
    if (!ctx || !left || !right || !disp) return MPV_ERR_INVALID_ARG;
    const int D = ctx->p.max_disparity;
    mpv_status st = validate_pair(ctx->p, width, height, pitch, disp_pitch, D);
    if (st != MPV_OK) return st;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // device copies of the pair and of the map live in a context-owned staging buffer
    const size_t img = (size_t)height * width;
    const size_t need = 2 * ((img + 255) & ~(size_t)255) + sizeof(uint16_t) * img;
    if (ctx->stage_bytes < need) {
        if (ctx->stage) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->stage);
        }
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (cudaMalloc(&ctx->stage, need) != cudaSuccess) {
            cudaGetLastError();
            return MPV_ERR_OOM;
        }
        ctx->stage_bytes = need;
    }
    uint8_t *dl = (uint8_t *)ctx->stage;
    uint8_t *dr = dl + ((img + 255) & ~(size_t)255);
    uint16_t *dd = (uint16_t *)(dr + ((img + 255) & ~(size_t)255));
    cudaMemcpy2DAsync(dl, width, left, pitch, width, height, cudaMemcpyHostToDevice, s);
    cudaMemcpy2DAsync(dr, width, right, pitch, width, height, cudaMemcpyHostToDevice, s);
    st = mpv_match(ctx, dl, dr, width, height, width, dd, width, cuda_stream);
    if (st != MPV_OK) return st;
    cudaMemcpy2DAsync(disp, sizeof(uint16_t) * disp_pitch, dd, sizeof(uint16_t) * width,
                      sizeof(uint16_t) * width, height, cudaMemcpyDeviceToHost, s);
    return cuda_status(cudaStreamSynchronize(s));
}

mpv_status mpv_load_proposal_weights(mpv_ctx *ctx, const char *path)
{
    if (!ctx || !path) return MPV_ERR_INVALID_ARG;
    return MPV_ERR_UNSUPPORTED;
}

mpv_status mpv_sync(mpv_ctx *ctx)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    const mpv_status st = (mpv_status)ctx->latched;
    ctx->latched = MPV_OK;
    return st;
}

mpv_status mpv_workspace_bytes(const mpv_ctx *ctx, int32_t width, int32_t height, size_t *bytes)
{
    if (!ctx || !bytes || width < 1 || height < 1) return MPV_ERR_INVALID_ARG;
    Geometry g;
    geometry(ctx->p, width, height, ctx->p.max_disparity, g);
    *bytes = layout(g, ctx->p.lr_check ? 2 : 1).total;
    return MPV_OK;
}

mpv_status mpv_set_workspace_limit(mpv_ctx *ctx, size_t bytes)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    ctx->ws_limit = bytes;
    return MPV_OK;
}

mpv_status mpv_debug_stage(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                           int32_t width, int32_t height, int32_t pitch, int32_t view,
                           int32_t level, uint16_t *lo, uint16_t *cost, uint32_t *sum,
                           uint16_t *disp, void *cuda_stream)
{
    if (!ctx || !left || !right) return MPV_ERR_INVALID_ARG;
    if (view < 0 || view > 1 || level < 0 || level >= ctx->p.num_scales)
        return MPV_ERR_INVALID_ARG;
    const mpv_status st =
        validate_pair(ctx->p, width, height, pitch, width, ctx->p.max_disparity);
    if (st != MPV_OK) return st;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    StageOut dbg;
    dbg.view = view;
    dbg.level = level;
    dbg.lo = lo;
    dbg.cost = cost;
    dbg.sum = sum;
    dbg.disp = disp;
    Job j{left, right, width, height, pitch, ctx->p.max_disparity, nullptr, width, nullptr};
    mpv_status r = enqueue_pair(ctx, j, s, &dbg);
    if (r != MPV_OK) return r;
    return cuda_status(cudaStreamSynchronize(s));
}

mpv_status mpv_level_info(const mpv_ctx *ctx, int32_t width, int32_t height, int32_t level,
                          int32_t *w, int32_t *h, int32_t *range, int32_t *window)
{
    if (!ctx || level < 0 || level >= ctx->p.num_scales || width < 1 || height < 1)
        return MPV_ERR_INVALID_ARG;
    Geometry g;
    geometry(ctx->p, width, height, ctx->p.max_disparity, g);
    if (w) *w = g.W[level];
    if (h) *h = g.H[level];
    if (range) *range = g.D[level];
    if (window) *window = g.Dw[level];
    return MPV_OK;
}

mpv_status mpv_profile_enable(mpv_ctx *ctx, int32_t on)
{
    if (!ctx || (on != 0 && on != 1)) return MPV_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (!on) {
        for (auto &r : ctx->recs) {
            cudaEventSynchronize(r.b);
            ctx->pool.push_back(r.a);
            ctx->pool.push_back(r.b);
        }
        ctx->recs.clear();
    }
    ctx->profiling = on != 0;
    return MPV_OK;
}

mpv_status mpv_profile_read(mpv_ctx *ctx, double *ms, int64_t *launches, int32_t n)
{
    if (!ctx || n < 0) return MPV_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    double tot[MPV_NUM_STAGES] = {};
    mpv_status st = MPV_OK;
    for (auto &r : ctx->recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) st = MPV_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) tot[r.stage] += t;
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    for (int k = 0; k < n && k < MPV_NUM_STAGES; ++k) {
        if (ms) ms[k] = tot[k];
        if (launches) launches[k] = ctx->launches[k];
    }
    for (int k = 0; k < MPV_NUM_STAGES; ++k) ctx->launches[k] = 0;
    cudaGetLastError();
    return st;
}

const char *mpv_status_string(mpv_status s)
{
    switch (s) {
    case MPV_OK: return "ok";
    case MPV_ERR_INVALID_ARG: return "invalid argument";
    case MPV_ERR_UNSUPPORTED: return "unsupported";
    case MPV_ERR_OOM: return "out of device memory";
    case MPV_ERR_CUDA: return "CUDA error";
    case MPV_ERR_TIMEOUT: return "device wait timed out";
    case MPV_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

void mpv_destroy(mpv_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceGuard guard(ctx->device);
        for (auto &r : ctx->recs) {
            cudaEventSynchronize(r.b);
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : ctx->pool) cudaEventDestroy(e);
    }
    if (ctx->ws || ctx->stage) {
        DeviceGuard guard(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->stage) cudaFree(ctx->stage);
    }
    delete ctx;
}

}  // extern "C"
