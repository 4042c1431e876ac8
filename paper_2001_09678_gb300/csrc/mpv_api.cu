// mpv_api.cu -- C ABI of the matcher: contexts, validation, workspace, launch sequence.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

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

void hook_begin(void *user, int stage, int nkernels, cudaStream_t s)
{
    mpv_ctx *ctx = (mpv_ctx *)user;
    ctx->launches[stage] += nkernels;
    if (!ctx->profiling) return;
    mpv_ctx::Rec r{stage, pool_event(ctx), pool_event(ctx)};
    cudaEventRecord(r.a, s);
    ctx->recs.push_back(r);
}

void hook_end(void *user, int stage, cudaStream_t s)
{
    mpv_ctx *ctx = (mpv_ctx *)user;
    (void)stage;
    if (!ctx->profiling || ctx->recs.empty()) return;
    cudaEventRecord(ctx->recs.back().b, s);
}

// Enqueues one pair with the context's workspace and profiler.
mpv_status enqueue(mpv_ctx *ctx, const PairJob &job, cudaStream_t s, const StageSink *dbg)
{
    Geometry g;
    make_geometry(ctx->p, job.W, job.H, job.D, g);
    const Layout L = make_layout(g, views_needed(ctx->p, job, dbg));
    const mpv_status st = ensure_workspace(ctx, L.total);
    if (st != MPV_OK) return st;
    StageHook hook{hook_begin, hook_end, ctx};
    return enqueue_pair(ctx->p, job, (uint8_t *)ctx->ws, s, &hook, dbg);
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
        PairJob j{q.left, q.right, q.width, q.height, q.pitch,
                  q.max_disparity > 0 ? q.max_disparity : ctx->p.max_disparity,
                  q.disp, q.disp_pitch, q.disp_right};
        const mpv_status st = enqueue(ctx, j, s, nullptr);
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
    make_geometry(ctx->p, width, height, ctx->p.max_disparity, g);
    *bytes = make_layout(g, ctx->p.lr_check ? 2 : 1).total;
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
    StageSink dbg;
    dbg.view = view;
    dbg.level = level;
    dbg.lo = lo;
    dbg.cost = cost;
    dbg.sum = sum;
    dbg.disp = disp;
    PairJob j{left, right, width, height, pitch, ctx->p.max_disparity, nullptr, width, nullptr};
    mpv_status r = enqueue(ctx, j, s, &dbg);
    if (r != MPV_OK) return r;
    return cuda_status(cudaStreamSynchronize(s));
}

mpv_status mpv_level_info(const mpv_ctx *ctx, int32_t width, int32_t height, int32_t level,
                          int32_t *w, int32_t *h, int32_t *range, int32_t *window)
{
    if (!ctx || level < 0 || level >= ctx->p.num_scales || width < 1 || height < 1)
        return MPV_ERR_INVALID_ARG;
    Geometry g;
    make_geometry(ctx->p, width, height, ctx->p.max_disparity, g);
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
