// server.cu -- continuous-batching request loop for several camera streams.
//
// Each camera owns resident device state: a matcher context (its workspace keeps the
// pyramid levels and volumes of that frame size allocated between frames), device
// copies of the pair and of the map, pinned host staging and a CUDA stream.  Frames wait
// in a per-camera FIFO.  poll() retires finished frames and admits waiting frames while
// in-flight slots and the device-memory budget allow; an admitted frame's copies and
// kernels are enqueued on its camera's stream at once, so frames of different cameras
// overlap on the GPU while later frames keep arriving.  A camera's resident memory is
// charged to the budget when its first frame is admitted; idle cameras are evicted
// least-recently-used first when a new camera needs room.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mpv_internal.cuh"

namespace {

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id;
    int camera;
    const uint8_t *left, *right;
    int pitch;
    uint16_t *disp;
    int disp_pitch;
    double t_submit, t_start;
    std::atomic<double> t_done{0.0};
    std::atomic<int> done{0};
    mpv_status status = MPV_OK;
};

struct Camera {
    int id, W, H, D;
    mpv_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    uint8_t *dev = nullptr;          // left, right, disp
    uint8_t *pinned = nullptr;       // left, right, disp staging
    size_t resident = 0;             // bytes charged to the budget
    std::deque<Request *> queue;
    Request *inflight = nullptr;
    double last_use = 0.0;
};

void CUDART_CB stamp_done(void *p)
{
    Request *r = (Request *)p;
    r->t_done.store(now_ms());
    r->done.store(1);
}

}  // namespace

struct mpv_server {
    int device = 0;
    mpv_params params{};
    size_t budget = 0, used = 0;
    int max_inflight = 1, inflight = 0;
    std::map<int, Camera> cams;
    std::deque<mpv_completion> completed;
    uint64_t admitted = 0, evictions = 0;
    int peak_inflight = 0;
    std::string proposal;            // weights of the learned proposal ("" = pyramid only)
};

namespace {

size_t frame_bytes(int W, int H) { return (size_t)W * H * 2 + (size_t)W * H * 2; }

void release(Camera &c)
{
    if (c.ctx) mpv_destroy(c.ctx);
    if (c.dev) cudaFree(c.dev);
    if (c.pinned) cudaFreeHost(c.pinned);
    if (c.stream) cudaStreamDestroy(c.stream);
    c.ctx = nullptr;
    c.dev = nullptr;
    c.pinned = nullptr;
    c.stream = nullptr;
    c.resident = 0;
}

// Makes the camera's state resident, within the budget; false if it cannot yet.
bool make_resident(mpv_server *s, Camera &c, mpv_status &err)
{
    if (c.ctx) return true;
    size_t ws = 0;
    mpv_ctx *ctx = nullptr;
    if ((err = mpv_create(s->device, &ctx)) != MPV_OK) return false;
    mpv_params p = s->params;
    p.max_disparity = c.D;
    if ((err = mpv_set_params(ctx, &p)) != MPV_OK) {
        mpv_destroy(ctx);
        return false;
    }
    if (!s->proposal.empty()) {
        // the learned proposal where the network fits the camera's range, else the pyramid
        mpv_params q = p;
        q.proposal = MPV_PROPOSAL_LEARNED;
        if (mpv_set_params(ctx, &q) != MPV_OK ||
            mpv_load_proposal_weights(ctx, s->proposal.c_str()) != MPV_OK ||
            !mpv::proposal_fits(ctx, c.D))
            mpv_set_params(ctx, &p);
    }
    if ((err = mpv_workspace_bytes(ctx, c.W, c.H, &ws)) != MPV_OK) {
        mpv_destroy(ctx);
        return false;
    }
    const size_t need = ws + frame_bytes(c.W, c.H);
    while (s->budget && s->used + need > s->budget) {
        // evict the least recently used idle camera
        Camera *victim = nullptr;
        for (auto &kv : s->cams) {
            Camera &o = kv.second;
            if (o.ctx && !o.inflight && o.queue.empty() && (!victim || o.last_use < victim->last_use))
                victim = &o;
        }
        if (!victim) {
            mpv_destroy(ctx);
            // nothing left to evict: wait for in-flight frames, unless none can free memory
            bool busy = false;
            for (auto &kv : s->cams) busy = busy || kv.second.inflight != nullptr;
            err = busy ? MPV_OK : MPV_ERR_OOM;
            return false;
        }
        s->used -= victim->resident;
        release(*victim);
        ++s->evictions;
    }
    c.ctx = ctx;
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&c.dev, frame_bytes(c.W, c.H)) != cudaSuccess ||
        cudaMallocHost(&c.pinned, frame_bytes(c.W, c.H)) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        err = MPV_ERR_OOM;
        return false;
    }
    c.resident = need;
    s->used += need;
    return true;
}

void admit(mpv_server *s, Camera &c, Request *r)
{
    const size_t img = (size_t)c.W * c.H;
    uint8_t *hl = c.pinned, *hr = c.pinned + img;
    uint16_t *hd = (uint16_t *)(c.pinned + 2 * img);
    uint8_t *dl = c.dev, *dr = c.dev + img;
    uint16_t *dd = (uint16_t *)(c.dev + 2 * img);
    for (int y = 0; y < c.H; ++y) {
        std::memcpy(hl + (size_t)y * c.W, r->left + (size_t)y * r->pitch, c.W);
        std::memcpy(hr + (size_t)y * c.W, r->right + (size_t)y * r->pitch, c.W);
    }
    r->t_start = now_ms();
    cudaMemcpyAsync(dl, hl, img, cudaMemcpyHostToDevice, c.stream);
    cudaMemcpyAsync(dr, hr, img, cudaMemcpyHostToDevice, c.stream);
    r->status = mpv_match(c.ctx, dl, dr, c.W, c.H, c.W, dd, c.W, c.stream);
    cudaMemcpyAsync(hd, dd, img * sizeof(uint16_t), cudaMemcpyDeviceToHost, c.stream);
    if (cudaLaunchHostFunc(c.stream, stamp_done, r) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(c.stream);
        stamp_done(r);
        if (r->status == MPV_OK) r->status = MPV_ERR_CUDA;
    }
    c.inflight = r;
    c.last_use = r->t_start;
    ++s->inflight;
    ++s->admitted;
    if (s->inflight > s->peak_inflight) s->peak_inflight = s->inflight;
}

void retire(mpv_server *s, Camera &c)
{
    Request *r = c.inflight;
    const size_t img = (size_t)c.W * c.H;
    const uint16_t *hd = (const uint16_t *)(c.pinned + 2 * img);
    for (int y = 0; y < c.H; ++y)
        std::memcpy(r->disp + (size_t)y * r->disp_pitch, hd + (size_t)y * c.W, c.W * sizeof(uint16_t));
    mpv_completion out{};
    out.request_id = r->id;
    out.camera = r->camera;
    out.status = r->status;
    out.t_submit_ms = r->t_submit;
    out.t_start_ms = r->t_start;
    out.t_done_ms = r->t_done.load();
    s->completed.push_back(out);
    c.inflight = nullptr;
    c.last_use = now_ms();
    --s->inflight;
    delete r;
}

}  // namespace

extern "C" {

mpv_status mpv_server_create(int device, const mpv_params *p, size_t hbm_budget,
                             int32_t max_inflight, mpv_server **out)
{
    if (!out || !p || max_inflight < 1) return MPV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mpv::params_valid(*p) || p->proposal != MPV_PROPOSAL_PYRAMID) return MPV_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return MPV_ERR_INVALID_ARG;
    }
    mpv_server *s = new (std::nothrow) mpv_server();
    if (!s) return MPV_ERR_OOM;
    s->device = device;
    s->params = *p;
    s->budget = hbm_budget;
    s->max_inflight = max_inflight;
    *out = s;
    return MPV_OK;
}

mpv_status mpv_server_set_proposal(mpv_server *s, const char *weights_path)
{
    if (!s) return MPV_ERR_INVALID_ARG;
    s->proposal = weights_path ? weights_path : "";
    return MPV_OK;
}

mpv_status mpv_server_add_camera(mpv_server *s, int32_t camera, int32_t width, int32_t height,
                                 int32_t max_disparity)
{
    if (!s || s->cams.count(camera)) return MPV_ERR_INVALID_ARG;
    mpv_params p = s->params;
    p.max_disparity = max_disparity;
    if (!mpv::params_valid(p)) return MPV_ERR_INVALID_ARG;
    const mpv_status v = mpv::validate_pair(p, width, height, width, width, max_disparity);
    if (v != MPV_OK) return v;
    Camera c;
    c.id = camera;
    c.W = width;
    c.H = height;
    c.D = max_disparity;
    s->cams.emplace(camera, std::move(c));
    return MPV_OK;
}

mpv_status mpv_server_submit(mpv_server *s, int32_t camera, const uint8_t *left,
                             const uint8_t *right, int32_t pitch, uint16_t *disp,
                             int32_t disp_pitch, uint64_t request_id)
{
    if (!s || !left || !right || !disp) return MPV_ERR_INVALID_ARG;
    auto it = s->cams.find(camera);
    if (it == s->cams.end()) return MPV_ERR_INVALID_ARG;
    Camera &c = it->second;
    if (pitch < c.W || disp_pitch < c.W) return MPV_ERR_INVALID_ARG;
    Request *r = new (std::nothrow) Request();
    if (!r) return MPV_ERR_OOM;
    r->id = request_id;
    r->camera = camera;
    r->left = left;
    r->right = right;
    r->pitch = pitch;
    r->disp = disp;
    r->disp_pitch = disp_pitch;
    r->t_submit = now_ms();
    c.queue.push_back(r);
    return MPV_OK;
}

mpv_status mpv_server_poll(mpv_server *s, mpv_completion *out, int32_t max, int32_t *n)
{
    if (!s || (max > 0 && !out) || max < 0) return MPV_ERR_INVALID_ARG;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    mpv_status err = MPV_OK;
    // retire
    for (auto &kv : s->cams) {
        Camera &c = kv.second;
        if (c.inflight && c.inflight->done.load()) retire(s, c);
    }
    // admit: oldest waiting frame first, while slots and memory allow; a camera that
    // must wait for memory does not hold back the others
    while (s->inflight < s->max_inflight) {
        std::vector<Camera *> cand;
        for (auto &kv : s->cams) {
            Camera &c = kv.second;
            if (!c.inflight && !c.queue.empty()) cand.push_back(&c);
        }
        std::sort(cand.begin(), cand.end(), [](const Camera *a, const Camera *b) {
            return a->queue.front()->t_submit < b->queue.front()->t_submit;
        });
        bool progressed = false;
        for (Camera *c : cand) {
            if (make_resident(s, *c, err)) {
                Request *r = c->queue.front();
                c->queue.pop_front();
                admit(s, *c, r);
                progressed = true;
                break;
            }
            if (err == MPV_ERR_OOM) {
                // this camera can never fit the budget: its frame fails
                Request *r = c->queue.front();
                c->queue.pop_front();
                mpv_completion o{};
                o.request_id = r->id;
                o.camera = r->camera;
                o.status = MPV_ERR_OOM;
                o.t_submit_ms = o.t_start_ms = o.t_done_ms = r->t_submit;
                s->completed.push_back(o);
                delete r;
                err = MPV_OK;
                progressed = true;
                break;
            }
        }
        if (!progressed) break;
    }
    int k = 0;
    while (k < max && !s->completed.empty()) {
        out[k++] = s->completed.front();
        s->completed.pop_front();
    }
    if (n) *n = k;
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
    return err;
}

mpv_status mpv_server_stats(const mpv_server *s, int32_t *inflight, int32_t *waiting,
                            size_t *resident_bytes, uint64_t *evictions, int32_t *peak_inflight)
{
    if (!s) return MPV_ERR_INVALID_ARG;
    int w = 0;
    for (const auto &kv : s->cams) w += (int)kv.second.queue.size();
    if (inflight) *inflight = s->inflight;
    if (waiting) *waiting = w;
    if (resident_bytes) *resident_bytes = s->used;
    if (evictions) *evictions = s->evictions;
    if (peak_inflight) *peak_inflight = s->peak_inflight;
    return MPV_OK;
}

void mpv_server_destroy(mpv_server *s)
{
    if (!s) return;
    for (auto &kv : s->cams) {
        Camera &c = kv.second;
        if (c.stream) cudaStreamSynchronize(c.stream);
        if (c.inflight) delete c.inflight;
        for (Request *r : c.queue) delete r;
        release(c);
    }
    delete s;
}

}  // extern "C"
