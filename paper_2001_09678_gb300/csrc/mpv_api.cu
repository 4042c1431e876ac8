// mpv_api.cu -- C ABI of the matcher: contexts, validation, workspace, launch sequence.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
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
    // batches: worker streams, capture stream, fork/join events, per-worker workspaces,
    // instantiated graphs keyed by batch signature, autotuned launch shapes per shape
    std::vector<cudaStream_t> workers;
    cudaStream_t cap = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    void *bws = nullptr;
    size_t bws_bytes = 0;
    struct Graph {
        uint64_t sig;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    std::vector<Graph> singles;   // single pairs (mpv_match), keyed like batches
    // MPV_NO_GRAPHS set in the environment: single pairs launch directly (profilers that
    // replay graph nodes one by one)
    bool single_graphs = std::getenv("MPV_NO_GRAPHS") == nullptr;
    std::map<uint64_t, Tuning> tuning;
    // learned proposal
    ProposalNet net;
    void *net_mem = nullptr;
    // pinned: window-edge hits and pixels of the last learned frame, learned frames and
    // fallbacks since creation, and the network's wait status (copied from counters_dev
    // after every learned frame)
    unsigned long long *edge_host = nullptr;
    // device: learned frames, fallbacks, the network's wait status (non-zero: the wait for
    // the tensor cores ran out)
    unsigned long long *counters_dev = nullptr;
    // gradient-weighted penalty: host copy and device copy of the 256 slopes
    bool grad_on = false;
    int32_t grad_host[256] = {};
    int *grad_dev = nullptr;
    // persistent batches: per signature the uploaded plan (device), its tuned shapes and
    // graph; the status word of the last launch (pinned); the bounded wait in clock cycles
    struct PBatch {
        uint64_t sig;
        void *dev;
        cudaGraphExec_t exec;
        BatchTune tune;
    };
    std::vector<PBatch> pbatches;
    std::map<uint64_t, BatchTune> btuning;
    int *bstatus_host = nullptr;
    long long wait_cycles = 4000000000ll;   // about 2 s at the GPU's clock
    bool stall_next = false;                // test hook (mpv_debug_batch_stall)
    long long stall_wait_cycles = 0;
    bool persistent = std::getenv("MPV_BATCH_STREAMS") == nullptr;
    BatchTune last_batch;                   // the last batch's path and shapes
    int *err_dev = nullptr;                 // bounds-checked builds: the device error word
    int batch_mode = MPV_BATCH_AUTO;
    // road detection: steps back of the profile when they do not fit in shared memory
    void *road_scratch = nullptr;
    size_t road_scratch_bytes = 0;

    const int *lut() const { return grad_on ? grad_dev : nullptr; }
};

namespace mpv {

// The loaded network takes the top level of range D under the context's parameters.
bool proposal_fits(const mpv_ctx *ctx, int D)
{
    const int S = ctx->p.num_scales;
    if (!ctx->net.layers || S < 2) return false;
    const int top = (D + (1 << (S - 1)) - 1) >> (S - 1);
    return ctx->net.cin[0] == 2 + top;
}

}  // namespace mpv

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
        for (auto &g : ctx->singles) cudaGraphExecDestroy(g.exec);   // they use the old one
        ctx->singles.clear();
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


constexpr int kBatchStreams = 16;
constexpr size_t kMaxGraphs = 8;

uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h * 0xFF51AFD7ED558CCDull;
}

uint64_t shape_key(const mpv_params &p, int W, int H, int D)
{
    uint64_t h = mix64(0, (uint64_t)W);
    h = mix64(h, (uint64_t)H);
    h = mix64(h, (uint64_t)D);
    const uint32_t *w = (const uint32_t *)&p;
    for (size_t i = 0; i < sizeof(mpv_params) / 4; ++i) h = mix64(h, w[i]);
    return h;
}

mpv_status ensure_batch_streams(mpv_ctx *ctx)
{
    if (!ctx->workers.empty()) return MPV_OK;
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    for (int i = 0; i < kBatchStreams; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return MPV_ERR_CUDA;
        }
        ctx->workers.push_back(s);
        ctx->joins.push_back(e);
    }
    return MPV_OK;
}

// The gradient table's slopes must not exceed p1 (the energy bounds are derived from p1).
mpv_status check_grad(const mpv_ctx *ctx)
{
    if (!ctx->grad_on) return MPV_OK;
    for (int g = 0; g < 256; ++g)
        if (ctx->grad_host[g] < 0 || ctx->grad_host[g] > ctx->p.p1) return MPV_ERR_INVALID_ARG;
    return MPV_OK;
}

void drop_pbatches(mpv_ctx *ctx)
{
    if (ctx->pbatches.empty()) return;
    cudaDeviceSynchronize();
    for (auto &b : ctx->pbatches) {
        if (b.exec) cudaGraphExecDestroy(b.exec);
        if (b.dev) cudaFree(b.dev);
    }
    ctx->pbatches.clear();
}

void drop_graphs(mpv_ctx *ctx)
{
    drop_pbatches(ctx);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    for (auto &g : ctx->singles) cudaGraphExecDestroy(g.exec);
    ctx->singles.clear();
}

// Autotuner: times the whole matcher on `job` once per candidate launch shape (after a
// warm-up run) on the context's workspace, and keeps the fastest.  Every candidate gives
// the same bit-exact result; only the time differs.
mpv_status autotune(mpv_ctx *ctx, const PairJob &job, Tuning &out)
{
    if (check_grad(ctx) != MPV_OK) return MPV_ERR_INVALID_ARG;
    const uint64_t key = shape_key(ctx->p, job.W, job.H, job.D);
    auto it = ctx->tuning.find(key);
    if (it != ctx->tuning.end()) {
        out = it->second;
        return MPV_OK;
    }
    mpv_status st = ensure_batch_streams(ctx);
    if (st != MPV_OK) return st;
    // earlier calls may still use the context workspace on the caller's stream
    cudaStreamSynchronize(ctx->last_stream);
    Geometry g;
    make_geometry(ctx->p, job.W, job.H, job.D, g);
    st = ensure_workspace(ctx, make_layout(g, views_needed(ctx->p, job, nullptr), ctx->p).total);
    if (st != MPV_OK) return st;
    cudaStream_t s = ctx->workers[0];
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cands[2] = {8, 4};
    float best = 1e30f;
    Tuning bt;
    for (int c : cands) {
        Tuning t;
        t.lanes = c;
        t.err = ctx->err_dev;
        enqueue_pair(ctx->p, job, (uint8_t *)ctx->ws, s, nullptr, nullptr, t, &ctx->net,
                     ctx->lut());
        float tot = 0.f;
        for (int r = 0; r < 2; ++r) {
            cudaEventRecord(e0, s);
            enqueue_pair(ctx->p, job, (uint8_t *)ctx->ws, s, nullptr, nullptr, t, &ctx->net,
                         ctx->lut());
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (tot < best) {
            best = tot;
            bt = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    ctx->tuning[key] = bt;
    out = bt;
    return MPV_OK;
}

mpv_status run_batch_streams(mpv_ctx *ctx, const PairJob *jobs, int n, cudaStream_t stream);

// The batch through one persistent kernel over a device work list (batch.cu): every pair
// gets its own workspace region; the plan is uploaded once per batch signature and its
// launch (state clear, kernel, status copy) captured as a CUDA graph that repeats replay.
// The launch shapes come from the batch autotuner, which times each candidate on the
// batch itself and keeps the fastest (all give the same bit-exact maps).
mpv_status run_batch_persistent(mpv_ctx *ctx, const PairJob *jobs, int n, cudaStream_t stream)
{
    mpv_status st = ensure_batch_streams(ctx);
    if (st != MPV_OK) return st;
    if (!ctx->bstatus_host) {
        if (cudaMallocHost(&ctx->bstatus_host, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return MPV_ERR_OOM;
        }
        *ctx->bstatus_host = 0;
    }
    std::vector<size_t> off(n);
    size_t total = 0;
    uint64_t shapes = 0;
    for (int i = 0; i < n; ++i) {
        off[i] = total;
        total += (batch_pair_bytes(ctx->p, jobs[i]) + 255) & ~(size_t)255;
        shapes = mix64(shapes, shape_key(ctx->p, jobs[i].W, jobs[i].H, jobs[i].D));
    }
    if (total > ctx->bws_bytes) {
        if (ctx->ws_limit && total > ctx->ws_limit) return MPV_ERR_OOM;
        drop_graphs(ctx);
        if (ctx->bws) {
            cudaDeviceSynchronize();
            cudaFree(ctx->bws);
            ctx->bws = nullptr;
            ctx->bws_bytes = 0;
        }
        const cudaError_t e = cudaMalloc(&ctx->bws, total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
        ctx->bws_bytes = total;
    }
    uint64_t sig = mix64(shapes, (uint64_t)(uintptr_t)ctx->bws);
    for (int i = 0; i < n; ++i) {
        const PairJob &j = jobs[i];
        sig = mix64(sig, (uint64_t)(uintptr_t)j.left);
        sig = mix64(sig, (uint64_t)(uintptr_t)j.right);
        sig = mix64(sig, (uint64_t)(uintptr_t)j.disp);
        sig = mix64(sig, (uint64_t)(uintptr_t)j.disp_right);
        sig = mix64(sig, ((uint64_t)j.pitch << 32) | (uint32_t)j.disp_pitch);
    }
    const bool stall = ctx->stall_next;
    ctx->stall_next = false;
    if (!stall)
        for (auto &b : ctx->pbatches)
            if (b.sig == sig && ctx->batch_mode != MPV_BATCH_STREAMS &&
                (b.tune.persistent || ctx->batch_mode == MPV_BATCH_PERSISTENT)) {
                ctx->last_batch = b.tune;
                ctx->last_batch.persistent = true;
                return cuda_status(cudaGraphLaunch(b.exec, stream));
            }

    auto build = [&](const BatchTune &t0, void **dev, BatchDevice &bd) -> mpv_status {
        BatchTune t = t0;
        t.err = ctx->err_dev;
        BatchPlan plan;
        mpv_status r = plan_batch(ctx->p, jobs, n, (uint8_t *)ctx->bws, off.data(), t, plan);
        if (r != MPV_OK) return r;
        const cudaError_t e = cudaMalloc(dev, batch_device_bytes(plan));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
        r = upload_batch(plan, *dev, bd);
        bd.occupancy = t.occupancy;
        return r;
    };

    // the launch shapes: tuned once per set of pair shapes
    BatchTune tune;
    auto tit = ctx->btuning.find(shapes);
    if (tit != ctx->btuning.end()) {
        tune = tit->second;
    } else {
        cudaStreamSynchronize(stream);
        cudaStream_t s = ctx->workers[0];
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        // times one candidate; false when the batch failed (status in r)
        auto trial = [&](const BatchTune &t, mpv_status &r) {
            void *dev = nullptr;
            BatchDevice bd;
            r = build(t, &dev, bd);
            float ms = 1e30f;
            if (r == MPV_OK) {
                r = launch_batch(bd, ctx->wait_cycles, ctx->bstatus_host, s);   // warm
                cudaEventRecord(e0, s);
                if (r == MPV_OK) r = launch_batch(bd, ctx->wait_cycles, ctx->bstatus_host, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                if (r == MPV_OK && *ctx->bstatus_host == MPV_OK) cudaEventElapsedTime(&ms, e0, e1);
            }
            if (dev) cudaFree(dev);
            if (r == MPV_OK && ms < best) {
                best = ms;
                tune = t;
            }
            return r == MPV_OK;
        };
        mpv_status tr = MPV_OK;
        bool ok = true;
        for (int lanes : {8, 4})
            for (int queues : {16, 32})
                for (int cb : {2, 8}) {
                    BatchTune t;
                    t.lanes = lanes;
                    t.queues = queues;
                    t.cost_blocks = cb;
                    if (ok) ok = trial(t, tr);
                }
        // then the register budget, with the best shapes
        for (int occ : {3, 4}) {
            BatchTune t = tune;
            t.occupancy = occ;
            if (ok) ok = trial(t, tr);
        }
        if (!ok) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return tr;
        }
        // the same batch as a graph of per-pair launch sequences over worker streams
        float streams_ms = 1e30f;
        {
            mpv_status r = run_batch_streams(ctx, jobs, n, s);   // captures its graph
            cudaEventRecord(e0, s);
            if (r == MPV_OK) r = run_batch_streams(ctx, jobs, n, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            if (r == MPV_OK) cudaEventElapsedTime(&streams_ms, e0, e1);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *ctx->bstatus_host = 0;
        tune.persistent = best <= streams_ms;
        tune.ms = best;
        tune.streams_ms = streams_ms;
        ctx->btuning[shapes] = tune;
    }
    ctx->last_batch = tune;
    ctx->last_batch.persistent = ctx->batch_mode == MPV_BATCH_PERSISTENT ||
                                 (ctx->batch_mode == MPV_BATCH_AUTO && tune.persistent) || stall;
    if (!ctx->last_batch.persistent) return run_batch_streams(ctx, jobs, n, stream);
    BatchTune t = tune;
    t.stall = stall;
    void *dev = nullptr;
    BatchDevice bd;
    st = build(t, &dev, bd);
    if (st != MPV_OK) {
        if (dev) cudaFree(dev);
        return st;
    }
    if (stall) {   // a one-off launch with the test hook: not cached
        const mpv_status r = launch_batch(bd, ctx->stall_wait_cycles, ctx->bstatus_host, stream);
        cudaStreamSynchronize(stream);
        cudaFree(dev);
        return r;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dev);
        return MPV_ERR_CUDA;
    }
    const mpv_status lr = launch_batch(bd, ctx->wait_cycles, ctx->bstatus_host, ctx->cap);
    e = cudaStreamEndCapture(ctx->cap, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && lr == MPV_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || lr != MPV_OK) {
        cudaGetLastError();
        cudaFree(dev);
        return lr != MPV_OK ? lr : MPV_ERR_CUDA;
    }
    if (ctx->pbatches.size() >= 4) {   // keep a few signatures
        cudaDeviceSynchronize();
        cudaGraphExecDestroy(ctx->pbatches.front().exec);
        cudaFree(ctx->pbatches.front().dev);
        ctx->pbatches.erase(ctx->pbatches.begin());
    }
    ctx->pbatches.push_back({sig, dev, exec, tune});
    return cuda_status(cudaGraphLaunch(exec, stream));
}

// Runs a batch as one CUDA graph: pair i runs on worker stream w(i) (largest pairs
// first, round robin), pairs sharing a worker run one after another and share that
// worker's workspace region, and the workers run concurrently.  The instantiated graph
// is cached by the batch signature and replayed by a single graph launch.
mpv_status run_batch_streams(mpv_ctx *ctx, const PairJob *jobs, int n, cudaStream_t stream)
{
    if (check_grad(ctx) != MPV_OK) return MPV_ERR_INVALID_ARG;
    mpv_status st = ensure_batch_streams(ctx);
    if (st != MPV_OK) return st;
    std::vector<Tuning> tune(n);
    for (int i = 0; i < n; ++i) {
        st = autotune(ctx, jobs[i], tune[i]);
        if (st != MPV_OK) return st;
        tune[i].err = ctx->err_dev;
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)jobs[a].W * jobs[a].H * jobs[a].D > (int64_t)jobs[b].W * jobs[b].H * jobs[b].D;
    });
    const int nw = std::min(n, kBatchStreams);
    std::vector<int> worker(n);
    std::vector<size_t> wbytes(nw, 0), woff(nw, 0);
    for (int r = 0; r < n; ++r) {
        const int i = order[r];
        worker[i] = r % nw;
        Geometry g;
        make_geometry(ctx->p, jobs[i].W, jobs[i].H, jobs[i].D, g);
        const size_t b = make_layout(g, views_needed(ctx->p, jobs[i], nullptr), ctx->p).total;
        wbytes[worker[i]] = std::max(wbytes[worker[i]], b);
    }
    size_t total = 0;
    for (int w = 0; w < nw; ++w) {
        woff[w] = total;
        total += (wbytes[w] + 255) & ~(size_t)255;
    }
    if (total > ctx->bws_bytes) {
        if (ctx->ws_limit && total > ctx->ws_limit) return MPV_ERR_OOM;
        drop_graphs(ctx);
        if (ctx->bws) {
            cudaDeviceSynchronize();
            cudaFree(ctx->bws);
            ctx->bws = nullptr;
            ctx->bws_bytes = 0;
        }
        const cudaError_t e = cudaMalloc(&ctx->bws, total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
        ctx->bws_bytes = total;
    }
    uint64_t sig = mix64(shape_key(ctx->p, n, nw, 0), (uint64_t)(uintptr_t)ctx->bws);
    sig = mix64(sig, (uint64_t)(uintptr_t)ctx->lut());
    for (int i = 0; i < n; ++i) {
        const PairJob &j = jobs[i];
        sig = mix64(sig, (uint64_t)(uintptr_t)j.left);
        sig = mix64(sig, (uint64_t)(uintptr_t)j.right);
        sig = mix64(sig, (uint64_t)(uintptr_t)j.disp);
        sig = mix64(sig, (uint64_t)(uintptr_t)j.disp_right);
        sig = mix64(sig, ((uint64_t)j.W << 32) | (uint32_t)j.H);
        sig = mix64(sig, ((uint64_t)j.pitch << 32) | (uint32_t)j.disp_pitch);
        sig = mix64(sig, ((uint64_t)j.D << 32) | (uint32_t)tune[i].lanes);
    }
    for (size_t k = 0; k < ctx->graphs.size(); ++k)
        if (ctx->graphs[k].sig == sig) {
            const cudaError_t e = cudaGraphLaunch(ctx->graphs[k].exec, stream);
            return cuda_status(e);
        }

    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    cudaEventRecord(ctx->fork, ctx->cap);
    for (int w = 0; w < nw; ++w) cudaStreamWaitEvent(ctx->workers[w], ctx->fork, 0);
    mpv_status est = MPV_OK;
    for (int r = 0; r < n && est == MPV_OK; ++r) {
        const int i = order[r];
        const int w = worker[i];
        est = enqueue_pair(ctx->p, jobs[i], (uint8_t *)ctx->bws + woff[w], ctx->workers[w],
                           nullptr, nullptr, tune[i], &ctx->net, ctx->lut(), ctx->counters_dev);
    }
    for (int w = 0; w < nw; ++w) {
        cudaEventRecord(ctx->joins[w], ctx->workers[w]);
        cudaStreamWaitEvent(ctx->cap, ctx->joins[w], 0);
    }
    e = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != cudaSuccess || est != MPV_OK) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return est != MPV_OK ? est : MPV_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    if (ctx->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(ctx->graphs.front().exec);
        ctx->graphs.erase(ctx->graphs.begin());
    }
    ctx->graphs.push_back({sig, exec});
    return cuda_status(cudaGraphLaunch(exec, stream));
}

// Enqueues one pair with the context's workspace and profiler.
// The launches of one pair on stream s with the context's workspace (and, for the
// learned proposal, the copy of the window-edge counters to pinned host memory).
mpv_status enqueue_direct(mpv_ctx *ctx, const PairJob &job, cudaStream_t s, const StageSink *dbg,
                          const Tuning &t, const Layout &L, cudaStream_t aux = nullptr)
{
    StageHook hook{hook_begin, hook_end, ctx};
    mpv_status r = enqueue_pair(ctx->p, job, (uint8_t *)ctx->ws, s, &hook, dbg, t, &ctx->net,
                                ctx->lut(), ctx->counters_dev, nullptr, aux);
    if (r == MPV_OK && ctx->p.proposal == MPV_PROPOSAL_LEARNED && !dbg) {
        // with a fallback the workspace's counters may be reused by the fallback's
        // launches: the decision keeps its own copy
        const uint8_t *src = (const uint8_t *)ctx->ws + L.edge;
        if (ctx->p.fallback != MPV_FALLBACK_NONE)
            src = (const uint8_t *)ctx->ws + L.gate + offsetof(FallbackGate, hits);
        cudaMemcpyAsync(ctx->edge_host, src, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(ctx->edge_host + 2, ctx->counters_dev, 3 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s);
        r = cuda_status(cudaGetLastError());
    }
    return r;
}

// Enqueues one pair with the context's workspace and profiler.  Without profiling or a
// stage dump, the launches are captured once per signature (shape, parameters, buffers,
// tuning, tables) into a CUDA graph on the context's capture stream and replayed on s.
mpv_status enqueue(mpv_ctx *ctx, const PairJob &job, cudaStream_t s, const StageSink *dbg)
{
    if (check_grad(ctx) != MPV_OK) return MPV_ERR_INVALID_ARG;
    Geometry g;
    make_geometry(ctx->p, job.W, job.H, job.D, g);
    const Layout L = make_layout(g, views_needed(ctx->p, job, dbg), ctx->p);
    mpv_status st = ensure_workspace(ctx, L.total);
    if (st != MPV_OK) return st;
    Tuning t;
    const auto it = ctx->tuning.find(shape_key(ctx->p, job.W, job.H, job.D));
    if (it != ctx->tuning.end()) t = it->second;
    t.err = ctx->err_dev;
    const bool learned = ctx->p.proposal == MPV_PROPOSAL_LEARNED;
    if (learned && !ctx->net.layers) return MPV_ERR_INVALID_ARG;    // no weights loaded
    if (learned && !dbg && !ctx->edge_host) {
        if (cudaMallocHost(&ctx->edge_host, 5 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return MPV_ERR_OOM;
        }
        for (int i = 0; i < 5; ++i) ctx->edge_host[i] = 0;
        if (cudaMalloc(&ctx->counters_dev, 3 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemset(ctx->counters_dev, 0, 3 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(ctx->edge_host);
            ctx->edge_host = nullptr;
            if (ctx->counters_dev) cudaFree(ctx->counters_dev);
            ctx->counters_dev = nullptr;
            return MPV_ERR_OOM;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (dbg || ctx->profiling || !ctx->single_graphs ||
        cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return enqueue_direct(ctx, job, s, dbg, t, L);
    }
    st = ensure_batch_streams(ctx);
    if (st != MPV_OK) return st;
    uint64_t sig = mix64(shape_key(ctx->p, job.W, job.H, job.D), (uint64_t)(uintptr_t)ctx->ws);
    sig = mix64(sig, (uint64_t)(uintptr_t)job.left);
    sig = mix64(sig, (uint64_t)(uintptr_t)job.right);
    sig = mix64(sig, (uint64_t)(uintptr_t)job.disp);
    sig = mix64(sig, (uint64_t)(uintptr_t)job.disp_right);
    sig = mix64(sig, ((uint64_t)job.pitch << 32) | (uint32_t)job.disp_pitch);
    sig = mix64(sig, (uint64_t)t.lanes);
    sig = mix64(sig, (uint64_t)(uintptr_t)ctx->lut());
    sig = mix64(sig, (uint64_t)(uintptr_t)ctx->net_mem);
    sig = mix64(sig, (uint64_t)(uintptr_t)ctx->edge_host);
    for (const auto &gr : ctx->singles)
        if (gr.sig == sig) return cuda_status(cudaGraphLaunch(gr.exec, s));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return enqueue_direct(ctx, job, s, dbg, t, L);
    }
    // (a learned-proposal fallback becomes a conditional node, its body captured on the
    // first worker stream)
    const mpv_status est = enqueue_direct(ctx, job, ctx->cap, nullptr, t, L, ctx->workers[0]);
    e = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != cudaSuccess || est != MPV_OK) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return est != MPV_OK ? est : MPV_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    if (ctx->singles.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(ctx->singles.front().exec);
        ctx->singles.erase(ctx->singles.begin());
    }
    ctx->singles.push_back({sig, exec});
    return cuda_status(cudaGraphLaunch(exec, s));
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

// A batch: through the persistent kernel where it applies and the autotuner found it
// faster than the graph of worker streams, else through that graph.
mpv_status run_batch(mpv_ctx *ctx, const PairJob *jobs, int n, cudaStream_t stream)
{
    if (check_grad(ctx) != MPV_OK) return MPV_ERR_INVALID_ARG;
    if (ctx->persistent && !ctx->grad_on && ctx->batch_mode != MPV_BATCH_STREAMS) {
        bool ok = true;
        for (int i = 0; i < n && ok; ++i)
            ok = batch_supported(ctx->p, jobs[i].W, jobs[i].H, jobs[i].D);
        if (ok) return run_batch_persistent(ctx, jobs, n, stream);
    }
    ctx->last_batch = BatchTune();
    ctx->last_batch.persistent = false;
    return run_batch_streams(ctx, jobs, n, stream);
}

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
    p->top_block = 0;
    p->fallback = MPV_FALLBACK_PYRAMID;
    p->fallback_edge_bp = 1500;
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
#ifdef MPV_DEBUG_BOUNDS
    {
        DeviceGuard guard(device);
        if (cudaMalloc(&c->err_dev, sizeof(int)) != cudaSuccess ||
            cudaMemset(c->err_dev, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return MPV_ERR_OOM;
        }
    }
#endif
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
    std::vector<PairJob> jobs(n);
    for (int i = 0; i < n; ++i) {
        const mpv_pair &q = pairs[i];
        jobs[i] = PairJob{q.left, q.right, q.width, q.height, q.pitch,
                          q.max_disparity > 0 ? q.max_disparity : ctx->p.max_disparity,
                          q.disp, q.disp_pitch, q.disp_right};
    }
    if (n == 1) return enqueue(ctx, jobs[0], s, nullptr);
    if (n == 0) return MPV_OK;
    return run_batch(ctx, jobs.data(), n, s);
}

mpv_status mpv_autotune(mpv_ctx *ctx, const mpv_pair *pair, int32_t *lanes)
{
    if (!ctx || !pair || !pair->left || !pair->right || !pair->disp) return MPV_ERR_INVALID_ARG;
    const int D = pair->max_disparity > 0 ? pair->max_disparity : ctx->p.max_disparity;
    const mpv_status v = validate_pair(ctx->p, pair->width, pair->height, pair->pitch,
                                       pair->disp_pitch, D);
    if (v != MPV_OK) return v;
    DeviceGuard guard(ctx->device);
    const PairJob job{pair->left, pair->right, pair->width, pair->height, pair->pitch, D,
                      pair->disp, pair->disp_pitch, pair->disp_right};
    Tuning t;
    const mpv_status st = autotune(ctx, job, t);
    if (st == MPV_OK && lanes) *lanes = t.lanes;
    return st;
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
    FILE *f = std::fopen(path, "rb");
    if (!f) return MPV_ERR_INVALID_ARG;
    std::vector<unsigned char> data;
    unsigned char buf[65536];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) data.insert(data.end(), buf, buf + got);
    std::fclose(f);
    auto rd = [&](size_t off) -> int32_t {
        int32_t v;
        std::memcpy(&v, data.data() + off, 4);
        return v;
    };
    if (data.size() < 20 || std::memcmp(data.data(), "MPVP", 4) != 0 || rd(4) != 1 ||
        rd(8) != kProposalLayers)
        return MPV_ERR_INVALID_ARG;
    ProposalNet net;
    net.layers = kProposalLayers;
    net.train_D = rd(12);
    net.factor = rd(16);
    size_t off = 20, nw = 0, nb = 0;
    for (int k = 0; k < kProposalLayers; ++k, off += 12) {
        if (off + 12 > data.size()) return MPV_ERR_INVALID_ARG;
        net.cin[k] = rd(off);
        net.cout[k] = rd(off + 4);
        net.relu[k] = rd(off + 8);
        const bool lastk = k == kProposalLayers - 1;
        if (net.cin[k] < 1 || net.cin[k] > 1024 || net.cout[k] != (lastk ? 1 : 32) ||
            !conv3x3_tc_ok(net.cin[k], net.cout[k]) ||
            net.relu[k] != (lastk ? 0 : 1) || (k > 0 && net.cin[k] != net.cout[k - 1]))
            return MPV_ERR_INVALID_ARG;
        nw += (size_t)net.cout[k] * net.cin[k] * 9;
        nb += (size_t)net.cout[k];
    }
    if (off + 4 * (nw + nb) != data.size()) return MPV_ERR_INVALID_ARG;
    // device layout: all BF16 weights, then all FP32 biases (256-byte aligned)
    const size_t wbytes = ((nw * sizeof(__nv_bfloat16)) + 255) & ~(size_t)255;
    std::vector<__nv_bfloat16> hw(nw);
    std::vector<float> hb(nb);
    size_t iw = 0, ib = 0;
    for (int k = 0; k < kProposalLayers; ++k) {
        const size_t n = (size_t)net.cout[k] * net.cin[k] * 9;
        for (size_t i = 0; i < n; ++i, off += 4) {
            float v;
            std::memcpy(&v, data.data() + off, 4);
            hw[iw + i] = __float2bfloat16(v);
        }
        std::memcpy(hb.data() + ib, data.data() + off, 4 * (size_t)net.cout[k]);
        off += 4 * (size_t)net.cout[k];
        iw += n;
        ib += net.cout[k];
    }
    // the same weights in the tensor-core kernel's layout [9][planes][width][8] (zero
    // padded input and output channels), copied whole by the matcher's network
    std::vector<__nv_bfloat16> ht;
    size_t toff[kProposalLayers];
    {
        size_t iw2 = 0;
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        for (int k = 0; k < kProposalLayers; ++k) {
            const int Cin = net.cin[k], Cout = net.cout[k];
            const int planes = tc_planes(Cin), width = tc_width(Cout);
            toff[k] = ht.size();
            ht.resize(ht.size() + tc_weight_elems(Cin, Cout), zero);
            for (int co = 0; co < Cout; ++co)
                for (int c = 0; c < Cin; ++c)
                    for (int tap = 0; tap < 9; ++tap)
                        ht[toff[k] + ((size_t)(tap * planes + c / 8) * width + co) * 8 + c % 8] =
                            hw[iw2 + ((size_t)co * Cin + c) * 9 + tap];
            iw2 += (size_t)Cout * Cin * 9;
        }
    }
    const size_t bbytes = ((nb * sizeof(float)) + 255) & ~(size_t)255;
    DeviceGuard guard(ctx->device);
    void *mem = nullptr;
    if (cudaMalloc(&mem, wbytes + bbytes + ht.size() * sizeof(__nv_bfloat16)) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_OOM;
    }
    cudaMemcpy(mem, hw.data(), nw * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
    cudaMemcpy((uint8_t *)mem + wbytes, hb.data(), nb * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy((uint8_t *)mem + wbytes + bbytes, ht.data(), ht.size() * sizeof(__nv_bfloat16),
               cudaMemcpyHostToDevice);
    iw = ib = 0;
    for (int k = 0; k < kProposalLayers; ++k) {
        net.w[k] = (const __nv_bfloat16 *)mem + iw;
        net.b[k] = (const float *)((uint8_t *)mem + wbytes) + ib;
        net.wt[k] = (const __nv_bfloat16 *)((uint8_t *)mem + wbytes + bbytes) + toff[k];
        iw += (size_t)net.cout[k] * net.cin[k] * 9;
        ib += net.cout[k];
    }
    if (ctx->net_mem) {
        cudaDeviceSynchronize();
        cudaFree(ctx->net_mem);
    }
    drop_graphs(ctx);
    ctx->net_mem = mem;
    ctx->net = net;
    return cuda_status(cudaGetLastError());
}

mpv_status mpv_proposal_features(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                 int32_t width, int32_t height, int32_t pitch, int32_t view,
                                 void *out, void *cuda_stream)
{
    if (!ctx || !left || !right || !out || view < 0 || view > 1) return MPV_ERR_INVALID_ARG;
    mpv_params p = ctx->p;
    p.proposal = MPV_PROPOSAL_PYRAMID;
    const mpv_status v = validate_pair(p, width, height, pitch, width, p.max_disparity);
    if (v != MPV_OK) return v;
    DeviceGuard guard(ctx->device);
    Geometry g;
    make_geometry(p, width, height, p.max_disparity, g);
    const mpv_status st = ensure_workspace(ctx, make_layout(g, view == 1 ? 2 : 1, p).total);
    if (st != MPV_OK) return st;
    const PairJob job{left, right, width, height, pitch, p.max_disparity, nullptr, width, nullptr};
    return enqueue_features(p, job, (uint8_t *)ctx->ws, (cudaStream_t)cuda_stream, view,
                            (__nv_bfloat16 *)out);
}

mpv_status mpv_set_gradient_penalty(mpv_ctx *ctx, const int32_t *slopes)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    if (!slopes) {
        ctx->grad_on = false;   // cached batch graphs are keyed by the table pointer
        return MPV_OK;
    }
    for (int g = 0; g < 256; ++g)
        if (slopes[g] < 0) return MPV_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (!ctx->grad_dev) {
        const cudaError_t e = cudaMalloc(&ctx->grad_dev, 256 * sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->grad_dev = nullptr;
            return cuda_status(e);
        }
    }
    // earlier matches may still read the table on the caller's stream
    cudaStreamSynchronize(ctx->last_stream);
    const cudaError_t e =
        cudaMemcpy(ctx->grad_dev, slopes, 256 * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
    for (int g = 0; g < 256; ++g) ctx->grad_host[g] = slopes[g];
    ctx->grad_on = true;
    return MPV_OK;
}

mpv_status mpv_road_detect(mpv_ctx *ctx, const uint16_t *disp, int32_t width, int32_t height,
                           int32_t disp_pitch, int32_t max_disparity, int32_t eta,
                           uint32_t *vdisp, uint32_t *udisp, int32_t *profile, int64_t *energy,
                           void *cuda_stream)
{
    if (!ctx || !disp || !vdisp || !profile || !energy || width < 1 || height < 1 ||
        height > kRoadMaxRows || disp_pitch < width || max_disparity < 1 ||
        max_disparity > 1024 || eta < 2 || eta > 256)
        return MPV_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint8_t *scratch = nullptr;
    if (!road_back_in_smem(height, max_disparity)) {
        const size_t need = road_scratch_bytes(height, max_disparity);
        if (ctx->road_scratch_bytes < need) {
            if (ctx->road_scratch) {
                cudaDeviceSynchronize();
                cudaFree(ctx->road_scratch);
            }
            ctx->road_scratch = nullptr;
            ctx->road_scratch_bytes = 0;
            const cudaError_t e = cudaMalloc(&ctx->road_scratch, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return cuda_status(e);
            }
            ctx->road_scratch_bytes = need;
        }
        scratch = (uint8_t *)ctx->road_scratch;
    }
    launch_road(disp, width, height, disp_pitch, max_disparity, eta, vdisp, udisp, profile,
                energy, scratch, s);
    return cuda_status(cudaGetLastError());
}

mpv_status mpv_proposal_stats(const mpv_ctx *ctx, uint64_t *edge_hits, uint64_t *pixels)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    if (edge_hits) *edge_hits = ctx->edge_host ? ctx->edge_host[0] : 0;
    if (pixels) *pixels = ctx->edge_host ? ctx->edge_host[1] : 0;
    return MPV_OK;
}

mpv_status mpv_proposal_fallbacks(const mpv_ctx *ctx, uint64_t *frames, uint64_t *fallbacks)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    if (frames) *frames = ctx->edge_host ? ctx->edge_host[2] : 0;
    if (fallbacks) *fallbacks = ctx->edge_host ? ctx->edge_host[3] : 0;
    return MPV_OK;
}

mpv_status mpv_sync(mpv_ctx *ctx)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    if (ctx->err_dev) {   // bounds-checked builds: a device index check failed
        int site = 0;
        cudaMemcpy(&site, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
        if (site) {
            std::fprintf(stderr, "mpv: device bounds check failed at site %d\n", site);
            cudaMemset(ctx->err_dev, 0, sizeof(int));
            ctx->latched = MPV_ERR_INTERNAL;
        }
    }
    if (ctx->bstatus_host && *ctx->bstatus_host != MPV_OK) {   // a persistent batch's wait ran out
        ctx->latched = *ctx->bstatus_host;
        *ctx->bstatus_host = MPV_OK;
    }
    if (ctx->edge_host && ctx->edge_host[4] != 0) {   // the proposal network's wait ran out
        ctx->latched = MPV_ERR_TIMEOUT;
        ctx->edge_host[4] = 0;
        cudaMemset(ctx->counters_dev + 2, 0, sizeof(unsigned long long));
    }
    const mpv_status st = (mpv_status)ctx->latched;
    ctx->latched = MPV_OK;
    return st;
}

mpv_status mpv_set_batch_mode(mpv_ctx *ctx, int32_t mode)
{
    if (!ctx || mode < MPV_BATCH_AUTO || mode > MPV_BATCH_STREAMS) return MPV_ERR_INVALID_ARG;
    ctx->batch_mode = mode;
    return MPV_OK;
}

mpv_status mpv_debug_batch_stall(mpv_ctx *ctx, int64_t wait_cycles)
{
    if (!ctx || wait_cycles < 1) return MPV_ERR_INVALID_ARG;
    ctx->stall_next = true;
    ctx->stall_wait_cycles = wait_cycles;
    return MPV_OK;
}

mpv_status mpv_batch_info(const mpv_ctx *ctx, int32_t *persistent, int32_t *lanes,
                          int32_t *queues, int32_t *cost_blocks, float *persistent_ms,
                          float *streams_ms, int32_t *occupancy)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    const BatchTune &t = ctx->last_batch;
    if (persistent) *persistent = t.persistent ? 1 : 0;
    if (lanes) *lanes = t.lanes;
    if (queues) *queues = t.queues;
    if (occupancy) *occupancy = t.occupancy;
    if (cost_blocks) *cost_blocks = t.cost_blocks;
    if (persistent_ms) *persistent_ms = t.ms;
    if (streams_ms) *streams_ms = t.streams_ms;
    return MPV_OK;
}

mpv_status mpv_workspace_bytes(const mpv_ctx *ctx, int32_t width, int32_t height, size_t *bytes)
{
    if (!ctx || !bytes || width < 1 || height < 1) return MPV_ERR_INVALID_ARG;
    Geometry g;
    make_geometry(ctx->p, width, height, ctx->p.max_disparity, g);
    *bytes = make_layout(g, ctx->p.lr_check ? 2 : 1, ctx->p).total;
    return MPV_OK;
}

mpv_status mpv_set_workspace_limit(mpv_ctx *ctx, size_t bytes)
{
    if (!ctx) return MPV_ERR_INVALID_ARG;
    ctx->ws_limit = bytes;
    return MPV_OK;
}

mpv_status mpv_proposal_predict(mpv_ctx *ctx, const uint8_t *left, const uint8_t *right,
                                int32_t width, int32_t height, int32_t pitch, int32_t view,
                                float *out, void *cuda_stream)
{
    if (!ctx || !left || !right || !out || view < 0 || view > 1) return MPV_ERR_INVALID_ARG;
    if (ctx->p.proposal != MPV_PROPOSAL_LEARNED) return MPV_ERR_INVALID_ARG;
    const mpv_status st =
        validate_pair(ctx->p, width, height, pitch, width, ctx->p.max_disparity);
    if (st != MPV_OK) return st;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    StageSink dbg;
    dbg.view = view;
    dbg.level = 0;
    dbg.proposal = out;
    PairJob j{left, right, width, height, pitch, ctx->p.max_disparity, nullptr, width, nullptr};
    return enqueue(ctx, j, s, &dbg);
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
        drop_graphs(ctx);
        for (auto s : ctx->workers) cudaStreamDestroy(s);
        for (auto e : ctx->joins) cudaEventDestroy(e);
        if (ctx->cap) cudaStreamDestroy(ctx->cap);
        if (ctx->fork) cudaEventDestroy(ctx->fork);
        if (ctx->bws) {
            cudaDeviceSynchronize();
            cudaFree(ctx->bws);
        }
        if (ctx->net_mem) cudaFree(ctx->net_mem);
        if (ctx->grad_dev) cudaFree(ctx->grad_dev);
        if (ctx->road_scratch) cudaFree(ctx->road_scratch);
        drop_pbatches(ctx);
        if (ctx->err_dev) cudaFree(ctx->err_dev);
        if (ctx->bstatus_host) cudaFreeHost(ctx->bstatus_host);
        if (ctx->edge_host) cudaFreeHost(ctx->edge_host);
        if (ctx->counters_dev) cudaFree(ctx->counters_dev);
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
