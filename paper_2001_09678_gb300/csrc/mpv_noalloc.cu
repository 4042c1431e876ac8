// mpv_noalloc.cu -- the matcher for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running where the allocator is owned by
// someone else (a host framework with a fixed memory pool, a real-time loop that must
// not allocate after start-up, a plug-in loaded into a process whose device memory is
// budgeted).  mpv_match_noalloc serves them: it runs the same kernels as mpv_match, but
// every scratch buffer (pyramid levels, window starts, cost and summed volumes, WTA
// maps) is carved out of one file-scope __device__ array of fixed size that the CUDA
// runtime places when the library is loaded on a device; the call itself allocates
// nothing.  The array stays resident on every device that loads the library until the
// process exits.
#include <cstring>
#include <mutex>

#include "../../include/mpv.h"
#include "mpv_internal.cuh"

namespace mpv {
namespace {

// The scratch array.  In host code `g_scratch` is only a host-side stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[MPV_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
mpv_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return MPV_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MPV_ERR_CUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return MPV_OK;
}

struct Geo {
    int S, W[kMaxScales], H[kMaxScales], D[kMaxScales], Dw[kMaxScales], block[kMaxScales];
    int pitch[kMaxScales];
};

// Pyramid geometry (Section 3.4): the input is the finest level, each coarser level
// halves size and range, the top level searches its whole range and the others a
// window of Dw labels.
void geo_of(const mpv_params &p, int W, int H, Geo &g)
{
    g.S = p.num_scales;
    int w = W, h = H;
    for (int l = g.S - 1; l >= 0; --l) {
        g.W[l] = w;
        g.H[l] = h;
        const int sh = g.S - 1 - l;
        g.D[l] = (p.max_disparity + (1 << sh) - 1) >> sh;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    int Dw = p.window > 0 ? p.window : p.max_disparity / 4;
    if (Dw < 1) Dw = 1;
    for (int l = 0; l < g.S; ++l) {
        g.Dw[l] = l == 0 ? g.D[0] : (Dw < g.D[l] ? Dw : g.D[l]);
        const int b = l > 0 ? p.block[l - 1] : 0;
        g.block[l] = b > 0 ? b : (l == g.S - 1 ? 1 : 2);
        g.pitch[l] = (g.W[l] + 15) / 16 * 16;
    }
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    }
};

struct Plan {
    size_t img0[kMaxViews][kMaxScales], img1[kMaxViews][kMaxScales];
    size_t lo[kMaxViews][kMaxScales], d[kMaxViews][kMaxScales];
    size_t C[kMaxViews], S[kMaxViews];
    size_t total;
};

Plan plan_of(const Geo &g, int nviews)
{
    Plan P{};
    Carve c;
    size_t maxvol = 0;
    for (int l = 0; l < g.S; ++l) {
        const size_t v = (size_t)g.W[l] * g.H[l] * g.Dw[l];
        if (v > maxvol) maxvol = v;
    }
    for (int v = 0; v < nviews; ++v) {
        for (int l = 0; l < g.S; ++l) {
            const size_t img = (size_t)g.pitch[l] * g.H[l];
            const bool caller = (v == 0 && l == g.S - 1);
            P.img0[v][l] = caller ? 0 : c.take(img);
            P.img1[v][l] = caller ? 0 : c.take(img);
            P.lo[v][l] = c.take(sizeof(uint16_t) * (size_t)g.W[l] * g.H[l]);
            P.d[v][l] = c.take(sizeof(uint16_t) * (size_t)g.W[l] * g.H[l]);
        }
        P.C[v] = c.take(sizeof(uint16_t) * maxvol);
        P.S[v] = c.take(sizeof(uint32_t) * maxvol);
    }
    P.total = c.off;
    return P;
}

bool params_ok(const mpv_params &p, int W, int H, int pitch, int disp_pitch)
{
    if (p.struct_size != sizeof(mpv_params)) return false;
    if (p.ssim_window != 3 && p.ssim_window != 5) return false;
    if (p.num_scales < 1 || p.num_scales > kMaxScales) return false;
    if (p.num_paths != 4 && p.num_paths != 8) return false;
    if (p.p1 < 0 || p.trunc < 0 || p.window < 0 || p.lr_tol < 0) return false;
    if (p.lr_check != 0 && p.lr_check != 1) return false;
    if (p.merge_mode != MPV_MERGE_SUM || p.proposal != MPV_PROPOSAL_PYRAMID) return false;
    for (int i = 0; i < 4; ++i)
        if (p.block[i] < 0 || p.block[i] > 8) return false;
    const int N = p.ssim_window, D = p.max_disparity;
    if (W < N || H < N || D < 1 || D > W || D > 1024) return false;
    if (pitch < W || disp_pitch < W) return false;
    Geo g;
    geo_of(p, W, H, g);
    if (g.W[0] < N || g.H[0] < N) return false;
    const int64_t jump = (int64_t)p.p1 * (D - 1);
    const int64_t pen = p.trunc < jump ? p.trunc : jump;
    return (int64_t)p.num_paths * (255 + pen) < 65535;
}

}  // namespace
}  // namespace mpv

using namespace mpv;

extern "C" mpv_status mpv_match_noalloc(const mpv_params *params, const uint8_t *left,
                                        const uint8_t *right, int32_t width, int32_t height,
                                        int32_t pitch, uint16_t *disp, int32_t disp_pitch,
                                        void *cuda_stream)
{
    if (!params || !left || !right || !disp) return MPV_ERR_INVALID_ARG;
    const mpv_params &p = *params;
    if (!params_ok(p, width, height, pitch, disp_pitch)) return MPV_ERR_INVALID_ARG;
    Geo g;
    geo_of(p, width, height, g);
    const int nviews = p.lr_check ? 2 : 1;
    const Plan P = plan_of(g, nviews);
    if (P.total > (size_t)MPV_NOALLOC_SCRATCH_BYTES) return MPV_ERR_INVALID_ARG;

    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    void *addr = nullptr;
    const mpv_status st = scratch_address(device, &addr);
    if (st != MPV_OK) return st;
    uint8_t *base = (uint8_t *)addr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int top = g.S - 1;

    const uint8_t *I0[kMaxViews][kMaxScales];
    const uint8_t *I1[kMaxViews][kMaxScales];
    int P0[kMaxViews][kMaxScales], Pp[kMaxViews][kMaxScales];
    for (int v = 0; v < nviews; ++v)
        for (int l = 0; l < g.S; ++l) {
            I0[v][l] = base + P.img0[v][l];
            I1[v][l] = base + P.img1[v][l];
            P0[v][l] = Pp[v][l] = g.pitch[l];
        }
    I0[0][top] = left;
    I1[0][top] = right;
    P0[0][top] = Pp[0][top] = pitch;
    if (nviews == 2) {
        ImageJob m[2] = {{right, pitch, base + P.img0[1][top], g.pitch[top]},
                         {left, pitch, base + P.img1[1][top], g.pitch[top]}};
        launch_mirror(m, 2, width, height, s);
    }
    for (int l = top - 1; l >= 0; --l) {
        ImageJob jobs[4];
        int n = 0;
        for (int v = 0; v < nviews; ++v) {
            jobs[n++] = {I0[v][l + 1], P0[v][l + 1], base + P.img0[v][l], g.pitch[l]};
            jobs[n++] = {I1[v][l + 1], Pp[v][l + 1], base + P.img1[v][l], g.pitch[l]};
        }
        launch_down2(jobs, n, g.W[l + 1], g.H[l + 1], s);
    }
    const int Teff = p.trunc >= MPV_NO_TRUNC ? kInf : p.trunc;
    const int P1eff = p.trunc >= MPV_NO_TRUNC ? p.p1 : (p.p1 < p.trunc ? p.p1 : p.trunc);
    const int64_t n = (int64_t)p.ssim_window * p.ssim_window;
    for (int l = 0; l < g.S; ++l) {
        LevelArgs a{};
        a.W = g.W[l];
        a.H = g.H[l];
        a.D = g.D[l];
        a.Dw = g.Dw[l];
        a.nviews = nviews;
        a.N = p.ssim_window;
        a.c1 = (int)((65025 * n * n + 5000) / 10000);
        a.c2 = (int)((585225 * n * n + 5000) / 10000);
        a.p1 = P1eff;
        a.trunc = Teff;
        a.npaths = p.num_paths;
        for (int v = 0; v < nviews; ++v) {
            ViewLevel &vl = a.v[v];
            vl.I0 = I0[v][l];
            vl.I1 = I1[v][l];
            vl.pitch0 = P0[v][l];
            vl.pitch1 = Pp[v][l];
            vl.lo = l == 0 ? nullptr : (const uint16_t *)(base + P.lo[v][l]);
            vl.C = (uint16_t *)(base + P.C[v]);
            vl.S = (uint32_t *)(base + P.S[v]);
            vl.d = (uint16_t *)(base + P.d[v][l]);
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
                sa.dprev[v] = (const uint16_t *)(base + P.d[v][l - 1]);
                sa.lo[v] = (uint16_t *)(base + P.lo[v][l]);
            }
            launch_seed(sa, s);
        }
        launch_cost(a, s);
        // the array keeps the previous call's contents: the summed volume must start at 0
        const size_t vol = (size_t)a.W * a.H * a.Dw;
        for (int v = 0; v < nviews; ++v) cudaMemsetAsync(a.v[v].S, 0, vol * sizeof(uint32_t), s);
        launch_aggregate(a, s);
        launch_wta(a, s);
    }
    const uint16_t *dL = (const uint16_t *)(base + P.d[0][top]);
    const uint16_t *dRm = nviews == 2 ? (const uint16_t *)(base + P.d[1][top]) : dL;
    launch_lr(dL, dRm, width, height, p.lr_tol, p.lr_check, disp, disp_pitch, nullptr,
              disp_pitch, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPV_OK : MPV_ERR_CUDA;
}
