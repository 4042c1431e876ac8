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
#include <mutex>

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
    if (!params_valid(p) || p.proposal != MPV_PROPOSAL_PYRAMID) return MPV_ERR_INVALID_ARG;
    const mpv_status v = validate_pair(p, width, height, pitch, disp_pitch, p.max_disparity);
    if (v != MPV_OK) return v;
    const PairJob job{left, right, width, height, pitch, p.max_disparity, disp, disp_pitch,
                      nullptr};
    Geometry g;
    make_geometry(p, width, height, p.max_disparity, g);
    const Layout L = make_layout(g, views_needed(p, job, nullptr), p);
    if (L.total > (size_t)MPV_NOALLOC_SCRATCH_BYTES) return MPV_ERR_INVALID_ARG;

    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return MPV_ERR_CUDA;
    }
    void *addr = nullptr;
    const mpv_status st = scratch_address(device, &addr);
    if (st != MPV_OK) return st;
    // the pipeline clears what must start at zero (the summed volume of each level)
    return enqueue_pair(p, job, (uint8_t *)addr, (cudaStream_t)cuda_stream, nullptr, nullptr);
}
