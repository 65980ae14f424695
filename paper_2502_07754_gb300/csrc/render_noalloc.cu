// ms_render_noalloc: the forward render with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory: a plugin whose host application owns the
// GPU memory budget and hands out no allocations, or a service that reserves all of its
// device memory at start-up and forbids allocation afterwards.  They cannot provide the
// workspace that ms_render needs, so this entry point uses a file-scope device array
// instead.  Inputs and the output image are still the caller's.
//
// The array is kNoAllocWorkspaceBytes (64 MiB).  Every GPU that loads this library
// holds it until the process exits.  Its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current) on the first call made on that
// device; make that first call before any stream capture begins.  All calls share the
// one array: ms_render clears the part that must start at zero on every call, and two
// calls whose work overlaps on the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {
namespace {

constexpr size_t kNoAllocWorkspaceBytes = 64u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocWorkspaceBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" MS_API ms_status ms_render_noalloc(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans,
                                              int32_t K, const ms_camera *cam, const ms_render_params *params,
                                              float *out_rgba, ms_render_info *info, void *stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(MS_ERR_UNSUPPORTED, "device %d out of range", dev);
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_ws);
            if (e != cudaSuccess || !p)
                return set_error(MS_ERR_CUDA, "cudaGetSymbolAddress of the static workspace: %s",
                                      cudaGetErrorString(e));
            g_noalloc_addr[dev] = p;
        }
        ws = g_noalloc_addr[dev];
    }
    const size_t need = ms_render_workspace_size(n_fans, K, cam, params);
    if (need == 0) return set_error(MS_ERR_INVALID, "invalid render configuration");
    if (need > kNoAllocWorkspaceBytes)
        return set_error(MS_ERR_INVALID,
                              "this render needs a %zu-byte workspace; ms_render_noalloc holds %zu bytes "
                              "(use ms_render with a caller workspace)",
                              need, kNoAllocWorkspaceBytes);
    ms_status s = ms_render(xyz, rgb, alpha, n_fans, K, cam, params, out_rgba, ws, kNoAllocWorkspaceBytes, stream);
    if (s != MS_OK) return s;
    ms_render_info local;
    return ms_render_get_info(ws, info ? info : &local, stream);
}
