// ms_batch_autotune: picks the tile edge, the per-pixel pending buffer and the two list
// capacities (tile-pair list, fragment-record list) of the batch render by measurement.
//
// Host code only.  Every candidate goes through the public batch entry points, so what
// is timed is exactly what a caller runs.
#include <algorithm>
#include <string.h>
#include <vector>

#include "ms_common.cuh"
#include "ms_internal.h"

using namespace ms;

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int64_t with_headroom(int64_t n, float headroom, int64_t floor_) {
    const double v = (double)n * (1.0 + (double)headroom);
    return std::max<int64_t>((int64_t)v + 1, floor_);
}

}  // namespace

extern "C" MS_API ms_status ms_batch_autotune(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans,
                                              int32_t K, const ms_camera *cams, int32_t n_views,
                                              const ms_render_params *base, float *const *out_rgba,
                                              const float *const *dL_drgba, float *d_xyz, float *d_rgb,
                                              float *d_alpha, void *workspace, size_t ws_bytes, int32_t reps,
                                              float headroom, ms_render_params *best, ms_tune_result *res,
                                              void *stream) {
    if (!best || !res) return set_error(MS_ERR_INVALID, "best / res is NULL");
    if (reps < 1 || !(headroom >= 0.0f)) return set_error(MS_ERR_INVALID, "reps < 1 or headroom < 0");
    cudaStream_t st = (cudaStream_t)stream;
    memset(res, 0, sizeof(*res));
    res->best = -1;
    ms_render_params b0;
    if (base) {
        b0 = *base;
    } else {
        ms_render_params_default(&b0);
    }
    const int64_t V = n_fans * (int64_t)(K + 1);
    EventPair ev;
    cudaError_t e = cudaEventCreate(&ev.a);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "event create: %s", cudaGetErrorString(e));

    for (int c = 0; c < MS_TUNE_CANDIDATES; ++c) {
        ms_render_params p = b0;
        p.tile = 8 << (c / 2);
        p.kbuf = 8 << (c % 2);
        res->cand_ms[c] = -1.0f;
        // measure the two list lengths; grow the capacities until a render fits
        bool settled = false;
        for (int attempt = 0; attempt < 4 && !settled; ++attempt) {
            const size_t need = ms_batch_workspace_size(n_fans, K, cams, n_views, &p);
            res->cand_ws_bytes[c] = need;
            if (need == 0) return set_error(MS_ERR_INVALID, "invalid render configuration");
            if (need > ws_bytes) break;
            ms_status s = ms_batch_render(xyz, rgb, alpha, n_fans, K, cams, n_views, &p, out_rgba, workspace,
                                          ws_bytes, stream);
            if (s != MS_OK) return s;
            ms_render_info info;
            s = ms_render_get_info(workspace, &info, stream);
            if (s == MS_OK) {
                p.pair_capacity = with_headroom(info.pairs, headroom, 4096);
                p.frag_capacity = with_headroom(info.frags, headroom, 65536);
                settled = true;
            } else if (s == MS_ERR_CAPACITY) {
                if (info.pairs > info.pair_capacity) p.pair_capacity = with_headroom(info.pairs, 0.25f, 4096);
                if (info.frags > info.frag_capacity) p.frag_capacity = with_headroom(info.frags, 0.25f, 65536);
            } else {
                return s;
            }
        }
        if (!settled) {
            res->cand_ms[c] = res->cand_ws_bytes[c] > ws_bytes ? -2.0f : -3.0f;
            continue;
        }
        const size_t need = ms_batch_workspace_size(n_fans, K, cams, n_views, &p);
        res->cand_ws_bytes[c] = need;
        if (need > ws_bytes) {
            res->cand_ms[c] = -2.0f;
            continue;
        }
        // one warm step, then `reps` timed forward+backward steps
        std::vector<float> t;
        for (int r = -1; r < reps; ++r) {
            if (V > 0) {
                cudaMemsetAsync(d_xyz, 0, 12 * (size_t)V, st);
                cudaMemsetAsync(d_rgb, 0, 12 * (size_t)V, st);
                cudaMemsetAsync(d_alpha, 0, 4 * (size_t)V, st);
            }
            if ((e = cudaEventRecord(ev.a, st)) != cudaSuccess)
                return set_error(MS_ERR_CUDA, "event record: %s", cudaGetErrorString(e));
            ms_status s = ms_batch_render(xyz, rgb, alpha, n_fans, K, cams, n_views, &p, out_rgba, workspace,
                                          ws_bytes, stream);
            if (s == MS_OK)
                s = ms_batch_render_backward(xyz, rgb, alpha, n_fans, K, cams, n_views, &p, out_rgba, dL_drgba,
                                             d_xyz, d_rgb, d_alpha, workspace, ws_bytes, stream);
            if (s != MS_OK) return s;
            if ((e = cudaEventRecord(ev.b, st)) != cudaSuccess)
                return set_error(MS_ERR_CUDA, "event record: %s", cudaGetErrorString(e));
            if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess)
                return set_error(MS_ERR_CUDA, "event sync: %s", cudaGetErrorString(e));
            float ms_ = 0.0f;
            cudaEventElapsedTime(&ms_, ev.a, ev.b);
            if (r >= 0) t.push_back(ms_);
        }
        ms_render_info info;
        const ms_status s = ms_render_get_info(workspace, &info, stream);
        if (s == MS_ERR_CAPACITY) {   // lists grew past the headroom between runs (cannot for a fixed scene)
            res->cand_ms[c] = -3.0f;
            continue;
        }
        if (s != MS_OK) return s;
        std::sort(t.begin(), t.end());
        res->cand_ms[c] = t[t.size() / 2];
        if (res->best < 0 || res->cand_ms[c] < res->best_ms) {
            res->best = c;
            res->best_ms = res->cand_ms[c];
            res->pairs = info.pairs;
            res->frags = info.frags;
            *best = p;
        }
    }
    if (res->best < 0) return set_error(MS_ERR_CAPACITY, "no autotune candidate fits the %zu-byte workspace", ws_bytes);
    return MS_OK;
}
