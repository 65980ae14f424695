// C ABI entry points (include/meshsplats.h): argument checks, workspace layout and
// the launch sequence of each call.  Nothing here allocates device memory.
#include <math.h>
#include <stdarg.h>

#include <algorithm>
#include <atomic>
#include <vector>
#include <stdio.h>
#include <string.h>

#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

static thread_local char g_err[512] = "";

static ms_status fail(ms_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

ms_status set_error(ms_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

static ms_status cuda_fail(cudaError_t e, const char *what) {
    return fail(MS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ launch accounting
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches += n; }

// ------------------------------------------------------------------ stage profiler
struct EvPair {
    int stage;
    cudaEvent_t a, b;
};
static bool g_prof = false;
static std::vector<EvPair> g_ev;
static size_t g_ev_used = 0;

StageScope::StageScope(int s, cudaStream_t st_) : stage(s), st(st_), slot(-1) {
    if (!g_prof) return;
    if (g_ev_used == g_ev.size()) {
        EvPair p;
        p.stage = s;
        if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return;
        g_ev.push_back(p);
    }
    slot = (int)g_ev_used++;
    g_ev[slot].stage = s;
    cudaEventRecord(g_ev[slot].a, st);
}
StageScope::~StageScope() {
    if (slot >= 0) cudaEventRecord(g_ev[slot].b, st);
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int bits_for(int64_t n) {   // bits to hold values 0..n-1 (at least 1)
    int b = 1;
    while (b < 62 && (1ll << b) < n) ++b;
    return b;
}

static void params_or_default(const ms_render_params *p, ms_render_params &out) {
    if (p) {
        out = *p;
    } else {
        ms_render_params_default(&out);
    }
    // depth_bits 0: chosen by render_layout
    if (out.T_eps <= 0.0f) out.T_eps = 1e-5f;
}

RenderLayout render_layout(int64_t n_fans, int K, const ms_camera *cams, int n_views, const ms_render_params &p) {
    RenderLayout L;
    memset(&L, 0, sizeof(L));
    L.tile = p.tile;
    L.kbuf = p.kbuf;
    L.n_views = n_views;
    int64_t tiles = 0, npx = 0;
    for (int v = 0; v < n_views; ++v) {
        L.tiles_x[v] = (cams[v].width + p.tile - 1) / p.tile;
        const int ty = (cams[v].height + p.tile - 1) / p.tile;
        L.tile_base[v] = (int)tiles;
        L.pix_base[v] = npx;
        tiles += (int64_t)L.tiles_x[v] * ty;
        npx += (int64_t)cams[v].width * cams[v].height;
    }
    L.n_tiles = (int)tiles;
    L.npx = npx;
    L.tile_bits = bits_for(L.n_tiles);
    // A sort element is one 64-bit word: tile | quantised depth bound | fan id, the fan id in
    // the low fan_bits bits; the radix passes sort the tile and depth bits above them.
    // Automatic depth bits: at least 12 over the view's depth range, and as many more as fill
    // the sort key's last byte, within the word.
    L.fan_bits = bits_for(n_fans);
    L.depth_bits = p.depth_bits ? p.depth_bits
                                : std::min(std::min(31, 8 * ((L.tile_bits + 12 + 7) / 8) - L.tile_bits),
                                           64 - L.fan_bits - L.tile_bits);
    L.key_bits = L.tile_bits + L.depth_bits;
    L.passes = (L.key_bits + 7) / 8;
    L.n_fans = n_fans;
    L.V = n_fans * (K + 1);
    int64_t cap = p.pair_capacity;
    if (cap <= 0) {
        cap = 8 * n_fans * n_views;
        if (cap < 65536) cap = 65536;
        const int64_t most = n_fans * (int64_t)L.n_tiles;
        if (cap > most) cap = most > 0 ? most : 1;
    }
    L.cap = cap;
    int64_t fcap = p.frag_capacity;
    if (fcap <= 0) fcap = 8 * npx + 65536;
    L.frag_cap = fcap;
    L.bin_fan_blocks = (n_fans + 255) / 256;
    L.bin_blocks = L.bin_fan_blocks * n_views;
    L.sort_blocks = (cap + sort_tile_elems() - 1) / sort_tile_elems();
    L.scan_blocks = ((int64_t)L.n_tiles * L.tile * L.tile + 2047) / 2048;   // pixel slots in tile order
    L.max_items = L.n_tiles + (cap + kItemFans - 1) / kItemFans;
    L.tscan_blocks = ((int64_t)L.n_tiles + 2047) / 2048;
    size_t o = 0;
    L.off_status = o;            o = align_up(o + 256, 256);
    L.off_bin_state = o;         o = align_up(o + 8 * (size_t)L.bin_blocks, 256);
    L.off_hist = o;              o = align_up(o + 8 * 256 * 4, 256);
    L.off_lookback = o;          o = align_up(o + (size_t)L.passes * L.sort_blocks * 256 * 4, 256);
    L.off_ranges = o;            o = align_up(o + 8 * (size_t)L.n_tiles, 256);
    L.off_scan_state = o;        o = align_up(o + 8 * (size_t)L.scan_blocks, 256);
    L.off_tscan_state = o;       o = align_up(o + 8 * (size_t)L.tscan_blocks, 256);
    L.off_pbucket = o;           o = align_up(o + 2 * 256 * 4, 256);   // pixel-count histogram, fill cursors
    L.off_zrange = o;            o = align_up(o + 8 * (size_t)n_views, 256);   // per view: ~bits(zlo), bits(zhi)
    L.off_mask_cursor = o;       o = align_up(o + 4 * (size_t)kMaskRegions, 256);
    L.off_keys0 = o;             o = align_up(o + 8 * (size_t)cap, 256);   // (zeroed prefix ends here)
    L.off_keys1 = o;             o = align_up(o + 8 * (size_t)cap, 256);
    L.off_tile_nitems = o;       o = align_up(o + 4 * (size_t)L.n_tiles, 256);
    L.off_tile_ibase = o;        o = align_up(o + 4 * (size_t)L.n_tiles, 256);
    L.off_items = o;             o = align_up(o + 16 * (size_t)L.max_items, 256);
    L.off_icnt = o;              o = align_up(o + 4 * (size_t)L.max_items * p.tile * p.tile, 256);
    // coverage masks of the count pass (2 bytes per (pixel, fan) test) and each pair's first
    // mask, so that the fill pass reads its coverage instead of testing it again; tests
    // beyond the capacity fall back to testing
    L.mask_cap = std::min<int64_t>(16 * npx + 65536, 0xfffffffell);
    L.off_maskoff = o;           o = align_up(o + 8 * (size_t)cap, 256);   // per pair: mask index, rectangle
    L.off_masks = o;             o = align_up(o + 2 * (size_t)L.mask_cap, 256);
    L.off_counts = o;            o = align_up(o + 4 * (size_t)npx, 256);
    L.off_offsets = o;           o = align_up(o + 4 * (size_t)npx, 256);
    L.off_perm = o;              o = align_up(o + 8 * (size_t)npx, 256);   // forward, backward pixel orders
    L.off_frags = o;             o = align_up(o + 16 * kRecFwd * (size_t)fcap, 256);
    L.off_adj = o;               o = align_up(o + 32 * (size_t)fcap, 256);   // adjoint records
    L.off_corder = o;            o = align_up(o + 4 * (size_t)fcap, 256);
    L.off_tfinal = o;            o = align_up(o + 4 * (size_t)npx, 256);
    L.off_ncommit = o;           o = align_up(o + 4 * (size_t)npx, 256);
    L.off_grad = o;              o = align_up(o + 32 * (size_t)L.V, 256);
    L.off_dec = o;               o = align_up(o + 16 * (size_t)L.V * n_views, 256);   // decided vertices per view
    L.total = o;
    return L;
}

static ms_status check_cameras(const ms_camera *cams, int n_views) {
    if (!cams) return fail(MS_ERR_INVALID, "camera is NULL");
    if (n_views < 1 || n_views > kMaxViews) return fail(MS_ERR_INVALID, "n_views=%d outside 1..%d", n_views, kMaxViews);
    for (int v = 0; v < n_views; ++v) {
        const ms_camera *cam = cams + v;
        if (cam->width <= 0 || cam->height <= 0 || cam->width > 32768 || cam->height > 32768)
            return fail(MS_ERR_INVALID, "view %d: image size %dx%d", v, cam->width, cam->height);
        if (!(cam->znear > 0.0f)) return fail(MS_ERR_INVALID, "view %d: znear must be > 0", v);
        if (!(cam->fx != 0.0f && cam->fy != 0.0f)) return fail(MS_ERR_INVALID, "view %d: zero focal length", v);
    }
    return MS_OK;
}

static ms_status check_render_args(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int K,
                                   const ms_camera *cams, int n_views, const ms_render_params &p, const void *ws,
                                   size_t ws_bytes, RenderLayout &L) {
    ms_status s = check_cameras(cams, n_views);
    if (s != MS_OK) return s;
    if (K < 3 || K > kMaxK) return fail(MS_ERR_INVALID, "K=%d outside 3..%d", K, kMaxK);
    if (n_fans < 0) return fail(MS_ERR_INVALID, "n_fans < 0");
    if (n_fans > 0 && (!xyz || !rgb || !alpha)) return fail(MS_ERR_INVALID, "scene pointer is NULL");
    if (n_fans * (int64_t)(K + 1) >= (1ll << 32)) return fail(MS_ERR_INVALID, "too many vertices");
    if (p.tile != 8 && p.tile != 16 && p.tile != 32) return fail(MS_ERR_INVALID, "tile %d not in {8,16,32}", p.tile);
    if (p.kbuf != 8 && p.kbuf != 16) return fail(MS_ERR_INVALID, "kbuf %d not in {8,16}", p.kbuf);
    if (p.depth_bits != 0 && (p.depth_bits < 8 || p.depth_bits > 31))
        return fail(MS_ERR_INVALID, "depth_bits %d", p.depth_bits);
    L = render_layout(n_fans, K, cams, n_views, p);
    if (L.key_bits + L.fan_bits > 64 || L.depth_bits < 8)
        return fail(MS_ERR_INVALID, "sort element needs %d tile + %d depth + %d fan bits (> 64 or depth < 8)",
                    L.tile_bits, L.depth_bits, L.fan_bits);
    if (L.cap >= (1ll << 30)) return fail(MS_ERR_INVALID, "pair capacity %lld >= 2^30", (long long)L.cap);
    if (L.frag_cap >= (1ll << 32)) return fail(MS_ERR_INVALID, "fragment capacity %lld >= 2^32", (long long)L.frag_cap);
    if (L.npx >= (1ll << 32)) return fail(MS_ERR_INVALID, "%lld pixels over all views >= 2^32", (long long)L.npx);
    if (!ws) return fail(MS_ERR_INVALID, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(MS_ERR_INVALID, "workspace not 256-byte aligned");
    if (ws_bytes < L.total) return fail(MS_ERR_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    return MS_OK;
}

static ViewTable make_views(const ms_camera *cams, int n_views, const RenderLayout &L, float *const *out,
                            const float *const *out_fwd, const float *const *dL) {
    ViewTable t;
    memset(&t, 0, sizeof(t));
    t.n = n_views;
    for (int v = 0; v < n_views; ++v) {
        t.v[v].cam = make_cam(cams[v]);
        t.v[v].tile_base = (uint32_t)L.tile_base[v];
        t.v[v].tiles_x = (uint32_t)L.tiles_x[v];
        t.v[v].pix_base = (unsigned long long)L.pix_base[v];
        t.v[v].out = out ? out[v] : nullptr;
        t.v[v].out_fwd = out_fwd ? out_fwd[v] : nullptr;
        t.v[v].dL = dL ? dL[v] : nullptr;
    }
    return t;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Forward of any number of views: one binning launch, one sort, one rasterisation
// and one resolve over the concatenated tile / pixel index space.
static ms_status render_views(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int K,
                              const ms_camera *cams, int n_views, const ms_render_params *params, float *const *out,
                              void *workspace, size_t ws_bytes, cudaStream_t st) {
    ms_render_params p;
    params_or_default(params, p);
    RenderLayout L;
    ms_status s = check_render_args(xyz, rgb, alpha, n_fans, K, cams, n_views, p, workspace, ws_bytes, L);
    if (s != MS_OK) return s;
    if (!out) return fail(MS_ERR_INVALID, "output image list is NULL");
    for (int v = 0; v < n_views; ++v)
        if (!out[v] || !aligned16(out[v])) return fail(MS_ERR_INVALID, "view %d: output image NULL or not 16-byte aligned", v);
    char *ws = static_cast<char *>(workspace);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.off_keys0, st);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    RenderArgs a;
    memset(&a, 0, sizeof(a));
    a.xyz = xyz; a.rgb = rgb; a.alpha = alpha; a.n_fans = n_fans; a.K = K; a.prm = p; a.L = L; a.ws = ws;
    a.key_scale = 1.0f;
    a.vt = make_views(cams, n_views, L, out, nullptr, nullptr);
    {
        StageScope sc(MS_STAGE_BIN, st);
        if ((e = launch_bin(a, st)) != cudaSuccess) return cuda_fail(e, "bin launch");
    }
    {
        StageScope sc(MS_STAGE_SORT, st);
        if ((e = launch_sort(a, st)) != cudaSuccess) return cuda_fail(e, "sort launch");
    }
    {
        StageScope sc(MS_STAGE_RASTER, st);
        if ((e = launch_raster_count(a, st)) != cudaSuccess) return cuda_fail(e, "raster count launch");
        if ((e = launch_raster(a, true, st)) != cudaSuccess) return cuda_fail(e, "raster fill launch");
        if ((e = launch_resolve(a, false, st)) != cudaSuccess) return cuda_fail(e, "resolve launch");
    }
    if (n_fans > 0) count_launches(1 + 3 + L.passes);
    count_launches(1);   // resolve (raster kernels count themselves)
    return MS_OK;
}

static ms_status render_views_backward(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int K,
                                       const ms_camera *cams, int n_views, const ms_render_params *params,
                                       const float *const *out_fwd, const float *const *dL, float *d_xyz, float *d_rgb,
                                       float *d_alpha, void *workspace, size_t ws_bytes, cudaStream_t st) {
    ms_render_params p;
    params_or_default(params, p);
    RenderLayout L;
    ms_status s = check_render_args(xyz, rgb, alpha, n_fans, K, cams, n_views, p, workspace, ws_bytes, L);
    if (s != MS_OK) return s;
    if (!out_fwd || !dL) return fail(MS_ERR_INVALID, "image lists are NULL");
    for (int v = 0; v < n_views; ++v)
        if (!out_fwd[v] || !dL[v] || !aligned16(out_fwd[v]) || !aligned16(dL[v]))
            return fail(MS_ERR_INVALID, "view %d: image NULL or not 16-byte aligned", v);
    const bool keep_in_ws = !d_xyz && !d_rgb && !d_alpha;   // gradients stay in the workspace
    if (n_fans > 0 && !keep_in_ws && (!d_xyz || !d_rgb || !d_alpha))
        return fail(MS_ERR_INVALID, "gradient pointers must be all set or all NULL");
    char *ws = static_cast<char *>(workspace);
    StageScope sc(MS_STAGE_RASTER_BWD, st);
    // (the backward resolve writes every record's upstream gradient, zero where a record
    // was not composited, so only the vertex sums are cleared here)
    cudaError_t e = cudaMemsetAsync(ws + L.off_grad, 0, 32 * (size_t)L.V, st);
    if (e != cudaSuccess) return cuda_fail(e, "gradient clear");
    RenderArgs a;
    memset(&a, 0, sizeof(a));
    a.xyz = xyz; a.rgb = rgb; a.alpha = alpha; a.n_fans = n_fans; a.K = K; a.prm = p; a.L = L; a.ws = ws;
    a.d_xyz = d_xyz; a.d_rgb = d_rgb; a.d_alpha = d_alpha;
    a.key_scale = 1.0f;
    a.vt = make_views(cams, n_views, L, nullptr, out_fwd, dL);
    // the forward's composited fragments are replayed in commit order, recomputing
    // transmittance; the per-record upstream gradients are then chained to the vertices
    // record by record
    if ((e = launch_resolve(a, true, st)) != cudaSuccess) return cuda_fail(e, "resolve backward launch");
    if ((e = launch_record_chain(a, st)) != cudaSuccess) return cuda_fail(e, "record chain launch");
    if (!keep_in_ws && (e = launch_grad_scatter(a, st)) != cudaSuccess)
        return cuda_fail(e, "gradient scatter launch");
    count_launches(1 + (L.V > 0 && !keep_in_ws ? 1 : 0));   // resolve, scatter (the chain counts itself)
    return MS_OK;
}

// Source-Gaussian splat render: the polygons circumscribing the splats go through the
// same binning, sort and work-item machinery as fans; the splat passes then evaluate
// the Gaussians themselves.  The polygon soup lives after the render layout.
constexpr double kSplatTrunc = 2.7;           // truncation radius in scales (the fan's scale_mul)
constexpr float kSplatKeyScale = 0.9990234375f;   // 1 - 2^-10: depth keys stay below every hit

static size_t splat_poly_bytes(int64_t N) { return align_up((size_t)N * (kSplatK + 1) * 12, 256); }

static ms_status splat_views(const float *means, const float *log_scales, const float *quats, const float *opacity,
                             const float *rgb, int64_t N, int axis_rule, const ms_camera *cams, int n_views,
                             const ms_render_params *params, float *const *out, void *workspace, size_t ws_bytes,
                             cudaStream_t st) {
    ms_render_params p;
    params_or_default(params, p);
    if (axis_rule != 0 && axis_rule != 1) return fail(MS_ERR_INVALID, "axis_rule %d", axis_rule);
    if (N > 0 && (!means || !log_scales || !quats || !opacity || !rgb)) return fail(MS_ERR_INVALID, "NULL pointer");
    if (N > 0 && (reinterpret_cast<uintptr_t>(quats) & 15)) return fail(MS_ERR_INVALID, "quats must be 16-byte aligned");
    if (N >= (1ll << 31)) return fail(MS_ERR_INVALID, "too many Gaussians");
    RenderLayout L;
    // the layout check sees a placeholder soup pointer: the polygons are made below
    ms_status s = check_render_args(N > 0 ? means : nullptr, means, means, N, kSplatK, cams, n_views, p, workspace,
                                    ws_bytes > splat_poly_bytes(N) ? ws_bytes - splat_poly_bytes(N) : 0, L);
    if (s != MS_OK) return s;
    if (!out) return fail(MS_ERR_INVALID, "output image list is NULL");
    for (int v = 0; v < n_views; ++v)
        if (!out[v] || !aligned16(out[v])) return fail(MS_ERR_INVALID, "view %d: output image NULL or not 16-byte aligned", v);
    char *ws = static_cast<char *>(workspace);
    float *poly = reinterpret_cast<float *>(ws + L.total);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.off_keys0, st);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    RenderArgs a;
    memset(&a, 0, sizeof(a));
    a.xyz = poly; a.n_fans = N; a.K = kSplatK; a.prm = p; a.L = L; a.ws = ws;
    a.splat = true;
    a.key_scale = kSplatKeyScale;
    a.spl.means = means; a.spl.log_scales = log_scales; a.spl.quats = quats; a.spl.opacity = opacity;
    a.spl.rgb = rgb; a.spl.axis_rule = axis_rule; a.spl.trunc = kSplatTrunc;
    a.vt = make_views(cams, n_views, L, out, nullptr, nullptr);
    if ((e = launch_splat_polygons(a.spl, N, poly, st)) != cudaSuccess) return cuda_fail(e, "polygon launch");
    if ((e = launch_bin(a, st)) != cudaSuccess) return cuda_fail(e, "bin launch");
    if ((e = launch_sort(a, st)) != cudaSuccess) return cuda_fail(e, "sort launch");
    if ((e = launch_raster_count(a, st)) != cudaSuccess) return cuda_fail(e, "splat count launch");
    if ((e = launch_raster(a, true, st)) != cudaSuccess) return cuda_fail(e, "splat fill launch");
    if ((e = launch_resolve(a, false, st)) != cudaSuccess) return cuda_fail(e, "resolve launch");
    if (N > 0) count_launches(2 + 3 + L.passes);
    count_launches(1);
    return MS_OK;
}

}  // namespace ms

using namespace ms;

extern "C" {

MS_API const char *ms_version(void) { return "meshsplats-gb300 0.1 (sm_103a)"; }

MS_API const char *ms_last_error(void) { return g_err; }

MS_API void ms_render_params_default(ms_render_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->tile = 16;
    p->kbuf = 8;
    p->T_eps = 1e-5f;
    p->depth_bits = 0;
    p->face_mask = nullptr;
}

static ms_status mesh_build_common(const float *means, const float *log_scales, const float *quats,
                                   const float *opacity, const void *sh, int32_t sh_dtype, int32_t sh_degree, int64_t N,
                                   const ms_fan_params *fan, const float *cam_center, const float *corr, float *xyz,
                                   float *rgb, float *alpha, bool three, void *stream,
                                   const void *mlp_packed = nullptr) {
    if (!fan) return fail(MS_ERR_INVALID, "fan params NULL");
    if (mlp_packed && fan->K > 15) return fail(MS_ERR_INVALID, "K=%d: the initializer predicts K <= 15", fan->K);
    if (N < 0) return fail(MS_ERR_INVALID, "N < 0");
    if (fan->K < 3 || fan->K > kMaxK) return fail(MS_ERR_INVALID, "K=%d outside 3..%d", fan->K, kMaxK);
    if (sh_degree < 0 || sh_degree > 3) return fail(MS_ERR_INVALID, "sh_degree %d", sh_degree);
    if (sh_dtype != 0 && sh_dtype != 1) return fail(MS_ERR_INVALID, "sh_dtype %d", sh_dtype);
    if (fan->axis_rule != 0 && fan->axis_rule != 1) return fail(MS_ERR_INVALID, "axis_rule %d", fan->axis_rule);
    if (N == 0) return MS_OK;
    if (!means || !log_scales || !quats || !opacity || !sh || !xyz || !rgb || !alpha)
        return fail(MS_ERR_INVALID, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(quats) & 15) return fail(MS_ERR_INVALID, "quats must be 16-byte aligned");
    if (mlp_packed && (reinterpret_cast<uintptr_t>(mlp_packed) & 255))
        return fail(MS_ERR_INVALID, "packed weights must be 256-byte aligned");
    if (N * (int64_t)(fan->K + 1) * (three ? 3 : 1) >= (1ll << 32)) return fail(MS_ERR_INVALID, "too many vertices");
    MeshBuildConst kc;
    memset(&kc, 0, sizeof(kc));
    kc.K = fan->K;
    kc.scale_mul = fan->scale_mul;
    kc.opac_mul = fan->opac_mul;
    kc.axis_rule = fan->axis_rule;
    kc.three = three ? 1 : 0;
    const double PI = 3.14159265358979323846;
    for (int i = 0; i < fan->K; ++i) {
        const double th = -PI + 2.0 * PI * i / fan->K;
        kc.cs[i] = (float)cos(th);
        kc.sn[i] = (float)sin(th);
        if (three && (4 * i) % fan->K == 0) {   // a quarter turn: exact, so shared tips coincide
            static const float qc[4] = {-1.0f, 0.0f, 1.0f, 0.0f}, qs[4] = {0.0f, -1.0f, 0.0f, 1.0f};
            const int q = (4 * i) / fan->K;
            kc.cs[i] = qc[q & 3];
            kc.sn[i] = qs[q & 3];
        }
    }
    kc.shc[0] = (float)(0.5 * sqrt(1.0 / PI));
    kc.shc[1] = (float)sqrt(3.0 / (4.0 * PI));
    kc.shc[2] = (float)(0.5 * sqrt(15.0 / PI));
    kc.shc[3] = (float)(0.25 * sqrt(5.0 / PI));
    kc.shc[4] = (float)(0.25 * sqrt(15.0 / PI));
    kc.shc[5] = (float)(0.125 * sqrt(70.0 / PI));
    kc.shc[6] = (float)(0.25 * sqrt(105.0 / PI));
    kc.shc[7] = (float)(0.125 * sqrt(42.0 / PI));
    kc.shc[8] = (float)(0.25 * sqrt(7.0 / PI));
    if (cam_center) {
        kc.has_cam = 1;
        kc.cc[0] = cam_center[0];
        kc.cc[1] = cam_center[1];
        kc.cc[2] = cam_center[2];
    }
    kc.sh_vec_ok = (reinterpret_cast<uintptr_t>(sh) & 15) == 0;
    cudaError_t e;
    {
        // the fused kernel is the initializer's inference with the conversion in its epilogue
        StageScope sc(mlp_packed ? MS_STAGE_MLP : MS_STAGE_MESH_BUILD, (cudaStream_t)stream);
        if (mlp_packed) {
            const MlpSrc src{log_scales, quats, opacity, sh, sh_dtype, sh_degree};
            e = launch_mesh_build_mlp(means, src, N, static_cast<const char *>(mlp_packed), kc, xyz, rgb, alpha,
                                      (cudaStream_t)stream);
        } else {
            e = launch_mesh_build(means, log_scales, quats, opacity, sh, sh_dtype, sh_degree, N, kc, corr, xyz, rgb,
                                  alpha, (cudaStream_t)stream);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "mesh_build launch");
    count_launches(1);
    return MS_OK;
}

MS_API ms_status ms_mesh_build(const float *means, const float *log_scales, const float *quats, const float *opacity,
                               const void *sh, int32_t sh_dtype, int32_t sh_degree, int64_t N, const ms_fan_params *fan,
                               const float *cam_center, const float *corr, float *xyz, float *rgb, float *alpha,
                               void *stream) {
    return mesh_build_common(means, log_scales, quats, opacity, sh, sh_dtype, sh_degree, N, fan, cam_center, corr, xyz,
                             rgb, alpha, false, stream);
}

MS_API ms_status ms_mesh_build_mlp(const float *means, const float *log_scales, const float *quats,
                                   const float *opacity, const void *sh, int32_t sh_dtype, int32_t sh_degree, int64_t N,
                                   const ms_fan_params *fan, const float *cam_center, const void *packed, float *xyz,
                                   float *rgb, float *alpha, void *stream) {
    if (!packed) return fail(MS_ERR_INVALID, "packed weights NULL");
    return mesh_build_common(means, log_scales, quats, opacity, sh, sh_dtype, sh_degree, N, fan, cam_center, nullptr,
                             xyz, rgb, alpha, false, stream, packed);
}

MS_API int32_t ms_three_fan_copies(int32_t K, int32_t *first_copy) {
    if (K < 3 || K > kMaxK || !first_copy) return -1;
    const int KV = K + 1;
    // a slot of fan f (axes (1,2), (1,3), (2,3)) at angle i reaches the tip of axis c with
    // sign s when the angle is a quarter turn; the centre is slot 0 of every fan
    auto tip = [&](int f, int i, int &axis, int &sign) -> bool {
        if ((4 * i) % K != 0) return false;
        const int q = ((4 * i) / K) & 3;   // angle (q - 2) pi / 2
        const int a = f == 2 ? 1 : 0, b = f == 0 ? 1 : 2;
        if (q == 0 || q == 2) { axis = a; sign = q == 2 ? 1 : -1; }
        else { axis = b; sign = q == 3 ? 1 : -1; }
        return true;
    };
    int distinct = 1;
    for (int f = 0; f < 3; ++f) {
        first_copy[f * KV] = 0;
        for (int i = 0; i < K; ++i) {
            const int slot = f * KV + 1 + i;
            first_copy[slot] = slot;
            int ax, sg;
            if (tip(f, i, ax, sg)) {
                for (int g = 0; g < f && first_copy[slot] == slot; ++g)
                    for (int j = 0; j < K; ++j) {
                        int ax2, sg2;
                        if (tip(g, j, ax2, sg2) && ax2 == ax && sg2 == sg) {
                            first_copy[slot] = g * KV + 1 + j;
                            break;
                        }
                    }
            }
            if (first_copy[slot] == slot) ++distinct;
        }
    }
    return distinct;
}

MS_API ms_status ms_mesh_build_3d(const float *means, const float *log_scales, const float *quats,
                                  const float *opacity, const void *sh, int32_t sh_dtype, int32_t sh_degree, int64_t N,
                                  const ms_fan_params *fan, const float *cam_center, float *xyz, float *rgb,
                                  float *alpha, void *stream) {
    return mesh_build_common(means, log_scales, quats, opacity, sh, sh_dtype, sh_degree, N, fan, cam_center, nullptr,
                             xyz, rgb, alpha, true, stream);
}

MS_API size_t ms_render_workspace_size(int64_t n_fans, int32_t K, const ms_camera *cam, const ms_render_params *params) {
    return ms_batch_workspace_size(n_fans, K, cam, 1, params);
}

MS_API size_t ms_batch_workspace_size(int64_t n_fans, int32_t K, const ms_camera *cams, int32_t n_views,
                                      const ms_render_params *params) {
    if (!cams || K < 3 || K > kMaxK || n_fans < 0 || n_views < 1 || n_views > kMaxViews) return 0;
    ms_render_params p;
    params_or_default(params, p);
    return render_layout(n_fans, K, cams, n_views, p).total;
}

MS_API ms_status ms_render(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                           const ms_camera *cam, const ms_render_params *params, float *out_rgba, void *workspace,
                           size_t ws_bytes, void *stream) {
    float *out[1] = {out_rgba};
    return render_views(xyz, rgb, alpha, n_fans, K, cam, 1, params, out, workspace, ws_bytes, (cudaStream_t)stream);
}

MS_API ms_status ms_render_backward(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                                    const ms_camera *cam, const ms_render_params *params, const float *out_rgba,
                                    const float *dL_drgba, float *d_xyz, float *d_rgb, float *d_alpha, void *workspace,
                                    size_t ws_bytes, void *stream) {
    const float *of[1] = {out_rgba};
    const float *dl[1] = {dL_drgba};
    return render_views_backward(xyz, rgb, alpha, n_fans, K, cam, 1, params, of, dl, d_xyz, d_rgb, d_alpha, workspace,
                                 ws_bytes, (cudaStream_t)stream);
}

MS_API ms_status ms_batch_render(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                                 const ms_camera *cams, int32_t n_views, const ms_render_params *params,
                                 float *const *out_rgba, void *workspace, size_t ws_bytes, void *stream) {
    return render_views(xyz, rgb, alpha, n_fans, K, cams, n_views, params, out_rgba, workspace, ws_bytes,
                        (cudaStream_t)stream);
}

MS_API ms_status ms_batch_render_backward(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans,
                                          int32_t K, const ms_camera *cams, int32_t n_views,
                                          const ms_render_params *params, const float *const *out_rgba,
                                          const float *const *dL_drgba, float *d_xyz, float *d_rgb, float *d_alpha,
                                          void *workspace, size_t ws_bytes, void *stream) {
    return render_views_backward(xyz, rgb, alpha, n_fans, K, cams, n_views, params, out_rgba, dL_drgba, d_xyz, d_rgb,
                                 d_alpha, workspace, ws_bytes, (cudaStream_t)stream);
}

MS_API size_t ms_splat_workspace_size(int64_t N, const ms_camera *cams, int32_t n_views,
                                      const ms_render_params *params) {
    const size_t base = ms_batch_workspace_size(N, kSplatK, cams, n_views, params);
    return base ? base + splat_poly_bytes(N) : 0;
}

MS_API ms_status ms_splat_render(const float *means, const float *log_scales, const float *quats,
                                 const float *opacity, const float *rgb, int64_t N, int32_t axis_rule,
                                 const ms_camera *cams, int32_t n_views, const ms_render_params *params,
                                 float *const *out_rgba, void *workspace, size_t ws_bytes, void *stream) {
    return splat_views(means, log_scales, quats, opacity, rgb, N, axis_rule, cams, n_views, params, out_rgba,
                       workspace, ws_bytes, (cudaStream_t)stream);
}

MS_API size_t ms_render_grad_offset(int64_t n_fans, int32_t K, const ms_camera *cams, int32_t n_views,
                                    const ms_render_params *params) {
    if (!cams || K < 3 || K > kMaxK || n_fans < 0 || n_views < 1 || n_views > kMaxViews) return 0;
    ms_render_params p;
    params_or_default(params, p);
    return render_layout(n_fans, K, cams, n_views, p).off_grad;
}

MS_API ms_status ms_render_get_info(const void *workspace, ms_render_info *info, void *stream) {
    if (!workspace || !info) return fail(MS_ERR_INVALID, "NULL argument");
    Status st;
    cudaError_t e = cudaMemcpyAsync(&st, workspace, sizeof(Status), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    memset(info, 0, sizeof(*info));
    info->pairs = (int64_t)st.pairs;
    info->culled_tris = (int64_t)st.culled;
    info->extra_passes = (int64_t)st.extra_passes;
    info->timeouts = (int32_t)st.timeouts;
    info->pair_capacity = (int64_t)st.cap;
    info->n_tiles = (int32_t)st.n_tiles;
    info->sort_bits = (int32_t)st.sort_bits;
    info->overflow = st.pairs > st.cap ? 1 : 0;
    info->rect_tests = (int64_t)st.rect_tests;
    info->fragments = (int64_t)st.fragments;
    info->commits = (int64_t)st.commits;
    info->frags = (int64_t)st.frags;
    info->frag_capacity = (int64_t)st.frag_cap;
    if (st.frags > st.frag_cap) {
        info->overflow = 1;
        return fail(MS_ERR_CAPACITY, "%llu fragments exceed the workspace fragment capacity %llu", st.frags,
                    st.frag_cap);
    }
    if (info->overflow)
        return fail(MS_ERR_CAPACITY, "%llu (tile, fan) pairs exceed the workspace capacity %llu", st.pairs, st.cap);
    if (st.timeouts) return fail(MS_ERR_TIMEOUT, "%u bounded device waits expired", st.timeouts);
    return MS_OK;
}

MS_API ms_status ms_l1_loss(const float *img_rgba, const float *target_rgba, int64_t n_pixels, float *dL_drgba,
                            float *loss, void *stream) {
    if (n_pixels < 0 || !loss) return fail(MS_ERR_INVALID, "bad arguments");
    if (n_pixels > 0 && (!img_rgba || !target_rgba || !dL_drgba)) return fail(MS_ERR_INVALID, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(img_rgba) | reinterpret_cast<uintptr_t>(target_rgba) |
         reinterpret_cast<uintptr_t>(dL_drgba)) & 15)
        return fail(MS_ERR_INVALID, "images must be 16-byte aligned");
    cudaError_t e;
    {
        StageScope sc(MS_STAGE_LOSS, (cudaStream_t)stream);
        e = launch_l1(img_rgba, target_rgba, n_pixels, dL_drgba, loss, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "l1 launch");
    if (n_pixels > 0) count_launches(1);
    return MS_OK;
}

MS_API size_t ms_fine_tune_loss_workspace_size(int32_t height, int32_t width) {
    if (height < 0 || width < 0) return 0;
    return align_up(ssim_scratch_bytes(height, width), 256) + 256;
}

MS_API ms_status ms_fine_tune_loss(const float *img_rgba, const float *target_rgba, int32_t height, int32_t width,
                                   float lambda, float *dL_drgba, float *loss, void *workspace, size_t ws_bytes,
                                   void *stream) {
    if (height < 0 || width < 0 || height > 32768 || width > 32768 || !loss)
        return fail(MS_ERR_INVALID, "bad image size %dx%d or NULL loss", width, height);
    if (!(lambda >= 0.0f && lambda <= 1.0f)) return fail(MS_ERR_INVALID, "lambda %g outside [0, 1]", (double)lambda);
    const bool empty = height == 0 || width == 0;
    if (!empty && (!img_rgba || !target_rgba || !dL_drgba || !workspace)) return fail(MS_ERR_INVALID, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(img_rgba) | reinterpret_cast<uintptr_t>(target_rgba) |
         reinterpret_cast<uintptr_t>(dL_drgba)) & 15)
        return fail(MS_ERR_INVALID, "images must be 16-byte aligned");
    if (!empty && ws_bytes < ms_fine_tune_loss_workspace_size(height, width))
        return fail(MS_ERR_INVALID, "workspace %zu bytes < %zu needed", ws_bytes,
                    ms_fine_tune_loss_workspace_size(height, width));
    char *ws = static_cast<char *>(workspace);
    float *scratch = reinterpret_cast<float *>(ws + ((256 - (reinterpret_cast<uintptr_t>(ws) & 255)) & 255));
    cudaError_t e;
    {
        StageScope sc(MS_STAGE_LOSS, (cudaStream_t)stream);
        e = launch_ssim_loss(img_rgba, target_rgba, height, width, lambda, dL_drgba, loss, empty ? nullptr : scratch,
                             (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fine-tune loss launch");
    if (!empty) count_launches(2);
    return MS_OK;
}

MS_API size_t ms_prune_workspace_size(int64_t n_fans) {
    if (n_fans < 0) return 0;
    return align_up(prune_scratch_bytes(n_fans), 256) + 256;
}

MS_API ms_status ms_prune_faces(const float *xyz, const float *rgb, const float *alpha, const float *m, const float *v,
                                const uint32_t *face_mask_in, int64_t n_fans, int32_t K, float threshold,
                                float *xyz_out, float *rgb_out, float *alpha_out, float *m_out, float *v_out,
                                uint32_t *face_mask_out, int64_t *n_kept, void *workspace, size_t ws_bytes,
                                void *stream) {
    if (n_fans < 0 || K < 3 || K > kMaxK || !n_kept) return fail(MS_ERR_INVALID, "bad n_fans, K or NULL n_kept");
    if (n_fans * (int64_t)(K + 1) >= (1ll << 32)) return fail(MS_ERR_INVALID, "too many vertices");
    if (n_fans > 0 && (!xyz || !rgb || !alpha || !xyz_out || !rgb_out || !alpha_out || !workspace))
        return fail(MS_ERR_INVALID, "NULL pointer");
    if ((m == nullptr) != (m_out == nullptr) || (v == nullptr) != (v_out == nullptr))
        return fail(MS_ERR_INVALID, "a moment array and its output must be both set or both NULL");
    if (n_fans > 0 && ws_bytes < ms_prune_workspace_size(n_fans))
        return fail(MS_ERR_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, ms_prune_workspace_size(n_fans));
    char *ws = static_cast<char *>(workspace);
    void *scratch = ws ? ws + ((256 - (reinterpret_cast<uintptr_t>(ws) & 255)) & 255) : nullptr;
    cudaError_t e = launch_prune(xyz, rgb, alpha, m, v, face_mask_in, n_fans, K, threshold, xyz_out, rgb_out,
                                 alpha_out, m_out, v_out, face_mask_out, n_kept, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "prune launch");
    if (n_fans > 0) count_launches(3);
    return MS_OK;
}

MS_API ms_status ms_prune_fans(const float *xyz, const float *rgb, const float *alpha, const float *m, const float *v,
                               int64_t n_fans, int32_t K, float threshold, float *xyz_out, float *rgb_out,
                               float *alpha_out, float *m_out, float *v_out, int64_t *n_kept, void *workspace,
                               size_t ws_bytes, void *stream) {
    return ms_prune_faces(xyz, rgb, alpha, m, v, nullptr, n_fans, K, threshold, xyz_out, rgb_out, alpha_out, m_out,
                          v_out, nullptr, n_kept, workspace, ws_bytes, stream);
}

static ms_status adam_common(float *xyz, float *rgb, float *alpha, const float *d_xyz, const float *d_rgb,
                             const float *d_alpha, float *m, float *v, int64_t V, int32_t step, int32_t *d_step,
                             float lr_color, float lr_xyz, float beta1, float beta2, float eps, void *stream) {
    if (V > 0 && (!xyz || !rgb || !alpha || !d_xyz || !d_rgb || !d_alpha || !m || !v))
        return fail(MS_ERR_INVALID, "NULL pointer");
    cudaError_t e;
    {
        StageScope sc(MS_STAGE_ADAM, (cudaStream_t)stream);
        e = launch_adam(xyz, rgb, alpha, d_xyz, d_rgb, d_alpha, m, v, V, step, d_step, lr_color, lr_xyz, beta1, beta2,
                        eps, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "adam launch");
    count_launches((V > 0 ? 1 : 0) + (d_step ? 1 : 0));
    return MS_OK;
}

MS_API ms_status ms_adam_step(float *xyz, float *rgb, float *alpha, const float *d_xyz, const float *d_rgb,
                              const float *d_alpha, float *m, float *v, int64_t V, int32_t step, float lr_color,
                              float lr_xyz, float beta1, float beta2, float eps, void *stream) {
    if (V < 0 || step < 1) return fail(MS_ERR_INVALID, "bad V or step");
    return adam_common(xyz, rgb, alpha, d_xyz, d_rgb, d_alpha, m, v, V, step, nullptr, lr_color, lr_xyz, beta1, beta2,
                       eps, stream);
}

MS_API ms_status ms_adam_step_ws(float *xyz, float *rgb, float *alpha, const void *grad, float *m, float *v,
                                 int64_t V, int32_t step, int32_t *d_step, float lr_color, float lr_xyz, float beta1,
                                 float beta2, float eps, void *stream) {
    if (V < 0 || (!d_step && step < 1)) return fail(MS_ERR_INVALID, "bad V or step");
    if (V > 0 && (!xyz || !rgb || !alpha || !grad || !m || !v)) return fail(MS_ERR_INVALID, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(grad) & 15) return fail(MS_ERR_INVALID, "gradients not 16-byte aligned");
    cudaError_t e;
    {
        StageScope sc(MS_STAGE_ADAM, (cudaStream_t)stream);
        e = launch_adam_ws(xyz, rgb, alpha, static_cast<const float4 *>(grad), m, v, V, d_step ? 1 : step, d_step,
                           lr_color, lr_xyz, beta1, beta2, eps, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "adam launch");
    count_launches((V > 0 ? 1 : 0) + (d_step ? 1 : 0));
    return MS_OK;
}

MS_API ms_status ms_adam_step_counted(float *xyz, float *rgb, float *alpha, const float *d_xyz, const float *d_rgb,
                                      const float *d_alpha, float *m, float *v, int64_t V, int32_t *d_step,
                                      float lr_color, float lr_xyz, float beta1, float beta2, float eps,
                                      void *stream) {
    if (V < 0 || !d_step) return fail(MS_ERR_INVALID, "bad V or NULL step counter");
    return adam_common(xyz, rgb, alpha, d_xyz, d_rgb, d_alpha, m, v, V, 1, d_step, lr_color, lr_xyz, beta1, beta2,
                       eps, stream);
}

MS_API ms_status ms_mse(const float *img_rgba, const float *target_rgba, int64_t n_pixels, float *out, void *stream) {
    if (n_pixels < 0 || !out || (n_pixels > 0 && (!img_rgba || !target_rgba))) return fail(MS_ERR_INVALID, "bad arguments");
    if ((reinterpret_cast<uintptr_t>(img_rgba) | reinterpret_cast<uintptr_t>(target_rgba)) & 15)
        return fail(MS_ERR_INVALID, "images must be 16-byte aligned");
    cudaError_t e = launch_mse(img_rgba, target_rgba, n_pixels, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mse launch");
    if (n_pixels > 0) count_launches(1);
    return MS_OK;
}

MS_API ms_status ms_fan_corrections(const float *xyz0, const float *alpha0, const float *xyz1, const float *alpha1,
                                    int64_t N, int32_t K, float *corr, void *stream) {
    if (N < 0 || K < 3 || K > kMaxK) return fail(MS_ERR_INVALID, "bad N or K");
    if (N > 0 && (!xyz0 || !alpha0 || !xyz1 || !alpha1 || !corr)) return fail(MS_ERR_INVALID, "NULL pointer");
    cudaError_t e = launch_fan_corr(xyz0, alpha0, xyz1, alpha1, N, K, corr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fan corrections launch");
    if (N > 0) count_launches(1);
    return MS_OK;
}

MS_API size_t ms_mlp_packed_bytes(void) { return mlp_packed_bytes(); }

MS_API ms_status ms_mlp_pack(const float *W1, const float *W2, const float *W3, int32_t n_out, void *packed,
                             void *stream) {
    if (!W1 || !W2 || !W3 || !packed) return fail(MS_ERR_INVALID, "NULL pointer");
    if (n_out < 1 || n_out > 32) return fail(MS_ERR_INVALID, "n_out %d outside 1..32", n_out);
    if (reinterpret_cast<uintptr_t>(packed) & 255) return fail(MS_ERR_INVALID, "packed weights not 256-byte aligned");
    cudaError_t e = launch_mlp_pack(W1, W2, W3, n_out, static_cast<char *>(packed), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp pack launch");
    count_launches(1);
    return MS_OK;
}

static ms_status mlp_src(const float *log_scales, const float *quats, const float *opacity, const void *sh,
                         int32_t sh_dtype, int32_t sh_degree, int64_t N, MlpSrc &s) {
    if (N < 0) return fail(MS_ERR_INVALID, "N < 0");
    if (sh_degree < 0 || sh_degree > 3 || (sh_dtype != 0 && sh_dtype != 1))
        return fail(MS_ERR_INVALID, "sh_degree %d / sh_dtype %d", sh_degree, sh_dtype);
    if (N > 0 && (!log_scales || !quats || !opacity || !sh)) return fail(MS_ERR_INVALID, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(quats) & 15) return fail(MS_ERR_INVALID, "quats must be 16-byte aligned");
    s.log_scales = log_scales; s.quats = quats; s.opacity = opacity; s.sh = sh;
    s.sh_dtype = sh_dtype; s.sh_degree = sh_degree;
    return MS_OK;
}

MS_API ms_status ms_mlp_features(const float *log_scales, const float *quats, const float *opacity, const void *sh,
                                 int32_t sh_dtype, int32_t sh_degree, int64_t N, float *X, void *stream) {
    MlpSrc s;
    ms_status r = mlp_src(log_scales, quats, opacity, sh, sh_dtype, sh_degree, N, s);
    if (r != MS_OK) return r;
    if (N > 0 && !X) return fail(MS_ERR_INVALID, "X is NULL");
    cudaError_t e = launch_mlp_features(s, N, X, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp features launch");
    if (N > 0) count_launches(1);
    return MS_OK;
}

MS_API ms_status ms_mlp_forward(const float *log_scales, const float *quats, const float *opacity, const void *sh,
                                int32_t sh_dtype, int32_t sh_degree, int64_t N, const void *packed, int32_t n_out,
                                float *corr, void *stream) {
    MlpSrc s;
    ms_status r = mlp_src(log_scales, quats, opacity, sh, sh_dtype, sh_degree, N, s);
    if (r != MS_OK) return r;
    if (!packed || (N > 0 && !corr)) return fail(MS_ERR_INVALID, "NULL pointer");
    if (n_out < 1 || n_out > 32) return fail(MS_ERR_INVALID, "n_out %d outside 1..32", n_out);
    if (reinterpret_cast<uintptr_t>(packed) & 255) return fail(MS_ERR_INVALID, "packed weights not 256-byte aligned");
    cudaError_t e;
    {
        StageScope sc(MS_STAGE_MLP, (cudaStream_t)stream);
        e = launch_mlp_forward(s, N, static_cast<const char *>(packed), n_out, corr, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mlp forward launch");
    if (N > 0) count_launches(1);
    return MS_OK;
}

MS_API size_t ms_mlp_train_workspace_size(int64_t n) { return n < 0 ? 0 : mlp_act_bytes(n); }

MS_API ms_status ms_mlp_grads(const float *X, const float *T, int64_t n, int32_t n_out, const void *packed,
                              float *grads, float *loss, void *workspace, size_t ws_bytes, void *stream) {
    if (n < 0 || n_out < 1 || n_out > 32) return fail(MS_ERR_INVALID, "bad n or n_out");
    if (!packed || !grads || !loss || (n > 0 && (!X || !T || !workspace))) return fail(MS_ERR_INVALID, "NULL pointer");
    if (ws_bytes < mlp_act_bytes(n)) return fail(MS_ERR_INVALID, "workspace %zu < %zu", ws_bytes, mlp_act_bytes(n));
    if ((reinterpret_cast<uintptr_t>(packed) | reinterpret_cast<uintptr_t>(workspace)) & 255)
        return fail(MS_ERR_INVALID, "packed weights / workspace not 256-byte aligned");
    cudaError_t e = launch_mlp_grads(X, T, n, n_out, static_cast<const char *>(packed), static_cast<char *>(workspace),
                                     grads, loss, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp gradient launch");
    if (n > 0) count_launches(2);
    return MS_OK;
}

MS_API ms_status ms_mlp_adam(float *W, const float *grads, float *m, float *v, int32_t n_out, int32_t *d_step,
                             float lr, float beta1, float beta2, float eps, void *packed, void *stream) {
    if (!W || !grads || !m || !v || !d_step || !packed) return fail(MS_ERR_INVALID, "NULL pointer");
    if (n_out < 1 || n_out > 32) return fail(MS_ERR_INVALID, "n_out %d outside 1..32", n_out);
    cudaError_t e = launch_mlp_adam(W, grads, m, v, n_out, d_step, lr, beta1, beta2, eps, static_cast<char *>(packed),
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp adam launch");
    count_launches(3);
    return MS_OK;
}

MS_API ms_status ms_mlp_status(const void *packed, int32_t *timeouts, void *stream) {
    if (!packed || !timeouts) return fail(MS_ERR_INVALID, "NULL pointer");
    uint32_t t = 0;
    cudaError_t e = cudaMemcpyAsync(&t, static_cast<const char *>(packed) + mlp_status_offset(), 4,
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp status read");
    *timeouts = (int32_t)t;
    return t ? fail(MS_ERR_TIMEOUT, "%u bounded tensor-core waits expired", t) : MS_OK;
}

MS_API void ms_profile_enable(int32_t on) { g_prof = on != 0; }

MS_API ms_status ms_profile_read(double *ms_per_stage, int64_t *launches_per_stage, int32_t n) {
    if (n < 0 || n > MS_STAGE_COUNT) return fail(MS_ERR_INVALID, "n=%d", n);
    for (int i = 0; i < n; ++i) {
        if (ms_per_stage) ms_per_stage[i] = 0.0;
        if (launches_per_stage) launches_per_stage[i] = 0;
    }
    ms_status s = MS_OK;
    for (size_t i = 0; i < g_ev_used; ++i) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(g_ev[i].b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, g_ev[i].a, g_ev[i].b);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "profile event");
            continue;
        }
        const int st = g_ev[i].stage;
        if (st < n) {
            if (ms_per_stage) ms_per_stage[st] += t;
            if (launches_per_stage) launches_per_stage[st] += 1;
        }
    }
    g_ev_used = 0;
    return s;
}

MS_API int64_t ms_kernel_launches(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
