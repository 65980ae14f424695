// Internal launch interfaces between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/meshsplats.h"
#include "ms_common.cuh"

namespace ms {


struct MeshBuildConst {
    int K;
    float scale_mul, opac_mul;
    int axis_rule;
    float cs[16], sn[16];   // cos / sin of theta_i = -pi + 2 pi i / K
    float shc[9];           // SH normalisation constants (see sh_basis)
    int has_cam;
    float cc[3];
    int sh_vec_ok;          // SH base pointer 16-byte aligned
    int three;              // three fans per Gaussian (3D conversion), else one flat fan
};

cudaError_t launch_mesh_build(const float *means, const float *log_scales, const float *quats, const float *opacity,
                              const void *sh, int sh_dtype, int sh_degree, int64_t N, const MeshBuildConst &kc,
                              const float *corr, float *xyz, float *rgb, float *alpha, cudaStream_t st);

// Render workspace layout (byte offsets from the workspace base, 256-byte aligned).
// Tiles and pixels of all views form one index space (see ViewTable).
struct RenderLayout {
    int tile, n_views, n_tiles, tile_bits, depth_bits, key_bits, passes, kbuf;
    int fan_bits;              // low bits of a sort element holding the fan id
    int tiles_x[kMaxViews], tile_base[kMaxViews];
    int64_t pix_base[kMaxViews];
    int64_t npx, n_fans, V, cap, frag_cap, mask_cap;
    int64_t bin_fan_blocks, bin_blocks, sort_blocks, scan_blocks, tscan_blocks, max_items;
    size_t off_status, off_bin_state, off_keys0, off_keys1, off_hist, off_lookback,
        off_ranges, off_scan_state, off_tscan_state, off_pbucket, off_zrange, off_mask_cursor, off_perm, off_tile_nitems, off_tile_ibase, off_items, off_icnt,
        off_counts, off_offsets, off_maskoff, off_masks, off_frags, off_adj, off_corder, off_tfinal, off_ncommit, off_grad, off_dec, total;
};

RenderLayout render_layout(int64_t n_fans, int K, const ms_camera *cams, int n_views, const ms_render_params &p);

// Source Gaussians drawn by the splat passes (ms_splat_render); device pointers.
struct SplatSrc {
    const float *means, *log_scales, *quats, *opacity, *rgb;
    int axis_rule;
    double trunc;
};

struct RenderArgs {
    const float *xyz, *rgb, *alpha;
    int64_t n_fans;
    int K;
    ViewTable vt;              // cameras, index-space bases, per-view image pointers
    ms_render_params prm;
    RenderLayout L;
    char *ws;
    float *d_xyz, *d_rgb, *d_alpha;   // backward outputs
    bool splat;                // draw the source Gaussians of `spl` over the polygons in xyz
    float key_scale;           // binning: depth keys from key_scale * min Z (1 for fans)
    SplatSrc spl;
};

// Learned fan initializer (mlp.cu): Gaussian inputs, packed weights, kernels.
struct MlpSrc {
    const float *log_scales, *quats, *opacity;
    const void *sh;
    int sh_dtype, sh_degree;
};
size_t mlp_packed_bytes();
size_t mlp_act_bytes(int64_t n);
size_t mlp_param_count(int n_out);
uint32_t mlp_status_offset();
cudaError_t launch_mlp_pack(const float *W1, const float *W2, const float *W3, int n_out, char *packed,
                            cudaStream_t st);
cudaError_t launch_mlp_features(const MlpSrc &s, int64_t N, float *X, cudaStream_t st);
cudaError_t launch_mlp_forward(const MlpSrc &s, int64_t N, const char *packed, int n_out, float *corr,
                               cudaStream_t st);
// The conversion fused behind the initializer's inference (flat fans, n_out = 2(K+1)).
cudaError_t launch_mesh_build_mlp(const float *means, const MlpSrc &s, int64_t N, const char *packed,
                                  const MeshBuildConst &kc, float *xyz, float *rgb, float *alpha, cudaStream_t st);
cudaError_t launch_mlp_grads(const float *X, const float *T, int64_t n, int n_out, const char *packed, char *act,
                             float *grads, float *loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float *W, const float *grads, float *m, float *v, int n_out, int32_t *d_step, float lr,
                            float b1, float b2, float eps, char *packed, cudaStream_t st);

// Polygons circumscribing the splats' truncation ellipses (K = 8 fans), for binning.
constexpr int kSplatK = 8;
cudaError_t launch_splat_polygons(const SplatSrc &s, int64_t N, float *xyz, cudaStream_t st);

cudaError_t launch_bin(const RenderArgs &a, cudaStream_t st);
cudaError_t launch_sort(const RenderArgs &a, cudaStream_t st);
// Stable LSD sort of n 64-bit elements by bits [shift, shift + 8 passes): a and b are the two
// buffers, *result receives the one holding the sorted elements; scratch (device,
// sort_scratch_bytes, 16-byte aligned) is cleared and used for counts and look-back flags.
size_t sort_scratch_bytes(int64_t n, int passes);
// Elements of one sort tile (one look-back slot per tile and digit).
int64_t sort_tile_elems();
cudaError_t sort_u64(unsigned long long *a, unsigned long long *b, int64_t n, int shift, int passes, char *scratch,
                     cudaStream_t st, unsigned long long **result);
constexpr int kItemFans = 64;   // fans per raster work item

cudaError_t launch_raster(const RenderArgs &a, bool fill, cudaStream_t st);
cudaError_t launch_raster_count(const RenderArgs &a, cudaStream_t st);   // items, count, prefix, pixel scan
cudaError_t launch_record_chain(const RenderArgs &a, cudaStream_t st);   // adjoint: records -> fan vertices
constexpr int kRecFwd = 2;   // float4s per fragment record
cudaError_t launch_pixel_order(const RenderArgs &a, cudaStream_t st);   // resolve order of the pixels
cudaError_t launch_resolve(const RenderArgs &a, bool backward, cudaStream_t st);
cudaError_t launch_grad_scatter(const RenderArgs &a, cudaStream_t st);

// Records a host-side error message for ms_last_error() (api.cu).
ms_status set_error(ms_status s, const char *fmt, ...);

// Launch accounting and optional stage events (api.cu).
void count_launches(int n);
struct StageScope {
    int stage;
    cudaStream_t st;
    int slot;
    StageScope(int stage, cudaStream_t st);
    ~StageScope();
};

cudaError_t launch_l1(const float *img, const float *tgt, int64_t n_pixels, float *dL, float *loss, cudaStream_t st);
// Pruning of fans whose vertex opacities are all below a threshold (prune.cu).
size_t prune_scratch_bytes(int64_t n_fans);
cudaError_t launch_prune(const float *xyz, const float *rgb, const float *alpha, const float *m, const float *v,
                         const uint32_t *mask_in, int64_t n_fans, int K, float thr, float *xyz_o, float *rgb_o,
                         float *alpha_o, float *m_o, float *v_o, uint32_t *mask_o, int64_t *n_kept, void *scratch,
                         cudaStream_t st);
// Fine-tuning loss lambda L1 + (1 - lambda)(1 - SSIM) of one H x W RGBA image (ssim.cu).
size_t ssim_scratch_bytes(int H, int W);
cudaError_t launch_ssim_loss(const float *img, const float *tgt, int H, int W, float lam, float *dL, float *loss,
                             float *scratch, cudaStream_t st);
cudaError_t launch_adam_ws(float *xyz, float *rgb, float *alpha, const float4 *grad, float *m, float *v, int64_t V,
                           int step, int32_t *d_step, float lr_c, float lr_x, float b1, float b2, float eps,
                           cudaStream_t st);
cudaError_t launch_mse(const float *img, const float *tgt, int64_t n_pixels, float *out, cudaStream_t st);
cudaError_t launch_fan_corr(const float *xyz0, const float *a0, const float *xyz1, const float *a1, int64_t N, int K,
                            float *corr, cudaStream_t st);
cudaError_t launch_adam(float *xyz, float *rgb, float *alpha, const float *dx, const float *dc, const float *da,
                        float *m, float *v, int64_t V, int step, int32_t *d_step, float lr_c, float lr_x, float b1,
                        float b2, float eps, cudaStream_t st);

}  // namespace ms
