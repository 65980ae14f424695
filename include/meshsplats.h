/*
 * meshsplats.h -- C ABI of the GB300 (sm_103a) MeshSplats hot path.
 *
 * MeshSplats (arXiv 2502.07754) turns every Gaussian of a Gaussian-Splatting scene
 * into a disjoint triangle fan and renders and fine-tunes those fans with
 * order-correct alpha compositing.  This library implements, as CUDA kernels:
 *   ms_mesh_build       Gaussian -> fan conversion with SH colour (Sec. 3, Eq. 2 and the
 *                       vertex / colour / opacity rules that follow it)
 *   ms_render           MVP projection, tile binning, radix sort of (tile, depth) keys,
 *                       exact per-pixel depth order, perspective-correct barycentric
 *                       interpolation, front-to-back compositing (Sec. 3 "Rendering
 *                       MeshSplats in Nvdiffrast")
 *   ms_render_backward  adjoint of ms_render for vertex positions, colours and opacities
 *                       (Sec. 3 "Fine-tuning", "Optimization and Pruning")
 *   ms_l1_loss, ms_fine_tune_loss, ms_adam_step   the L1 term and the full loss of Eq. 3,
 *                       and the two-learning-rate update
 *   ms_batch_render     all of the above for up to 32 views in one index space
 *   ms_prune_faces      the pruning of Sec. 3 "Optimization and Pruning" (per face)
 *   ms_mesh_build_3d, ms_three_fan_sum_copies   the three-fan conversion of 3D Gaussians
 *   ms_mesh_render      explicit triangles over a shared vertex array (centroid fans),
 *   ms_mesh_prior_*     and the mesh-prior mode ("MeshSplats with Mesh Prior")
 *   ms_bvh_build, ms_raytrace   ray tracing of the triangles with shadows (the secondary
 *                       effects the mesh form is for)
 *   ms_mlp_*, ms_mesh_build_mlp   a learned fan initializer on the tensor cores, fused into
 *                       the conversion
 *   ms_spatial_order, ms_gather_rows   the Gaussians' storage order (Morton order of the
 *                       means), applied once when a scene is loaded
 *
 * Conventions (all entry points):
 *   - Every pointer named d_* or documented as "device" is caller-owned device memory;
 *     the library never allocates device memory.  Per-call scratch lives in a
 *     caller-provided workspace sized by the matching *_workspace_size function.
 *   - Calls are asynchronous on the given stream (cudaStream_t passed as void*; NULL
 *     is the legacy default stream).  Errors found on the host return immediately;
 *     errors found on the device (capacity overflow, bounded wait expired) are
 *     recorded in the workspace and reported by ms_render_get_info().
 *   - Arrays are row-major, little-endian.  Images are H x W x 4 float32 (R,G,B,A),
 *     row 0 at the top.  Fan soups are structure-of-arrays: xyz V x 3, rgb V x 3,
 *     alpha V, with V = N (K+1); vertex g(K+1) is the centre of fan g and vertex
 *     g(K+1)+1+i its i-th boundary vertex; triangle g K + j is
 *     (g(K+1), g(K+1)+1+j, g(K+1)+1+((j+1) mod K)).
 *   - Gradient outputs accumulate (+=); the caller zeroes them.
 *   - Camera: pinhole, OpenCV axes (x right, y down, z forward), X_cam = R_cw (p - C),
 *     pixel (fx X/Z + cx, fy Y/Z + cy); pixel (i, j) has its centre at (i+0.5, j+0.5).
 *
 * Decisions.  Coverage and per-pixel order follow their plain definitions: a triangle
 * covers a pixel centre when its three edge functions pass the top-left fill rule, and
 * the fragments of a pixel are composited in ascending depth 1 / sum_k (lambda_k / Z_k)
 * (the ray-plane depth of the triangle at the pixel centre; ties by ascending triangle
 * index).  The kernels take these decisions so that they agree with an FP64 evaluation:
 *   - each vertex is projected in double-float (d = p - C exact, the camera rotation and
 *     the pinhole division carried to ~2^-44 relative): X, Y, Z and x = fx X/Z + cx,
 *     y = fy Y/Z + cy;
 *   - a vertex is valid iff round(Z) > znear and |round(x)|, |round(y)| <= 2^17; a
 *     triangle with an invalid vertex is culled;
 *   - coverage is evaluated in binary32 on fan-relative coordinates: the fan's origin is
 *     o = floor of its centre's screen position, each vertex enters as the binary32 value
 *     nearest (x - o.x, y - o.y), the pixel centre as (px - o.x + 0.5, py - o.y + 0.5)
 *     (exact); area2(A,B,C) = (xB - xA)(yC - yA) - (yB - yA)(xC - xA), 0 never covers,
 *     < 0 swaps B, C; the edge of the vertex pair {a < b} (by vertex index) is
 *     F = (xb - xa)(py - ya) - (yb - ya)(px - xa), negated when the oriented edge runs
 *     b -> a; it passes if F > 0, or F == 0 and its direction (ex, ey) has ey < 0, or
 *     ey == 0 and ex > 0.  Near a fan the coordinates are small, so these binary32 edge
 *     values have the sign of the exact ones except within ~1e-6 px of an edge;
 *   - the depth is the double-float plane depth (n . P_c) / (n . r) with n the
 *     triangle's normal from its camera-space vertex offsets and r the pixel's ray,
 *     clamped to the triangle's vertex depths; fragments are ordered by (depth high part,
 *     low part, triangle index).
 * On the test scenes (1k to 1M Gaussians, full frames and windows) no pixel's fragment
 * list differs from the FP64 decisions; taking the order from binary32 depths instead
 * changes it on 1.6% to 39% of the pixels (nearly coplanar surfels).
 * Interpolation and compositing are FP32: mu_k = (E_k / Z_k) / sum_j (E_j / Z_j),
 * c = sum mu_k c_k, a = sum mu_k a_k; C += T a c, T *= 1 - a, stop once T < T_eps;
 * out = (C + T bg, 1 - T).
 */
#ifndef MESHSPLATS_H
#define MESHSPLATS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_API __attribute__((visibility("default")))

typedef enum {
    MS_OK = 0,
    MS_ERR_INVALID = 1,     /* bad argument (null pointer, size, K out of range, ...) */
    MS_ERR_CAPACITY = 2,    /* workspace pair capacity exceeded; see ms_render_info */
    MS_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    MS_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired (result invalid) */
    MS_ERR_UNSUPPORTED = 5  /* valid request this build does not implement */
} ms_status;

/* Fan conversion hyperparameters (Sec. 3: scale_mul, no_triag, opac_mul). */
typedef struct {
    int32_t K;          /* no_triag, 3..16 (paper: 8) */
    float scale_mul;    /* paper: 2.7 */
    float opac_mul;     /* paper: 0.2 */
    int32_t axis_rule;  /* 0: drop axis 0 (GaMeS epsilon axis); 1: drop the axis of smallest scale */
} ms_fan_params;

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R_cw[9];      /* row-major world -> camera rotation */
    float C[3];         /* camera centre, world */
    float znear;        /* triangles with a vertex at Z <= znear are culled */
} ms_camera;

typedef struct {
    int32_t tile;           /* screen tile edge in pixels: 8, 16 or 32 */
    int32_t kbuf;           /* per-pixel pending-fragment buffer: 8 or 16 */
    float T_eps;            /* early-termination transmittance (default 1e-5) */
    float bg[3];            /* background colour */
    int64_t pair_capacity;  /* (tile, fan) pair capacity of the workspace; 0 = default */
    int32_t depth_bits;     /* depth bits in the sort key, 8..31; 0 = automatic: the most (<= 27) that
                               keep the key within the bytes of tile bits + 20 */
    int64_t frag_capacity;  /* per-pixel fragment records of the workspace; 0 = 8 W H + 65536 */
    const uint32_t *face_mask;  /* NULL: every face of every fan is drawn; else device, one word per fan,
                                   bit j set = triangle j drawn (the faces ms_prune_faces keeps) */
} ms_render_params;

/* Device-side outcome of the last ms_render / ms_render_backward on a workspace. */
typedef struct {
    int64_t pairs;          /* (tile, fan) pairs the binning produced */
    int64_t pair_capacity;  /* capacity of the workspace */
    int64_t culled_tris;    /* triangles culled at the near plane / guard band */
    int64_t extra_passes;   /* pixel-passes re-run because the pending buffer overflowed */
    int32_t overflow;       /* 1 if pairs or fragments exceed their capacity (image invalid) */
    int32_t timeouts;       /* bounded waits that expired (image invalid) */
    int32_t sort_bits;      /* key bits sorted */
    int32_t n_tiles;
    int64_t rect_tests;     /* (pixel, fan) pairs the forward rasterisation evaluated */
    int64_t fragments;      /* covered (pixel, triangle) fragments it found */
    int64_t commits;        /* fragments composited by the forward resolve */
    int64_t frags;          /* fragment records the rasterisation produced */
    int64_t frag_capacity;  /* fragment record capacity of the workspace */
} ms_render_info;

/* Stages timed by the optional profiler (ms_profile_enable). */
typedef enum {
    MS_STAGE_MESH_BUILD = 0,
    MS_STAGE_BIN = 1,
    MS_STAGE_SORT = 2,
    MS_STAGE_RASTER = 3,          /* count, pixel scan, fill and resolve of the forward */
    MS_STAGE_RASTER_BWD = 4,      /* fill, adjoint resolve and gradient scatter */
    MS_STAGE_LOSS = 5,
    MS_STAGE_ADAM = 6,
    MS_STAGE_MLP = 7,             /* learned initializer inference */
    MS_STAGE_COUNT = 8
} ms_stage;

MS_API const char *ms_version(void);
/* Message of the last host-side error of this thread (static storage). */
MS_API const char *ms_last_error(void);
/* Fills the defaults (tile 16, kbuf 8, T_eps 1e-5, black background, capacities 0, depth bits 0 = automatic,
 * no face mask). */
MS_API void ms_render_params_default(ms_render_params *p);

/*
 * Gaussians -> fan soup (Sec. 3, "MeshSplats Transformation for Flat Gaussians": Eq. 2
 * a = scale_mul exp(s_a) r_a, b = scale_mul exp(s_b) r_b; v_0 = m,
 * v_{1+i} = m + cos(theta_i) a + sin(theta_i) b with theta_i = -pi + 2 pi i / K; every
 * vertex gets the Gaussian's colour; centre opacity sigma, boundary opacity
 * opac_mul sigma).
 *   means, log_scales: N x 3 f32; quats: N x 4 f32 (w,x,y,z), normalised here;
 *   opacity: N f32 (activated); sh: N x (deg+1)^2 x 3, f32 (sh_dtype 0) or bf16 (1);
 *   colour = max(0, 0.5 + sum_lm Y_lm(dir) f_lm), dir = normalize(m - cam_center), real SH
 *   basis of degree <= 3; cam_center (host, 3 floats) NULL -> degree 0 only.
 *   corr: NULL or device N x 2(K+1) f32: radial (first K+1, centre entry unused) and
 *   log-opacity corrections: v_{1+i} = m + (1 + corr_r) (...), alpha = clamp(alpha exp(corr_o), 0, 1).
 *   Outputs (device): xyz, rgb (V x 3), alpha (V), V = N (K+1).
 * All inputs and outputs are device memory.
 */
MS_API ms_status ms_mesh_build(const float *means, const float *log_scales, const float *quats,
                               const float *opacity, const void *sh, int32_t sh_dtype, int32_t sh_degree,
                               int64_t N, const ms_fan_params *fan, const float *cam_center,
                               const float *corr, float *xyz, float *rgb, float *alpha, void *stream);

/*
 * Three-fan conversion of 3D Gaussians (Sec. 3 "Transformation for 3D Gaussians"): all
 * three scaled axes sr_c = scale_mul exp(s_c) r_c are kept and each Gaussian becomes one
 * fan of K triangles per pair of axes, (1, 2), (1, 3), (2, 3), with the angles, colour
 * and opacity rules of ms_mesh_build (fan->axis_rule is ignored; no corrections).  The
 * fans meet at the centre and at the axis tips m +- sr_c that two fans both reach; the
 * output keeps the implicit fan layout the renderer takes, so those shared vertices appear
 * once in every fan that uses them (quarter-turn angles use exact cosine and sine, so the
 * copies are equal bit for bit).
 *   xyz, rgb, alpha: device, 3 N (K + 1) vertices: fan 3g + f of Gaussian g is vertices
 *   (3g + f)(K + 1) .. + K, centre first.  Render them as 3 N fans of K triangles.
 * Other arguments and errors as ms_mesh_build.
 */
/*
 * Copy map of the three-fan layout of ms_mesh_build_3d (host only, no device work): for
 * each of the 3 (K + 1) vertex slots of one Gaussian (fan f, vertex k at slot f (K + 1) + k)
 * writes to first_copy the slot of the first copy of the same vertex (a slot that is its
 * own first copy maps to itself; the centre of every fan maps to slot 0).  Summing the
 * gradients of a vertex's copies and giving every copy the sum keeps the copies equal
 * under a fine-tune.  Returns the number of distinct vertices per Gaussian (19 for
 * K = 8), or -1 for K outside 3..16 or a NULL pointer.
 */
MS_API int32_t ms_three_fan_copies(int32_t K, int32_t *first_copy);

/*
 * Gradients of the shared vertices of a three-fan soup (Sec. 3 "Transformation for 3D
 * Gaussians": the three fans of a Gaussian share the centre and the axis tips two fans
 * reach, i.e. one vertex appears as several copies in the implicit layout of
 * ms_mesh_build_3d).  For every Gaussian, each vertex slot receives the sum of the
 * gradients of all copies of its vertex (the gradient of the shared vertex), summed in slot
 * order, so every copy holds the same value and an optimiser step keeps the copies equal.
 *   Either grad (device, 16-byte aligned: the gradient sums ms_render_backward leaves in a
 *   render workspace, at ms_render_grad_offset; two float4 per vertex) or, when grad is
 *   NULL, d_xyz, d_rgb (3 N (K+1) x 3) and d_alpha (3 N (K+1)): device, updated in place.
 * One kernel launch on `stream`; MS_ERR_INVALID for K outside 3..16, N < 0 or NULL arrays.
 */
MS_API ms_status ms_three_fan_sum_copies(float *d_xyz, float *d_rgb, float *d_alpha, void *grad, int64_t N,
                                         int32_t K, void *stream);

MS_API ms_status ms_mesh_build_3d(const float *means, const float *log_scales, const float *quats,
                                  const float *opacity, const void *sh, int32_t sh_dtype, int32_t sh_degree, int64_t N,
                                  const ms_fan_params *fan, const float *cam_center, float *xyz, float *rgb,
                                  float *alpha, void *stream);

/*
 * Explicit triangles (the renderer's `tris` input; Sec. 3 renders meshes whose triangles
 * need not form fans: the three-fan conversion's shared vertices, the mesh prior's
 * secondary triangles).  Each triangle (v1, v2, v3) is drawn as a fan of K = 3 around its
 * centroid c, whose position, colour and opacity are the binary32 values nearest the exact
 * means of the vertices': the three sub-triangles (c, v_i, v_i+1) tile the triangle and an
 * attribute that is affine on the triangle interpolates to the same values on them.
 *   ms_tris_to_fans: xyz, rgb (V x 3), alpha (V) device vertex arrays; tris: device T x 3
 *     int32 vertex indices, or NULL for a triangle soup (triangle t = vertices 3t, 3t+1,
 *     3t+2); writes the fan soup fan_xyz, fan_rgb (4T x 3), fan_alpha (4T): fan t is
 *     vertices 4t (centroid), 4t+1 .. 4t+3.
 *   ms_fans_to_tris_grads: the adjoint, ADDED to d_xyz, d_rgb, d_alpha (V arrays, caller
 *     zeroes) with atomics: vertex k of triangle t receives fan vertex 4t+1+k's gradient and
 *     a third of the centroid's.  The fan gradients come from three arrays (4T) or, when
 *     grad_ws is non-NULL, from the sums a render backward left in its workspace
 *     (ms_render_grad_offset; 16-byte aligned).
 *   ms_mesh_render / ms_mesh_render_backward: the two steps around ms_render /
 *     ms_render_backward (T fans of K = 3) in one workspace of ms_mesh_workspace_size bytes
 *     (256-byte aligned; it holds the fan soup, then the render workspace).  Gradients are
 *     added to the vertex arrays.  Errors as ms_render, MS_ERR_INVALID for T >= 2^29.
 */
MS_API ms_status ms_tris_to_fans(const float *xyz, const float *rgb, const float *alpha, const int32_t *tris,
                                 int64_t T, float *fan_xyz, float *fan_rgb, float *fan_alpha, void *stream);
MS_API ms_status ms_fans_to_tris_grads(const float *g_fan_xyz, const float *g_fan_rgb, const float *g_fan_alpha,
                                       const void *grad_ws, const int32_t *tris, int64_t T, float *d_xyz,
                                       float *d_rgb, float *d_alpha, void *stream);
MS_API size_t ms_mesh_workspace_size(int64_t T, const ms_camera *cam, const ms_render_params *params);
MS_API ms_status ms_mesh_render(const float *xyz, const float *rgb, const float *alpha, const int32_t *tris, int64_t T,
                                const ms_camera *cam, const ms_render_params *params, float *out_rgba,
                                void *workspace, size_t ws_bytes, void *stream);
MS_API ms_status ms_mesh_render_backward(const float *xyz, const float *rgb, const float *alpha, const int32_t *tris,
                                         int64_t T, const ms_camera *cam, const ms_render_params *params,
                                         const float *out_rgba, const float *dL_drgba, float *d_xyz, float *d_rgb,
                                         float *d_alpha, void *workspace, size_t ws_bytes, void *stream);

/*
 * Mesh-prior mode (Sec. 3, the mesh-prior paragraphs): every face (m1, m2, m3) of a
 * geometry mesh carries S secondary triangles whose vertices are convex combinations
 * v_i = sum_k a_ik m_k of the face's corners, with a_ik = w_ik^2 / sum_j w_ij^2 of free
 * weights w (so a_i stays on the simplex), and per-vertex colour and opacity.
 *   faces: device F x 3 corners x 3 floats; w: device F x S x 3 vertices x 3 corners;
 *   rgb: device F x S x 3 x 3; alpha: device F x S x 3.
 *   ms_mesh_prior_build writes the secondary triangles as centroid fans (as
 *     ms_tris_to_fans: fan_xyz, fan_rgb 4FS x 3, fan_alpha 4FS), ready for ms_render with
 *     K = 3.
 *   ms_mesh_prior_backward ADDS to d_w (shape of w), d_rgb, d_alpha the gradients given
 *     the fan soup's (three arrays, or grad_ws as in ms_fans_to_tris_grads): the centroid's
 *     share goes a third to each vertex, then dL/da_ik = dL/dv_i . m_k and
 *     dL/dw_ij = (2 w_ij / Q_i)(dL/da_ij - sum_k a_ik dL/da_ik), Q_i = sum_j w_ij^2.
 *     (A vertex whose weights are all zero has no defined simplex point; callers keep w
 *     away from 0.)
 */
MS_API ms_status ms_mesh_prior_build(const float *faces, const float *w, const float *rgb, const float *alpha,
                                     int64_t F, int32_t S, float *fan_xyz, float *fan_rgb, float *fan_alpha,
                                     void *stream);
MS_API ms_status ms_mesh_prior_backward(const float *faces, const float *w, const float *g_fan_xyz,
                                        const float *g_fan_rgb, const float *g_fan_alpha, const void *grad_ws,
                                        int64_t F, int32_t S, float *d_w, float *d_rgb, float *d_alpha, void *stream);

/*
 * Ray tracing of the triangle soup with shadows (the motivation of Sec. 1: a mesh of
 * triangles is what ray tracers take, with secondary effects such as shadows; the paper
 * gives no shading model, so this one is stated here).  Primary rays: the pixel-centre ray
 * C + t d of the pinhole camera with d of unit view depth; every triangle crossed at
 * t > znear is a fragment with the ray's barycentrics (the rasteriser's perspective-correct
 * ones), ordered by t, ties by triangle index, composited front to back as ms_render does
 * (C += T a c, T *= 1 - a; out = (C + T bg, 1 - T)), stopping once T < T_eps (0: never).
 * Shadows (light non-NULL and ambient < 1): a point light L; the fragment at p takes the
 * product S of (1 - a_g) over every other triangle g crossed by the segment p -> L at a
 * segment parameter in (1e-9, 1 - 1e-9), and its colour becomes c (ambient + (1 - ambient) S);
 * a shadow ray stops once S < T_eps (so the factor moves by at most (1 - ambient) T_eps).
 * Crossings are decided in FP64 (Moller-Trumbore, closed edges).
 *   Triangles: tris (device T x 3 int32) or, when NULL, the implicit fan topology of K
 *   triangles a fan (T = n_fans K); xyz, rgb (V x 3), alpha (V) device.
 *   ms_bvh_build: a linear BVH over the triangles into `bvh` (device, >=
 *   ms_bvh_workspace_size(T) bytes, 256-byte aligned); rebuild after the vertices move.
 *   ms_raytrace: out_rgba device H x W x 4 (16-byte aligned); light, bg: host 3 floats
 *   (bg NULL = black).  Traversal stacks are bounded; ms_bvh_status synchronises the
 *   stream and returns MS_ERR_CAPACITY (with the count) if a traversal overflowed its stack.
 */
MS_API size_t ms_bvh_workspace_size(int64_t T);
MS_API ms_status ms_bvh_build(const float *xyz, const int32_t *tris, int64_t T, int32_t K, void *bvh, size_t bvh_bytes,
                              void *stream);
MS_API ms_status ms_raytrace(const float *xyz, const float *rgb, const float *alpha, const int32_t *tris, int64_t T,
                             int32_t K, const void *bvh, const ms_camera *cam, const float *light, float ambient,
                             float T_eps, const float *bg, float *out_rgba, void *stream);
MS_API ms_status ms_bvh_status(const void *bvh, int32_t *stack_overflows, void *stream);

/*
 * Storage order of the Gaussians (no counterpart in the paper, whose render does not
 * depend on the order of its inputs except for exact depth ties, which go to the lower
 * triangle index).  ms_spatial_order writes the permutation perm (device int32, N entries)
 * that sorts the Gaussians by the Morton code of their means: each coordinate quantised to
 * 10 bits over the means' bounding box, q = min(max(floor((m - lo) / (hi - lo) * 1024), 0),
 * 1023) in binary32 (an axis of zero extent counts as 1), bits interleaved x, y, z from the
 * top; equal codes keep the input order.  Gaussians stored in that order (ms_gather_rows
 * on each attribute array, once, when a scene is loaded) put the fans that meet in one
 * screen tile near each other in memory, which the render's gathers and the adjoint's
 * gradient sums profit from.
 *   means: device N x 3; N < 2^31.  workspace: device, 256-byte aligned, at least
 *   ms_spatial_order_workspace_size(N) bytes (0 for an invalid N).  Kernel launches on `stream`
 *   only (the library's radix sort among them), no host synchronisation.
 * ms_gather_rows: dst row i = src row perm[i] for n_rows rows of row_bytes bytes (a multiple
 *   of 4; src and dst device, 4-byte aligned, not overlapping; perm device, every entry in
 *   0..n_rows-1, which the caller guarantees).  One kernel launch.
 * Errors: MS_ERR_INVALID for bad sizes, NULL or misaligned pointers.
 */
MS_API size_t ms_spatial_order_workspace_size(int64_t N);
MS_API ms_status ms_spatial_order(const float *means, int64_t N, int32_t *perm, void *workspace, size_t ws_bytes,
                                  void *stream);
MS_API ms_status ms_gather_rows(const void *src, int64_t n_rows, int64_t row_bytes, const int32_t *perm, void *dst,
                                void *stream);

/* Bytes of workspace ms_render / ms_render_backward need for n_fans fans of K triangles. */
MS_API size_t ms_render_workspace_size(int64_t n_fans, int32_t K, const ms_camera *cam,
                                       const ms_render_params *params);

/*
 * Forward render of an implicit-topology fan soup (see Conventions) with exact
 * per-pixel depth order (Sec. 3 "Rendering MeshSplats in Nvdiffrast": the
 * depth-peeled layers composited front to back, here with an unbounded layer count).
 *   xyz, rgb, alpha: device fan soup; n_fans fans of K (3..16) triangles.
 *   out_rgba: device H x W x 4.
 *   workspace: device, >= ms_render_workspace_size bytes, 256-byte aligned; it keeps
 *   the sorted tile lists and per-pixel transmittance that ms_render_backward reuses.
 * MS_ERR_INVALID for bad sizes or pointers, including 2^32 or more pixels over all views
 * of a call (pixel indices are 32-bit in the fragment records).
 * Returns once the work is queued; call ms_render_get_info for device-side errors.
 */
MS_API ms_status ms_render(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                           const ms_camera *cam, const ms_render_params *params, float *out_rgba,
                           void *workspace, size_t ws_bytes, void *stream);

/*
 * Adjoint of the last ms_render on this workspace (same scene, camera and params; the
 * scene must not have changed).  Replays the front-to-back traversal, recomputing
 * transmittance, and accumulates dL/dxyz, dL/drgb, dL/dalpha (device, +=) from dL/drgba
 * (device H x W x 4) and the forward output out_rgba.  Visibility (coverage and order)
 * is held fixed.  With d_xyz, d_rgb and d_alpha all NULL the gradients are left in the
 * workspace instead (see ms_render_grad_offset).
 */
MS_API ms_status ms_render_backward(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans,
                                    int32_t K, const ms_camera *cam, const ms_render_params *params,
                                    const float *out_rgba, const float *dL_drgba, float *d_xyz, float *d_rgb,
                                    float *d_alpha, void *workspace, size_t ws_bytes, void *stream);

/*
 * Byte offset, within a render workspace, of the gradient sums that ms_render_backward /
 * ms_batch_render_backward leave there when called with d_xyz = d_rgb = d_alpha = NULL:
 * per vertex two float4s, (dL/dxyz, dL/dalpha) and (dL/drgb, 0), overwritten by each call.
 * ms_adam_step_ws consumes them without a separate gradient array.  0 for an invalid
 * request.
 */
MS_API size_t ms_render_grad_offset(int64_t n_fans, int32_t K, const ms_camera *cams, int32_t n_views,
                                    const ms_render_params *params);

/* Synchronises the stream and reads the device-side outcome recorded in the workspace.
 * Returns MS_ERR_CAPACITY or MS_ERR_TIMEOUT when the last render (single or batch) on it
 * was invalid; the counters then cover all views of a batch together. */
MS_API ms_status ms_render_get_info(const void *workspace, ms_render_info *info, void *stream);

/* Largest number of views of one batch call. */
#define MS_MAX_VIEWS 32

/* Bytes of workspace ms_batch_render / ms_batch_render_backward need for n_views
 * (1..MS_MAX_VIEWS) cameras of any resolutions; 0 for an invalid request.
 * ms_batch_workspace_size(n, K, cam, 1, p) == ms_render_workspace_size(n, K, cam, p). */
MS_API size_t ms_batch_workspace_size(int64_t n_fans, int32_t K, const ms_camera *cams, int32_t n_views,
                                      const ms_render_params *params);

/*
 * Forward render of one fan soup into n_views images of (possibly) different sizes in
 * one pass of the pipeline: the tiles of all views form one index space, so binning,
 * the key sort, rasterisation and the per-pixel resolve each launch once for the whole
 * batch (the multi-view renders of fine-tuning, Sec. 3 "Fine-tuning", and of the
 * evaluation in Sec. 4).  Image v equals ms_render with cams[v] bit for bit.
 *   cams: host array of n_views cameras (read during the call only).
 *   out_rgba: host array of n_views device pointers, image v H_v x W_v x 4, 16-byte aligned.
 *   workspace: device, >= ms_batch_workspace_size bytes, 256-byte aligned.
 * The call does no host synchronisation and no allocation, so it can be captured in a
 * CUDA graph (the host arrays are copied into the kernel parameters at capture).
 */
MS_API ms_status ms_batch_render(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                                 const ms_camera *cams, int32_t n_views, const ms_render_params *params,
                                 float *const *out_rgba, void *workspace, size_t ws_bytes, void *stream);

/*
 * Adjoint of the last ms_batch_render on this workspace (same scene, cameras and params),
 * summed over all views into d_xyz, d_rgb, d_alpha (device, +=).  out_rgba and dL_drgba
 * are host arrays of n_views device images.
 */
MS_API ms_status ms_batch_render_backward(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans,
                                          int32_t K, const ms_camera *cams, int32_t n_views,
                                          const ms_render_params *params, const float *const *out_rgba,
                                          const float *const *dL_drgba, float *d_xyz, float *d_rgb, float *d_alpha,
                                          void *workspace, size_t ws_bytes, void *stream);

/*
 * Source-Gaussian render: the flat Gaussians themselves, drawn as truncated splats on
 * their planes and composited in depth order -- the image the fans approximate (the
 * Gaussian component of Sec. 3 with mean m, rotation R, scales S and opacity sigma in the
 * flat GaMeS form).  For pixel ray x = C + t d (d with unit camera z) meeting the plane of
 * the two kept unit axes u_a, u_b (axis_rule as in ms_fan_params) at local (u, v):
 * alpha = sigma exp(-(u^2/s_a^2 + v^2/s_b^2)/2), kept where (u/(2.7 s_a))^2 + (v/(2.7 s_b))^2
 * <= 1 (the ellipse the fan is inscribed in) and t > znear; colour rgb[g]; fragments of a
 * pixel ordered by (binary32 t, Gaussian index); compositing as in ms_render.  The hit
 * test runs in FP64.
 *   means N x 3, log_scales N x 3, quats N x 4 (w, x, y, z; 16-byte aligned), opacity N,
 *   rgb N x 3: device.  cams: host array of n_views cameras.  out_rgba: host array of
 *   n_views device images H_v x W_v x 4.  workspace >= ms_splat_workspace_size bytes.
 * Device-side outcome through ms_render_get_info.
 */
MS_API size_t ms_splat_workspace_size(int64_t N, const ms_camera *cams, int32_t n_views,
                                      const ms_render_params *params);
MS_API ms_status ms_splat_render(const float *means, const float *log_scales, const float *quats,
                                 const float *opacity, const float *rgb, int64_t N, int32_t axis_rule,
                                 const ms_camera *cams, int32_t n_views, const ms_render_params *params,
                                 float *const *out_rgba, void *workspace, size_t ws_bytes, void *stream);

/*
 * Learned fan initializer (the project's addition standing in for part of the
 * fine-tuning of Sec. 3 "Fine-tuning": vertex positions and opacities are optimised
 * after the conversion).  A perceptron 16 -> 128 -> 128 -> n_out (n_out = 2 (K+1) <= 32)
 * with exact GELU after the hidden layers, run on the tensor cores (tcgen05.mma, BF16
 * operands, FP32 accumulation).  Inputs per Gaussian: log-scales (3), normalised
 * quaternion (4), opacity (1), degree-0 SH (3), scales sorted descending over the largest
 * (3), log(s_min / s_mid) (1), constant 1.  Outputs: radial corrections dr_0..dr_K then
 * log-opacity corrections do_0..do_K, the `corr` input of ms_mesh_build.
 * Weights: FP32 masters W1 (16 x 128), W2 (128 x 128), W3 (128 x n_out), row-major, and a
 * packed bf16 copy (device, ms_mlp_packed_bytes(), 256-byte aligned, zeroed before first
 * use: its tail counts expired tensor-core waits, read by ms_mlp_status).
 */
MS_API size_t ms_mlp_packed_bytes(void);
MS_API ms_status ms_mlp_pack(const float *W1, const float *W2, const float *W3, int32_t n_out, void *packed,
                             void *stream);
/* X: device N x 16 FP32 inputs. */
MS_API ms_status ms_mlp_features(const float *log_scales, const float *quats, const float *opacity, const void *sh,
                                 int32_t sh_dtype, int32_t sh_degree, int64_t N, float *X, void *stream);
/* corr: device N x n_out FP32 (inputs computed in the kernel from the Gaussians). */
MS_API ms_status ms_mlp_forward(const float *log_scales, const float *quats, const float *opacity, const void *sh,
                                int32_t sh_dtype, int32_t sh_degree, int64_t N, const void *packed, int32_t n_out,
                                float *corr, void *stream);
/* The conversion of ms_mesh_build (flat fans) fused behind the inference: one kernel runs
 * the perceptron on each 128-Gaussian tile and converts the tile's Gaussians with their
 * corrections taken from on-chip registers, so the N x 2(K+1) corrections never reach device
 * memory.  The result equals ms_mlp_forward followed by ms_mesh_build with corr bit for bit.
 * packed: weights packed with n_out = 2(K+1) (K <= 15); other arguments as ms_mesh_build.
 * Errors: MS_ERR_INVALID for NULL or misaligned pointers, K outside 3..15. */
MS_API ms_status ms_mesh_build_mlp(const float *means, const float *log_scales, const float *quats,
                                   const float *opacity, const void *sh, int32_t sh_dtype, int32_t sh_degree, int64_t N,
                                   const ms_fan_params *fan, const float *cam_center, const void *packed, float *xyz,
                                   float *rgb, float *alpha, void *stream);
/* Training: mean squared error of the outputs for inputs X (n x 16) against targets T
 * (n x n_out).  ms_mlp_grads overwrites grads (device FP32, the sizes of W1, W2, W3 in that
 * order) and *loss (device).  ms_mlp_adam updates the masters W (same flat order) with
 * Adam at step *d_step + 1, advances *d_step and repacks. */
MS_API size_t ms_mlp_train_workspace_size(int64_t n);
MS_API ms_status ms_mlp_grads(const float *X, const float *T, int64_t n, int32_t n_out, const void *packed,
                              float *grads, float *loss, void *workspace, size_t ws_bytes, void *stream);
MS_API ms_status ms_mlp_adam(float *W, const float *grads, float *m, float *v, int32_t n_out, int32_t *d_step,
                             float lr, float beta1, float beta2, float eps, void *packed, void *stream);
/* Synchronises and reads the expired-wait counter: MS_ERR_TIMEOUT if non-zero. */
MS_API ms_status ms_mlp_status(const void *packed, int32_t *timeouts, void *stream);

/* Mean over n_pixels x RGB of (img - target)^2 into *out (device float, overwritten);
 * PSNR = -10 log10(*out) for images in [0, 1]. */
MS_API ms_status ms_mse(const float *img_rgba, const float *target_rgba, int64_t n_pixels, float *out, void *stream);

/* Training targets of the learned initializer from one fine-tune: the corrections (the
 * corr layout of ms_mesh_build, N x 2(K+1)) that map the converted soup (xyz0, alpha0)
 * to the fine-tuned one (xyz1, alpha1): dr_i = <o1_i, o0_i> / |o0_i|^2 - 1 with o the
 * boundary offsets from the original centre (dr_0 = 0), do_k = log(alpha1_k / alpha0_k)
 * (0 where either is 0).  All device arrays. */
MS_API ms_status ms_fan_corrections(const float *xyz0, const float *alpha0, const float *xyz1, const float *alpha1,
                                    int64_t N, int32_t K, float *corr, void *stream);

/* Candidates the autotuner times: tile in {8, 16, 32} x kbuf in {8, 16}. */
#define MS_TUNE_CANDIDATES 6

typedef struct {
    /* per candidate c (tile = 8 << (c / 2), kbuf = 8 << (c % 2)): median milliseconds of one
     * forward+backward batch step, or -2 workspace too small,
     * -3 capacity did not settle */
    float cand_ms[MS_TUNE_CANDIDATES];
    size_t cand_ws_bytes[MS_TUNE_CANDIDATES];   /* workspace each candidate needs (0 if unknown) */
    int32_t best;                               /* index of the chosen candidate, -1 if none */
    float best_ms;
    int64_t pairs, frags;                       /* measured list lengths of the chosen candidate */
} ms_tune_result;

/*
 * Autotuner of the batch render (no counterpart in the paper, whose renderer has fixed
 * settings).  For every candidate (tile edge, per-pixel buffer) it renders once to
 * measure the (tile, fan) pair list and the fragment-record list, sets both capacities
 * to the measured length times (1 + headroom) (headroom >= 0; the "list capacity" of the
 * batch), then times `reps` (>= 1) forward+backward batch steps with CUDA events and
 * keeps the median.  *best receives `base` with the fastest candidate's tile, kbuf and
 * capacities.  Candidates whose workspace exceeds ws_bytes are skipped and report their
 * size in res->cand_ws_bytes.  out_rgba / dL_drgba as in ms_batch_render(_backward);
 * d_xyz, d_rgb, d_alpha are overwritten with scratch values.  This call synchronises the
 * stream (it reads list lengths and event times on the host), so run it before any graph
 * capture.  Returns MS_ERR_CAPACITY if no candidate fits the workspace.
 */
MS_API ms_status ms_batch_autotune(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                                   const ms_camera *cams, int32_t n_views, const ms_render_params *base,
                                   float *const *out_rgba, const float *const *dL_drgba, float *d_xyz, float *d_rgb,
                                   float *d_alpha, void *workspace, size_t ws_bytes, int32_t reps, float headroom,
                                   ms_render_params *best, ms_tune_result *res, void *stream);

/*
 * L1 term of Eq. 3: loss = mean over H x W x 3 of |C - C*|.  img_rgba: device H x W x 4;
 * target_rgba: device H x W x 4 (alpha ignored).  Writes dL_drgba (device H x W x 4,
 * alpha gradient 0) and loss (device, 1 float; overwritten).
 */
MS_API ms_status ms_l1_loss(const float *img_rgba, const float *target_rgba, int64_t n_pixels,
                            float *dL_drgba, float *loss, void *stream);

/*
 * Full fine-tuning loss of Eq. 3 (Sec. 3 "Loss Function"), read as
 *   loss = lambda L1 + (1 - lambda)(1 - SSIM),  lambda = 0.6 in the paper,
 * with L1 = mean |C - C*| and SSIM the mean over the pixels and the three colour channels
 * of the local structural similarity under an 11 x 11 Gaussian window (sigma 1.5, zero
 * padding outside the image, C1 = 0.01^2, C2 = 0.03^2).  (The equation as printed adds
 * SSIM itself; the text says the loss follows 3DGS, whose SSIM term is 1 - SSIM.)
 *   img_rgba, target_rgba: device height x width x 4 floats, 16-byte aligned (alpha
 *     ignored).
 *   dL_drgba: device height x width x 4, written (alpha gradient 0).
 *   loss: device, 1 float, overwritten.
 *   workspace: device scratch of ms_fine_tune_loss_workspace_size bytes (any alignment);
 *     its contents need not be initialised and are not kept.
 * MS_ERR_INVALID for a size outside 0..32768, lambda outside [0, 1], NULL or misaligned
 * pointers or a short workspace.  Two kernel launches on `stream`.
 */
MS_API size_t ms_fine_tune_loss_workspace_size(int32_t height, int32_t width);
MS_API ms_status ms_fine_tune_loss(const float *img_rgba, const float *target_rgba, int32_t height, int32_t width,
                                   float lambda, float *dL_drgba, float *loss, void *workspace, size_t ws_bytes,
                                   void *stream);

/*
 * Pruning step of Sec. 3 ("Optimization and Pruning"): a face goes when all three of its
 * vertex opacities are below `threshold` (exp(-4) in the paper), and vertices no face
 * uses any more go with it.  With the implicit fan layout this is applied per fan: a fan
 * whose faces all go -- exactly when all K + 1 of its vertex opacities are below the
 * threshold -- is removed; every other fan is kept whole.  (A fan whose centre is below
 * the threshold but some boundary vertex is not keeps the faces that Sec. 3 would drop
 * between two dim boundary vertices.)  Kept fans are compacted in their order.
 *   xyz, rgb, alpha: device soup of n_fans fans of K triangles (read only).
 *   m, v: optional device Adam moments in the ms_adam_step layout [xyz 3V | rgb 3V |
 *     alpha V], compacted with the soup; NULL together with m_out / v_out to skip.
 *   *_out: device arrays of the input sizes (the kept soup fills their front); they must
 *     not overlap the inputs.
 *   n_kept: device int64, written with the number of kept fans.
 *   workspace: device scratch of ms_prune_workspace_size bytes (any alignment).
 * Three kernel launches on `stream`.
 */
MS_API size_t ms_prune_workspace_size(int64_t n_fans);
/*
 * The pruning step of Sec. 3 per face: bit j of a fan's face mask (face (c, b_j, b_j+1),
 * the face_mask of ms_render_params) stays set while some vertex of the face has opacity
 * at or above `threshold`, ANDed with the fan's earlier mask (face_mask_in, device, one
 * word per fan; NULL = all faces).  Fans left with no face are removed with their K + 1
 * vertices (with no earlier mask, exactly the fans ms_prune_fans removes); the others are
 * kept whole and compacted in order, and face_mask_out (device, one word per input fan,
 * the kept fans' masks at its front; NULL to skip) receives their masks.  Other arguments,
 * workspace and errors as ms_prune_fans.
 */
MS_API ms_status ms_prune_faces(const float *xyz, const float *rgb, const float *alpha, const float *m,
                                const float *v, const uint32_t *face_mask_in, int64_t n_fans, int32_t K,
                                float threshold, float *xyz_out, float *rgb_out, float *alpha_out, float *m_out,
                                float *v_out, uint32_t *face_mask_out, int64_t *n_kept, void *workspace,
                                size_t ws_bytes, void *stream);
MS_API ms_status ms_prune_fans(const float *xyz, const float *rgb, const float *alpha, const float *m, const float *v,
                               int64_t n_fans, int32_t K, float threshold, float *xyz_out, float *rgb_out,
                               float *alpha_out, float *m_out, float *v_out, int64_t *n_kept, void *workspace,
                               size_t ws_bytes, void *stream);

/*
 * Adam step on the fan soup (Sec. 3 "Optimization and Pruning": colours and opacities at
 * lr_color, positions at lr_xyz = exp(-3) lr_color).  Parameters and gradients are
 * device SoA arrays of V vertices; m, v: device moments, 7 V floats each laid out like the
 * parameters ([xyz 3V | rgb 3V | alpha V]), zeroed before step 1.  step counts from 1.
 * Opacity is clamped to [0, 1].
 */
MS_API ms_status ms_adam_step(float *xyz, float *rgb, float *alpha, const float *d_xyz, const float *d_rgb,
                              const float *d_alpha, float *m, float *v, int64_t V, int32_t step,
                              float lr_color, float lr_xyz, float beta1, float beta2, float eps, void *stream);

/*
 * ms_adam_step reading the gradients from a render workspace (grad = workspace +
 * ms_render_grad_offset(...), device, 16-byte aligned; layout as stated there).  With
 * d_step non-NULL the step number is kept on the device as in ms_adam_step_counted and
 * `step` is ignored.
 */
MS_API ms_status ms_adam_step_ws(float *xyz, float *rgb, float *alpha, const void *grad, float *m, float *v,
                                 int64_t V, int32_t step, int32_t *d_step, float lr_color, float lr_xyz, float beta1,
                                 float beta2, float eps, void *stream);

/*
 * ms_adam_step with the step number kept on the device: *d_step (device int32, 0 before
 * the first step) is advanced by one on the stream and the bias corrections use the new
 * value.  A captured CUDA graph of a fine-tune step therefore replays with the right
 * step number on every launch.
 */
MS_API ms_status ms_adam_step_counted(float *xyz, float *rgb, float *alpha, const float *d_xyz, const float *d_rgb,
                                      const float *d_alpha, float *m, float *v, int64_t V, int32_t *d_step,
                                      float lr_color, float lr_xyz, float beta1, float beta2, float eps,
                                      void *stream);

/*
 * Forward render without a caller workspace.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- a plugin whose host
 * application owns the GPU memory budget and hands out no allocations, or a service that
 * reserves all of its device memory at start-up and forbids allocation afterwards.  It
 * behaves like
 * ms_render (same inputs, output, camera and params; everything in device memory owned
 * by the caller) but its scratch is a 64 MiB file-scope device array inside the library,
 * held by every GPU that loads the library until the process exits.  Renders whose
 * workspace (ms_render_workspace_size) exceeds 64 MiB are rejected with MS_ERR_INVALID
 * and a message naming both sizes.  The first call on a device looks up the array's
 * device address with that device current; make it before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU race.  The call waits for
 * the stream, then reports device-side errors like ms_render_get_info and fills *info
 * (optional).  It allocates nothing.
 */
MS_API ms_status ms_render_noalloc(const float *xyz, const float *rgb, const float *alpha, int64_t n_fans, int32_t K,
                                   const ms_camera *cam, const ms_render_params *params, float *out_rgba,
                                   ms_render_info *info, void *stream);

/*
 * Optional stage profiler (host-side instrumentation, not part of the method).  While
 * enabled, every entry point records a CUDA event pair around each of its stages on
 * the caller's stream.  ms_profile_read waits for those events, writes the summed
 * milliseconds and the number of timed launches per stage (arrays of n entries,
 * n <= MS_STAGE_COUNT) and clears the record.  Not thread-safe.
 */
MS_API void ms_profile_enable(int32_t on);
MS_API ms_status ms_profile_read(double *ms_per_stage, int64_t *launches_per_stage, int32_t n);

/* Number of CUDA kernels this library has launched in this process. */
MS_API int64_t ms_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif
