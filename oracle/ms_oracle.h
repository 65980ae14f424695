/*
 * MeshSplats plain CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load this
 * library.  It shares no code, header or constant with the CUDA library: it is an
 * independent, slow, direct statement of what the method computes.
 *
 * Precision.  Every value (fan geometry, SH colour, barycentrics, interpolated
 * attributes, compositing, gradients) is computed in FP64 from exactly widened
 * FP32/BF16 inputs.  The two discrete decisions of the renderer -- whether a pixel
 * centre is covered by a triangle, and the front-to-back order of the fragments of
 * a pixel -- are taken in one of three ways (`decide`): 1, the plain definition in
 * FP64; 0, both in IEEE FP32 by the formulas written out in ms_oracle.c (section
 * "Decisions"); 2, coverage by those binary32 edge formulas on the vertices' FP64
 * projections rounded to binary32, and the order by the FP64 depth (the split the
 * library's header states for its kernels), so that both sides can take each decision
 * in the same precision.  Comparing the modes pixel by pixel measures what
 * deciding in binary32 changes.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R_cw[9];   /* row-major world->camera rotation, rows = camera x (right), y (down), z (forward) */
    float C[3];      /* camera centre in world coordinates */
    float znear;
} orc_camera;

/* Number of worker threads the last parallel call used. */
int orc_last_threads(void);

/* Unit quaternion (w,x,y,z), normalised first -> row-major 3x3 rotation R; columns r1,r2,r3. */
void orc_quat_to_rot(const double q[4], double R[9]);

/* Real spherical-harmonic basis of degree <= 3 at unit direction d; writes (deg+1)^2 values. */
int orc_sh_basis(int degree, const double d[3], double *Y);

/* Projection of one world point: decided binary32 (xs, ys, Z, valid) and FP64 (xs, ys, Z). */
void orc_project(const orc_camera *cam, const double p[3], float dec[4], double val[3]);

/* Fan topology: triangle g*K+j = (g(K+1), g(K+1)+1+j, g(K+1)+1+((j+1) mod K)). */
void orc_fan_tris(int64_t N, int32_t K, int32_t *tris);

/*
 * Conversion of Gaussians into triangle fans (Sec. 3 "MeshSplats Transformation for
 * Flat Gaussians", Eq. 2 and the vertex equation that follows it).
 *   sh_dtype 0: float32 coefficients, 1: bfloat16 bits (uint16); layout N x (deg+1)^2 x 3.
 *   axis_rule 0: drop axis 0 (the epsilon axis of GaMeS); 1: drop the axis of smallest scale.
 *   cam_center NULL: colour from the degree-0 coefficient only.
 *   corr NULL or N x 2(K+1): per-vertex radial (first K+1) and log-opacity (next K+1) corrections.
 * Outputs: xyz, rgb (N(K+1) x 3), alpha (N(K+1)).  Returns 0 on success.
 */
int orc_mesh_build(int64_t N, const float *means, const float *log_scales, const float *quats,
                   const float *opacity, const void *sh, int sh_dtype, int sh_degree,
                   int K, double scale_mul, double opac_mul, int axis_rule,
                   const float *cam_center, const double *corr,
                   double *xyz, double *rgb, double *alpha);

/*
 * Render (Sec. 3 "Rendering MeshSplats in Nvdiffrast" and "Fine-tuning": MVP
 * transform, rasterisation with exact per-pixel depth order, interpolation of vertex
 * colour and opacity, front-to-back alpha blending).
 * The window [x0,x1) x [y0,y1) of the image is rendered; out_rgba is
 * (y1-y0) x (x1-x0) x 4, row-major, RGB then alpha.  brute=1 tests every pixel of the
 * window against every triangle; brute=0 first restricts each triangle to its
 * screen bounding box widened by 2 pixels.  nthreads 0 = all online cores.
 * out_nfrag (optional): fragments per pixel.  n_culled (optional): triangles with a
 * vertex at or behind the near plane or outside the guard band.
 */
int orc_render(int64_t V, const double *xyz, const double *rgb, const double *alpha,
               int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
               int x0, int y0, int x1, int y1, int brute, int nthreads,
               double *out_rgba, int32_t *out_nfrag, int64_t *n_culled);

/*
 * orc_render with the decisions chosen (decide: 0 binary32, 1 FP64, 2 binary32 coverage
 * and FP64 order; any other value returns 4) and, when
 * out_sig is non-NULL, a 64-bit FNV-1a hash per pixel of its ordered list of triangle ids
 * (the pixel's decisions: equal hashes mean the same fragments in the same order).
 */
int orc_render_ex(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                  int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                  int x0, int y0, int x1, int y1, int brute, int nthreads, int decide,
                  double *out_rgba, int32_t *out_nfrag, uint64_t *out_sig, int64_t *n_culled);

/*
 * Exact reverse pass of orc_render over the full fragment lists (no early
 * termination).  dL_drgba has the window's shape; gradients ACCUMULATE into
 * d_xyz (V x 3), d_rgb (V x 3), d_alpha (V).  Coverage and order are held fixed.
 */
int orc_render_backward(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                        int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                        int x0, int y0, int x1, int y1, int nthreads,
                        const double *dL_drgba, double *d_xyz, double *d_rgb, double *d_alpha);

/* orc_render_backward with the decision precision chosen as in orc_render_ex. */
int orc_render_backward_ex(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                           int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                           int x0, int y0, int x1, int y1, int nthreads, int decide,
                           const double *dL_drgba, double *d_xyz, double *d_rgb, double *d_alpha);

/*
 * Source-Gaussian render (ms_oracle_splat.c): the scene's flat Gaussians drawn as
 * truncated Gaussian splats on their planes and composited in depth order -- the image
 * the fans approximate.  rgb: N x 3 colour per Gaussian.  trunc: truncation radius in
 * units of the scale (2.7, the fan's scale_mul).  Window and outputs as orc_render.
 */
int orc_splat_render(int64_t N, const float *means, const float *log_scales, const float *quats,
                     const float *opacity, const double *rgb, int axis_rule, double trunc,
                     const orc_camera *cam, const double bg[3], int x0, int y0, int x1, int y1,
                     int nthreads, double *out_rgba, int32_t *out_nfrag);

#ifdef __cplusplus
}
#endif
#endif
