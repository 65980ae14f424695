/*
 * MeshSplats plain CPU oracle -- TEST INFRASTRUCTURE ONLY (see ms_oracle.h).
 *
 * What it computes, and where the paper says so:
 *   - Gaussian record (m, R, S, sigma, c): Sec. 3, Eq. 1 and the GaMeS flat form
 *     S = diag(eps, s2, s3), R = [r1 r2 r3].
 *   - Fan conversion: Sec. 3 "MeshSplats Transformation for Flat Gaussians", Eq. 2
 *     (scaled axes = scale_mul * exp(s) * r), the boundary vertex equation
 *     v_i = m + cos(theta_i) a + sin(theta_i) b, the fan of no_triag triangles sharing the
 *     centre, per-vertex colour inherited from the Gaussian, centre opacity sigma and
 *     boundary opacity opac_mul * sigma.
 *   - Rendering: Sec. 3 "Rendering MeshSplats in Nvdiffrast" (MVP to clip space,
 *     depth-peeled layers, interpolation of vertex colours, blending through alpha)
 *     and "Fine-tuning" (the same render inside the optimisation loop).  Depth
 *     peeling with an unbounded number of layers composites every fragment of a
 *     pixel in depth order; this file does exactly that with a full sort.
 *
 * Readings where the paper is silent:
 *   angles theta_i = -pi + 2 pi i / K (K distinct angles in [-pi, pi));
 *   quaternion (w,x,y,z) normalised before use; s are log-scales;
 *   colour = max(0, 0.5 + sum_lm Y_lm(dir) f_lm), dir = normalize(m - camera centre);
 *   pinhole camera with OpenCV axes, pixel centres at (i+0.5, j+0.5), two-sided
 *   triangles, top-left fill rule, perspective-correct interpolation, non-premultiplied
 *   colours, C += T a c then T *= (1 - a), output RGB = C + T bg and alpha = 1 - T;
 *   triangles with a vertex at Z <= znear or beyond the +-2^17 px guard band are culled.
 *
 * Decisions.  Coverage and fragment order are taken in one of two precisions:
 *   binary32 (decide = 0): IEEE binary32 with round-to-nearest-even and no fused
 *     multiply-add (built with -ffp-contract=off), evaluating left to right exactly the
 *     expressions in decide_vertex(), tri_area2(), edge_canon(), oriented_edge() and
 *     frag_depth() below;
 *   FP64 (decide = 1): the plain definition in FP64 -- the FP64 projection of each
 *     vertex, the three edge functions with the top-left rule, and the fragment depth
 *     Z_f = 1 / sum_k (lambda_k / Z_k) -- in frag_depth64();
 *   mixed (decide = 2): culling on each vertex's FP64 projection rounded to binary32
 *     (round_vertex()); coverage by the binary32 formulas of tri_area2(), edge_canon(),
 *     oriented_edge() and frag_depth() applied to positions relative to an integer origin
 *     o = floor of the FP64 screen position of the triangle's first vertex (a fan's centre,
 *     shared by all of its triangles): each vertex at the binary32 rounding of its FP64
 *     position minus o, the pixel centre at (i + 0.5 - o.x, j + 0.5 - o.y) exactly; and the
 *     order by the FP64 depth of value_depth() -- the split the library's kernels implement.
 * The FP64 depth is clamped to the range of its triangle's vertex depths, where a covered
 * centre lies; the clamp acts only where rounding puts a decided centre just outside the
 * exact triangle.  Everything else is FP64 in every mode.
 */
#include "ms_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static int g_last_threads = 1;
int orc_last_threads(void) { return g_last_threads; }

static int resolve_threads(int n) {
    if (n > 0) return n;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* ------------------------------------------------------------------------------------ */
/* Rotation and spherical harmonics                                                     */
/* ------------------------------------------------------------------------------------ */

void orc_quat_to_rot(const double q_in[4], double R[9]) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/*
 * Real SH, bands l = 0..3, index l*l + (m + l).  Y_{l,m} = sqrt2 Im(Y_l^|m|) for m < 0,
 * Y_l^0 for m = 0, sqrt2 Re(Y_l^m) for m > 0, where Y_l^m is the complex harmonic with
 * the Condon-Shortley phase (the layout used by common Gaussian-splatting codes).
 * Written out as polynomials in the unit direction (x, y, z).
 */
int orc_sh_basis(int degree, const double d[3], double *Y) {
    const double PI = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    if (degree < 0 || degree > 3) return 1;
    Y[0] = 0.5 * sqrt(1.0 / PI);
    if (degree >= 1) {
        double c1 = sqrt(3.0 / (4.0 * PI));
        Y[1] = -c1 * y;
        Y[2] = c1 * z;
        Y[3] = -c1 * x;
    }
    if (degree >= 2) {
        double a = 0.5 * sqrt(15.0 / PI), b = 0.25 * sqrt(5.0 / PI), c = 0.25 * sqrt(15.0 / PI);
        Y[4] = a * x * y;
        Y[5] = -a * y * z;
        Y[6] = b * (2 * z * z - x * x - y * y);
        Y[7] = -a * x * z;
        Y[8] = c * (x * x - y * y);
    }
    if (degree >= 3) {
        double k33 = 0.125 * sqrt(70.0 / PI);   /* |m| = 3 */
        double k32 = 0.25 * sqrt(105.0 / PI);   /* |m| = 2 (times 2 for the xyz term) */
        double k31 = 0.125 * sqrt(42.0 / PI);   /* |m| = 1 */
        double k30 = 0.25 * sqrt(7.0 / PI);     /* m = 0 */
        double t = 4 * z * z - x * x - y * y;
        Y[9] = -k33 * y * (3 * x * x - y * y);
        Y[10] = 2 * k32 * x * y * z;
        Y[11] = -k31 * y * t;
        Y[12] = k30 * z * (2 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = -k31 * x * t;
        Y[14] = k32 * z * (x * x - y * y);
        Y[15] = -k33 * x * (x * x - 3 * y * y);
    }
    return 0;
}

static double sh_coef(const void *sh, int sh_dtype, int64_t idx) {
    if (sh_dtype == 0) return (double)((const float *)sh)[idx];
    uint32_t bits = ((uint32_t)((const uint16_t *)sh)[idx]) << 16;
    float f;
    memcpy(&f, &bits, 4);
    return (double)f;
}

/* ------------------------------------------------------------------------------------ */
/* Fan conversion                                                                       */
/* ------------------------------------------------------------------------------------ */

void orc_fan_tris(int64_t N, int32_t K, int32_t *tris) {
    for (int64_t g = 0; g < N; ++g)
        for (int32_t j = 0; j < K; ++j) {
            int64_t t = g * K + j, c = g * (K + 1);
            tris[3 * t + 0] = (int32_t)c;
            tris[3 * t + 1] = (int32_t)(c + 1 + j);
            tris[3 * t + 2] = (int32_t)(c + 1 + (j + 1) % K);
        }
}

int orc_mesh_build(int64_t N, const float *means, const float *log_scales, const float *quats,
                   const float *opacity, const void *sh, int sh_dtype, int sh_degree,
                   int K, double scale_mul, double opac_mul, int axis_rule,
                   const float *cam_center, const double *corr,
                   double *xyz, double *rgb, double *alpha) {
    const double PI = 3.14159265358979323846;
    if (K < 3 || sh_degree < 0 || sh_degree > 3) return 1;
    int nb = (sh_degree + 1) * (sh_degree + 1);
    for (int64_t g = 0; g < N; ++g) {
        double m[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
        double s[3] = {log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]};
        double q[4] = {quats[4 * g], quats[4 * g + 1], quats[4 * g + 2], quats[4 * g + 3]};
        double R[9];
        orc_quat_to_rot(q, R);
        /* The two kept axes: GaMeS drops the epsilon axis (axis 0); the general rule
         * drops the axis of smallest scale (ties: the lower index is dropped). */
        int drop = 0;
        if (axis_rule == 1) {
            if (s[1] < s[drop]) drop = 1;
            if (s[2] < s[drop]) drop = 2;
        }
        int ia = drop == 0 ? 1 : 0;
        int ib = drop == 2 ? 1 : 2;
        double a[3], b[3];
        for (int r = 0; r < 3; ++r) {
            a[r] = scale_mul * exp(s[ia]) * R[3 * r + ia];   /* scaled_rot_1 = scale_mul exp(s_2) r_2 */
            b[r] = scale_mul * exp(s[ib]) * R[3 * r + ib];   /* scaled_rot_2 = scale_mul exp(s_3) r_3 */
        }
        /* Colour: every vertex inherits the Gaussian's colour. */
        double col[3];
        double Y[16];
        int use_deg = 0;
        double dir[3] = {0, 0, 0};
        if (cam_center) {
            double dv[3] = {m[0] - cam_center[0], m[1] - cam_center[1], m[2] - cam_center[2]};
            double n = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            if (n > 0) {
                dir[0] = dv[0] / n; dir[1] = dv[1] / n; dir[2] = dv[2] / n;
                use_deg = sh_degree;
            }
        }
        orc_sh_basis(use_deg, dir, Y);
        int nuse = (use_deg + 1) * (use_deg + 1);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.5;
            for (int i = 0; i < nuse; ++i) acc += Y[i] * sh_coef(sh, sh_dtype, ((int64_t)g * nb + i) * 3 + ch);
            col[ch] = acc > 0 ? acc : 0;
        }
        double sig = opacity[g];
        const double *cr = corr ? corr + (int64_t)g * 2 * (K + 1) : 0;
        int64_t v0 = g * (K + 1);
        for (int k = 0; k <= K; ++k) {
            int64_t v = v0 + k;
            double op = k == 0 ? sig : opac_mul * sig;
            if (k == 0) {
                for (int r = 0; r < 3; ++r) xyz[3 * v + r] = m[r];
            } else {
                int i = k - 1;
                double th = -PI + 2.0 * PI * i / K;
                double rs = cr ? 1.0 + cr[k] : 1.0;
                for (int r = 0; r < 3; ++r) xyz[3 * v + r] = m[r] + rs * (cos(th) * a[r] + sin(th) * b[r]);
            }
            if (cr) {
                op = op * exp(cr[K + 1 + k]);
                op = op < 0 ? 0 : (op > 1 ? 1 : op);
            }
            alpha[v] = op;
            for (int ch = 0; ch < 3; ++ch) rgb[3 * v + ch] = col[ch];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Decisions (binary32, see the header comment)                                         */
/* ------------------------------------------------------------------------------------ */

#define GUARD_PX 131072.0f

typedef struct {
    float xs, ys, Z, iz;
    int valid;
} dvert;

static void decide_vertex(const orc_camera *cam, float px, float py, float pz, dvert *o) {
    const float *R = cam->R_cw;
    float dx = px - cam->C[0];
    float dy = py - cam->C[1];
    float dz = pz - cam->C[2];
    float X = (R[0] * dx + R[1] * dy) + R[2] * dz;
    float Y = (R[3] * dx + R[4] * dy) + R[5] * dz;
    float Z = (R[6] * dx + R[7] * dy) + R[8] * dz;
    float u = X / Z;
    float v = Y / Z;
    o->xs = cam->fx * u + cam->cx;
    o->ys = cam->fy * v + cam->cy;
    o->Z = Z;
    o->iz = 1.0f / Z;
    o->valid = (Z > cam->znear) && (fabsf(o->xs) <= GUARD_PX) && (fabsf(o->ys) <= GUARD_PX);
}

static float tri_area2(const dvert *A, const dvert *B, const dvert *C) {
    return (B->xs - A->xs) * (C->ys - A->ys) - (B->ys - A->ys) * (C->xs - A->xs);
}

/* Edge value of the unordered vertex pair, evaluated from the lower vertex index. */
static float edge_canon(const dvert *lo, const dvert *hi, float px, float py) {
    return (hi->xs - lo->xs) * (py - lo->ys) - (hi->ys - lo->ys) * (px - lo->xs);
}

/* Oriented edge u->v at pixel centre p: value (exact negation of the canonical value when
 * u has the higher index) and the top-left test on its direction. */
static int oriented_edge(const dvert *vu, int64_t iu, const dvert *vv, int64_t iv,
                         float px, float py, float *E) {
    float e, ex, ey;
    if (iu < iv) {
        e = edge_canon(vu, vv, px, py);
        ex = vv->xs - vu->xs;
        ey = vv->ys - vu->ys;
    } else {
        e = -edge_canon(vv, vu, px, py);
        ex = -(vu->xs - vv->xs);
        ey = -(vu->ys - vv->ys);
    }
    *E = e;
    return e > 0.0f || (e == 0.0f && (ey < 0.0f || (ey == 0.0f && ex > 0.0f)));
}

/* Coverage of pixel centre (px,py) by triangle (ids ia,ib,ic; decided vertices A,B,C),
 * given area2 = tri_area2(A,B,C) != 0; on coverage writes the fragment depth. */
static int frag_depth(const dvert *A, int64_t ia, const dvert *B, int64_t ib, const dvert *C, int64_t ic,
                      float area2, float px, float py, float *Zf) {
    const dvert *P0 = A, *P1 = B, *P2 = C;
    int64_t i0 = ia, i1 = ib, i2 = ic;
    if (area2 < 0.0f) {
        P1 = C; i1 = ic;
        P2 = B; i2 = ib;
        area2 = -area2;
    }
    float E0, E1, E2;
    if (!oriented_edge(P1, i1, P2, i2, px, py, &E0)) return 0;
    if (!oriented_edge(P2, i2, P0, i0, px, py, &E1)) return 0;
    if (!oriented_edge(P0, i0, P1, i1, px, py, &E2)) return 0;
    float w = (E0 * P0->iz + E1 * P1->iz) + E2 * P2->iz;
    float z = area2 / w;
    float zlo = fminf(fminf(A->Z, B->Z), C->Z);
    float zhi = fmaxf(fmaxf(A->Z, B->Z), C->Z);
    *Zf = fminf(fmaxf(z, zlo), zhi);
    return 1;
}

/* FP64 decisions: the same rules without the binary32 rounding.  A vertex is valid when
 * Z > znear and its FP64 screen position lies within the guard band; the edge value of a
 * vertex pair is evaluated from the lower vertex index and negated for the other
 * direction, so two triangles sharing an edge see exactly opposite values (watertight);
 * an edge passes when E > 0, or E == 0 and it is a top or left edge (direction with
 * ey < 0, or ey == 0 and ex > 0, in y-down screen space for the positively oriented
 * triangle); the depth is area2 / sum_k (E_k / Z_k) = 1 / sum_k (lambda_k / Z_k). */
typedef struct {
    double xs, ys, Z;
    int valid;
} dvert64;

static double tri_area2_64(const dvert64 *A, const dvert64 *B, const dvert64 *C) {
    return (B->xs - A->xs) * (C->ys - A->ys) - (B->ys - A->ys) * (C->xs - A->xs);
}

static int oriented_edge64(const dvert64 *vu, int64_t iu, const dvert64 *vv, int64_t iv,
                           double px, double py, double *E) {
    const dvert64 *lo = iu < iv ? vu : vv, *hi = iu < iv ? vv : vu;
    double e = (hi->xs - lo->xs) * (py - lo->ys) - (hi->ys - lo->ys) * (px - lo->xs);
    double ex = vv->xs - vu->xs, ey = vv->ys - vu->ys;
    if (!(iu < iv)) e = -e;
    *E = e;
    return e > 0.0 || (e == 0.0 && (ey < 0.0 || (ey == 0.0 && ex > 0.0)));
}

static int frag_depth64(const dvert64 *A, int64_t ia, const dvert64 *B, int64_t ib, const dvert64 *C,
                        int64_t ic, double area2, double px, double py, double *Zf) {
    const dvert64 *P0 = A, *P1 = B, *P2 = C;
    int64_t i0 = ia, i1 = ib, i2 = ic;
    if (area2 < 0.0) {
        P1 = C; i1 = ic;
        P2 = B; i2 = ib;
        area2 = -area2;
    }
    double E0, E1, E2;
    if (!oriented_edge64(P1, i1, P2, i2, px, py, &E0)) return 0;
    if (!oriented_edge64(P2, i2, P0, i0, px, py, &E1)) return 0;
    if (!oriented_edge64(P0, i0, P1, i1, px, py, &E2)) return 0;
    double z = area2 / (E0 / P0->Z + E1 / P1->Z + E2 / P2->Z);
    double zlo = fmin(fmin(A->Z, B->Z), C->Z), zhi = fmax(fmax(A->Z, B->Z), C->Z);
    *Zf = fmin(fmax(z, zlo), zhi);
    return 1;
}

/* ------------------------------------------------------------------------------------ */
/* Values (FP64)                                                                        */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double X, Y, Z, xs, ys;
} vvert;

static void value_vertex(const orc_camera *cam, const double *p, vvert *o) {
    double R[9], C[3];
    for (int i = 0; i < 9; ++i) R[i] = cam->R_cw[i];
    for (int i = 0; i < 3; ++i) C[i] = cam->C[i];
    double d[3] = {p[0] - C[0], p[1] - C[1], p[2] - C[2]};
    o->X = R[0] * d[0] + R[1] * d[1] + R[2] * d[2];
    o->Y = R[3] * d[0] + R[4] * d[1] + R[5] * d[2];
    o->Z = R[6] * d[0] + R[7] * d[1] + R[8] * d[2];
    o->xs = (double)cam->fx * o->X / o->Z + (double)cam->cx;
    o->ys = (double)cam->fy * o->Y / o->Z + (double)cam->cy;
}

/* Perspective-correct barycentrics of pixel centre p in triangle (A,B,C):
 * lambda_k = E_k / area (screen space), mu_k = (lambda_k / Z_k) / sum_j (lambda_j / Z_j). */
static void persp_bary(const vvert *A, const vvert *B, const vvert *C, double px, double py,
                       double E[3], double mu[3], double *Wsum) {
    E[0] = (C->xs - B->xs) * (py - B->ys) - (C->ys - B->ys) * (px - B->xs);
    E[1] = (A->xs - C->xs) * (py - C->ys) - (A->ys - C->ys) * (px - C->xs);
    E[2] = (B->xs - A->xs) * (py - A->ys) - (B->ys - A->ys) * (px - A->xs);
    double w0 = E[0] / A->Z, w1 = E[1] / B->Z, w2 = E[2] / C->Z;
    double W = w0 + w1 + w2;
    mu[0] = w0 / W;
    mu[1] = w1 / W;
    mu[2] = w2 / W;
    *Wsum = W;
}

/* FP64 depth of pixel centre p on triangle (A,B,C): 1 / sum_k (lambda_k / Z_k) with
 * lambda_k = E_k / area2 (orientation cancels), clamped to the vertices' depth range. */
static double value_depth(const vvert *A, const vvert *B, const vvert *C, double px, double py) {
    double E[3], mu[3], W;
    persp_bary(A, B, C, px, py, E, mu, &W);
    double z = (E[0] + E[1] + E[2]) / W;
    double zlo = fmin(fmin(A->Z, B->Z), C->Z), zhi = fmax(fmax(A->Z, B->Z), C->Z);
    return fmin(fmax(z, zlo), zhi);
}

/* Per-vertex projection as seen by the renderer: decided binary32 screen position and
 * depth (dec[4] = xs, ys, Z, valid) and the FP64 values (val[3] = xs, ys, Z). */
void orc_project(const orc_camera *cam, const double p[3], float dec[4], double val[3]) {
    dvert d;
    vvert v;
    decide_vertex(cam, (float)p[0], (float)p[1], (float)p[2], &d);
    value_vertex(cam, p, &v);
    dec[0] = d.xs; dec[1] = d.ys; dec[2] = d.Z; dec[3] = (float)d.valid;
    val[0] = v.xs; val[1] = v.ys; val[2] = v.Z;
}

/* ------------------------------------------------------------------------------------ */
/* Fragment collection                                                                  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int32_t pix;   /* index within the band */
    double z;      /* decided depth (a binary32 value in binary32 mode) */
    int64_t tri;
} frag;

typedef struct {
    frag *f;
    size_t n, cap;
} fragvec;

static int fv_push(fragvec *v, int32_t pix, double z, int64_t tri) {
    if (v->n == v->cap) {
        size_t nc = v->cap ? v->cap * 2 : 4096;
        frag *nf = (frag *)realloc(v->f, nc * sizeof(frag));
        if (!nf) return 1;
        v->f = nf;
        v->cap = nc;
    }
    v->f[v->n].pix = pix;
    v->f[v->n].z = z;
    v->f[v->n].tri = tri;
    v->n++;
    return 0;
}

/* Gradient contributions of one worker, (vertex, dxyz[3], drgb[3], dalpha) per entry,
 * summed into the caller's arrays in worker order once all workers are done. */
typedef struct {
    int64_t v;
    double g[7];
} gradent;

typedef struct {
    gradent *e;
    size_t n, cap;
} gradvec;

/* Appends three zeroed entries for the vertices of one triangle (one allocation step, so
 * the three pointers stay valid together). */
static int gv_add3(gradvec *v, const int64_t vid[3], double *out[3]) {
    if (v->n + 3 > v->cap) {
        size_t nc = v->cap ? v->cap * 2 : 4096;
        gradent *ne = (gradent *)realloc(v->e, nc * sizeof(gradent));
        if (!ne) return 1;
        v->e = ne;
        v->cap = nc;
    }
    for (int k = 0; k < 3; ++k) {
        gradent *g = &v->e[v->n++];
        g->v = vid[k];
        for (int i = 0; i < 7; ++i) g->g[i] = 0.0;
        out[k] = g->g;
    }
    return 0;
}

static int frag_cmp(const void *pa, const void *pb) {
    const frag *a = (const frag *)pa, *b = (const frag *)pb;
    if (a->pix != b->pix) return a->pix < b->pix ? -1 : 1;
    if (a->z != b->z) return a->z < b->z ? -1 : 1;
    if (a->tri != b->tri) return a->tri < b->tri ? -1 : 1;
    return 0;
}

typedef struct {
    /* scene */
    int64_t V, T;
    const double *xyz, *rgb, *alpha;
    const int32_t *tris;
    const orc_camera *cam;
    const double *bg;
    const dvert *dv;
    const dvert64 *dv64;    /* FP64 coverage when non-NULL */
    int order64;            /* binary32 coverage: order by the FP64 depth */
    const vvert *vv;
    int x0, x1, by0, by1, brute;
    /* forward outputs */
    double *out_rgba;       /* full window buffer */
    int32_t *out_nfrag;
    int wx0, wy0, ww;       /* window origin and width for output indexing */
    /* backward */
    uint64_t *out_sig;      /* per pixel: hash of the ordered triangle ids (optional) */
    const double *dL;
    gradvec gl;             /* backward: this worker's per-(fragment, vertex) contributions */
    int err;
} band_job;

/* collect() in FP64 decisions. */
static int collect64(band_job *j, fragvec *fv) {
    int bw = j->x1 - j->x0;
    for (int64_t t = 0; t < j->T; ++t) {
        int64_t ia = j->tris[3 * t], ib = j->tris[3 * t + 1], ic = j->tris[3 * t + 2];
        const dvert64 *A = &j->dv64[ia], *B = &j->dv64[ib], *C = &j->dv64[ic];
        if (!(A->valid && B->valid && C->valid)) continue;
        double area2 = tri_area2_64(A, B, C);
        if (!(area2 != 0.0)) continue;
        int px0 = j->x0, px1 = j->x1 - 1, py0 = j->by0, py1 = j->by1 - 1;
        if (!j->brute) {
            double mnx = fmin(fmin(A->xs, B->xs), C->xs), mxx = fmax(fmax(A->xs, B->xs), C->xs);
            double mny = fmin(fmin(A->ys, B->ys), C->ys), mxy = fmax(fmax(A->ys, B->ys), C->ys);
            int bx0 = (int)floor(mnx) - 2, bx1 = (int)floor(mxx) + 2;
            int by0 = (int)floor(mny) - 2, by1 = (int)floor(mxy) + 2;
            if (bx0 > px0) px0 = bx0;
            if (bx1 < px1) px1 = bx1;
            if (by0 > py0) py0 = by0;
            if (by1 < py1) py1 = by1;
        }
        for (int py = py0; py <= py1; ++py)
            for (int px = px0; px <= px1; ++px) {
                double zf;
                if (frag_depth64(A, ia, B, ib, C, ic, area2, px + 0.5, py + 0.5, &zf))
                    if (fv_push(fv, (py - j->by0) * bw + (px - j->x0), zf, t)) return 1;
            }
    }
    qsort(fv->f, fv->n, sizeof(frag), frag_cmp);
    return 0;
}

/* Mixed mode: a vertex relative to the integer origin (ox, oy), rounded to binary32. */
static dvert rel_vertex(const dvert *d, const vvert *w, double ox, double oy) {
    dvert r = *d;
    r.xs = (float)(w->xs - ox);
    r.ys = (float)(w->ys - oy);
    return r;
}

static int collect(band_job *j, fragvec *fv) {
    if (j->dv64) return collect64(j, fv);
    int bw = j->x1 - j->x0;
    for (int64_t t = 0; t < j->T; ++t) {
        int64_t ia = j->tris[3 * t], ib = j->tris[3 * t + 1], ic = j->tris[3 * t + 2];
        const dvert *A0 = &j->dv[ia], *B0 = &j->dv[ib], *C0 = &j->dv[ic];
        if (!(A0->valid && B0->valid && C0->valid)) continue;
        double ox = 0.0, oy = 0.0;
        dvert Ar = *A0, Br = *B0, Cr = *C0;
        if (j->order64) {
            ox = floor(j->vv[ia].xs);
            oy = floor(j->vv[ia].ys);
            Ar = rel_vertex(A0, &j->vv[ia], ox, oy);
            Br = rel_vertex(B0, &j->vv[ib], ox, oy);
            Cr = rel_vertex(C0, &j->vv[ic], ox, oy);
        }
        const dvert *A = &Ar, *B = &Br, *C = &Cr;
        float area2 = tri_area2(A, B, C);
        if (!(area2 != 0.0f)) continue;
        int px0 = j->x0, px1 = j->x1 - 1, py0 = j->by0, py1 = j->by1 - 1;
        if (!j->brute) {
            float mnx = fminf(fminf(A0->xs, B0->xs), C0->xs), mxx = fmaxf(fmaxf(A0->xs, B0->xs), C0->xs);
            float mny = fminf(fminf(A0->ys, B0->ys), C0->ys), mxy = fmaxf(fmaxf(A0->ys, B0->ys), C0->ys);
            int bx0 = (int)floorf(mnx) - 2, bx1 = (int)floorf(mxx) + 2;
            int by0 = (int)floorf(mny) - 2, by1 = (int)floorf(mxy) + 2;
            if (bx0 > px0) px0 = bx0;
            if (bx1 < px1) px1 = bx1;
            if (by0 > py0) py0 = by0;
            if (by1 < py1) py1 = by1;
        }
        for (int py = py0; py <= py1; ++py)
            for (int px = px0; px <= px1; ++px) {
                float zf;
                if (frag_depth(A, ia, B, ib, C, ic, area2, (float)(px - ox) + 0.5f, (float)(py - oy) + 0.5f,
                               &zf)) {
                    double z = j->order64 ? value_depth(&j->vv[ia], &j->vv[ib], &j->vv[ic], px + 0.5, py + 0.5)
                                          : (double)zf;
                    if (fv_push(fv, (py - j->by0) * bw + (px - j->x0), z, t)) return 1;
                }
            }
    }
    qsort(fv->f, fv->n, sizeof(frag), frag_cmp);
    return 0;
}

/* Interpolated colour and opacity of a fragment (Sec. 3: vertex colours interpolated
 * across the triangle; opacity interpolated linearly between centre and boundary). */
static void frag_value(const band_job *j, int64_t t, double px, double py,
                       double mu[3], double E[3], double *W, double c[3], double *a) {
    int64_t id[3] = {j->tris[3 * t], j->tris[3 * t + 1], j->tris[3 * t + 2]};
    persp_bary(&j->vv[id[0]], &j->vv[id[1]], &j->vv[id[2]], px, py, E, mu, W);
    c[0] = c[1] = c[2] = 0;
    *a = 0;
    for (int k = 0; k < 3; ++k) {
        for (int ch = 0; ch < 3; ++ch) c[ch] += mu[k] * j->rgb[3 * id[k] + ch];
        *a += mu[k] * j->alpha[id[k]];
    }
}

static void *fwd_worker(void *arg) {
    band_job *j = (band_job *)arg;
    fragvec fv = {0, 0, 0};
    if (collect(j, &fv)) { j->err = 1; free(fv.f); return 0; }
    int bw = j->x1 - j->x0;
    size_t i = 0;
    for (int py = j->by0; py < j->by1; ++py)
        for (int px = j->x0; px < j->x1; ++px) {
            int32_t pix = (py - j->by0) * bw + (px - j->x0);
            double T = 1.0, C[3] = {0, 0, 0};
            int32_t n = 0;
            uint64_t h = 1469598103934665603ull;   /* FNV-1a over the ordered triangle ids */
            while (i < fv.n && fv.f[i].pix == pix) {
                for (int b = 0; b < 8; ++b) {
                    h ^= (uint64_t)(((uint64_t)fv.f[i].tri >> (8 * b)) & 0xff);
                    h *= 1099511628211ull;
                }
                double mu[3], E[3], W, c[3], a;
                frag_value(j, fv.f[i].tri, px + 0.5, py + 0.5, mu, E, &W, c, &a);
                for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * c[ch];
                T *= (1.0 - a);
                ++n;
                ++i;
            }
            size_t o = ((size_t)(py - j->wy0) * j->ww + (px - j->wx0)) * 4;
            for (int ch = 0; ch < 3; ++ch) j->out_rgba[o + ch] = C[ch] + T * j->bg[ch];
            j->out_rgba[o + 3] = 1.0 - T;
            if (j->out_nfrag) j->out_nfrag[(size_t)(py - j->wy0) * j->ww + (px - j->wx0)] = n;
            if (j->out_sig) j->out_sig[(size_t)(py - j->wy0) * j->ww + (px - j->wx0)] = h;
        }
    free(fv.f);
    return 0;
}

/* Reverse pass for one pixel's sorted fragment list (exact, FP64).
 * out = R_0 with R_f = a_f c_f + (1 - a_f) R_{f+1}, R_n = bg, so
 * d out/d c_f = T_f a_f and d out/d a_f = T_f (c_f - R_{f+1}); the alpha channel is the
 * same recursion with colour 1 and background 0. */
static void pixel_backward(band_job *j, const frag *fl, int n, int px, int py) {
    enum { MAXF = 4096 };
    static __thread double Tf[MAXF], cf[MAXF][3], af[MAXF], muf[MAXF][3], Ef[MAXF][3], Wf[MAXF];
    if (n > MAXF) { j->err = 2; return; }
    double T = 1.0;
    for (int f = 0; f < n; ++f) {
        Tf[f] = T;
        frag_value(j, fl[f].tri, px + 0.5, py + 0.5, muf[f], Ef[f], &Wf[f], cf[f], &af[f]);
        T *= (1.0 - af[f]);
    }
    size_t o = ((size_t)(py - j->wy0) * j->ww + (px - j->wx0)) * 4;
    const double *g = j->dL + o;
    double Rc[3] = {j->bg[0], j->bg[1], j->bg[2]}, Ra = 0.0;
    const orc_camera *cam = j->cam;
    for (int f = n - 1; f >= 0; --f) {
        double dc[3], da = 0;
        for (int ch = 0; ch < 3; ++ch) {
            dc[ch] = g[ch] * Tf[f] * af[f];
            da += g[ch] * Tf[f] * (cf[f][ch] - Rc[ch]);
        }
        da += g[3] * Tf[f] * (1.0 - Ra);
        for (int ch = 0; ch < 3; ++ch) Rc[ch] = af[f] * cf[f][ch] + (1.0 - af[f]) * Rc[ch];
        Ra = af[f] + (1.0 - af[f]) * Ra;

        int64_t t = fl[f].tri;
        int64_t id[3] = {j->tris[3 * t], j->tris[3 * t + 1], j->tris[3 * t + 2]};
        double *gvk[3];
        if (gv_add3(&j->gl, id, gvk)) { j->err = 3; return; }
        double gmu[3];
        for (int k = 0; k < 3; ++k) {
            double *gv = gvk[k];
            gmu[k] = da * j->alpha[id[k]];
            for (int ch = 0; ch < 3; ++ch) {
                gv[3 + ch] += muf[f][k] * dc[ch];
                gmu[k] += dc[ch] * j->rgb[3 * id[k] + ch];
            }
            gv[6] += muf[f][k] * da;
        }
        /* mu_k = w_k / W with w_k = E_k / Z_k. */
        double s = gmu[0] * muf[f][0] + gmu[1] * muf[f][1] + gmu[2] * muf[f][2];
        double gw[3], gE[3], gZ[3] = {0, 0, 0}, gx[3] = {0, 0, 0}, gy[3] = {0, 0, 0};
        const vvert *Vv[3] = {&j->vv[id[0]], &j->vv[id[1]], &j->vv[id[2]]};
        for (int k = 0; k < 3; ++k) {
            gw[k] = (gmu[k] - s) / Wf[f];
            gE[k] = gw[k] / Vv[k]->Z;
            gZ[k] -= gw[k] * Ef[f][k] / (Vv[k]->Z * Vv[k]->Z);
        }
        /* E_k is the edge function of the edge (a -> b) opposite vertex k:
         * E = (xb - xa)(py - ya) - (yb - ya)(px - xa). */
        double ppx = px + 0.5, ppy = py + 0.5;
        for (int k = 0; k < 3; ++k) {
            int a = (k + 1) % 3, b = (k + 2) % 3;
            const vvert *A = Vv[a], *B = Vv[b];
            gx[a] += gE[k] * (B->ys - ppy);
            gy[a] += gE[k] * (ppx - B->xs);
            gx[b] += gE[k] * (ppy - A->ys);
            gy[b] += gE[k] * (A->xs - ppx);
        }
        /* Screen position and depth -> view space -> world space. */
        for (int k = 0; k < 3; ++k) {
            const vvert *P = Vv[k];
            double gX = gx[k] * cam->fx / P->Z;
            double gY = gy[k] * cam->fy / P->Z;
            double gZv = gZ[k] - gx[k] * cam->fx * P->X / (P->Z * P->Z) - gy[k] * cam->fy * P->Y / (P->Z * P->Z);
            double *gv = gvk[k];
            for (int r = 0; r < 3; ++r)
                gv[r] += (double)cam->R_cw[r] * gX + (double)cam->R_cw[3 + r] * gY + (double)cam->R_cw[6 + r] * gZv;
        }
    }
}

static void *bwd_worker(void *arg) {
    band_job *j = (band_job *)arg;
    fragvec fv = {0, 0, 0};
    if (collect(j, &fv)) { j->err = 1; free(fv.f); return 0; }
    int bw = j->x1 - j->x0;
    size_t i = 0;
    for (int py = j->by0; py < j->by1; ++py)
        for (int px = j->x0; px < j->x1; ++px) {
            int32_t pix = (py - j->by0) * bw + (px - j->x0);
            size_t s = i;
            while (i < fv.n && fv.f[i].pix == pix) ++i;
            if (i > s) pixel_backward(j, fv.f + s, (int)(i - s), px, py);
        }
    free(fv.f);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Driver                                                                               */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    const orc_camera *cam;
    const double *xyz;
    dvert *dv;
    dvert64 *dv64;
    vvert *vv;
    int64_t v0, v1;
    int rounded;            /* decided vertices from the rounded FP64 projection */
} vert_job;

/* Decided vertex of the mixed mode: the FP64 screen position and depth rounded to
 * binary32 (round to nearest), 1/Z of the rounded depth, validity on the rounded values. */
static void round_vertex(const orc_camera *cam, const vvert *w, dvert *o) {
    o->xs = (float)w->xs;
    o->ys = (float)w->ys;
    o->Z = (float)w->Z;
    o->iz = 1.0f / o->Z;
    o->valid = (o->Z > cam->znear) && (fabsf(o->xs) <= GUARD_PX) && (fabsf(o->ys) <= GUARD_PX);
}

static void *vert_worker(void *arg) {
    vert_job *j = (vert_job *)arg;
    for (int64_t v = j->v0; v < j->v1; ++v) {
        const double *p = j->xyz + 3 * v;
        value_vertex(j->cam, p, &j->vv[v]);
        if (j->rounded)
            round_vertex(j->cam, &j->vv[v], &j->dv[v]);
        else
            decide_vertex(j->cam, (float)p[0], (float)p[1], (float)p[2], &j->dv[v]);
        if (j->dv64) {
            const vvert *w = &j->vv[v];
            dvert64 *d = &j->dv64[v];
            d->xs = w->xs;
            d->ys = w->ys;
            d->Z = w->Z;
            d->valid = (w->Z > (double)j->cam->znear) && (fabs(w->xs) <= (double)GUARD_PX) &&
                       (fabs(w->ys) <= (double)GUARD_PX);
        }
    }
    return 0;
}

static int run_pass(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                    int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                    int x0, int y0, int x1, int y1, int brute, int nthreads, int decide,
                    double *out_rgba, int32_t *out_nfrag, uint64_t *out_sig, int64_t *n_culled,
                    const double *dL, double *d_xyz, double *d_rgb, double *d_alpha) {
    if (x1 <= x0 || y1 <= y0) return 0;
    if (decide < 0 || decide > 2) return 4;
    const int decide64 = decide == 1;
    int nt = resolve_threads(nthreads);
    int backward = dL != 0;
    if (nt > y1 - y0) nt = y1 - y0;
    g_last_threads = nt;
    dvert *dv = (dvert *)malloc(sizeof(dvert) * (V > 0 ? V : 1));
    vvert *vv = (vvert *)malloc(sizeof(vvert) * (V > 0 ? V : 1));
    dvert64 *dv64 = decide64 ? (dvert64 *)malloc(sizeof(dvert64) * (V > 0 ? V : 1)) : 0;
    if (!dv || !vv || (decide64 && !dv64)) { free(dv); free(vv); free(dv64); return 3; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
    vert_job *vj = (vert_job *)malloc(sizeof(vert_job) * nt);
    for (int i = 0; i < nt; ++i) {
        vj[i].cam = cam; vj[i].xyz = xyz; vj[i].dv = dv; vj[i].dv64 = dv64; vj[i].vv = vv;
        vj[i].v0 = V * i / nt; vj[i].v1 = V * (i + 1) / nt;
        vj[i].rounded = decide == 2;
        pthread_create(&th[i], 0, vert_worker, &vj[i]);
    }
    for (int i = 0; i < nt; ++i) pthread_join(th[i], 0);
    if (n_culled) {
        int64_t c = 0;
        for (int64_t t = 0; t < T; ++t) {
            int64_t a = tris[3 * t], b = tris[3 * t + 1], cc = tris[3 * t + 2];
            int ok = decide64 ? (dv64[a].valid && dv64[b].valid && dv64[cc].valid)
                              : (dv[a].valid && dv[b].valid && dv[cc].valid);
            if (!ok) ++c;
        }
        *n_culled = c;
    }
    band_job *bj = (band_job *)calloc(nt, sizeof(band_job));
    int err = 0;
    for (int i = 0; i < nt; ++i) {
        band_job *j = &bj[i];
        j->V = V; j->T = T; j->xyz = xyz; j->rgb = rgb; j->alpha = alpha; j->tris = tris;
        j->cam = cam; j->bg = bg; j->dv = dv; j->dv64 = dv64; j->vv = vv; j->order64 = decide == 2;
        j->x0 = x0; j->x1 = x1; j->brute = brute;
        j->by0 = y0 + (int)((int64_t)(y1 - y0) * i / nt);
        j->by1 = y0 + (int)((int64_t)(y1 - y0) * (i + 1) / nt);
        j->out_rgba = out_rgba; j->out_nfrag = out_nfrag; j->out_sig = out_sig;
        j->wx0 = x0; j->wy0 = y0; j->ww = x1 - x0;
        j->dL = dL;
    }
    for (int i = 0; i < nt; ++i) pthread_create(&th[i], 0, backward ? bwd_worker : fwd_worker, &bj[i]);
    for (int i = 0; i < nt; ++i) pthread_join(th[i], 0);
    for (int i = 0; i < nt; ++i)
        if (bj[i].err) err = bj[i].err;
    if (backward && !err) {
        /* contributions summed in band order, then fragment order: deterministic */
        for (int i = 0; i < nt; ++i)
            for (size_t e = 0; e < bj[i].gl.n; ++e) {
                const gradent *g = &bj[i].gl.e[e];
                int64_t v = g->v;
                for (int r = 0; r < 3; ++r) d_xyz[3 * v + r] += g->g[r];
                for (int r = 0; r < 3; ++r) d_rgb[3 * v + r] += g->g[3 + r];
                d_alpha[v] += g->g[6];
            }
    }
    for (int i = 0; i < nt; ++i) free(bj[i].gl.e);
    free(bj); free(vj); free(th); free(dv); free(vv); free(dv64);
    return err;
}

int orc_render_ex(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                  int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                  int x0, int y0, int x1, int y1, int brute, int nthreads, int decide,
                  double *out_rgba, int32_t *out_nfrag, uint64_t *out_sig, int64_t *n_culled) {
    return run_pass(V, xyz, rgb, alpha, T, tris, cam, bg, x0, y0, x1, y1, brute, nthreads, decide,
                    out_rgba, out_nfrag, out_sig, n_culled, 0, 0, 0, 0);
}

int orc_render(int64_t V, const double *xyz, const double *rgb, const double *alpha,
               int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
               int x0, int y0, int x1, int y1, int brute, int nthreads,
               double *out_rgba, int32_t *out_nfrag, int64_t *n_culled) {
    return orc_render_ex(V, xyz, rgb, alpha, T, tris, cam, bg, x0, y0, x1, y1, brute, nthreads, 0,
                         out_rgba, out_nfrag, 0, n_culled);
}

int orc_render_backward_ex(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                           int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                           int x0, int y0, int x1, int y1, int nthreads, int decide,
                           const double *dL_drgba, double *d_xyz, double *d_rgb, double *d_alpha) {
    return run_pass(V, xyz, rgb, alpha, T, tris, cam, bg, x0, y0, x1, y1, 0, nthreads, decide,
                    0, 0, 0, 0, dL_drgba, d_xyz, d_rgb, d_alpha);
}

int orc_render_backward(int64_t V, const double *xyz, const double *rgb, const double *alpha,
                        int64_t T, const int32_t *tris, const orc_camera *cam, const double bg[3],
                        int x0, int y0, int x1, int y1, int nthreads,
                        const double *dL_drgba, double *d_xyz, double *d_rgb, double *d_alpha) {
    return orc_render_backward_ex(V, xyz, rgb, alpha, T, tris, cam, bg, x0, y0, x1, y1, nthreads, 0,
                                  dL_drgba, d_xyz, d_rgb, d_alpha);
}
