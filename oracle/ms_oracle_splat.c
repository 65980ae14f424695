/*
 * Source-Gaussian render -- TEST INFRASTRUCTURE ONLY (see ms_oracle.h).
 *
 * The image the fans stand in for: every flat Gaussian (m, R, S, sigma, colour) of the
 * scene drawn as itself (Sec. 3: the Gaussian component with mean m, rotation R, scale
 * S and opacity sigma, in the GaMeS flat form whose thin axis is dropped), composited in
 * depth order exactly like the fans.  Readings:
 *   - the pixel ray x = C + t d, d = R_cw^T ((px - cx)/fx, (py - cy)/fy, 1), meets the
 *     plane through m spanned by the two kept unit axes u_a, u_b (same axis rule as the
 *     fan conversion) at local coordinates u = (x - m).u_a, v = (x - m).u_b;
 *   - opacity alpha = sigma exp(-(u^2 / s_a^2 + v^2 / s_b^2) / 2) with s = exp(log-scale),
 *     kept only where (u / (T s_a))^2 + (v / (T s_b))^2 <= 1 with T = scale_mul = 2.7,
 *     the ellipse whose inscribed polygon is the fan, and only for t > znear;
 *   - the colour is the Gaussian's colour (the value every vertex of its fan carries);
 *   - order: ascending (float) t, which is the view depth Z of the hit point since d has
 *     unit z, rounded to binary32, ties by ascending Gaussian index; then C += T a c,
 *     T *= 1 - a, out = (C + T bg, 1 - T) as for the fans.
 * All arithmetic is FP64; the only binary32 step is the rounding of the depth key.
 */
#include "ms_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
    double mc[3], ua[3], ub[3], n[3];   /* camera-space centre, kept axes, plane normal */
    double sa, sb, sigma, col[3];
    double mcn;                         /* mc . n */
    int bx0, bx1, by0, by1;             /* pixel bounding box (inclusive), or the window */
} splat;

typedef struct {
    int32_t pix;
    float z;
    int64_t g;
} sfrag;

typedef struct {
    const splat *sp;
    int64_t N;
    const orc_camera *cam;
    const double *bg;
    double trunc;
    int x0, x1, y0, y1;     /* band */
    int wx0, wy0, ww;       /* window */
    double *out;
    int32_t *nfrag;
    int err;
} sjob;

static int sfrag_cmp(const void *pa, const void *pb) {
    const sfrag *a = (const sfrag *)pa, *b = (const sfrag *)pb;
    if (a->pix != b->pix) return a->pix < b->pix ? -1 : 1;
    if (a->z != b->z) return a->z < b->z ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return 0;
}

/* Hit of pixel centre (px, py) with splat s: returns 1 and (t, alpha) when kept. */
static int splat_hit(const splat *s, const orc_camera *cam, double trunc, double px, double py, double *t,
                     double *alpha) {
    const double d[3] = {(px - cam->cx) / cam->fx, (py - cam->cy) / cam->fy, 1.0};
    const double den = d[0] * s->n[0] + d[1] * s->n[1] + d[2] * s->n[2];
    if (den == 0.0) return 0;
    const double tt = s->mcn / den;
    if (!(tt > (double)cam->znear)) return 0;
    const double w[3] = {tt * d[0] - s->mc[0], tt * d[1] - s->mc[1], tt * d[2] - s->mc[2]};
    const double u = w[0] * s->ua[0] + w[1] * s->ua[1] + w[2] * s->ua[2];
    const double v = w[0] * s->ub[0] + w[1] * s->ub[1] + w[2] * s->ub[2];
    const double ru = u / (trunc * s->sa), rv = v / (trunc * s->sb);
    if (!(ru * ru + rv * rv <= 1.0)) return 0;
    *t = tt;
    *alpha = s->sigma * exp(-0.5 * (u * u / (s->sa * s->sa) + v * v / (s->sb * s->sb)));
    return 1;
}

static void *splat_worker(void *arg) {
    sjob *j = (sjob *)arg;
    const int bw = j->x1 - j->x0;
    size_t n = 0, cap = 4096;
    sfrag *f = (sfrag *)malloc(cap * sizeof(sfrag));
    if (!f) { j->err = 1; return 0; }
    for (int64_t g = 0; g < j->N; ++g) {
        const splat *s = &j->sp[g];
        const int px0 = s->bx0 > j->x0 ? s->bx0 : j->x0, px1 = s->bx1 < j->x1 - 1 ? s->bx1 : j->x1 - 1;
        const int py0 = s->by0 > j->y0 ? s->by0 : j->y0, py1 = s->by1 < j->y1 - 1 ? s->by1 : j->y1 - 1;
        for (int py = py0; py <= py1; ++py)
            for (int px = px0; px <= px1; ++px) {
                double t, a;
                if (!splat_hit(s, j->cam, j->trunc, px + 0.5, py + 0.5, &t, &a)) continue;
                if (n == cap) {
                    cap *= 2;
                    sfrag *nf = (sfrag *)realloc(f, cap * sizeof(sfrag));
                    if (!nf) { free(f); j->err = 1; return 0; }
                    f = nf;
                }
                f[n].pix = (py - j->y0) * bw + (px - j->x0);
                f[n].z = (float)t;
                f[n].g = g;
                ++n;
            }
    }
    qsort(f, n, sizeof(sfrag), sfrag_cmp);
    size_t i = 0;
    for (int py = j->y0; py < j->y1; ++py)
        for (int px = j->x0; px < j->x1; ++px) {
            const int32_t pix = (py - j->y0) * bw + (px - j->x0);
            double T = 1.0, C[3] = {0, 0, 0};
            int32_t cnt = 0;
            while (i < n && f[i].pix == pix) {
                double t, a;
                const splat *s = &j->sp[f[i].g];
                splat_hit(s, j->cam, j->trunc, px + 0.5, py + 0.5, &t, &a);
                for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * s->col[ch];
                T *= (1.0 - a);
                ++cnt;
                ++i;
            }
            const size_t o = ((size_t)(py - j->wy0) * j->ww + (px - j->wx0)) * 4;
            for (int ch = 0; ch < 3; ++ch) j->out[o + ch] = C[ch] + T * j->bg[ch];
            j->out[o + 3] = 1.0 - T;
            if (j->nfrag) j->nfrag[(size_t)(py - j->wy0) * j->ww + (px - j->wx0)] = cnt;
        }
    free(f);
    return 0;
}

int orc_splat_render(int64_t N, const float *means, const float *log_scales, const float *quats,
                     const float *opacity, const double *rgb, int axis_rule, double trunc,
                     const orc_camera *cam, const double bg[3], int x0, int y0, int x1, int y1,
                     int nthreads, double *out_rgba, int32_t *out_nfrag) {
    if (N < 0 || x1 < x0 || y1 < y0 || !(trunc > 0)) return 1;
    splat *sp = (splat *)malloc((size_t)(N > 0 ? N : 1) * sizeof(splat));
    if (!sp) return 2;
    double Rc[9];
    for (int i = 0; i < 9; ++i) Rc[i] = cam->R_cw[i];
    for (int64_t g = 0; g < N; ++g) {
        splat *s = &sp[g];
        double q[4] = {quats[4 * g], quats[4 * g + 1], quats[4 * g + 2], quats[4 * g + 3]}, R[9];
        orc_quat_to_rot(q, R);
        const double ls[3] = {log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]};
        int drop = 0;
        if (axis_rule == 1) {
            if (ls[1] < ls[drop]) drop = 1;
            if (ls[2] < ls[drop]) drop = 2;
        }
        const int ia = drop == 0 ? 1 : 0, ib = drop == 2 ? 1 : 2;
        const double dm[3] = {means[3 * g] - (double)cam->C[0], means[3 * g + 1] - (double)cam->C[1],
                              means[3 * g + 2] - (double)cam->C[2]};
        for (int r = 0; r < 3; ++r) {
            s->mc[r] = Rc[3 * r] * dm[0] + Rc[3 * r + 1] * dm[1] + Rc[3 * r + 2] * dm[2];
            s->ua[r] = Rc[3 * r] * R[ia] + Rc[3 * r + 1] * R[3 + ia] + Rc[3 * r + 2] * R[6 + ia];
            s->ub[r] = Rc[3 * r] * R[ib] + Rc[3 * r + 1] * R[3 + ib] + Rc[3 * r + 2] * R[6 + ib];
        }
        s->n[0] = s->ua[1] * s->ub[2] - s->ua[2] * s->ub[1];
        s->n[1] = s->ua[2] * s->ub[0] - s->ua[0] * s->ub[2];
        s->n[2] = s->ua[0] * s->ub[1] - s->ua[1] * s->ub[0];
        s->mcn = s->mc[0] * s->n[0] + s->mc[1] * s->n[1] + s->mc[2] * s->n[2];
        s->sa = exp(ls[ia]);
        s->sb = exp(ls[ib]);
        s->sigma = opacity[g];
        for (int ch = 0; ch < 3; ++ch) s->col[ch] = rgb[3 * g + ch];
        /* bounding box: the projected corners of the rectangle circumscribing the
         * truncation ellipse, widened by 2 px; the whole window if a corner is not in
         * front of the camera */
        double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300;
        int front = 1;
        for (int c = 0; c < 4; ++c) {
            const double ea = (c & 1 ? 1.0 : -1.0) * trunc * s->sa, eb = (c & 2 ? 1.0 : -1.0) * trunc * s->sb;
            double P[3];
            for (int r = 0; r < 3; ++r) P[r] = s->mc[r] + ea * s->ua[r] + eb * s->ub[r];
            if (!(P[2] > 1e-9)) { front = 0; break; }
            const double xs = cam->fx * P[0] / P[2] + cam->cx, ys = cam->fy * P[1] / P[2] + cam->cy;
            if (xs < mnx) mnx = xs;
            if (xs > mxx) mxx = xs;
            if (ys < mny) mny = ys;
            if (ys > mxy) mxy = ys;
        }
        if (front && mnx > -1e9 && mxx < 1e9 && mny > -1e9 && mxy < 1e9) {
            s->bx0 = (int)floor(mnx) - 2; s->bx1 = (int)floor(mxx) + 2;
            s->by0 = (int)floor(mny) - 2; s->by1 = (int)floor(mxy) + 2;
        } else {
            s->bx0 = x0; s->bx1 = x1 - 1; s->by0 = y0; s->by1 = y1 - 1;
        }
    }
    int nt = nthreads > 0 ? nthreads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nt < 1) nt = 1;
    const int H = y1 - y0;
    if (nt > H) nt = H > 0 ? H : 1;
    sjob *jobs = (sjob *)calloc((size_t)nt, sizeof(sjob));
    pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    if (!jobs || !th) { free(sp); free(jobs); free(th); return 2; }
    for (int k = 0; k < nt; ++k) {
        sjob *j = &jobs[k];
        j->sp = sp; j->N = N; j->cam = cam; j->bg = bg; j->trunc = trunc;
        j->x0 = x0; j->x1 = x1;
        j->y0 = y0 + (int)((int64_t)H * k / nt);
        j->y1 = y0 + (int)((int64_t)H * (k + 1) / nt);
        j->wx0 = x0; j->wy0 = y0; j->ww = x1 - x0;
        j->out = out_rgba; j->nfrag = out_nfrag;
    }
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], 0, splat_worker, &jobs[k]);
    int err = 0;
    for (int k = 0; k < nt; ++k) {
        pthread_join(th[k], 0);
        err |= jobs[k].err;
    }
    free(sp); free(jobs); free(th);
    return err ? 3 : 0;
}
