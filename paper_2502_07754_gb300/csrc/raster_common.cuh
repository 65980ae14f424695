// Shared pieces of the rasterisation kernels: double-float projection of a fan
// centre (value path), the shared-memory stage of a chunk of fans, the per-pixel
// coverage walk over a staged fan's K triangles with the binary32 decision formulas on
// fan-relative vertex positions, and the double-float fragment depth that orders them.
#pragma once

#include "fan_geom.cuh"
#include "ms_internal.h"

namespace ms {

// Pixels are resolved in descending order of their fragment counts, clamped here.
constexpr int kCountBuckets = 256;
__device__ __forceinline__ int count_bucket(uint32_t n) {
    return n < (uint32_t)kCountBuckets ? (int)n : kCountBuckets - 1;
}

struct SceneDev {
    const float *xyz, *rgb, *alpha;
    int K;
    const CamDev *cam;   // points into the kernel's __grid_constant__ view table
    int W, H;
    const float4 *dec;   // this view's decided vertices (xr, yr, Z or -1, origin), written by binning
    const uint32_t *face_mask;   // per fan, bit j = face j drawn; NULL = all
};

// ------------------------------------------------------------------------------------
// Double-float helpers of the value path (Knuth two-sum, FMA two-product)
// ------------------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}
// Row of R_cw applied to (d_hi + d_lo), as hi + lo.
__device__ __forceinline__ void df_dot(const float *R, const float dh[3], const float dl[3], float &h, float &l) {
    float p0, q0, p1, q1, p2, q2, s, e1, e2;
    two_prod(R[0], dh[0], p0, q0);
    two_prod(R[1], dh[1], p1, q1);
    two_prod(R[2], dh[2], p2, q2);
    two_sum(p0, p1, s, e1);
    two_sum(s, p2, h, e2);
    l = ((e1 + e2) + (q0 + q1 + q2)) + (R[0] * dl[0] + R[1] * dl[1] + R[2] * dl[2]);
}
// f * (X / Z) + c as hi + lo, with X, Z given as hi + lo.
__device__ __forceinline__ void df_screen(float Xh, float Xl, float Zh, float Zl, float f, float c, float &h,
                                          float &l) {
    const float q1 = Xh / Zh;
    const float r = fmaf(-q1, Zh, Xh) + (Xl - q1 * Zl);
    const float q2 = r / Zh;
    float a1, a2, e;
    two_prod(f, q1, a1, a2);
    a2 = fmaf(f, q2, a2);
    two_sum(a1, c, h, e);
    l = e + a2;
}

// View-space centre of a fan (hi parts) and its double-float screen position.  The
// other vertices are placed by their exact world offsets from the centre, so screen
// positions relative to a pixel carry ~1e-6 px error instead of the ~1e-4 px of a
// plain binary32 projection at 1080p.
struct CentreProj {
    float Xh, Yh, Zh, Xl, Yl, Zl;
    float xh, xl, yh, yl;
};
__device__ __forceinline__ CentreProj project_centre(const CamDev &c, const float m[3]) {
    float dh[3], dl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) two_sum(m[r], -c.C[r], dh[r], dl[r]);
    CentreProj o;
    df_dot(c.R, dh, dl, o.Xh, o.Xl);
    df_dot(c.R + 3, dh, dl, o.Yh, o.Yl);
    df_dot(c.R + 6, dh, dl, o.Zh, o.Zl);
    df_screen(o.Xh, o.Xl, o.Zh, o.Zl, c.fx, c.cx, o.xh, o.xl);
    df_screen(o.Yh, o.Yl, o.Zh, o.Zl, c.fy, c.cy, o.yh, o.yl);
    return o;
}
__device__ __forceinline__ void vertex_offset(const CamDev &c, const CentreProj &cp, const float d[3], float &du,
                                              float &dv, float &X, float &Y, float &Z) {
    const float dX = c.R[0] * d[0] + c.R[1] * d[1] + c.R[2] * d[2];
    const float dY = c.R[3] * d[0] + c.R[4] * d[1] + c.R[5] * d[2];
    const float dZ = c.R[6] * d[0] + c.R[7] * d[1] + c.R[8] * d[2];
    X = cp.Xh + dX;
    Y = cp.Yh + dY;
    Z = cp.Zh + dZ;
    const float den = 1.0f / (Z * cp.Zh);
    du = c.fx * (dX * cp.Zh - cp.Xh * dZ) * den;
    dv = c.fy * (dY * cp.Zh - cp.Yh * dZ) * den;
}

// Camera-space offset R (p - m) of a vertex from its fan centre, in double-float (the
// world difference of two binary32 values is exact as a two-sum).
struct DfVec {
    dfl x, y, z;
};
__device__ __forceinline__ DfVec df_view_offset(const CamDev &c, const float m[3], const float *p) {
    const dfl d0 = df_two_sum(__ldg(p), -m[0]), d1 = df_two_sum(__ldg(p + 1), -m[1]);
    const dfl d2 = df_two_sum(__ldg(p + 2), -m[2]);
    return DfVec{df_row_dot(c.R, d0, d1, d2), df_row_dot(c.R + 3, d0, d1, d2), df_row_dot(c.R + 6, d0, d1, d2)};
}

// ------------------------------------------------------------------------------------
// Shared-memory stage (structure of arrays over CH slots)
// ------------------------------------------------------------------------------------

struct Stage {
    int4 *rect;                   // [CH] i0, i1, j0, j1
    uint32_t *flags;              // [CH] bits 0..15 valid triangle, 16..31 negative orientation
    uint32_t *q;                  // [CH] quantised depth bound
    uint32_t *fan;                // [CH] fan id
    uint32_t *stie, *rtie;        // [CH] top-left tie bits of the spoke / rim directions
    float *ox, *oy;               // [CH] integer origin of the fan's relative positions
    float *vx, *vy;               // [KV][CH] decided vertices relative to the origin
    float *sdx, *sdy;             // [K][CH] spoke directions b_i - c
    float *rdx, *rdy;             // [K][CH] rim directions, lower index to higher
    float *area;                  // [K][CH] |area2|
    float *cxh, *cxl, *cyh, *cyl; // [CH] double-float screen position of the centre (values)
    float *du, *dv;               // [K][CH] screen offsets of the boundary vertices (values)
    float *cr, *cg, *cb, *ca;     // [KV][CH] vertex colour and opacity (values)
    float *viz;                   // [KV][CH] 1 / depth (values: barycentric weights)
    // exact-order depth (frag_depth_df), double-float (high, low):
    float *pc;                    // [6][CH] fx X_c, fy Y_c, Z_c of the centre
    float *exh, *exl, *eyh, *eyl, *ezh, *ezl;   // [K][CH] view offsets R (b_i - c) of the boundary vertices
};

// What a stage holds: decisions only (count), or decisions and values (fill).
enum StageLevel { kStageDecide = 0, kStageValues = 1 };

__host__ __device__ __forceinline__ size_t stage_bytes(int CH, int K, int level) {
    const int dec = 2 * (K + 1) + 5 * K;
    const int val = level >= kStageValues ? 4 + 2 * K + 4 * (K + 1) + (K + 1) + 6 + 6 * K : 0;
    return (size_t)CH * (16 + 20 + 8 + 4 * (dec + val));
}

__device__ __forceinline__ Stage stage_ptrs(char *base, int CH, int K, int level) {
    const int KV = K + 1;
    Stage s;
    s.rect = reinterpret_cast<int4 *>(base);
    s.flags = reinterpret_cast<uint32_t *>(s.rect + CH);
    s.q = s.flags + CH;
    s.fan = s.q + CH;
    s.stie = s.fan + CH;
    s.rtie = s.stie + CH;
    float *f = reinterpret_cast<float *>(s.rtie + CH);
    s.ox = f; f += CH;
    s.oy = f; f += CH;
    s.vx = f; f += KV * CH;
    s.vy = f; f += KV * CH;
    s.sdx = f; f += K * CH;
    s.sdy = f; f += K * CH;
    s.rdx = f; f += K * CH;
    s.rdy = f; f += K * CH;
    s.area = f; f += K * CH;
    if (level >= kStageValues) {
        s.cxh = f; f += CH;
        s.cxl = f; f += CH;
        s.cyh = f; f += CH;
        s.cyl = f; f += CH;
        s.du = f; f += K * CH;
        s.dv = f; f += K * CH;
        s.cr = f; f += KV * CH;
        s.cg = f; f += KV * CH;
        s.cb = f; f += KV * CH;
        s.ca = f; f += KV * CH;
        s.viz = f; f += KV * CH;
        s.pc = f; f += 6 * CH;
        s.exh = f; f += K * CH;
        s.exl = f; f += K * CH;
        s.eyh = f; f += K * CH;
        s.eyl = f; f += K * CH;
        s.ezh = f; f += K * CH;
        s.ezl = f;
    }
    return s;
}

// OR / min / max over the LPF lanes of a fan's group (lanes lane & ~(LPF-1) .. + LPF-1).
template <int LPF>
__device__ __forceinline__ uint32_t group_or(uint32_t x) {
#pragma unroll
    for (int o = LPF / 2; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <int LPF>
__device__ __forceinline__ float group_min(float x) {
#pragma unroll
    for (int o = LPF / 2; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
template <int LPF>
__device__ __forceinline__ float group_max(float x) {
#pragma unroll
    for (int o = LPF / 2; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// The decision part of stage_fans: decided vertices, spoke and rim directions, areas,
// tie bits, valid-triangle flags and the pixel rectangle of every slot.
template <int LPF>
__device__ __forceinline__ void stage_decisions(const SceneDev &a, const Stage &s, int K, int slot, int sub,
                                                bool active, uint32_t fan, uint32_t q) {
    constexpr int CH = 32 / LPF;
    const int KV = K + 1;
    const float4 *dv = a.dec + (size_t)fan * KV;

    uint32_t vmask = 0;
    if (active)
        for (int k = sub; k < KV; k += LPF) {
            const float4 d = __ldg(dv + k);   // the binning pass's decide_vertex, bit for bit
            s.vx[k * CH + slot] = d.x;
            s.vy[k * CH + slot] = d.y;
            if (d.z > 0.0f) vmask |= 1u << k;   // binning marks invalid vertices with Z = -1
            if (k == 0) s.ox[slot] = d.w;
            if (k == 1) s.oy[slot] = d.w;
        }
    vmask = group_or<LPF>(vmask);
    __syncwarp();   // the group's vertex rows are complete
    uint32_t tmask = tri_valid_mask(vmask, K);
    if (a.face_mask && active) tmask &= __ldg(a.face_mask + fan);   // the same word in every lane of the fan
    float mnx = 3.0e38f, mxx = -3.0e38f, mny = 3.0e38f, mxy = -3.0e38f;
    uint32_t flags = 0, stie = 0, rtie = 0;
    if (active) {
        for (int k = sub; k < KV; k += LPF) {
            if (!vertex_used(tmask, k, K)) continue;
            const float x = s.vx[k * CH + slot], y = s.vy[k * CH + slot];
            mnx = fminf(mnx, x); mxx = fmaxf(mxx, x);
            mny = fminf(mny, y); mxy = fmaxf(mxy, y);
        }
        const float xc = s.vx[slot], yc = s.vy[slot];
        for (int j = sub; j < K; j += LPF) {
            const int b = 1 + j, c = 1 + (j + 1 == K ? 0 : j + 1);
            const float xb = s.vx[b * CH + slot], yb = s.vy[b * CH + slot];
            const float xn = s.vx[c * CH + slot], yn = s.vy[c * CH + slot];
            const float sx = __fsub_rn(xb, xc), sy = __fsub_rn(yb, yc);
            float rx, ry;
            if (j + 1 == K) {   // rim (b_{K-1}, b_0): the lower index is b_0
                rx = __fsub_rn(xb, xn);
                ry = __fsub_rn(yb, yn);
            } else {
                rx = __fsub_rn(xn, xb);
                ry = __fsub_rn(yn, yb);
            }
            s.sdx[j * CH + slot] = sx;
            s.sdy[j * CH + slot] = sy;
            s.rdx[j * CH + slot] = rx;
            s.rdy[j * CH + slot] = ry;
            const float ar = dec_area2(xc, yc, xb, yb, xn, yn);
            s.area[j * CH + slot] = fabsf(ar);
            if (((tmask >> j) & 1u) && ar != 0.0f) flags |= 1u << j;
            if (ar < 0.0f) flags |= 1u << (16 + j);
            // tie acceptance (E == 0) of each direction and of its reverse
            if (sy < 0.0f || (sy == 0.0f && sx > 0.0f)) stie |= 1u << j;
            if (sy > 0.0f || (sy == 0.0f && sx < 0.0f)) stie |= 1u << (16 + j);
            if (ry < 0.0f || (ry == 0.0f && rx > 0.0f)) rtie |= 1u << j;
            if (ry > 0.0f || (ry == 0.0f && rx < 0.0f)) rtie |= 1u << (16 + j);
        }
    }
    mnx = group_min<LPF>(mnx);
    mxx = group_max<LPF>(mxx);
    mny = group_min<LPF>(mny);
    mxy = group_max<LPF>(mxy);
    flags = group_or<LPF>(flags);
    stie = group_or<LPF>(stie);
    rtie = group_or<LPF>(rtie);
    if (active && sub == 0) {
        const FanRect r = rect_from_bounds_rel(mnx, mxx, mny, mxy, (int)s.ox[slot], (int)s.oy[slot], a.W, a.H);
        s.stie[slot] = stie;
        s.rtie[slot] = rtie;
        s.flags[slot] = (tmask == 0 || r.empty) ? 0u : flags;
        s.q[slot] = q;
        s.fan[slot] = fan;
        s.rect[slot] = make_int4(r.i0, r.i1, r.j0, r.j1);
    }
}
// The value part of stage_fans (fill passes): the double-float centre projection, the
// boundary vertices' screen offsets and view offsets, 1 / depth, colours and opacities.
template <int LPF>
__device__ __forceinline__ void stage_values(const SceneDev &a, const Stage &s, int K, int slot, int sub, uint32_t fan,
                                             const float *p) {
    constexpr int CH = 32 / LPF;
    const int KV = K + 1;
    const float m[3] = {__ldg(p), __ldg(p + 1), __ldg(p + 2)};
    const CentreProj cp = project_centre(*a.cam, m);
    const dfl zc = df_fast_two_sum(cp.Zh, cp.Zl);
    if (sub == 0) {
        s.cxh[slot] = cp.xh;
        s.cxl[slot] = cp.xl;
        s.cyh[slot] = cp.yh;
        s.cyl[slot] = cp.yl;
        s.viz[slot] = 1.0f / zc.h;
        const dfl xf = df_mul_f(df_fast_two_sum(cp.Xh, cp.Xl), a.cam->fx);
        const dfl yf = df_mul_f(df_fast_two_sum(cp.Yh, cp.Yl), a.cam->fy);
        s.pc[slot] = xf.h;
        s.pc[CH + slot] = xf.l;
        s.pc[2 * CH + slot] = yf.h;
        s.pc[3 * CH + slot] = yf.l;
        s.pc[4 * CH + slot] = zc.h;
        s.pc[5 * CH + slot] = zc.l;
    }
    for (int i = sub; i < K; i += LPF) {
        const float *pi = p + 3 * (1 + i);
        const float d[3] = {__ldg(pi) - m[0], __ldg(pi + 1) - m[1], __ldg(pi + 2) - m[2]};
        float du, dv, X, Y, Z;
        vertex_offset(*a.cam, cp, d, du, dv, X, Y, Z);
        s.du[i * CH + slot] = du;
        s.dv[i * CH + slot] = dv;
        // the exact view offset e = R (b_i - c) in double-float, for the fragment depths
        const DfVec e = df_view_offset(*a.cam, m, pi);
        s.viz[(1 + i) * CH + slot] = 1.0f / df_add(zc, e.z).h;
        const int u = i * CH + slot;
        s.exh[u] = e.x.h;
        s.exl[u] = e.x.l;
        s.eyh[u] = e.y.h;
        s.eyl[u] = e.y.l;
        s.ezh[u] = e.z.h;
        s.ezl[u] = e.z.l;
    }
    const float *col = a.rgb + (size_t)fan * KV * 3;
    const float *al = a.alpha + (size_t)fan * KV;
    for (int k = sub; k < KV; k += LPF) {
        s.cr[k * CH + slot] = __ldg(col + 3 * k);
        s.cg[k * CH + slot] = __ldg(col + 3 * k + 1);
        s.cb[k * CH + slot] = __ldg(col + 3 * k + 2);
        s.ca[k * CH + slot] = __ldg(al + k);
    }
}

// Stages CH = 32 / LPF fans into slots 0..CH-1 with the whole warp: the LPF lanes of slot
// lane / LPF share the fan's vertices, triangles and colours (every lane of the warp
// calls this; a lane whose slot is not active does no loads or stores but takes part in
// the shuffles).  The staged words are the same as one lane per fan would write.  With
// `decide` false (warp-uniform) only the fan id, depth bound and the values are staged:
// the caller already holds the fans' coverage masks and pixel rectangles.
template <int LPF>
__device__ __forceinline__ void stage_fans(const SceneDev &a, const Stage &s, int K, int lane, bool active,
                                           uint32_t fan, uint32_t q, int level, bool decide = true) {
    const int slot = lane / LPF, sub = lane % LPF;
    const float *p = a.xyz + (size_t)fan * (K + 1) * 3;
    if (decide)
        stage_decisions<LPF>(a, s, K, slot, sub, active, fan, q);
    else if (active && sub == 0) {
        s.q[slot] = q;
        s.fan[slot] = fan;
    }
    if (level < kStageValues || !active) return;
    stage_values<LPF>(a, s, K, slot, sub, fan, p);
}
// Coverage of the pixel centre (pxc, pyc) by staged fan f: bit j is set when triangle j
// covers it.  Each spoke value is computed once and turned into two pass bits (as the
// edge c -> b_i and as its reverse; the top-left tie bit of each direction was staged),
// so a triangle's two spoke tests are a bit test; only triangles passing both get the
// rim edge.  The result is the conjunction of the three edge tests, as stated.
template <int KT>
__device__ __forceinline__ uint32_t cover_mask(const Stage &S, int CH, int K, int f, uint32_t flags, float pxc,
                                               float pyc) {
    const float xc = S.vx[f], yc = S.vy[f];
    const float qx = __fsub_rn(pxc, xc), qy = __fsub_rn(pyc, yc);
    const uint32_t stie = S.stie[f];
    uint32_t P = 0, N = 0;
#pragma unroll(KT > 0 ? KT : 1)
    for (int i = 0; i < K; ++i) {
        const float Si = __fsub_rn(__fmul_rn(S.sdx[i * CH + f], qy), __fmul_rn(S.sdy[i * CH + f], qx));
        const bool z = Si == 0.0f;
        P |= (uint32_t)(Si > 0.0f || (z && ((stie >> i) & 1u))) << i;
        N |= (uint32_t)(Si < 0.0f || (z && ((stie >> (16 + i)) & 1u))) << i;
    }
    const uint32_t full = (1u << K) - 1u;
    const uint32_t Pn = ((P >> 1) | (P << (K - 1))) & full;   // bit j: spoke j+1
    const uint32_t Nn = ((N >> 1) | (N << (K - 1))) & full;
    const uint32_t negm = flags >> 16;
    uint32_t cand = ((P & Nn & ~negm) | (N & Pn & negm)) & flags & full;
    uint32_t hits = 0;
    const uint32_t rtie = S.rtie[f];
    while (cand) {
        const int j = __ffs(cand) - 1;
        cand &= cand - 1;
        const bool neg = (negm >> j) & 1u;
        const bool wrap = (j + 1 == K);
        const int lo = wrap ? 0 : j;
        const float Rc = dec_edge(S.rdx[j * CH + f], S.rdy[j * CH + f], S.vx[(1 + lo) * CH + f],
                                  S.vy[(1 + lo) * CH + f], pxc, pyc);
        // oriented rim: b_j -> b_{j+1} for positive orientation, reversed otherwise
        const bool flip = wrap != neg;
        const float E0 = flip ? -Rc : Rc;
        if (E0 > 0.0f || (E0 == 0.0f && ((rtie >> (flip ? 16 + j : j)) & 1u))) hits |= 1u << j;
    }
    return hits;
}

// Depth of triangle j = (c, b_j, b_j+1) of staged fan f at the pixel centre (pxc, pyc)
// (absolute screen coordinates), in double-float: the view depth where the pixel's ray
// r = ((x - cx) / fx, (y - cy) / fy, 1) meets the triangle's plane, Z = n . P_c / n . r with
// n = e_j x e_j+1 the normal from the vertices' exact view offsets and P_c the centre's
// view position (numerator and denominator both scaled by fx fy), which equals
// 1 / sum_k (lambda_k / Z_k) of the perspective-correct barycentrics.  Clamped to the
// triangle's vertex depths, where a covered centre lies (the clamp acts only where the
// decided coverage and the exact plane differ by rounding; a ray parallel to the plane
// takes the least vertex depth).
__device__ __forceinline__ dfl frag_depth_df(const Stage &S, int CH, int K, int f, int j, float pxc, float pyc,
                                             const CamDev &c) {
    const int jn = (j + 1 == K) ? 0 : j + 1;
    const int u = j * CH + f, w = jn * CH + f;
    const dfl e1x = {S.exh[u], S.exl[u]}, e1y = {S.eyh[u], S.eyl[u]}, e1z = {S.ezh[u], S.ezl[u]};
    const dfl e2x = {S.exh[w], S.exl[w]}, e2y = {S.eyh[w], S.eyl[w]}, e2z = {S.ezh[w], S.ezl[w]};
    const dfl xf = {S.pc[f], S.pc[CH + f]}, yf = {S.pc[2 * CH + f], S.pc[3 * CH + f]};
    const dfl zc = {S.pc[4 * CH + f], S.pc[5 * CH + f]};
    const dfl nx = df_add_fast(df_mul(e1y, e2z), df_neg(df_mul(e1z, e2y)));
    const dfl ny = df_add_fast(df_mul(e1z, e2x), df_neg(df_mul(e1x, e2z)));
    const dfl nz = df_add_fast(df_mul(e1x, e2y), df_neg(df_mul(e1y, e2x)));
    const dfl pa = df_mul_f(nx, c.fy), pb = df_mul_f(ny, c.fx), pn = df_mul_f(df_mul_f(nz, c.fx), c.fy);
    const dfl num = df_add_fast(df_add_fast(df_mul(pa, xf), df_mul(pb, yf)), df_mul(pn, zc));
    const dfl den = df_add_fast(df_add_fast(df_mul(pa, df_two_sum(pxc, -c.cx)), df_mul(pb, df_two_sum(pyc, -c.cy))),
                                pn);
    const dfl z1 = df_add_fast(zc, e1z), z2 = df_add_fast(zc, e2z);
    dfl lo = zc, hi = zc;
    if (df_lt(z1, lo)) lo = z1;
    if (df_lt(z2, lo)) lo = z2;
    if (df_lt(hi, z1)) hi = z1;
    if (df_lt(hi, z2)) hi = z2;
    if (den.h == 0.0f) return lo;
    dfl z = df_div_rcp(num, den);
    if (!(z.h == z.h)) return lo;   // NaN
    if (df_lt(z, lo)) z = lo;
    if (df_lt(hi, z)) z = hi;
    return z;
}

// ------------------------------------------------------------------------------------
// Source-Gaussian splats (FP64: the splat image is the reference the fans approximate,
// drawn once per view, so precision is worth more than speed here)
// ------------------------------------------------------------------------------------

struct SplatSlot {
    double mc[3], ua[3], ub[3], n[3];   // camera-space centre, kept unit axes, plane normal
    double mcn, sa, sb;                 // mc . n, the two kept scales
    float sigma, col[3];
};

// The flat Gaussian g in the camera frame: rotation from the normalised quaternion
// (w, x, y, z), the two kept axes by the same rule as the fan conversion.
__device__ __forceinline__ SplatSlot splat_setup(const SplatSrc &src, const CamDev &c, uint32_t g) {
    SplatSlot o;
    const float4 qf = *reinterpret_cast<const float4 *>(src.quats + 4 * (size_t)g);
    const double qn = sqrt((double)qf.x * qf.x + (double)qf.y * qf.y + (double)qf.z * qf.z + (double)qf.w * qf.w);
    const double w = qf.x / qn, x = qf.y / qn, y = qf.z / qn, z = qf.w / qn;
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                         2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
    const float *ls = src.log_scales + 3 * (size_t)g;
    const float s0 = ls[0], s1 = ls[1], s2 = ls[2];
    int drop = 0;
    if (src.axis_rule == 1) {
        float sm = s0;
        if (s1 < sm) { drop = 1; sm = s1; }
        if (s2 < sm) drop = 2;
    }
    const int ia = drop == 0 ? 1 : 0, ib = drop == 2 ? 1 : 2;
    const float *m = src.means + 3 * (size_t)g;
    const double dm[3] = {(double)m[0] - (double)c.C[0], (double)m[1] - (double)c.C[1], (double)m[2] - (double)c.C[2]};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double R0 = c.R[3 * r], R1 = c.R[3 * r + 1], R2 = c.R[3 * r + 2];
        o.mc[r] = R0 * dm[0] + R1 * dm[1] + R2 * dm[2];
        o.ua[r] = R0 * R[ia] + R1 * R[3 + ia] + R2 * R[6 + ia];
        o.ub[r] = R0 * R[ib] + R1 * R[3 + ib] + R2 * R[6 + ib];
    }
    o.n[0] = o.ua[1] * o.ub[2] - o.ua[2] * o.ub[1];
    o.n[1] = o.ua[2] * o.ub[0] - o.ua[0] * o.ub[2];
    o.n[2] = o.ua[0] * o.ub[1] - o.ua[1] * o.ub[0];
    o.mcn = o.mc[0] * o.n[0] + o.mc[1] * o.n[1] + o.mc[2] * o.n[2];
    o.sa = exp((double)(ia == 0 ? s0 : s1));
    o.sb = exp((double)(ib == 2 ? s2 : s1));
    o.sigma = src.opacity[g];
    o.col[0] = src.rgb[3 * (size_t)g];
    o.col[1] = src.rgb[3 * (size_t)g + 1];
    o.col[2] = src.rgb[3 * (size_t)g + 2];
    return o;
}

// Ray of pixel centre (px, py) against splat s: kept when the hit lies in front of the
// near plane and inside the truncation ellipse; t = view depth of the hit (rounded to
// binary32 as the order key), a = sigma exp(-(u^2/sa^2 + v^2/sb^2)/2).
__device__ __forceinline__ bool splat_hit(const SplatSlot &s, const CamDev &c, double trunc, double px, double py,
                                          float &t, float &a) {
    const double d0 = (px - (double)c.cx) / (double)c.fx, d1 = (py - (double)c.cy) / (double)c.fy;
    const double den = d0 * s.n[0] + d1 * s.n[1] + s.n[2];
    if (den == 0.0) return false;
    const double tt = s.mcn / den;
    if (!(tt > (double)c.znear)) return false;
    const double w0 = tt * d0 - s.mc[0], w1 = tt * d1 - s.mc[1], w2 = tt - s.mc[2];
    const double u = w0 * s.ua[0] + w1 * s.ua[1] + w2 * s.ua[2];
    const double v = w0 * s.ub[0] + w1 * s.ub[1] + w2 * s.ub[2];
    const double ru = u / (trunc * s.sa), rv = v / (trunc * s.sb);
    if (!(ru * ru + rv * rv <= 1.0)) return false;
    t = (float)tt;
    a = (float)((double)s.sigma * exp(-0.5 * (u * u / (s.sa * s.sa) + v * v / (s.sb * s.sb))));
    return true;
}

}  // namespace ms
