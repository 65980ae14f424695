// Shared device helpers of the MeshSplats CUDA library (sm_103a).
//
// The "decision" functions evaluate the coverage formulas stated in
// include/meshsplats.h in IEEE binary32 with the round-to-nearest intrinsics (which the
// compiler never fuses into FMAs), on vertex positions taken from a double-float
// projection; the fragment order uses a double-float depth.  The value functions
// (barycentrics, interpolation, compositing, gradients) are free FP32 arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/meshsplats.h"
#include "dfloat.cuh"

namespace ms {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr float kGuardPx = 131072.0f;   // |xs|, |ys| <= 2^17
constexpr int kMaxK = 16;
constexpr uint32_t kSpinLimit = 1u << 20;   // polls before a bounded wait gives up

// Device-side outcome block at the start of every render workspace.
struct Status {
    unsigned long long pairs;        // pairs produced by binning
    unsigned long long culled;       // culled triangles
    unsigned long long extra_passes; // pixel passes re-run after buffer overflow
    unsigned long long cap;          // pair capacity of the workspace
    unsigned int timeouts;           // bounded waits that expired
    unsigned int bin_ticket;         // virtual block ids of the binning scan
    unsigned int sort_ticket[8];     // virtual block ids of each sort pass
    unsigned int n_tiles;
    unsigned int sort_bits;
    unsigned long long rect_tests;   // forward rasterisation / resolve work counters
    unsigned long long fragments;
    unsigned long long commits;
    unsigned long long frags;        // fragment records the pixel scan counted
    unsigned long long frag_cap;     // fragment record capacity of the workspace
    unsigned int scan_ticket;        // virtual block ids of the pixel scan
    unsigned int tscan_ticket;       // virtual block ids of the tile work-item scan
    unsigned int n_items;            // raster work items (<= 64 fans of one tile each)
    unsigned long long items_total;  // work items the tile scan counted
};
// The count pass's coverage masks live in this many equal regions, each with its own cursor.
constexpr int kMaskRegions = 256;
static_assert(sizeof(Status) <= 256, "status block");

struct CamDev {
    float R[9];
    float C[3];
    float fx, fy, cx, cy, znear;
    int width, height;
};

inline CamDev make_cam(const ms_camera &c) {
    CamDev d;
    for (int i = 0; i < 9; ++i) d.R[i] = c.R_cw[i];
    for (int i = 0; i < 3; ++i) d.C[i] = c.C[i];
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.znear = c.znear;
    d.width = c.width; d.height = c.height;
    return d;
}

// Views of one render call.  Tiles and pixels of all views form one index space: view v
// owns global tiles [tile_base, tile_base + tiles) and pixels [pix_base, pix_base + W H).
// The table travels to the kernels as a __grid_constant__ parameter.
constexpr int kMaxViews = MS_MAX_VIEWS;
struct ViewDev {
    CamDev cam;
    uint32_t tile_base, tiles_x;
    unsigned long long pix_base;
    float *out;               // forward output image, H x W x 4
    const float *dL;          // backward: dL / d image
    const float *out_fwd;     // backward: the forward image
};
struct ViewTable {
    int n;
    ViewDev v[kMaxViews];
};

__device__ __forceinline__ int view_of_tile(const ViewTable &t, uint32_t tile) {
    int lo = 0, hi = t.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t.v[mid].tile_base <= tile) lo = mid; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int view_of_pixel(const ViewTable &t, unsigned long long pix) {
    int lo = 0, hi = t.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t.v[mid].pix_base <= pix) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------------
// Decisions
// ---------------------------------------------------------------------------------

// Double-float dot product of a binary32 row R with the double-float vector d: exact
// products of the high parts (FMA residuals), their sum by two-sums, and the remaining
// error terms summed in binary32.
__device__ __forceinline__ dfl df_row_dot(const float *R, dfl d0, dfl d1, dfl d2) {
    const dfl p0 = df_two_prod(R[0], d0.h), p1 = df_two_prod(R[1], d1.h), p2 = df_two_prod(R[2], d2.h);
    const dfl s = df_two_sum(p0.h, p1.h);
    const dfl t = df_two_sum(s.h, p2.h);
    const float l = __fadd_rn(__fadd_rn(__fadd_rn(s.l, t.l), __fadd_rn(__fadd_rn(p0.l, p1.l), p2.l)),
                              fmaf(R[0], d0.l, fmaf(R[1], d1.l, __fmul_rn(R[2], d2.l))));
    return df_fast_two_sum(t.h, l);
}

// f (N / Z) + c in double-float, the quotient from one reciprocal of Z.h and a
// double-float residual correction.
__device__ __forceinline__ dfl df_screen_coord(dfl N, dfl Z, float rz, float f, float c) {
    const float q1 = __fmul_rn(N.h, rz);
    const float r = __fadd_rn(fmaf(-q1, Z.h, N.h), fmaf(-q1, Z.l, N.l));
    const dfl q = df_fast_two_sum(q1, __fmul_rn(r, rz));
    dfl a = df_mul_f(q, f);
    return df_add_f(a, c);
}

// Camera-space position (X, Y, Z) and screen position (x, y) of a world point, all in
// double-float: d = p - C is exact, then the rotation and the pinhole division.
struct DfVert {
    dfl X, Y, Z, x, y;
};
__device__ __forceinline__ DfVert df_project(const CamDev &c, float px, float py, float pz) {
    const dfl d0 = df_two_sum(px, -c.C[0]), d1 = df_two_sum(py, -c.C[1]), d2 = df_two_sum(pz, -c.C[2]);
    DfVert o;
    o.X = df_row_dot(c.R, d0, d1, d2);
    o.Y = df_row_dot(c.R + 3, d0, d1, d2);
    o.Z = df_row_dot(c.R + 6, d0, d1, d2);
    const float rz = __frcp_rn(o.Z.h);
    o.x = df_screen_coord(o.X, o.Z, rz, c.fx, c.cx);
    o.y = df_screen_coord(o.Y, o.Z, rz, c.fy, c.cy);
    return o;
}

// A vertex as the coverage decisions see it: the double-float screen position rounded to
// binary32 (xs, ys) and relative to its fan's integer origin (xr, yr) = nearest binary32
// value of (x - ox, y - oy), its rounded depth Z, and the validity rule on the rounded
// values (Z > znear, |xs|, |ys| <= 2^17).
struct DVert {
    float xs, ys, xr, yr, Z;
    bool valid;
};

// Nearest binary32 value of v - o for an integer-valued binary32 o (exact two-sum of the
// high part, then the low parts).
__device__ __forceinline__ float df_offset(dfl v, float o) {
    const dfl s = df_two_sum(v.h, -o);
    return __fadd_rn(s.h, __fadd_rn(s.l, v.l));
}

__device__ __forceinline__ DVert decide_vertex(const CamDev &c, const DfVert &v, float ox, float oy) {
    DVert o;
    o.xs = df_round(v.x);
    o.ys = df_round(v.y);
    o.xr = df_offset(v.x, ox);
    o.yr = df_offset(v.y, oy);
    o.Z = df_round(v.Z);
    o.valid = (o.Z > c.znear) && (fabsf(o.xs) <= kGuardPx) && (fabsf(o.ys) <= kGuardPx);
    return o;
}

__device__ __forceinline__ float dec_area2(float xa, float ya, float xb, float yb, float xc, float yc) {
    return __fsub_rn(__fmul_rn(__fsub_rn(xb, xa), __fsub_rn(yc, ya)),
                     __fmul_rn(__fsub_rn(yb, ya), __fsub_rn(xc, xa)));
}

// Canonical edge value from vertex lo (lower index) to hi, with the direction
// (ex, ey) = (hi - lo) precomputed.
__device__ __forceinline__ float dec_edge(float ex, float ey, float lx, float ly, float px, float py) {
    return __fsub_rn(__fmul_rn(ex, __fsub_rn(py, ly)), __fmul_rn(ey, __fsub_rn(px, lx)));
}

// Top-left acceptance of an oriented edge value E with direction (ex, ey).
__device__ __forceinline__ bool edge_pass(float E, float ex, float ey) {
    return E > 0.0f || (E == 0.0f && (ey < 0.0f || (ey == 0.0f && ex > 0.0f)));
}

// Quantised depth used in sort keys and in the commit test.  A view's vertex depths span
// [zlo, zhi] (a pre-pass over the vertices); the key is the offset of the binary32 pattern
// of z from that of zlo (lowered by a margin), shifted right so that the span fits `bits`
// bits, clamped to [0, 2^bits - 1].  Positive binary32 patterns order like their values,
// so the map is monotone non-decreasing in z; it spends the bits on the view's depth range
// instead of on the whole exponent range.  zr[2 v] holds the complement of zlo's pattern
// (maximised atomically), zr[2 v + 1] zhi's pattern.
struct DepthQ {
    uint32_t base, shift, qmax;
};
__device__ __forceinline__ DepthQ depth_quant(const uint32_t *zr, int view, int bits) {
    const uint32_t lo = ~zr[2 * view], hi = zr[2 * view + 1];
    DepthQ d;
    d.qmax = (1u << bits) - 1u;
    if (hi < lo) {   // no vertex in front of the view: any monotone map
        d.base = 0;
        d.shift = 31u - (uint32_t)bits;
        return d;
    }
    constexpr uint32_t kMargin = 256;   // ulps below zlo / above zhi (keys sit 2^-20 below)
    d.base = lo > kMargin ? lo - kMargin : 0u;
    const uint32_t span = (hi + kMargin) - d.base;
    const int need = 32 - __clz(span);   // bits of the span
    d.shift = (uint32_t)max(0, need - bits);
    return d;
}
__device__ __forceinline__ uint32_t depth_qv(const DepthQ &d, float z) {
    const uint32_t b = __float_as_uint(z);
    return b <= d.base ? 0u : min((b - d.base) >> d.shift, d.qmax);
}

// ---------------------------------------------------------------------------------
// Bounded waits
// ---------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace ms
