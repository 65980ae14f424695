// Shared device helpers of the MeshSplats CUDA library (sm_103a).
//
// The "decision" functions evaluate, in IEEE binary32 with the round-to-nearest
// intrinsics (which the compiler never fuses into FMAs), exactly the coverage and
// depth formulas stated in include/meshsplats.h; the value functions (barycentrics,
// interpolation, compositing, gradients) are free FP32 arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/meshsplats.h"

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
// Decisions (binary32, no contraction)
// ---------------------------------------------------------------------------------

struct DVert {
    float xs, ys, Z, iz;
    bool valid;
};

__device__ __forceinline__ DVert decide_vertex(const CamDev &c, float px, float py, float pz) {
    float dx = __fsub_rn(px, c.C[0]);
    float dy = __fsub_rn(py, c.C[1]);
    float dz = __fsub_rn(pz, c.C[2]);
    float X = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], dx), __fmul_rn(c.R[1], dy)), __fmul_rn(c.R[2], dz));
    float Y = __fadd_rn(__fadd_rn(__fmul_rn(c.R[3], dx), __fmul_rn(c.R[4], dy)), __fmul_rn(c.R[5], dz));
    float Z = __fadd_rn(__fadd_rn(__fmul_rn(c.R[6], dx), __fmul_rn(c.R[7], dy)), __fmul_rn(c.R[8], dz));
    DVert o;
    o.xs = __fadd_rn(__fmul_rn(c.fx, __fdiv_rn(X, Z)), c.cx);
    o.ys = __fadd_rn(__fmul_rn(c.fy, __fdiv_rn(Y, Z)), c.cy);
    o.Z = Z;
    o.iz = __frcp_rn(Z);
    o.valid = (Z > c.znear) && (fabsf(o.xs) <= kGuardPx) && (fabsf(o.ys) <= kGuardPx);
    return o;
}

// The validity rule of decide_vertex, from stored decided values.
__device__ __forceinline__ bool vertex_valid(const CamDev &c, float xs, float ys, float Z) {
    return (Z > c.znear) && (fabsf(xs) <= kGuardPx) && (fabsf(ys) <= kGuardPx);
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

__device__ __forceinline__ float dec_depth(float area2, float E0, float iz0, float E1, float iz1, float E2,
                                           float iz2, float Za, float Zb, float Zc) {
    float w = __fadd_rn(__fadd_rn(__fmul_rn(E0, iz0), __fmul_rn(E1, iz1)), __fmul_rn(E2, iz2));
    float z = __fdiv_rn(area2, w);
    float zlo = fminf(fminf(Za, Zb), Zc);
    float zhi = fmaxf(fmaxf(Za, Zb), Zc);
    return fminf(fmaxf(z, zlo), zhi);
}

// Quantised depth used in sort keys and in the commit test: the top `bits` bits of
// the (positive) binary32 pattern; monotone non-decreasing in z.
__device__ __forceinline__ uint32_t depth_q(float z, int bits) {
    return __float_as_uint(z) >> (31 - bits);
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
