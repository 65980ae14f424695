// Per-fan screen-space setup shared by binning and the composite kernels, so that
// both derive bit-identical pixel rectangles and depth keys for a fan.
#pragma once

#include "ms_common.cuh"

namespace ms {

struct FanRect {
    int i0, i1, j0, j1;   // inclusive pixel range that may hold covered pixel centres
    bool empty;
};

// Pixel centres i + 0.5 within [min x - 0.25, max x + 0.25] (and the same in y) of the
// vertices of the fan's valid triangles.  Bound on the binary32 edge test: a centre p it
// accepts lies within 2.1 * 2^-24 * (|p - a|_1) of each edge line (a = the edge's lower
// vertex), plus the turn of the rounded edge direction, < 0.07 + 0.03 px for anything in
// the +-2^17 guard band; the quarter-pixel margin exceeds that, so no covered centre
// falls outside.  min/max are order independent, so every caller that feeds the same
// vertex set gets the same rectangle.
__device__ __forceinline__ FanRect rect_from_bounds(float mnx, float mxx, float mny, float mxy, int W, int H) {
    FanRect r;
    r.i0 = max((int)ceilf(mnx - 0.75f), 0);
    r.i1 = min((int)floorf(mxx - 0.25f), W - 1);
    r.j0 = max((int)ceilf(mny - 0.75f), 0);
    r.j1 = min((int)floorf(mxy - 0.25f), H - 1);
    r.empty = r.i0 > r.i1 || r.j0 > r.j1;
    return r;
}

// rect_from_bounds for bounds given relative to the integer origin (ox, oy): identical
// pixel arithmetic in the relative frame, shifted by the origin.
__device__ __forceinline__ FanRect rect_from_bounds_rel(float mnx, float mxx, float mny, float mxy, int ox, int oy,
                                                        int W, int H) {
    FanRect r;
    r.i0 = max((int)ceilf(mnx - 0.75f) + ox, 0);
    r.i1 = min((int)floorf(mxx - 0.25f) + ox, W - 1);
    r.j0 = max((int)ceilf(mny - 0.75f) + oy, 0);
    r.j1 = min((int)floorf(mxy - 0.25f) + oy, H - 1);
    r.empty = r.i0 > r.i1 || r.j0 > r.j1;
    return r;
}

// Triangle j of a fan is valid when the centre and both of its boundary vertices are.
__device__ __forceinline__ uint32_t tri_valid_mask(uint32_t vmask, int K) {
    uint32_t t = 0;
    if (vmask & 1u)
        for (int j = 0; j < K; ++j) {
            const int jn = j + 1 == K ? 0 : j + 1;
            if (((vmask >> (1 + j)) & 1u) && ((vmask >> (1 + jn)) & 1u)) t |= 1u << j;
        }
    return t;
}

// Whether vertex k (0 = centre, 1 + i = boundary i) belongs to a valid triangle.
__device__ __forceinline__ bool vertex_used(uint32_t tmask, int k, int K) {
    if (k == 0) return tmask != 0;
    const int i = k - 1, ip = i == 0 ? K - 1 : i - 1;
    return ((tmask >> i) & 1u) || ((tmask >> ip) & 1u);
}

}  // namespace ms
