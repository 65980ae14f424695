// Per-fan screen-space setup shared by binning and the composite kernels, so that
// both derive bit-identical pixel rectangles and depth keys for a fan.
#pragma once

#include "ms_common.cuh"

namespace ms {

struct FanRect {
    int i0, i1, j0, j1;   // inclusive pixel range that may hold covered pixel centres
    float zmin;           // smallest decided vertex depth of the valid triangles
    uint32_t valid;       // bit j: triangle j has three valid vertices
    bool empty;
};

// Pixel centres i + 0.5 within [min x - 0.5, max x + 0.5] (and the same in y) of the
// valid triangles' vertices.  The half-pixel margin exceeds the binary32 rounding of
// the edge test for coordinates within the +-2^17 guard band, so no covered centre
// falls outside.
__device__ __forceinline__ FanRect fan_rect(const DVert *v, int K, int W, int H) {
    FanRect r;
    r.valid = 0;
    float mnx = 3.0e38f, mxx = -3.0e38f, mny = 3.0e38f, mxy = -3.0e38f, zmin = 3.0e38f;
    const bool cv = v[0].valid;
    for (int j = 0; j < K; ++j) {
        const int b = 1 + j, c = 1 + (j + 1 == K ? 0 : j + 1);
        if (cv && v[b].valid && v[c].valid) {
            r.valid |= 1u << j;
            mnx = fminf(mnx, fminf(v[b].xs, v[c].xs));
            mxx = fmaxf(mxx, fmaxf(v[b].xs, v[c].xs));
            mny = fminf(mny, fminf(v[b].ys, v[c].ys));
            mxy = fmaxf(mxy, fmaxf(v[b].ys, v[c].ys));
            zmin = fminf(zmin, fminf(v[b].Z, v[c].Z));
        }
    }
    if (r.valid) {
        mnx = fminf(mnx, v[0].xs);
        mxx = fmaxf(mxx, v[0].xs);
        mny = fminf(mny, v[0].ys);
        mxy = fmaxf(mxy, v[0].ys);
        zmin = fminf(zmin, v[0].Z);
    }
    r.zmin = zmin;
    if (!r.valid) {
        r.empty = true;
        r.i0 = r.j0 = 1;
        r.i1 = r.j1 = 0;
        return r;
    }
    r.i0 = max((int)floorf(mnx - 1.0f), 0);
    r.i1 = min((int)floorf(mxx), W - 1);
    r.j0 = max((int)floorf(mny - 1.0f), 0);
    r.j1 = min((int)floorf(mxy), H - 1);
    r.empty = r.i0 > r.i1 || r.j0 > r.j1;
    return r;
}

}  // namespace ms
