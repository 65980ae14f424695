// Per-Gaussian body of the Gaussian -> triangle-fan conversion (Sec. 3, "MeshSplats
// Transformation for Flat Gaussians", Eq. 2 and the vertex equation after it; and
// "Transformation for 3D Gaussians"), shared by the plain conversion kernel and the
// conversion fused behind the learned initializer's inference.  One thread converts one
// Gaussian into shared-memory staging; the caller stores the block's staging coalesced.
#pragma once

#include <math.h>

#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {
namespace mb {

struct Gaussians {
    const float *means, *log_scales, *quats, *opacity;
    const void *sh;
};

__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float(((uint32_t)b) << 16); }

// Real SH basis (degree <= 3) at a unit direction, FP32.  Y_{l,m} = sqrt2 Im(Y_l^|m|)
// for m < 0, Y_l^0, sqrt2 Re(Y_l^m) for m > 0 (complex harmonics with the
// Condon-Shortley phase), written as polynomials in (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_basis(const MeshBuildConst &k, float x, float y, float z, float *Y) {
    Y[0] = k.shc[0];
    if (DEG >= 1) {
        Y[1] = -k.shc[1] * y;
        Y[2] = k.shc[1] * z;
        Y[3] = -k.shc[1] * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = k.shc[2] * x * y;
        Y[5] = -k.shc[2] * y * z;
        Y[6] = k.shc[3] * (2.0f * zz - xx - yy);
        Y[7] = -k.shc[2] * x * z;
        Y[8] = k.shc[4] * (xx - yy);
        if (DEG >= 3) {
            float t = 4.0f * zz - xx - yy;
            Y[9] = -k.shc[5] * y * (3.0f * xx - yy);
            Y[10] = 2.0f * k.shc[6] * x * y * z;
            Y[11] = -k.shc[7] * y * t;
            Y[12] = k.shc[8] * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -k.shc[7] * x * t;
            Y[14] = k.shc[6] * z * (xx - yy);
            Y[15] = -k.shc[5] * x * (xx - 3.0f * yy);
        }
    }
}

// Colour from the SH coefficients of Gaussian g: col[ch] = max(0, 0.5 + sum_{i < nuse}
// Y_i f_{i,ch}), accumulated in coefficient order.  The coefficients stream through
// registers 16 bytes at a time (flat index 3 i + ch), so only Y and the accumulators stay
// live.
template <int DEG, bool BF16>
__device__ __forceinline__ void sh_colour(const void *sh, int64_t g, bool vec_ok, const float *Y, int nuse,
                                          float col[3]) {
    constexpr int NC = 3 * (DEG + 1) * (DEG + 1);
    float acc[3] = {0.5f, 0.5f, 0.5f};
    auto add = [&](int idx, float v) {
        if (idx / 3 < nuse) acc[idx % 3] = fmaf(Y[idx / 3], v, acc[idx % 3]);
    };
    if (BF16) {
        const uint16_t *p = reinterpret_cast<const uint16_t *>(sh) + g * NC;
        if (NC % 8 == 0 && vec_ok) {
#pragma unroll
            for (int i = 0; i < NC / 8; ++i) {
                uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + i);
                uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    add(8 * i + 2 * j, __uint_as_float(w[j] << 16));
                    add(8 * i + 2 * j + 1, __uint_as_float(w[j] & 0xFFFF0000u));
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NC; ++i) add(i, bf16_to_f32(__ldg(p + i)));
        }
    } else {
        const float *p = reinterpret_cast<const float *>(sh) + g * NC;
        if (NC % 4 == 0 && vec_ok) {
#pragma unroll
            for (int i = 0; i < NC / 4; ++i) {
                float4 u = __ldg(reinterpret_cast<const float4 *>(p) + i);
                add(4 * i, u.x); add(4 * i + 1, u.y); add(4 * i + 2, u.z); add(4 * i + 3, u.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NC; ++i) add(i, __ldg(p + i));
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(acc[ch], 0.0f);
}

// Copies n floats from shared to global with the threads of the block; 16-byte stores
// when both ends allow it.
__device__ __forceinline__ void block_store(float *dst, const float *src, int n) {
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (n & 3) == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        for (int i = threadIdx.x; i < n / 4; i += blockDim.x) d4[i] = s4[i];
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
}

// Converts Gaussian g into staging vertices lv .. lv + GV - 1 (s_xyz, s_rgb: 3 floats per
// vertex; s_a: one).  cr: NULL, or the 2(K+1) corrections of g (radial dr_0..dr_K, then
// log-opacity do_0..do_K; flat fans only): boundary vertex i moves to
// m + (1 + dr_i)(cos th_i a + sin th_i b) and alpha_i <- clamp(alpha_i exp(do_i), 0, 1).
template <int DEG, bool BF16>
__device__ __forceinline__ void convert_gaussian(const Gaussians &G, const MeshBuildConst &kc, int64_t g,
                                                 const float *cr, float *s_xyz, float *s_rgb, float *s_a,
                                                 int lv) {
    const int KV = kc.K + 1;
    float m[3] = {__ldg(G.means + 3 * g), __ldg(G.means + 3 * g + 1), __ldg(G.means + 3 * g + 2)};
    float s[3] = {__ldg(G.log_scales + 3 * g), __ldg(G.log_scales + 3 * g + 1), __ldg(G.log_scales + 3 * g + 2)};
    float4 q = __ldg(reinterpret_cast<const float4 *>(G.quats) + g);
    float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
    // Rotation matrix, row-major; column c of R is the principal axis r_{c+1}.
    float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                  2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                  2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    int drop = 0;
    if (kc.axis_rule == 1) {
        if (s[1] < s[drop]) drop = 1;
        if (s[2] < s[drop]) drop = 2;
    }
    const int ia = drop == 0 ? 1 : 0, ib = drop == 2 ? 1 : 2;
    const float sa = kc.scale_mul * expf(s[ia]), sb = kc.scale_mul * expf(s[ib]);
    float a[3], b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        a[r] = sa * R[3 * r + ia];
        b[r] = sb * R[3 * r + ib];
    }
    constexpr int NB = (DEG + 1) * (DEG + 1);
    float Y[NB];
    int nuse = 1;
    float dx = m[0] - kc.cc[0], dy = m[1] - kc.cc[1], dz = m[2] - kc.cc[2];
    float dn = dx * dx + dy * dy + dz * dz;
    if (DEG > 0 && kc.has_cam && dn > 0.0f) {
        float inv = rsqrtf(dn);
        sh_basis<DEG>(kc, dx * inv, dy * inv, dz * inv, Y);
        nuse = NB;
    } else {
        Y[0] = kc.shc[0];
    }
    float col[3];   // one per Gaussian, inherited by all its vertices
    sh_colour<DEG, BF16>(G.sh, g, kc.sh_vec_ok, Y, nuse, col);
    const float sig = __ldg(G.opacity + g);
    if (kc.three) {
        float sr[3][3];   // sr[c] = scale_mul exp(s_c) r_c
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float sc = kc.scale_mul * expf(s[c]);
#pragma unroll
            for (int r = 0; r < 3; ++r) sr[c][r] = sc * R[3 * r + c];
        }
        for (int fan = 0; fan < 3; ++fan) {
            const int fa = fan == 2 ? 1 : 0, fb = fan == 0 ? 1 : 2;
            for (int k = 0; k < KV; ++k) {
                const int v = lv + fan * KV + k;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    s_xyz[3 * v + r] = k == 0 ? m[r]
                                              : m[r] + (kc.cs[k - 1] * sr[fa][r] + kc.sn[k - 1] * sr[fb][r]);
                    s_rgb[3 * v + r] = col[r];
                }
                s_a[v] = k == 0 ? sig : kc.opac_mul * sig;
            }
        }
        return;
    }
    for (int k = 0; k < KV; ++k) {
        float p[3];
        if (k == 0) {
            p[0] = m[0]; p[1] = m[1]; p[2] = m[2];
        } else {
            const float c = kc.cs[k - 1], sn = kc.sn[k - 1];
            const float rs = cr ? 1.0f + cr[k] : 1.0f;
#pragma unroll
            for (int r = 0; r < 3; ++r) p[r] = m[r] + rs * (c * a[r] + sn * b[r]);
        }
        float op = k == 0 ? sig : kc.opac_mul * sig;
        if (cr) op = fminf(fmaxf(op * expf(cr[KV + k]), 0.0f), 1.0f);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            s_xyz[3 * (lv + k) + r] = p[r];
            s_rgb[3 * (lv + k) + r] = col[r];
        }
        s_a[lv + k] = op;
    }
}

}  // namespace mb
}  // namespace ms
