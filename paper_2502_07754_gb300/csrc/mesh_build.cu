// Gaussian -> triangle-fan conversion with SH colour (Sec. 3, "MeshSplats
// Transformation for Flat Gaussians", Eq. 2 and the vertex equation after it; and
// "Transformation for 3D Gaussians": all three scaled axes kept, one fan per pair of axes
// (1, 2), (1, 3), (2, 3), written as three implicit fans of K triangles per Gaussian whose
// shared vertices -- the centre and the axis tips two fans reach -- are copies; the
// angle table then holds exact cosine and sine at quarter turns, so the copies are equal
// bit for bit).
//
// One thread per Gaussian.  The block's vertices are assembled in shared memory and
// leave in 16-byte coalesced stores, so each output byte crosses HBM once:
// read 44 B + SH, write 28 (K+1) B per fan.
#include <math.h>

#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kMBThreads = 128;

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

template <int DEG, bool BF16>
__device__ __forceinline__ void load_sh(const void *sh, int64_t g, bool vec_ok, float *f) {
    constexpr int NC = 3 * (DEG + 1) * (DEG + 1);
    if (BF16) {
        const uint16_t *p = reinterpret_cast<const uint16_t *>(sh) + g * NC;
        if (NC % 8 == 0 && vec_ok) {
#pragma unroll
            for (int i = 0; i < NC / 8; ++i) {
                uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + i);
                uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    f[8 * i + 2 * j] = __uint_as_float(w[j] << 16);
                    f[8 * i + 2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NC; ++i) f[i] = bf16_to_f32(__ldg(p + i));
        }
    } else {
        const float *p = reinterpret_cast<const float *>(sh) + g * NC;
        if (NC % 4 == 0 && vec_ok) {
#pragma unroll
            for (int i = 0; i < NC / 4; ++i) {
                float4 u = __ldg(reinterpret_cast<const float4 *>(p) + i);
                f[4 * i] = u.x; f[4 * i + 1] = u.y; f[4 * i + 2] = u.z; f[4 * i + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NC; ++i) f[i] = __ldg(p + i);
        }
    }
}

// Copies n floats from shared to global; 16-byte stores when both ends allow it.
__device__ __forceinline__ void block_store(float *dst, const float *src, int n) {
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (n & 3) == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        for (int i = threadIdx.x; i < n / 4; i += blockDim.x) d4[i] = s4[i];
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
}

template <int DEG, bool BF16>
__global__ void __launch_bounds__(kMBThreads) mesh_build_kernel(
    const float *__restrict__ means, const float *__restrict__ log_scales, const float *__restrict__ quats,
    const float *__restrict__ opacity, const void *__restrict__ sh, int64_t N, MeshBuildConst kc,
    const float *__restrict__ corr, float *__restrict__ xyz, float *__restrict__ rgb, float *__restrict__ alpha) {
    extern __shared__ float smem[];
    const int K = kc.K, KV = K + 1;
    const int GV = (kc.three ? 3 : 1) * KV;      // vertices per Gaussian
    float *s_xyz = smem;                          // kMBThreads * GV * 3
    float *s_rgb = s_xyz + kMBThreads * GV * 3;   // kMBThreads * GV * 3
    float *s_a = s_rgb + kMBThreads * GV * 3;     // kMBThreads * GV

    const int64_t g0 = (int64_t)blockIdx.x * kMBThreads;
    const int64_t g = g0 + threadIdx.x;
    const int nloc = (int)min64(kMBThreads, N - g0);
    if (g < N) {
        float m[3] = {__ldg(means + 3 * g), __ldg(means + 3 * g + 1), __ldg(means + 3 * g + 2)};
        float s[3] = {__ldg(log_scales + 3 * g), __ldg(log_scales + 3 * g + 1), __ldg(log_scales + 3 * g + 2)};
        float4 q = __ldg(reinterpret_cast<const float4 *>(quats) + g);
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
        // Colour (one per Gaussian, inherited by all its vertices).
        constexpr int NB = (DEG + 1) * (DEG + 1);
        float f[3 * NB];
        load_sh<DEG, BF16>(sh, g, kc.sh_vec_ok, f);
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
        float col[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (i < nuse) acc = fmaf(Y[i], f[3 * i + ch], acc);
            col[ch] = fmaxf(acc, 0.0f);
        }
        const float sig = __ldg(opacity + g);
        const int lv = threadIdx.x * GV;
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
        }
        const float *cr = corr ? corr + g * 2 * KV : nullptr;
        for (int k = 0; k < KV && !kc.three; ++k) {
            float p[3];
            if (k == 0) {
                p[0] = m[0]; p[1] = m[1]; p[2] = m[2];
            } else {
                const float c = kc.cs[k - 1], sn = kc.sn[k - 1];
                const float rs = cr ? 1.0f + __ldg(cr + k) : 1.0f;
#pragma unroll
                for (int r = 0; r < 3; ++r) p[r] = m[r] + rs * (c * a[r] + sn * b[r]);
            }
            float op = k == 0 ? sig : kc.opac_mul * sig;
            if (cr) op = fminf(fmaxf(op * expf(__ldg(cr + KV + k)), 0.0f), 1.0f);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                s_xyz[3 * (lv + k) + r] = p[r];
                s_rgb[3 * (lv + k) + r] = col[r];
            }
            s_a[lv + k] = op;
        }
    }
    __syncthreads();
    const int64_t v0 = g0 * GV;
    block_store(xyz + 3 * v0, s_xyz, 3 * nloc * GV);
    block_store(rgb + 3 * v0, s_rgb, 3 * nloc * GV);
    block_store(alpha + v0, s_a, nloc * GV);
}

template <int DEG>
cudaError_t launch_deg(bool bf16, const float *means, const float *log_scales, const float *quats,
                       const float *opacity, const void *sh, int64_t N, const MeshBuildConst &kc, const float *corr,
                       float *xyz, float *rgb, float *alpha, cudaStream_t st) {
    const int GV = (kc.three ? 3 : 1) * (kc.K + 1);
    const size_t smem = sizeof(float) * kMBThreads * GV * 7;
    const unsigned grid = (unsigned)((N + kMBThreads - 1) / kMBThreads);
    if (bf16) {
        auto fn = mesh_build_kernel<DEG, true>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fn<<<grid, kMBThreads, smem, st>>>(means, log_scales, quats, opacity, sh, N, kc, corr, xyz, rgb, alpha);
    } else {
        auto fn = mesh_build_kernel<DEG, false>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fn<<<grid, kMBThreads, smem, st>>>(means, log_scales, quats, opacity, sh, N, kc, corr, xyz, rgb, alpha);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mesh_build(const float *means, const float *log_scales, const float *quats, const float *opacity,
                              const void *sh, int sh_dtype, int sh_degree, int64_t N, const MeshBuildConst &kc,
                              const float *corr, float *xyz, float *rgb, float *alpha, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    const bool bf16 = sh_dtype == 1;
    switch (sh_degree) {
        case 0: return launch_deg<0>(bf16, means, log_scales, quats, opacity, sh, N, kc, corr, xyz, rgb, alpha, st);
        case 1: return launch_deg<1>(bf16, means, log_scales, quats, opacity, sh, N, kc, corr, xyz, rgb, alpha, st);
        case 2: return launch_deg<2>(bf16, means, log_scales, quats, opacity, sh, N, kc, corr, xyz, rgb, alpha, st);
        default: return launch_deg<3>(bf16, means, log_scales, quats, opacity, sh, N, kc, corr, xyz, rgb, alpha, st);
    }
}

}  // namespace ms
