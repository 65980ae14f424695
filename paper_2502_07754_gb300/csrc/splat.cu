// Polygons that circumscribe the source Gaussians' truncation ellipses, for binning the
// splat passes (ms_splat_render).  The regular 8-gon whose inscribed circle is the unit
// circle, mapped by the Gaussian's scaled kept axes, contains the ellipse; the extra
// 1e-4 relative margin keeps it containing the ellipse after binary32 rounding, so the
// polygon's pixel rectangle and minimum depth bound every hit of the splat.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {
namespace {

constexpr int kPolyThreads = 128;

__global__ void __launch_bounds__(kPolyThreads) splat_polygon_kernel(const SplatSrc s, int64_t N, float radius,
                                                                     float *__restrict__ xyz) {
    const int64_t g = (int64_t)blockIdx.x * kPolyThreads + threadIdx.x;
    if (g >= N) return;
    const float4 q4 = *reinterpret_cast<const float4 *>(s.quats + 4 * g);
    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    const float R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                        2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                        2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
    const float s0 = s.log_scales[3 * g], s1 = s.log_scales[3 * g + 1], s2 = s.log_scales[3 * g + 2];
    int drop = 0;
    if (s.axis_rule == 1) {
        float sm = s0;
        if (s1 < sm) { drop = 1; sm = s1; }
        if (s2 < sm) drop = 2;
    }
    const int ia = drop == 0 ? 1 : 0, ib = drop == 2 ? 1 : 2;
    const float ea = radius * expf(ia == 0 ? s0 : s1), eb = radius * expf(ib == 2 ? s2 : s1);
    const float m[3] = {s.means[3 * g], s.means[3 * g + 1], s.means[3 * g + 2]};
    float *o = xyz + g * (kSplatK + 1) * 3;
    o[0] = m[0];
    o[1] = m[1];
    o[2] = m[2];
#pragma unroll
    for (int i = 0; i < kSplatK; ++i) {
        float sn, cs;
        sincospif(-1.0f + 2.0f * (float)i / (float)kSplatK, &sn, &cs);
#pragma unroll
        for (int r = 0; r < 3; ++r) o[3 * (1 + i) + r] = m[r] + cs * ea * R[3 * r + ia] + sn * eb * R[3 * r + ib];
    }
}

}  // namespace

cudaError_t launch_splat_polygons(const SplatSrc &s, int64_t N, float *xyz, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    const double kPi = 3.14159265358979323846;
    const float radius = (float)(s.trunc / cos(kPi / kSplatK) * (1.0 + 1e-4));
    splat_polygon_kernel<<<(unsigned)((N + kPolyThreads - 1) / kPolyThreads), kPolyThreads, 0, st>>>(s, N, radius,
                                                                                                    xyz);
    return cudaGetLastError();
}

}  // namespace ms
