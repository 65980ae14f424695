// Gaussian -> triangle-fan conversion with SH colour (Sec. 3, "MeshSplats
// Transformation for Flat Gaussians", Eq. 2 and the vertex equation after it; and
// "Transformation for 3D Gaussians": all three scaled axes kept, one fan per pair of axes
// (1, 2), (1, 3), (2, 3), written as three implicit fans of K triangles per Gaussian whose
// shared vertices -- the centre and the axis tips two fans reach -- are copies; the
// angle table then holds exact cosine and sine at quarter turns, so the copies are equal
// bit for bit).
//
// One thread per Gaussian (the body is mb::convert_gaussian).  The block's vertices are
// assembled in shared memory and leave in 16-byte coalesced stores, so each output byte
// crosses HBM once: read 44 B + SH, write 28 (K+1) B per fan.
#include "mesh_build.cuh"

namespace ms {

namespace {

constexpr int kMBThreads = 128;

template <int DEG, bool BF16>
__global__ void __launch_bounds__(kMBThreads) mesh_build_kernel(const mb::Gaussians G, int64_t N, MeshBuildConst kc,
                                                                const float *__restrict__ corr,
                                                                float *__restrict__ xyz, float *__restrict__ rgb,
                                                                float *__restrict__ alpha) {
    extern __shared__ float smem[];
    const int KV = kc.K + 1;
    const int GV = (kc.three ? 3 : 1) * KV;      // vertices per Gaussian
    float *s_xyz = smem;                          // kMBThreads * GV * 3
    float *s_rgb = s_xyz + kMBThreads * GV * 3;   // kMBThreads * GV * 3
    float *s_a = s_rgb + kMBThreads * GV * 3;     // kMBThreads * GV

    const int64_t g0 = (int64_t)blockIdx.x * kMBThreads;
    const int64_t g = g0 + threadIdx.x;
    const int nloc = (int)min64(kMBThreads, N - g0);
    if (g < N)
        mb::convert_gaussian<DEG, BF16>(G, kc, g, corr ? corr + g * 2 * KV : nullptr, s_xyz, s_rgb, s_a,
                                        threadIdx.x * GV);
    __syncthreads();
    const int64_t v0 = g0 * GV;
    mb::block_store(xyz + 3 * v0, s_xyz, 3 * nloc * GV);
    mb::block_store(rgb + 3 * v0, s_rgb, 3 * nloc * GV);
    mb::block_store(alpha + v0, s_a, nloc * GV);
}

template <int DEG>
cudaError_t launch_deg(bool bf16, const float *means, const float *log_scales, const float *quats,
                       const float *opacity, const void *sh, int64_t N, const MeshBuildConst &kc, const float *corr,
                       float *xyz, float *rgb, float *alpha, cudaStream_t st) {
    const int GV = (kc.three ? 3 : 1) * (kc.K + 1);
    const size_t smem = sizeof(float) * kMBThreads * GV * 7;
    const unsigned grid = (unsigned)((N + kMBThreads - 1) / kMBThreads);
    const mb::Gaussians G{means, log_scales, quats, opacity, sh};
    if (bf16) {
        auto fn = mesh_build_kernel<DEG, true>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fn<<<grid, kMBThreads, smem, st>>>(G, N, kc, corr, xyz, rgb, alpha);
    } else {
        auto fn = mesh_build_kernel<DEG, false>;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fn<<<grid, kMBThreads, smem, st>>>(G, N, kc, corr, xyz, rgb, alpha);
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
