// Fine-tuning of three-fan meshes (Sec. 3 "Transformation for 3D Gaussians"): the fans of a
// 3D Gaussian share their centre and the axis tips that two fans reach.  The renderer draws
// them as 3 implicit fans with the shared vertices copied bit for bit into every fan, so
// the adjoint gives each copy its own share of the gradient.  The gradient of the shared
// vertex is the sum of its copies' gradients; giving every copy that sum makes the copies
// take identical optimiser steps, so they stay one vertex.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kCopyMax = 3 * (kMaxK + 1);

struct CopyMap {
    int32_t first[kCopyMax];   // first copy of every slot of one Gaussian
    int slots;                 // 3 (K + 1)
};

constexpr int kCopyThreads = 256;

// One block covers whole Gaussians (blockDim / slots of them); each thread loads its slot's
// seven gradient values into shared memory, then writes back the sum over the slots with
// the same first copy.  grad (workspace layout, two float4 per vertex: (xyz, alpha),
// (rgb, 0)) when non-null, else the three arrays.
__global__ void __launch_bounds__(kCopyThreads) sum_copies_kernel(const __grid_constant__ CopyMap cm, int64_t n_gauss,
                                                                  float *__restrict__ dx, float *__restrict__ dc,
                                                                  float *__restrict__ da, float4 *__restrict__ grad) {
    __shared__ float s_g[kCopyThreads][7];
    const int per_block = kCopyThreads / cm.slots;
    const int t = threadIdx.x;
    const int gl = t / cm.slots, slot = t - gl * cm.slots;
    const int64_t g = (int64_t)blockIdx.x * per_block + gl;
    const bool live = gl < per_block && g < n_gauss;
    const int64_t v = g * cm.slots + slot;
    if (live) {
        float w[7];
        if (grad) {
            const float4 a = grad[2 * v], b = grad[2 * v + 1];
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[6] = a.w;
            w[3] = b.x; w[4] = b.y; w[5] = b.z;
        } else {
            w[0] = dx[3 * v]; w[1] = dx[3 * v + 1]; w[2] = dx[3 * v + 2];
            w[3] = dc[3 * v]; w[4] = dc[3 * v + 1]; w[5] = dc[3 * v + 2];
            w[6] = da[v];
        }
#pragma unroll
        for (int i = 0; i < 7; ++i) s_g[t][i] = w[i];
    }
    __syncthreads();
    if (!live) return;
    const int root = cm.first[slot];
    float sum[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int u = 0; u < cm.slots; ++u)   // slots in order: every copy sums identically
        if (cm.first[u] == root) {
            const int tu = gl * cm.slots + u;
#pragma unroll
            for (int i = 0; i < 7; ++i) sum[i] += s_g[tu][i];
        }
    if (grad) {
        grad[2 * v] = make_float4(sum[0], sum[1], sum[2], sum[6]);
        grad[2 * v + 1] = make_float4(sum[3], sum[4], sum[5], 0.0f);
    } else {
        dx[3 * v] = sum[0]; dx[3 * v + 1] = sum[1]; dx[3 * v + 2] = sum[2];
        dc[3 * v] = sum[3]; dc[3 * v + 1] = sum[4]; dc[3 * v + 2] = sum[5];
        da[v] = sum[6];
    }
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" MS_API ms_status ms_three_fan_sum_copies(float *d_xyz, float *d_rgb, float *d_alpha, void *grad, int64_t N,
                                                    int32_t K, void *stream) {
    if (K < 3 || K > kMaxK) return set_error(MS_ERR_INVALID, "K=%d outside 3..%d", K, kMaxK);
    if (N < 0) return set_error(MS_ERR_INVALID, "N < 0");
    if (N == 0) return MS_OK;
    if (!grad && (!d_xyz || !d_rgb || !d_alpha)) return set_error(MS_ERR_INVALID, "gradient pointer is NULL");
    if (grad && (reinterpret_cast<uintptr_t>(grad) & 15)) return set_error(MS_ERR_INVALID, "grad not 16-byte aligned");
    CopyMap cm;
    cm.slots = 3 * (K + 1);
    if (ms_three_fan_copies(K, cm.first) < 0) return set_error(MS_ERR_INVALID, "copy map");
    const int per_block = kCopyThreads / cm.slots;
    const int64_t blocks = (N + per_block - 1) / per_block;
    sum_copies_kernel<<<(unsigned)blocks, kCopyThreads, 0, (cudaStream_t)stream>>>(cm, N, d_xyz, d_rgb, d_alpha,
                                                                                   static_cast<float4 *>(grad));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "sum_copies_kernel: %s", cudaGetErrorString(e));
    count_launches(1);
    return MS_OK;
}
