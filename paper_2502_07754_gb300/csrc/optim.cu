// L1 image loss (the L1 term of Eq. 3) and the two-learning-rate Adam update of the
// fan soup (Sec. 3 "Optimization and Pruning": colours and opacities at lr_color,
// positions at exp(-3) lr_color).  Both are elementwise and HBM-bound.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

__global__ void l1_kernel(const float4 *__restrict__ img, const float4 *__restrict__ tgt, int64_t n,
                          float4 *__restrict__ dL, float *loss) {
    const float sc = 1.0f / (3.0f * (float)n);
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = img[i], b = tgt[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2);
        dL[i] = make_float4(d0 > 0 ? sc : (d0 < 0 ? -sc : 0.0f), d1 > 0 ? sc : (d1 < 0 ? -sc : 0.0f),
                            d2 > 0 ? sc : (d2 < 0 ? -sc : 0.0f), 0.0f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(loss, v * sc);
    }
}

// One Adam update of a flat parameter segment (p, g, m, v of n floats each); clamp01
// clamps the result to [0, 1] (opacities).  With a device step counter the bias
// corrections come from *step (already advanced by step_advance).  Moments are laid out
// like the parameters: [xyz 3V | rgb 3V | alpha V].
__device__ __forceinline__ float adam1(float p, float g, float &m, float &v, float lr, float b1, float b2, float eps,
                                       float bc1, float bc2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    return p - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

struct AdamSeg {
    float *p;
    const float *g;
    float *m, *v;
    int64_t n;
    float lr;
    int clamp01;
};

__global__ void adam_kernel(AdamSeg s0, AdamSeg s1, AdamSeg s2, float b1, float b2, float eps, float bc1, float bc2,
                            const int32_t *step) {
    if (step) {
        const float t = (float)*step;
        bc1 = 1.0f - powf(b1, t);
        bc2 = 1.0f - powf(b2, t);
    }
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const AdamSeg segs[3] = {s0, s1, s2};
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        const AdamSeg &s = segs[k];
        const bool vec = ((reinterpret_cast<uintptr_t>(s.p) | reinterpret_cast<uintptr_t>(s.g) |
                           reinterpret_cast<uintptr_t>(s.m) | reinterpret_cast<uintptr_t>(s.v)) & 15) == 0;
        int64_t done = 0;
        if (vec) {   // 16-byte accesses over the aligned body
            const int64_t n4 = s.n / 4;
            for (int64_t i = tid; i < n4; i += nth) {
                float4 p = reinterpret_cast<float4 *>(s.p)[i];
                const float4 g = reinterpret_cast<const float4 *>(s.g)[i];
                float4 m = reinterpret_cast<float4 *>(s.m)[i], v = reinterpret_cast<float4 *>(s.v)[i];
                p.x = adam1(p.x, g.x, m.x, v.x, s.lr, b1, b2, eps, bc1, bc2);
                p.y = adam1(p.y, g.y, m.y, v.y, s.lr, b1, b2, eps, bc1, bc2);
                p.z = adam1(p.z, g.z, m.z, v.z, s.lr, b1, b2, eps, bc1, bc2);
                p.w = adam1(p.w, g.w, m.w, v.w, s.lr, b1, b2, eps, bc1, bc2);
                if (s.clamp01) {
                    p.x = fminf(fmaxf(p.x, 0.0f), 1.0f);
                    p.y = fminf(fmaxf(p.y, 0.0f), 1.0f);
                    p.z = fminf(fmaxf(p.z, 0.0f), 1.0f);
                    p.w = fminf(fmaxf(p.w, 0.0f), 1.0f);
                }
                reinterpret_cast<float4 *>(s.p)[i] = p;
                reinterpret_cast<float4 *>(s.m)[i] = m;
                reinterpret_cast<float4 *>(s.v)[i] = v;
            }
            done = n4 * 4;
        }
        for (int64_t i = done + tid; i < s.n; i += nth) {
            float m = s.m[i], v = s.v[i];
            float p = adam1(s.p[i], s.g[i], m, v, s.lr, b1, b2, eps, bc1, bc2);
            if (s.clamp01) p = fminf(fmaxf(p, 0.0f), 1.0f);
            s.p[i] = p;
            s.m[i] = m;
            s.v[i] = v;
        }
    }
}

__global__ void step_advance_kernel(int32_t *step) { *step += 1; }

// Adam straight from a render workspace's gradient sums: per vertex (dxyz, dalpha) and
// (drgb, 0) as two float4s; parameters and moments as in adam_kernel.
__global__ void adam_ws_kernel(float *__restrict__ xyz, float *__restrict__ rgb, float *__restrict__ alpha,
                               const float4 *__restrict__ grad, float *__restrict__ m, float *__restrict__ v,
                               int64_t V, float lr_c, float lr_x, float b1, float b2, float eps, float bc1, float bc2,
                               const int32_t *step) {
    if (step) {
        const float t = (float)*step;
        bc1 = 1.0f - powf(b1, t);
        bc2 = 1.0f - powf(b2, t);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 g0 = grad[2 * i], g1 = grad[2 * i + 1];
        const float gx[3] = {g0.x, g0.y, g0.z}, gc[3] = {g1.x, g1.y, g1.z};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float mm = m[3 * i + r], vv = v[3 * i + r];
            xyz[3 * i + r] = adam1(xyz[3 * i + r], gx[r], mm, vv, lr_x, b1, b2, eps, bc1, bc2);
            m[3 * i + r] = mm;
            v[3 * i + r] = vv;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int64_t k = 3 * V + 3 * i + r;
            float mm = m[k], vv = v[k];
            rgb[3 * i + r] = adam1(rgb[3 * i + r], gc[r], mm, vv, lr_c, b1, b2, eps, bc1, bc2);
            m[k] = mm;
            v[k] = vv;
        }
        const int64_t k = 6 * V + i;
        float mm = m[k], vv = v[k];
        alpha[i] = fminf(fmaxf(adam1(alpha[i], g0.w, mm, vv, lr_c, b1, b2, eps, bc1, bc2), 0.0f), 1.0f);
        m[k] = mm;
        v[k] = vv;
    }
}

// Mean squared error over the RGB channels of n pixels, accumulated into *out (zeroed by
// the launcher): the PSNR of a render is -10 log10 of it.
__global__ void mse_kernel(const float4 *__restrict__ img, const float4 *__restrict__ tgt, int64_t n, float *out) {
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = img[i], b = tgt[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z;
        acc += d0 * d0 + d1 * d1 + d2 * d2;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(out, v / (3.0f * (float)n));
    }
}

// Per-fan corrections that turn the conversion (xyz0, a0) into a fine-tuned soup (xyz1,
// a1): for boundary vertex i the radial component of its new offset from the original
// centre relative to the original offset, minus 1; for every vertex k the log ratio of
// the opacities (0 where either is 0).  Row layout as the corr input of mesh_build.
__global__ void fan_corr_kernel(const float *__restrict__ xyz0, const float *__restrict__ a0,
                                const float *__restrict__ xyz1, const float *__restrict__ a1, int64_t N, int K,
                                float *__restrict__ corr) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const int KV = K + 1;
    const float *p0 = xyz0 + g * KV * 3, *p1 = xyz1 + g * KV * 3;
    float *c = corr + g * 2 * KV;
    c[0] = 0.0f;
    for (int i = 1; i <= K; ++i) {
        const float o0x = p0[3 * i] - p0[0], o0y = p0[3 * i + 1] - p0[1], o0z = p0[3 * i + 2] - p0[2];
        const float o1x = p1[3 * i] - p0[0], o1y = p1[3 * i + 1] - p0[1], o1z = p1[3 * i + 2] - p0[2];
        const float nn = o0x * o0x + o0y * o0y + o0z * o0z;
        c[i] = nn > 0.0f ? (o1x * o0x + o1y * o0y + o1z * o0z) / nn - 1.0f : 0.0f;
    }
    for (int k = 0; k < KV; ++k) {
        const float x = a0[g * KV + k], y = a1[g * KV + k];
        c[KV + k] = (x > 0.0f && y > 0.0f) ? logf(y / x) : 0.0f;
    }
}

}  // namespace

cudaError_t launch_adam_ws(float *xyz, float *rgb, float *alpha, const float4 *grad, float *m, float *v, int64_t V,
                           int step, int32_t *d_step, float lr_c, float lr_x, float b1, float b2, float eps,
                           cudaStream_t st) {
    if (d_step) {
        step_advance_kernel<<<1, 1, 0, st>>>(d_step);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (V == 0) return cudaSuccess;
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    const int grid = (int)min64((V + 255) / 256, 16 * 152);
    adam_ws_kernel<<<grid, 256, 0, st>>>(xyz, rgb, alpha, grad, m, v, V, lr_c, lr_x, b1, b2, eps, bc1, bc2, d_step);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float *img, const float *tgt, int64_t n, float *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, sizeof(float), st);
    if (n == 0) return cudaGetLastError();
    const int grid = (int)min64((n + 255) / 256, 8 * 152);
    mse_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(img), reinterpret_cast<const float4 *>(tgt), n,
                                     out);
    return cudaGetLastError();
}

cudaError_t launch_fan_corr(const float *xyz0, const float *a0, const float *xyz1, const float *a1, int64_t N, int K,
                            float *corr, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    fan_corr_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(xyz0, a0, xyz1, a1, N, K, corr);
    return cudaGetLastError();
}

cudaError_t launch_l1(const float *img, const float *tgt, int64_t n, float *dL, float *loss, cudaStream_t st) {
    cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (n == 0) return cudaGetLastError();
    const int grid = (int)min64((n + 255) / 256, 8 * 152);
    l1_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(img), reinterpret_cast<const float4 *>(tgt), n,
                                    reinterpret_cast<float4 *>(dL), loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *xyz, float *rgb, float *alpha, const float *dx, const float *dc, const float *da,
                        float *m, float *v, int64_t V, int step, int32_t *d_step, float lr_c, float lr_x, float b1,
                        float b2, float eps, cudaStream_t st) {
    if (d_step) {
        step_advance_kernel<<<1, 1, 0, st>>>(d_step);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (V == 0) return cudaSuccess;
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    const AdamSeg sx = {xyz, dx, m, v, 3 * V, lr_x, 0};
    const AdamSeg sc = {rgb, dc, m + 3 * V, v + 3 * V, 3 * V, lr_c, 0};
    const AdamSeg sa = {alpha, da, m + 6 * V, v + 6 * V, V, lr_c, 1};
    const int grid = (int)min64((V + 255) / 256, 16 * 152);
    adam_kernel<<<grid, 256, 0, st>>>(sx, sc, sa, b1, b2, eps, bc1, bc2, d_step);
    return cudaGetLastError();
}

}  // namespace ms
