// Fine-tuning loss of Sec. 3 (Eq. 3), read as lambda L1 + (1 - lambda)(1 - SSIM): SSIM
// per colour channel under an 11 x 11 Gaussian window (sigma 1.5, zero padding outside
// the image, C1 = 0.01^2, C2 = 0.03^2) averaged over the pixels and the three channels.
//
// Two launches over 16 x 16 output tiles, each staging a 26 x 26 window of its inputs in
// shared memory (the forward stages the three channels of image and target in one pass)
// and applying the separable window as a row pass then a column pass:
//
// ssim_fwd_kernel: per channel the raw local moments (x, y, x^2, y^2, xy), the SSIM map,
//   and the three per-pixel factors of its gradient (with A = 2 mu_x mu_y + C1,
//   B = 2 s_xy + C2, C = mu_x^2 + mu_y^2 + C1, D = s_xx + s_yy + C2, S = AB/(CD)):
//     G2 = dS/ds_xx = -S/D,  G3 = dS/ds_xy = 2A/(CD),
//     G1 = dS/dmu_x - 2 mu_x G2 - mu_y G3,  dS/dmu_x = 2 mu_y B/(CD) - 2 mu_x S/C,
//   written as nine planes; the block's share of the loss is added to *loss.  The
//   moments are taken of x - r_x and y - r_y with one reference value per tile (a pixel
//   near its centre; outside the image the padded zeros become -r): the local
//   (co)variances do not depend on the shift, and E[x^2] - mu^2 then cancels against the
//   local contrast instead of against the brightness.
// ssim_bwd_kernel: dSSIM/dx_p = (1/N) [(w * G1)(p) + 2 x_p (w * G2)(p) + y_p (w * G3)(p)],
//   w * G the window sum of a plane over the image's pixels (zero outside), and
//   dL/dx = lambda sign(x - y)/N - (1 - lambda) dSSIM/dx, N = 3 H W.
#include <cmath>

#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kT = 16;            // output tile edge
constexpr int kR = 5;             // window radius
constexpr int kIn = kT + 2 * kR;  // staged tile edge (26)
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;

struct Window {
    float w[2 * kR + 1];
};

__device__ __forceinline__ float chan(const float4 &v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

__device__ __forceinline__ float block_sum(float v, float *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * kT + threadIdx.x;
    if ((tid & 31) == 0) s_red[tid >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    if (tid < 32) {
        t = tid < (kT * kT) / 32 ? s_red[tid] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(kT *kT) ssim_fwd_kernel(const float4 *__restrict__ img, const float4 *__restrict__ tgt,
                                                          int H, int W, float lam, float inv_n, Window win,
                                                          float *__restrict__ G, float *__restrict__ loss) {
    __shared__ float sx[3][kIn][kIn + 1], sy[3][kIn][kIn + 1];   // the three channels, shifted
    __shared__ float sh[5][kIn][kT + 1];
    __shared__ float s_red[(kT * kT) / 32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kT + tx;
    const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
    const int px = x0 + tx, py = y0 + ty;
    const bool inside = px < W && py < H;
    const size_t plane = (size_t)H * W;
    float acc = 0.0f;
    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f), yv = xv;
    if (inside) {
        xv = img[(size_t)py * W + px];
        yv = tgt[(size_t)py * W + px];
        acc += lam * (fabsf(xv.x - yv.x) + fabsf(xv.y - yv.y) + fabsf(xv.z - yv.z));
    }
    const size_t ref = (size_t)min(y0 + kT / 2, H - 1) * W + min(x0 + kT / 2, W - 1);
    const float4 rxv = img[ref], ryv = tgt[ref];
    // one pass over the window stages all three channels (each RGBA pixel loaded once)
    for (int i = tid; i < kIn * kIn; i += kT * kT) {
        const int lx = i % kIn, ly = i / kIn;
        const int gx = x0 - kR + lx, gy = y0 - kR + ly;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            a = img[(size_t)gy * W + gx];
            b = tgt[(size_t)gy * W + gx];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sx[c][ly][lx] = chan(a, c) - chan(rxv, c);
            sy[c][ly][lx] = chan(b, c) - chan(ryv, c);
        }
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        const float rx = chan(rxv, c), ry = chan(ryv, c);
        for (int i = tid; i < kIn * kT; i += kT * kT) {
            const int r = i / kT, q = i % kT;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * kR; ++t) {
                const float a = sx[c][r][q + t], b = sy[c][r][q + t], wt = win.w[t];
                s0 += wt * a;
                s1 += wt * b;
                s2 += wt * a * a;
                s3 += wt * b * b;
                s4 += wt * a * b;
            }
            sh[0][r][q] = s0;
            sh[1][r][q] = s1;
            sh[2][r][q] = s2;
            sh[3][r][q] = s3;
            sh[4][r][q] = s4;
        }
        __syncthreads();
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t <= 2 * kR; ++t) {
            const float wt = win.w[t];
#pragma unroll
            for (int k = 0; k < 5; ++k) m[k] += wt * sh[k][ty + t][tx];
        }
        if (inside) {
            const float sxx = m[2] - m[0] * m[0], syy = m[3] - m[1] * m[1], sxy = m[4] - m[0] * m[1];
            const float mx = m[0] + rx, my = m[1] + ry;
            const float A = 2.0f * mx * my + kC1, B = 2.0f * sxy + kC2;
            const float Cc = mx * mx + my * my + kC1, D = sxx + syy + kC2;
            const float iCD = 1.0f / (Cc * D);
            const float S = A * B * iCD;
            const float g2 = -S / D;
            const float g3 = 2.0f * A * iCD;
            const float g1 = 2.0f * my * B * iCD - 2.0f * mx * S / Cc - 2.0f * mx * g2 - my * g3;
            const size_t o = (size_t)py * W + px;
            G[(3 * c + 0) * plane + o] = g1;
            G[(3 * c + 1) * plane + o] = g2;
            G[(3 * c + 2) * plane + o] = g3;
            acc += (1.0f - lam) * (1.0f - S);
        }
        __syncthreads();   // the next channel's row pass overwrites sh
    }
    const float t = block_sum(acc, s_red);
    if (tid == 0) atomicAdd(loss, t * inv_n);
}

__global__ void __launch_bounds__(kT *kT) ssim_bwd_kernel(const float4 *__restrict__ img, const float4 *__restrict__ tgt,
                                                          int H, int W, float lam, float inv_n, Window win,
                                                          const float *__restrict__ G, float4 *__restrict__ dL) {
    __shared__ float sg[3][kIn][kIn + 1];
    __shared__ float sh[3][kIn][kT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kT + tx;
    const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
    const int px = x0 + tx, py = y0 + ty;
    const bool inside = px < W && py < H;
    const size_t plane = (size_t)H * W;
    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f), yv = xv;
    if (inside) {
        xv = img[(size_t)py * W + px];
        yv = tgt[(size_t)py * W + px];
    }
    float out[3];
    for (int c = 0; c < 3; ++c) {
        for (int i = tid; i < kIn * kIn; i += kT * kT) {
            const int lx = i % kIn, ly = i / kIn;
            const int gx = x0 - kR + lx, gy = y0 - kR + ly;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const size_t o = (size_t)gy * W + gx;
#pragma unroll
            for (int k = 0; k < 3; ++k) sg[k][ly][lx] = in ? G[(3 * c + k) * plane + o] : 0.0f;
        }
        __syncthreads();
        for (int i = tid; i < kIn * kT; i += kT * kT) {
            const int r = i / kT, q = i % kT;
            float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t <= 2 * kR; ++t) {
                const float wt = win.w[t];
#pragma unroll
                for (int k = 0; k < 3; ++k) s[k] += wt * sg[k][r][q + t];
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) sh[k][r][q] = s[k];
        }
        __syncthreads();
        float b[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t <= 2 * kR; ++t) {
            const float wt = win.w[t];
#pragma unroll
            for (int k = 0; k < 3; ++k) b[k] += wt * sh[k][ty + t][tx];
        }
        const float x = chan(xv, c), y = chan(yv, c);
        const float dS = (b[0] + 2.0f * x * b[1] + y * b[2]) * inv_n;
        const float d = x - y;
        const float sg1 = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
        out[c] = lam * sg1 * inv_n - (1.0f - lam) * dS;
        __syncthreads();   // the next channel restages the tiles
    }
    if (inside) dL[(size_t)py * W + px] = make_float4(out[0], out[1], out[2], 0.0f);
}

Window make_window() {
    Window w;
    double g[2 * kR + 1], z = 0.0;
    for (int t = -kR; t <= kR; ++t) {
        g[t + kR] = std::exp(-(double)(t * t) / (2.0 * 1.5 * 1.5));
        z += g[t + kR];
    }
    for (int t = 0; t <= 2 * kR; ++t) w.w[t] = (float)(g[t] / z);
    return w;
}

}  // namespace

size_t ssim_scratch_bytes(int H, int W) { return (size_t)9 * sizeof(float) * (size_t)H * (size_t)W; }

cudaError_t launch_ssim_loss(const float *img, const float *tgt, int H, int W, float lam, float *dL, float *loss,
                             float *scratch, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess || H == 0 || W == 0) return e;
    const dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT), block(kT, kT);
    const float inv_n = (float)(1.0 / (3.0 * (double)H * (double)W));
    const Window win = make_window();
    ssim_fwd_kernel<<<grid, block, 0, st>>>(reinterpret_cast<const float4 *>(img), reinterpret_cast<const float4 *>(tgt),
                                            H, W, lam, inv_n, win, scratch, loss);
    ssim_bwd_kernel<<<grid, block, 0, st>>>(reinterpret_cast<const float4 *>(img), reinterpret_cast<const float4 *>(tgt),
                                            H, W, lam, inv_n, win, scratch, reinterpret_cast<float4 *>(dL));
    return cudaGetLastError();
}

}  // namespace ms
