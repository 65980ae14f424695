// Learned fan initializer: a 16 -> 128 -> 128 -> n_out (<= 32) GELU perceptron on the
// 5th-generation tensor cores (tcgen05.mma, BF16 operands in shared memory, FP32
// accumulators in tensor memory), standing in for part of the fine-tuning of Sec. 3 by
// predicting per-vertex radial and log-opacity corrections of each fan.
//
//   inference  mlp_fwd_kernel: persistent CTAs of 512 threads (two per SM), one 128-row
//              tile at a time: features -> X (smem) -> Z1 = X W1 (TMEM) -> H1 = bf16(gelu)
//              (smem) -> Z2 -> H2 -> Z3 -> corrections (global FP32), or, fused, the
//              conversion of each row's Gaussian with its corrections still in registers
//              (the corrections never reach HBM).
//   training   mlp_act_kernel: the same forward plus the activation adjoint of the mean
//              squared error (dY, dZ2 = (dY W3^T) gelu'(Z2), dZ1 = (dZ2 W2^T) gelu'(Z1)),
//              writing the per-tile operands of the weight gradients transposed;
//              mlp_wgrad_kernel: dW1^T, dW2^T, dW3 summed over tiles in tensor memory
//              (operands brought in by one bulk copy per tile), added atomically.
// Every product is BF16 x BF16 with FP32 accumulation; the bf16 rounding points are the
// operands (inputs, weights, h1, h2, dy, dz2, dz1).  Weights are kept as FP32 masters and
// packed to bf16 tiles in the canonical K-major layout of tc05.cuh.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include "mesh_build.cuh"
#include "ms_common.cuh"
#include "ms_internal.h"
#include "gelu_poly.h"
#include "tc05.cuh"

namespace ms {
namespace {

constexpr int kIn = 16, kHid = 128, kOutPad = 32, kRows = 128;
constexpr uint32_t kTcWaitLimit = 1u << 20;

// Packed bf16 weight tiles (byte offsets); B operands are [N][K] K-major.
constexpr uint32_t kW1f = 0;                            // [128 h1][16 in]
constexpr uint32_t kW2f = kW1f + kHid * kIn * 2;        // [128 h2][128 h1]
constexpr uint32_t kW3f = kW2f + kHid * kHid * 2;       // [32 out][128 h2]
constexpr uint32_t kW3b = kW3f + kOutPad * kHid * 2;    // [128 h2][32 out]
constexpr uint32_t kW2b = kW3b + kHid * kOutPad * 2;    // [128 h1][128 h2]
constexpr uint32_t kPackedBytes = kW2b + kHid * kHid * 2;
constexpr uint32_t kStatusOff = kPackedBytes;           // uint32 timeouts, then pad
constexpr uint32_t kPackedTotal = kPackedBytes + 256;

// Per-tile operands of the weight gradients, [feature][row] K-major (K = the 128 rows).
constexpr uint32_t kTXt = 0;                            // X^T   [16][128]
constexpr uint32_t kTH1t = kTXt + kIn * kRows * 2;      // H1^T  [128][128]
constexpr uint32_t kTH2t = kTH1t + kHid * kRows * 2;    // H2^T
constexpr uint32_t kTdYt = kTH2t + kHid * kRows * 2;    // dY^T  [32][128]
constexpr uint32_t kTdZ2t = kTdYt + kOutPad * kRows * 2;   // dZ2^T [128][128]
constexpr uint32_t kTdZ1t = kTdZ2t + kHid * kRows * 2;     // dZ1^T [128][128]
constexpr uint32_t kTileBytes = kTdZ1t + kHid * kRows * 2;

// GELU x Phi(x) in binary32.  With z = |x| / sqrt 2 and E = erfc(z) / 2, Phi(x) is 1 - E
// for x >= 0 and E for x < 0, written Phi = fma(1 - 2 step, E, step) with step = [x >= 0];
// E = t 2^(G(t) - x^2 log2(e) / 2), t = 1 / (1 + z / 2), with G the degree-7 polynomial of
// gelu_poly.h (a least-squares fit): one reciprocal, one ex2, no branch.  The complementary
// form keeps the tail (x < -5) that 1 + erf(x / sqrt 2) would cancel to zero.  Relative
// error: below 3e-6 for x >= -5.6 and 1e-5 beyond (where |GELU| < 1e-8).  Pairs of values
// go through the packed f32x2 FMA and multiply of sm_100-class GPUs, which halves the
// instruction count of everything but the reciprocal and the exponential.
__device__ __forceinline__ float ex2_approx(float a) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rcp_approx(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ uint64_t f2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unf2(uint64_t r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
constexpr float kGeluT = 0.35355339059327376f;        // (1 / 2) / sqrt 2: t = 1 / (1 + |x| kGeluT)
constexpr float kGeluX2 = -0.72134752044448170f;      // -log2(e) / 2
__device__ __forceinline__ float gelu_step(float x) { return x >= 0.0f ? 1.0f : 0.0f; }

// Phi(x), one value (the derivative's first term).
__device__ __forceinline__ float gelu_phi(float x) {
    constexpr float c[] = {MS_GELU_POLY};
    const float t = rcp_approx(fmaf(fabsf(x), kGeluT, 1.0f));
    float q = c[kGeluDeg];
#pragma unroll
    for (int i = kGeluDeg - 1; i >= 0; --i) q = fmaf(q, t, c[i]);
    const float E = t * ex2_approx(fmaf(x * x, kGeluX2, q));
    const float st = gelu_step(x);
    return fmaf(fmaf(st, -2.0f, 1.0f), E, st);
}
// GELU of a pair, in place; the same roundings as x * gelu_phi(x) for each value.
__device__ __forceinline__ void gelu2(float &a, float &b) {
    constexpr float c[] = {MS_GELU_POLY};
    const uint64_t t = f2(rcp_approx(fmaf(fabsf(a), kGeluT, 1.0f)), rcp_approx(fmaf(fabsf(b), kGeluT, 1.0f)));
    const uint64_t x = f2(a, b);
    uint64_t q = f2(c[kGeluDeg], c[kGeluDeg]);
#pragma unroll
    for (int i = kGeluDeg - 1; i >= 0; --i) q = fma2(q, t, f2(c[i], c[i]));
    float ga, gb;
    unf2(fma2(mul2(x, x), f2(kGeluX2, kGeluX2), q), ga, gb);
    const uint64_t E = mul2(t, f2(ex2_approx(ga), ex2_approx(gb)));
    const uint64_t st = f2(gelu_step(a), gelu_step(b));
    const uint64_t phi = fma2(fma2(st, f2(-2.0f, -2.0f), f2(1.0f, 1.0f)), E, st);
    unf2(mul2(x, phi), a, b);
}
__device__ __forceinline__ float gelu_grad(float x) {
    return gelu_phi(x) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}
__device__ __forceinline__ void gelu16(float v[16]) {
#pragma unroll
    for (int i = 0; i < 16; i += 2) gelu2(v[i], v[i + 1]);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    return (uint32_t)bf16_bits(a) | ((uint32_t)bf16_bits(b) << 16);
}

// Eight consecutive K-values of row r of a K-major tile (one 16-byte core-matrix row).
__device__ __forceinline__ void put8(char *tile, int Kc, int r, int k0, const float *v) {
    uint4 u;
    u.x = pack2(v[0], v[1]);
    u.y = pack2(v[2], v[3]);
    u.z = pack2(v[4], v[5]);
    u.w = pack2(v[6], v[7]);
    *reinterpret_cast<uint4 *>(tile + tc::cm_offset(r, k0, Kc)) = u;
}

// The 16 inputs of a Gaussian: log-scales, normalised quaternion, opacity, degree-0 SH,
// scales sorted descending over the largest, and log(s_min / s_mid), then the constant 1.
__device__ __forceinline__ void features_from(float l0, float l1, float l2, float4 q, float op, const float dc[3],
                                              float f[kIn]) {
    const float qn = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float a = l0, b = l1, c = l2, t;   // sort descending
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    f[0] = l0; f[1] = l1; f[2] = l2;
    f[3] = q.x * qn; f[4] = q.y * qn; f[5] = q.z * qn; f[6] = q.w * qn;
    f[7] = op;
    f[8] = dc[0]; f[9] = dc[1]; f[10] = dc[2];
    f[11] = 1.0f;
    f[12] = expf(b - a);
    f[13] = expf(c - a);
    f[14] = c - b;
    f[15] = 1.0f;
}

__device__ __forceinline__ void gaussian_features(const MlpSrc &s, int64_t g, float f[kIn]) {
    const int nb = (s.sh_degree + 1) * (s.sh_degree + 1);
    float dc[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t i = g * nb * 3 + c;
        dc[c] = s.sh_dtype == 0 ? reinterpret_cast<const float *>(s.sh)[i]
                                : __uint_as_float((uint32_t)reinterpret_cast<const uint16_t *>(s.sh)[i] << 16);
    }
    features_from(s.log_scales[3 * g], s.log_scales[3 * g + 1], s.log_scales[3 * g + 2],
                  *reinterpret_cast<const float4 *>(s.quats + 4 * g), s.opacity[g], dc, f);
}

// The raw inputs of a row's features, brought into shared memory by asynchronous copies
// one tile ahead (48 bytes a row: log-scales at 0, opacity at 12, quaternion at 16, the
// first SH coefficients at 32: three f32, or four bf16 of which three are used).  Each
// thread copies and later reads its own row only, so the copies need no barrier.
constexpr int kRawRow = 48;
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Whether the raw inputs can be copied in 4-byte pieces: 4-byte aligned arrays, and for
// bf16 SH an even number of coefficients per Gaussian (degree 1 or 3).
__host__ __device__ __forceinline__ bool raw_copy_ok(const MlpSrc &s) {
    const int nb = (s.sh_degree + 1) * (s.sh_degree + 1);
    const uintptr_t mis = (reinterpret_cast<uintptr_t>(s.sh) | reinterpret_cast<uintptr_t>(s.log_scales) |
                           reinterpret_cast<uintptr_t>(s.opacity)) & 3;
    return mis == 0 && (s.sh_dtype == 0 || (nb % 2) == 0);
}
__device__ __forceinline__ void raw_fetch(const MlpSrc &s, int64_t g, char *row) {
    const int nb = (s.sh_degree + 1) * (s.sh_degree + 1);
    for (int i = 0; i < 3; ++i) cp_async4(row + 4 * i, s.log_scales + 3 * g + i);
    cp_async4(row + 12, s.opacity + g);
    cp_async16(row + 16, s.quats + 4 * g);
    if (s.sh_dtype == 0) {
        const float *p = reinterpret_cast<const float *>(s.sh) + g * nb * 3;
        for (int i = 0; i < 3; ++i) cp_async4(row + 32 + 4 * i, p + i);
    } else {
        const uint16_t *p = reinterpret_cast<const uint16_t *>(s.sh) + g * nb * 3;
        cp_async4(row + 32, p);
        cp_async4(row + 36, p + 2);
    }
}
__device__ __forceinline__ void raw_features(const MlpSrc &s, const char *row, float f[kIn]) {
    const float *r = reinterpret_cast<const float *>(row);
    float dc[3];
    if (s.sh_dtype == 0) {
        dc[0] = r[8]; dc[1] = r[9]; dc[2] = r[10];
    } else {
        const uint32_t w0 = reinterpret_cast<const uint32_t *>(row)[8], w1 = reinterpret_cast<const uint32_t *>(row)[9];
        dc[0] = __uint_as_float(w0 << 16);
        dc[1] = __uint_as_float(w0 & 0xFFFF0000u);
        dc[2] = __uint_as_float(w1 << 16);
    }
    features_from(r[0], r[1], r[2], *reinterpret_cast<const float4 *>(row + 16), r[3], dc, f);
}

struct TcState {
    uint64_t mbar;
    uint32_t tmem;
};

// Issue the K-slices of one product D (+)= A B^T by thread 0 and commit it.
__device__ __forceinline__ void issue(uint32_t d, const char *A, const char *B, int Kc, int N, bool acc_first,
                                      uint64_t *mbar) {
    const uint32_t id = tc::idesc_bf16_f32(128, N);
    const uint32_t a = tc::smem_u32(A), b = tc::smem_u32(B);
    for (int s = 0; s < Kc / 16; ++s)
        tc::mma_bf16(d, tc::kslice_desc(a, Kc, s), tc::kslice_desc(b, Kc, s), id, acc_first || s > 0);
    if (mbar) tc::commit(mbar);
}

// Shared-memory operands were written: make them visible to the tensor cores, order
// against earlier tensor-memory reads, and (thread 0) issue the product.
__device__ __forceinline__ void sync_then(bool issuer) {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (issuer) tc::fence_after_sync();
}

// Every thread tracks the barrier's phase parity in its own register.
__device__ __forceinline__ bool wait_mma(TcState *S, uint32_t &phase, uint32_t *timeouts) {
    const bool ok = tc::mbar_wait(&S->mbar, phase, kTcWaitLimit);
    phase ^= 1u;
    if (!ok && threadIdx.x == 0) atomicAdd(timeouts, 1u);
    tc::fence_after_sync();
    return ok;
}

// Slot version: every thread of the slot waits on the slot's mbarrier.
__device__ __forceinline__ bool wait_mma_slot(uint64_t *mbar, uint32_t &phase, uint32_t *timeouts, bool counter) {
    const bool ok = tc::mbar_wait(mbar, phase, kTcWaitLimit);
    phase ^= 1u;
    if (!ok && counter) atomicAdd(timeouts, 1u);
    tc::fence_after_sync();
    return ok;
}

// Shared prologue: weights into shared memory, barrier, tensor memory.
__device__ __forceinline__ void setup(char *smem, const char *packed, uint32_t wbytes_lo, uint32_t wbytes_hi,
                                      char *wdst, TcState *S, uint32_t ncols) {
    const uint4 *src = reinterpret_cast<const uint4 *>(packed + wbytes_lo);
    uint4 *dst = reinterpret_cast<uint4 *>(wdst);
    for (uint32_t i = threadIdx.x; i < (wbytes_hi - wbytes_lo) / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        tc::mbar_init(&S->mbar, 1);
        tc::mbar_init_fence();
    }
    if (threadIdx.x < 32) tc::tmem_alloc(&S->tmem, ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    (void)smem;
}

__device__ __forceinline__ void teardown(TcState *S, uint32_t ncols) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(S->tmem, ncols);
}

// ------------------------------------------------------------------ inference

// One CTA per SM holds the three forward weight tiles once and runs kSlots independent
// 128-row tiles ("slots"), each with 8 warps, its own X / H operands, raw-input buffer,
// mbarrier, named barrier and 128 tensor-memory columns (Z1, Z2 and Z3 of a tile reuse the
// same columns: each product is issued after the previous accumulator has been read).  While
// one slot waits for its product on the tensor cores, the other slots' GELU epilogues run.
constexpr int kSlots = 4;
constexpr int kSlotThreads = 256;
constexpr int kFwdThreads = kSlots * kSlotThreads;
constexpr uint32_t kFwdW = kW1f, kFwdWEnd = kW3b;        // W1f, W2f, W3f
constexpr uint32_t kSlotX = 0;                           // X  [128][16]
constexpr uint32_t kSlotH = kSlotX + kRows * kIn * 2;    // H1, then H2 [128][128]
constexpr uint32_t kSlotRaw = kSlotH + kRows * kHid * 2; // [128][kRawRow] raw inputs
constexpr uint32_t kSlotBytes = kSlotRaw + kRows * kRawRow;
constexpr uint32_t kFSlots = kFwdWEnd - kFwdW;
constexpr uint32_t kFState = kFSlots + kSlots * kSlotBytes;   // kSlots mbarriers, TMEM base
constexpr uint32_t kFwdSmem = kFState + 8 * kSlots + 16;
// After the last product of a tile, the slot's X and H are free: the fused conversion
// stages the tile's vertices there.
constexpr uint32_t kStageFloats = (kSlotRaw - kSlotX) / 4;
static_assert(kSlotBytes % 1024 == 0, "slot operands keep the 1024-byte alignment");
static_assert(kFwdSmem <= 227 * 1024, "shared memory");

// Named barrier of one slot (ids 1..kSlots; 0 is the CTA barrier), optionally AND-reducing.
__device__ __forceinline__ void slot_sync(int slot) {
    asm volatile("bar.sync %0, %1;" ::"r"(slot + 1), "r"(kSlotThreads) : "memory");
}
__device__ __forceinline__ bool slot_sync_and(int slot, bool v) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(out) : "r"((uint32_t)v), "r"(slot + 1), "r"(kSlotThreads) : "memory");
    return out != 0;
}
// The slot's operands were written: visible to the tensor cores, ordered after earlier
// tensor-memory reads; the slot's first thread then issues.
__device__ __forceinline__ void slot_sync_then(int slot, bool issuer) {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    slot_sync(slot);
    if (issuer) tc::fence_after_sync();
}

// Warp w of a slot reads tensor-memory lanes 32 (w % 4) .. + 31 (rows of the tile) and
// columns 64 (w / 4) .. + 63.
__device__ __forceinline__ void gelu_cols64(uint32_t tz, char *H, int r, int c0) {
#pragma unroll 1
    for (int h = 0; h < 64; h += 16) {
        float v[16];
        tc::tmem_ld16(tz + c0 + h, v);
        gelu16(v);
        put8(H, kHid, r, c0 + h, v);
        put8(H, kHid, r, c0 + h + 8, v + 8);
    }
}

// Copies n floats from shared to global with the 256 threads of a slot (16-byte stores
// when both ends allow it).
__device__ __forceinline__ void slot_store(float *dst, const float *src, int n, int st) {
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0 && (n & 3) == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        for (int i = st; i < n / 4; i += kSlotThreads) d4[i] = s4[i];
    } else {
        for (int i = st; i < n; i += kSlotThreads) dst[i] = src[i];
    }
}

// Where the outputs go: the corrections (N x n_out FP32), or, fused, the fan soup of
// the conversion with the row's corrections taken from registers.
struct FwdOut {
    float *corr;
    mb::Gaussians G;
    MeshBuildConst kc;
    float *xyz, *rgb, *alpha;
};

template <bool FUSED, int DEG, bool BF16>
__global__ void __launch_bounds__(kFwdThreads, 1) mlp_fwd_kernel(const MlpSrc s, int64_t N,
                                                                const char *__restrict__ packed, int n_out,
                                                                const FwdOut out) {
    extern __shared__ __align__(1024) char smem[];
    uint64_t *mbars = reinterpret_cast<uint64_t *>(smem + kFState);
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(smem + kFState + 8 * kSlots);
    uint32_t *timeouts = reinterpret_cast<uint32_t *>(const_cast<char *>(packed) + kStatusOff);
    {   // weights, barriers, tensor memory
        const uint4 *src = reinterpret_cast<const uint4 *>(packed + kFwdW);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (uint32_t i = threadIdx.x; i < (kFwdWEnd - kFwdW) / 16; i += blockDim.x) dst[i] = src[i];
        if (threadIdx.x == 0) {
            for (int k = 0; k < kSlots; ++k) tc::mbar_init(&mbars[k], 1);
            tc::mbar_init_fence();
        }
        if (threadIdx.x < 32) tc::tmem_alloc(tmem_base, 128 * kSlots);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    const char *W1 = smem + (kW1f - kFwdW), *W2 = smem + (kW2f - kFwdW), *W3 = smem + (kW3f - kFwdW);
    const int tid = threadIdx.x, slot = tid / kSlotThreads, st = tid % kSlotThreads;
    const int w = st >> 5, lane = tid & 31;
    char *X = smem + kFSlots + slot * kSlotBytes + kSlotX;
    char *H = smem + kFSlots + slot * kSlotBytes + kSlotH;
    char *raw = smem + kFSlots + slot * kSlotBytes + kSlotRaw;
    uint64_t *mbar = &mbars[slot];
    const int r = 32 * (w & 3) + lane;   // the row (tensor-memory lane) this thread reads
    const int c0 = 64 * (w >> 2);        // its accumulator columns
    const bool row_owner = w < 4;
    const bool issuer = st == 0;
    const uint32_t tz = *tmem_base + 128u * slot + ((uint32_t)(32 * (w & 3)) << 16);
    const uint32_t tz0 = *tmem_base + 128u * slot;
    const int64_t tiles = (N + kRows - 1) / kRows;
    const int64_t stride = (int64_t)gridDim.x * kSlots;
    const bool pre = raw_copy_ok(s);
    int64_t t = (int64_t)blockIdx.x * kSlots + slot;
    if (pre && row_owner) {   // this slot's first tile; later ones are fetched a tile ahead
        const int64_t g = t * kRows + r;
        if (t < tiles && g < N) raw_fetch(s, g, raw + r * kRawRow);
        cp_async_commit();
    }
    uint32_t phase = 0;
    bool ok = true;
    for (; t < tiles; t += stride) {
        const int64_t g = t * kRows + r;
        if (row_owner) {
            float f[kIn];
            if (g >= N) {
#pragma unroll
                for (int i = 0; i < kIn; ++i) f[i] = 0.0f;
            } else if (pre) {
                cp_async_wait_all();
                raw_features(s, raw + r * kRawRow, f);
            } else {
                gaussian_features(s, g, f);
            }
            put8(X, kIn, r, 0, f);
            put8(X, kIn, r, 8, f + 8);
            if (pre) {   // the row was read: the next tile's raw inputs replace it
                const int64_t gn = g + stride * kRows;
                if (gn < N) raw_fetch(s, gn, raw + r * kRawRow);
                cp_async_commit();
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        ok = slot_sync_and(slot, ok);
        if (!ok) break;
        if (issuer) {
            tc::fence_after_sync();
            issue(tz0, X, W1, kIn, kHid, false, mbar);
        }
        ok = wait_mma_slot(mbar, phase, timeouts, issuer);
        gelu_cols64(tz, H, r, c0);
        slot_sync_then(slot, issuer);
        if (issuer) issue(tz0, H, W2, kHid, kHid, false, mbar);
        ok = wait_mma_slot(mbar, phase, timeouts, issuer) && ok;
        gelu_cols64(tz, H, r, c0);   // the product has read H1: H2 replaces it
        slot_sync_then(slot, issuer);
        if (issuer) issue(tz0, H, W3, kHid, kOutPad, false, mbar);
        ok = wait_mma_slot(mbar, phase, timeouts, issuer) && ok;
        float y[32];
        if (row_owner) {
            tc::tmem_ld16(tz, *reinterpret_cast<float(*)[16]>(y));
            tc::tmem_ld16(tz + 16, *reinterpret_cast<float(*)[16]>(y + 16));
        }
        if (!FUSED) {
            if (row_owner && g < N) {
#pragma unroll
                for (int o = 0; o < kOutPad; ++o)   // unrolled: y stays in registers
                    if (o < n_out) out.corr[g * n_out + o] = y[o];
            }
        } else {
            // The tile's fans, staged in X and H (free now: every product has completed)
            // in chunks of whole Gaussians, each chunk stored coalesced by the slot.
            const int KV = out.kc.K + 1;
            const int per_chunk = min((int)(kStageFloats / (7 * KV)), kRows);
            const int64_t g0 = t * kRows;
            const int nloc = (int)min64(kRows, N - g0);
            float *stg = reinterpret_cast<float *>(X);
            for (int r0 = 0; r0 < nloc; r0 += per_chunk) {
                const int nc = min(per_chunk, nloc - r0);
                float *s_xyz = stg, *s_rgb = stg + 3 * nc * KV, *s_a = stg + 6 * nc * KV;
                if (row_owner && r >= r0 && r < r0 + nc)
                    mb::convert_gaussian<DEG, BF16>(out.G, out.kc, g, y, s_xyz, s_rgb, s_a, (r - r0) * KV);
                slot_sync(slot);
                const int64_t v0 = (g0 + r0) * KV;
                slot_store(out.xyz + 3 * v0, s_xyz, 3 * nc * KV, st);
                slot_store(out.rgb + 3 * v0, s_rgb, 3 * nc * KV, st);
                slot_store(out.alpha + v0, s_a, nc * KV, st);
                slot_sync(slot);
            }
        }
        // the next tile's features overwrite X and its first product Z3's columns: the
        // barrier at the top of the next iteration orders them after these reads
    }
    if (!ok) tc::mbar_wait(mbar, phase, kTcWaitLimit);   // let an unfinished product drain
    cp_async_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(*tmem_base, 128 * kSlots);
}

// ------------------------------------------------------------------ training: activations

constexpr uint32_t kAW = kW1f, kAWEnd = kPackedBytes;    // all five weight tiles
constexpr uint32_t kAX = kAWEnd - kAW;                   // X  [128][16]
constexpr uint32_t kAH1 = kAX + kRows * kIn * 2;         // H1, later dZ2 [128][128]
constexpr uint32_t kAH2 = kAH1 + kRows * kHid * 2;       // H2
constexpr uint32_t kAdY = kAH2 + kRows * kHid * 2;       // dY [128][32]
constexpr uint32_t kAT = kAdY + kRows * kOutPad * 2;     // transpose staging [128][128]
constexpr uint32_t kAState = kAT + kHid * kRows * 2;
constexpr uint32_t kActSmem = kAState + 64;

// Writes column values v[0..n) of this thread's row r into the staging tile laid out as
// [feature][row] (K = rows), at features f0..f0+n.
__device__ __forceinline__ void stage_t(char *T, int r, int f0, const float *v, int n) {
    for (int i = 0; i < n; ++i)
        *reinterpret_cast<uint16_t *>(T + tc::cm_offset(f0 + i, r, kRows)) = bf16_bits(v[i]);
}
// Copies `bytes` of the staging tile to global (all threads, after a barrier).
__device__ __forceinline__ void flush_t(const char *T, char *dst, uint32_t bytes) {
    __syncthreads();
    const uint4 *s = reinterpret_cast<const uint4 *>(T);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

__global__ void __launch_bounds__(128, 1) mlp_act_kernel(const float *__restrict__ Xin, const float *__restrict__ Tgt,
                                                         int64_t n, int n_out, const char *__restrict__ packed,
                                                         char *__restrict__ act, float *__restrict__ loss) {
    extern __shared__ __align__(1024) char smem[];
    TcState *S = reinterpret_cast<TcState *>(smem + kAState);
    uint32_t *timeouts = reinterpret_cast<uint32_t *>(const_cast<char *>(packed) + kStatusOff);
    setup(smem, packed, kAW, kAWEnd, smem, S, 512);
    const char *W1 = smem + kW1f, *W2 = smem + kW2f, *W3 = smem + kW3f, *W3b = smem + kW3b, *W2b = smem + kW2b;
    char *X = smem + kAX, *H1 = smem + kAH1, *H2 = smem + kAH2, *dY = smem + kAdY, *T = smem + kAT;
    const int r = threadIdx.x, warp = r >> 5;
    const uint32_t lo = (uint32_t)(warp * 32) << 16;
    const uint32_t tZ1 = S->tmem, tZ2 = S->tmem + 128, tZ3 = S->tmem + 256, tdH2 = S->tmem + 384,
                   tdH1 = S->tmem + 128;
    const int64_t tiles = (n + kRows - 1) / kRows;
    const float dscale = 2.0f / ((float)n * (float)n_out);
    float my_loss = 0.0f;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int64_t g = t * kRows + r;
        const bool live = g < n;
        char *out = act + (size_t)t * kTileBytes;
        float f[kIn];
#pragma unroll
        for (int i = 0; i < kIn; ++i) f[i] = live ? Xin[g * kIn + i] : 0.0f;
        put8(X, kIn, r, 0, f);
        put8(X, kIn, r, 8, f + 8);
        stage_t(T, r, 0, f, kIn);
        flush_t(T, out + kTXt, kIn * kRows * 2);
        // forward
        sync_then(r == 0);
        if (r == 0) issue(tZ1, X, W1, kIn, kHid, false, &S->mbar);
        ok = wait_mma(S, phase, timeouts) && ok;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tZ1 + lo + c0, v);
            gelu16(v);
            put8(H1, kHid, r, c0, v);
            put8(H1, kHid, r, c0 + 8, v + 8);
            stage_t(T, r, c0, v, 16);
        }
        flush_t(T, out + kTH1t, kHid * kRows * 2);
        sync_then(r == 0);
        if (r == 0) issue(tZ2, H1, W2, kHid, kHid, false, &S->mbar);
        ok = wait_mma(S, phase, timeouts) && ok;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tZ2 + lo + c0, v);
            gelu16(v);
            put8(H2, kHid, r, c0, v);
            put8(H2, kHid, r, c0 + 8, v + 8);
            stage_t(T, r, c0, v, 16);
        }
        flush_t(T, out + kTH2t, kHid * kRows * 2);
        sync_then(r == 0);
        if (r == 0) issue(tZ3, H2, W3, kHid, kOutPad, false, &S->mbar);
        ok = wait_mma(S, phase, timeouts) && ok;
        {
            float y[32];
            tc::tmem_ld16(tZ3 + lo, *reinterpret_cast<float(*)[16]>(y));
            tc::tmem_ld16(tZ3 + lo + 16, *reinterpret_cast<float(*)[16]>(y + 16));
            for (int o = 0; o < kOutPad; ++o) {
                float d = 0.0f;
                if (live && o < n_out) {
                    const float e = y[o] - Tgt[g * n_out + o];
                    my_loss += e * e;
                    d = dscale * e;
                }
                y[o] = d;
            }
            for (int c0 = 0; c0 < kOutPad; c0 += 8) put8(dY, kOutPad, r, c0, y + c0);
            stage_t(T, r, 0, y, kOutPad);
            flush_t(T, out + kTdYt, kOutPad * kRows * 2);
        }
        // adjoint: dH2 = dY W3^T, dZ2 = dH2 gelu'(Z2)
        sync_then(r == 0);
        if (r == 0) issue(tdH2, dY, W3b, kOutPad, kHid, false, &S->mbar);
        ok = wait_mma(S, phase, timeouts) && ok;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float z[16], d[16];
            tc::tmem_ld16(tZ2 + lo + c0, z);
            tc::tmem_ld16(tdH2 + lo + c0, d);
            for (int i = 0; i < 16; ++i) d[i] *= gelu_grad(z[i]);
            put8(H1, kHid, r, c0, d);          // H1's product finished: the buffer now holds dZ2
            put8(H1, kHid, r, c0 + 8, d + 8);
            stage_t(T, r, c0, d, 16);
        }
        flush_t(T, out + kTdZ2t, kHid * kRows * 2);
        // dH1 = dZ2 W2^T, dZ1 = dH1 gelu'(Z1)
        sync_then(r == 0);
        if (r == 0) issue(tdH1, H1, W2b, kHid, kHid, false, &S->mbar);
        ok = wait_mma(S, phase, timeouts) && ok;
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float z[16], d[16];
            tc::tmem_ld16(tZ1 + lo + c0, z);
            tc::tmem_ld16(tdH1 + lo + c0, d);
            for (int i = 0; i < 16; ++i) d[i] *= gelu_grad(z[i]);
            stage_t(T, r, c0, d, 16);
        }
        flush_t(T, out + kTdZ1t, kHid * kRows * 2);
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
    }
    for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
    if ((r & 31) == 0) atomicAdd(loss, my_loss / ((float)n * (float)n_out));
    if (!ok) tc::mbar_wait(&S->mbar, phase, kTcWaitLimit);
    teardown(S, 512);
}

// ------------------------------------------------------------------ training: weight gradients

constexpr uint32_t kGState = kTileBytes;
constexpr uint32_t kGradSmem = kGState + 64;

__global__ void __launch_bounds__(128, 1) mlp_wgrad_kernel(const char *__restrict__ act, int64_t tiles, int n_out,
                                                           uint32_t *timeouts, float *__restrict__ dW1,
                                                           float *__restrict__ dW2, float *__restrict__ dW3) {
    extern __shared__ __align__(1024) char smem[];
    TcState *S = reinterpret_cast<TcState *>(smem + kGState);
    __shared__ uint64_t load_bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&S->mbar, 1);
        tc::mbar_init(&load_bar, 1);
        tc::mbar_init_fence();
    }
    if (threadIdx.x < 32) tc::tmem_alloc(&S->tmem, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tD1 = S->tmem, tD2 = S->tmem + 32, tD3 = S->tmem + 160;
    uint32_t load_phase = 0, phase = 0;
    bool ok = true, first = true;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // one bulk copy brings the tile's six operands (all laid out K-major, K = rows)
        if (threadIdx.x == 0) {
            tc::mbar_expect_tx(&load_bar, kTileBytes);
            const char *src = act + (size_t)t * kTileBytes;
            const uint32_t parts[7] = {kTXt, kTH1t, kTH2t, kTdYt, kTdZ2t, kTdZ1t, kTileBytes};
            for (int i = 0; i < 6; ++i) tc::bulk_g2s(smem + parts[i], src + parts[i], parts[i + 1] - parts[i], &load_bar);
        }
        const bool loaded = tc::mbar_wait(&load_bar, load_phase, kTcWaitLimit);
        load_phase ^= 1u;
        if (!__syncthreads_and(loaded)) {
            if (threadIdx.x == 0) atomicAdd(timeouts, 1u);
            // the copy may still land: wait for it once more before the smem is released
            tc::mbar_wait(&load_bar, load_phase ^ 1u, kTcWaitLimit);
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            issue(tD1, smem + kTdZ1t, smem + kTXt, kRows, kIn, !first, nullptr);       // dW1^T
            issue(tD2, smem + kTdZ2t, smem + kTH1t, kRows, kHid, !first, nullptr);     // dW2^T
            issue(tD3, smem + kTH2t, smem + kTdYt, kRows, kOutPad, !first, &S->mbar);  // dW3
        }
        const bool done = wait_mma(S, phase, timeouts);
        first = false;
        if (!__syncthreads_and(done)) {
            ok = false;
            break;
        }
    }
    if (ok && !first) {
        const int r = threadIdx.x, warp = r >> 5;
        const uint32_t lo = (uint32_t)(warp * 32) << 16;
        float v[16];
        tc::tmem_ld16(tD1 + lo, v);                    // row r = h1 unit, columns = inputs
        for (int i = 0; i < kIn; ++i) atomicAdd(&dW1[i * kHid + r], v[i]);
        for (int c0 = 0; c0 < kHid; c0 += 16) {         // row r = h2 unit, columns = h1 units
            tc::tmem_ld16(tD2 + lo + c0, v);
            for (int i = 0; i < 16; ++i) atomicAdd(&dW2[(c0 + i) * kHid + r], v[i]);
        }
        for (int c0 = 0; c0 < kOutPad; c0 += 16) {      // row r = h2 unit, columns = outputs
            tc::tmem_ld16(tD3 + lo + c0, v);
            for (int i = 0; i < 16; ++i)
                if (c0 + i < n_out) atomicAdd(&dW3[r * n_out + c0 + i], v[i]);
        }
    }
    if (!ok) tc::mbar_wait(&S->mbar, phase, kTcWaitLimit);   // let an unfinished product drain
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(S->tmem, 256);
}

// ------------------------------------------------------------------ packing and Adam

__global__ void mlp_pack_kernel(const float *__restrict__ W1, const float *__restrict__ W2,
                                const float *__restrict__ W3, int n_out, char *__restrict__ packed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    auto put = [&](uint32_t base, int Kc, int row, int k, float v) {
        *reinterpret_cast<uint16_t *>(packed + base + tc::cm_offset(row, k, Kc)) = bf16_bits(v);
    };
    if (i < kHid * kIn) {                         // W1f[h][in] = W1[in][h]
        const int h = i / kIn, k = i % kIn;
        put(kW1f, kIn, h, k, W1[k * kHid + h]);
    }
    if (i < kHid * kHid) {
        const int a = i / kHid, b = i % kHid;
        put(kW2f, kHid, a, b, W2[b * kHid + a]);  // W2f[h2][h1] = W2[h1][h2]
        put(kW2b, kHid, a, b, W2[a * kHid + b]);  // W2b[h1][h2] = W2[h1][h2]
    }
    if (i < kOutPad * kHid) {
        const int o = i / kHid, h = i % kHid;     // W3f[o][h2] = W3[h2][o]
        put(kW3f, kHid, o, h, o < n_out ? W3[h * n_out + o] : 0.0f);
        const int h2 = i / kOutPad, o2 = i % kOutPad;   // W3b[h2][o] = W3[h2][o]
        put(kW3b, kOutPad, h2, o2, o2 < n_out ? W3[h2 * n_out + o2] : 0.0f);
    }
}

__global__ void flat_adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                                 float *__restrict__ v, int64_t n, const int32_t *step, float lr, float b1, float b2,
                                 float eps) {
    const float t = (float)(*step + 1);
    const float bc1 = 1.0f - powf(b1, t), bc2 = 1.0f - powf(b2, t);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mm = b1 * m[i] + (1.0f - b1) * gi;
        const float vv = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mm;
        v[i] = vv;
        p[i] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

__global__ void step_inc_kernel(int32_t *step) { *step += 1; }

__global__ void mlp_features_kernel(const MlpSrc s, int64_t N, float *__restrict__ X) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    float f[kIn];
    gaussian_features(s, g, f);
    for (int i = 0; i < kIn; ++i) X[g * kIn + i] = f[i];
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

size_t mlp_packed_bytes() { return kPackedTotal; }
size_t mlp_act_bytes(int64_t n) { return (size_t)((n + kRows - 1) / kRows) * kTileBytes; }
size_t mlp_param_count(int n_out) { return (size_t)kIn * kHid + (size_t)kHid * kHid + (size_t)kHid * n_out; }
uint32_t mlp_status_offset() { return kStatusOff; }

cudaError_t launch_mlp_pack(const float *W1, const float *W2, const float *W3, int n_out, char *packed,
                            cudaStream_t st) {
    mlp_pack_kernel<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(W1, W2, W3, n_out, packed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_features(const MlpSrc &s, int64_t N, float *X, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    mlp_features_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(s, N, X);
    return cudaGetLastError();
}

namespace {

template <bool FUSED, int DEG, bool BF16>
cudaError_t launch_fwd(const MlpSrc &s, int64_t N, const char *packed, int n_out, const FwdOut &out,
                       cudaStream_t st) {
    auto fn = mlp_fwd_kernel<FUSED, DEG, BF16>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (N + kRows - 1) / kRows;
    const int grid = (int)min64((tiles + kSlots - 1) / kSlots, (int64_t)sm_count());
    fn<<<grid, kFwdThreads, kFwdSmem, st>>>(s, N, packed, n_out, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_forward(const MlpSrc &s, int64_t N, const char *packed, int n_out, float *corr,
                               cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    FwdOut out;
    memset(&out, 0, sizeof(out));
    out.corr = corr;
    return launch_fwd<false, 0, false>(s, N, packed, n_out, out, st);
}

cudaError_t launch_mesh_build_mlp(const float *means, const MlpSrc &s, int64_t N, const char *packed,
                                  const MeshBuildConst &kc, float *xyz, float *rgb, float *alpha, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    FwdOut out;
    memset(&out, 0, sizeof(out));
    out.G = mb::Gaussians{means, s.log_scales, s.quats, s.opacity, s.sh};
    out.kc = kc;
    out.xyz = xyz;
    out.rgb = rgb;
    out.alpha = alpha;
    const int n_out = 2 * (kc.K + 1);
    const bool bf16 = s.sh_dtype == 1;
    switch (s.sh_degree) {
        case 0: return bf16 ? launch_fwd<true, 0, true>(s, N, packed, n_out, out, st)
                            : launch_fwd<true, 0, false>(s, N, packed, n_out, out, st);
        case 1: return bf16 ? launch_fwd<true, 1, true>(s, N, packed, n_out, out, st)
                            : launch_fwd<true, 1, false>(s, N, packed, n_out, out, st);
        case 2: return bf16 ? launch_fwd<true, 2, true>(s, N, packed, n_out, out, st)
                            : launch_fwd<true, 2, false>(s, N, packed, n_out, out, st);
        default: return bf16 ? launch_fwd<true, 3, true>(s, N, packed, n_out, out, st)
                             : launch_fwd<true, 3, false>(s, N, packed, n_out, out, st);
    }
}

cudaError_t launch_mlp_grads(const float *X, const float *T, int64_t n, int n_out, const char *packed, char *act,
                             float *grads, float *loss, cudaStream_t st) {
    const size_t np = mlp_param_count(n_out);
    cudaError_t e = cudaMemsetAsync(grads, 0, np * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess || n == 0) return e;
    const int64_t tiles = (n + kRows - 1) / kRows;
    const int grid = (int)min64(tiles, sm_count());
    cudaFuncSetAttribute(mlp_act_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kActSmem);
    mlp_act_kernel<<<grid, 128, kActSmem, st>>>(X, T, n, n_out, packed, act, loss);
    cudaFuncSetAttribute(mlp_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    uint32_t *timeouts = reinterpret_cast<uint32_t *>(const_cast<char *>(packed) + kStatusOff);
    mlp_wgrad_kernel<<<grid, 128, kGradSmem, st>>>(act, tiles, n_out, timeouts, grads, grads + kIn * kHid,
                                                   grads + kIn * kHid + kHid * kHid);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *W, const float *grads, float *m, float *v, int n_out, int32_t *d_step, float lr,
                            float b1, float b2, float eps, char *packed, cudaStream_t st) {
    const int64_t np = (int64_t)mlp_param_count(n_out);
    flat_adam_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(W, grads, m, v, np, d_step, lr, b1, b2, eps);
    step_inc_kernel<<<1, 1, 0, st>>>(d_step);
    return launch_mlp_pack(W, W + kIn * kHid, W + kIn * kHid + kHid * kHid, n_out, packed, st);
}

}  // namespace ms
