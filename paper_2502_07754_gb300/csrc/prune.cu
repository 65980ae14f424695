// Pruning step of Sec. 3 ("Optimization and Pruning") at fan granularity: a face goes
// when all three of its vertex opacities are below the threshold (exp(-4) in the paper);
// a fan goes when all of its faces do -- exactly when all K + 1 of its vertices are below
// the threshold, since every face holds the centre and each boundary vertex lies in a
// face.  Kept fans are compacted in order, with their vertices' Adam moments (layout
// [xyz 3V | rgb 3V | alpha V]).
//
// Three launches, no waits between blocks: per-block counts of kept fans; one block
// scanning the block counts (and writing the kept total); every block ranks its fans
// again and copies the kept ones to their new slots.
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kPThreads = 256, kPItems = 4, kPFans = kPThreads * kPItems;   // fans per block

__device__ __forceinline__ bool fan_kept(const float *__restrict__ alpha, int64_t f, int K, float thr) {
    const float *a = alpha + f * (K + 1);
    for (int k = 0; k <= K; ++k)
        if (!(a[k] < thr)) return true;
    return false;
}

// Exclusive prefix over the block's threads; returns it and the block total in *tot.
__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t *s_warp, uint32_t *tot) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();   // s_warp may still be read by an earlier call
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < kPThreads / 32; ++w) {
        if (w < warp) before += s_warp[w];
        all += s_warp[w];
    }
    *tot = all;
    return before + x - v;
}

__global__ void __launch_bounds__(kPThreads) prune_count_kernel(const float *__restrict__ alpha, int64_t n_fans, int K,
                                                                float thr, uint32_t *__restrict__ bsum) {
    __shared__ uint32_t s_warp[kPThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPFans;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < kPItems; ++i) {
        const int64_t f = base + i * kPThreads + threadIdx.x;
        if (f < n_fans && fan_kept(alpha, f, K, thr)) ++c;
    }
    uint32_t tot;
    block_excl(c, s_warp, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block: exclusive scan of the nblk block counts into boff, the total into *n_kept.
__global__ void __launch_bounds__(kPThreads) prune_scan_kernel(const uint32_t *__restrict__ bsum, int64_t nblk,
                                                               uint32_t *__restrict__ boff, int64_t *__restrict__ n_kept) {
    __shared__ uint32_t s_warp[kPThreads / 32];
    const int64_t per = (nblk + kPThreads - 1) / kPThreads;
    const int64_t b0 = threadIdx.x * per, b1 = min64(b0 + per, nblk);
    uint32_t local = 0;
    for (int64_t b = b0; b < b1; ++b) local += bsum[b];
    uint32_t tot;
    uint32_t run = block_excl(local, s_warp, &tot);
    for (int64_t b = b0; b < b1; ++b) {
        boff[b] = run;
        run += bsum[b];
    }
    if (threadIdx.x == 0) *n_kept = (int64_t)tot;
}

struct PruneIO {
    const float *xyz, *rgb, *alpha, *m, *v;
    float *xyz_o, *rgb_o, *alpha_o, *m_o, *v_o;
};

__device__ __forceinline__ void copy_moments(const float *__restrict__ src, float *__restrict__ dst, int64_t Vo,
                                             int64_t Vn, int64_t vo, int64_t vn) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        dst[3 * vn + r] = src[3 * vo + r];
        dst[3 * Vn + 3 * vn + r] = src[3 * Vo + 3 * vo + r];
    }
    dst[6 * Vn + vn] = src[6 * Vo + vo];
}

__global__ void __launch_bounds__(kPThreads) prune_scatter_kernel(PruneIO io, int64_t n_fans, int K, float thr,
                                                                  const uint32_t *__restrict__ boff,
                                                                  const int64_t *__restrict__ n_kept) {
    __shared__ uint32_t s_warp[kPThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPFans;
    const int KV = K + 1;
    const int64_t Vo = n_fans * KV, Vn = *n_kept * KV;
    uint32_t row_base = boff[blockIdx.x];
    for (int i = 0; i < kPItems; ++i) {   // rows of kPThreads consecutive fans, in order
        const int64_t f = base + i * kPThreads + threadIdx.x;
        const bool keep = f < n_fans && fan_kept(io.alpha, f, K, thr);
        uint32_t tot;
        const uint32_t rank = block_excl(keep ? 1u : 0u, s_warp, &tot);
        if (keep) {
            const int64_t nf = (int64_t)row_base + rank;
            for (int k = 0; k < KV; ++k) {
                const int64_t vo = f * KV + k, vn = nf * KV + k;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    io.xyz_o[3 * vn + r] = io.xyz[3 * vo + r];
                    io.rgb_o[3 * vn + r] = io.rgb[3 * vo + r];
                }
                io.alpha_o[vn] = io.alpha[vo];
                if (io.m) copy_moments(io.m, io.m_o, Vo, Vn, vo, vn);
                if (io.v) copy_moments(io.v, io.v_o, Vo, Vn, vo, vn);
            }
        }
        row_base += tot;
    }
}

}  // namespace

size_t prune_scratch_bytes(int64_t n_fans) {
    const int64_t nblk = (n_fans + kPFans - 1) / kPFans;
    return (size_t)(2 * nblk + 2) * sizeof(uint32_t);
}

cudaError_t launch_prune(const float *xyz, const float *rgb, const float *alpha, const float *m, const float *v,
                         int64_t n_fans, int K, float thr, float *xyz_o, float *rgb_o, float *alpha_o, float *m_o,
                         float *v_o, int64_t *n_kept, void *scratch, cudaStream_t st) {
    if (n_fans == 0) return cudaMemsetAsync(n_kept, 0, sizeof(int64_t), st);
    const int64_t nblk = (n_fans + kPFans - 1) / kPFans;
    uint32_t *bsum = static_cast<uint32_t *>(scratch);
    uint32_t *boff = bsum + nblk;
    prune_count_kernel<<<(unsigned)nblk, kPThreads, 0, st>>>(alpha, n_fans, K, thr, bsum);
    prune_scan_kernel<<<1, kPThreads, 0, st>>>(bsum, nblk, boff, n_kept);
    PruneIO io{xyz, rgb, alpha, m, v, xyz_o, rgb_o, alpha_o, m_o, v_o};
    prune_scatter_kernel<<<(unsigned)nblk, kPThreads, 0, st>>>(io, n_fans, K, thr, boff, n_kept);
    return cudaGetLastError();
}

}  // namespace ms
