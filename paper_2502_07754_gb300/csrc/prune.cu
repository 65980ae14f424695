// Pruning step of Sec. 3 ("Optimization and Pruning"): a face goes when all three of its
// vertex opacities are below the threshold (exp(-4) in the paper), and vertices that no
// face uses go with it.  Per fan this is a face mask: bit j (face (c, b_j, b_j+1)) stays
// set while some vertex of the face is at or above the threshold, ANDed with the mask the
// fan already had (faces once removed stay removed).  A fan whose mask becomes zero -- with
// no earlier mask, exactly when all K + 1 vertices are below the threshold -- is removed
// with its K + 1 vertices; the others are kept whole (a kept fan's vertices are all used by
// its kept faces or shared with them through the centre) and compacted in order, with
// their vertices' Adam moments (layout [xyz 3V | rgb 3V | alpha V]) and their masks.
//
// Three launches, no waits between blocks: per-block counts of kept fans; one block
// scanning the block counts (and writing the kept total); every block ranks its fans
// again and copies the kept ones to their new slots.  The copy is block-cooperative: the
// block's kept fans of a row are contiguous in the output, so consecutive threads write
// consecutive output words (each thread finds its source fan from a shared-memory map).
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kPThreads = 256, kPItems = 4, kPFans = kPThreads * kPItems;   // fans per block

// Face mask of fan f after this pruning step.
__device__ __forceinline__ uint32_t fan_faces(const float *__restrict__ alpha, const uint32_t *__restrict__ mask_in,
                                              int64_t f, int K, float thr) {
    const float *a = alpha + f * (K + 1);
    const bool c_low = a[0] < thr;
    const bool b0_low = a[1] < thr;
    uint32_t m = 0;
    for (int j = 0; j < K; ++j) {
        const bool bj_low = a[1 + j] < thr;
        const bool bn_low = (j + 1 == K) ? b0_low : (a[2 + j] < thr);
        if (!(c_low && bj_low && bn_low)) m |= 1u << j;
    }
    if (mask_in) m &= mask_in[f];
    return m & ((1u << K) - 1u);
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

__global__ void __launch_bounds__(kPThreads) prune_count_kernel(const float *__restrict__ alpha,
                                                                const uint32_t *__restrict__ mask_in, int64_t n_fans,
                                                                int K, float thr, uint32_t *__restrict__ bsum) {
    __shared__ uint32_t s_warp[kPThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPFans;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < kPItems; ++i) {
        const int64_t f = base + i * kPThreads + threadIdx.x;
        if (f < n_fans && fan_faces(alpha, mask_in, f, K, thr)) ++c;
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
    const uint32_t *mask_in;
    float *xyz_o, *rgb_o, *alpha_o, *m_o, *v_o;
    uint32_t *mask_o;
};

// Copies `per` consecutive words of every kept fan of the row from src (fan f at f * per)
// to dst (new fan nf at nf * per): consecutive threads take consecutive output words.
__device__ __forceinline__ void copy_rows(const float *__restrict__ src, float *__restrict__ dst, int per,
                                          const uint32_t *s_src, uint32_t kept, int64_t out0) {
    const uint32_t words = kept * (uint32_t)per;
    for (uint32_t o = threadIdx.x; o < words; o += kPThreads) {
        const uint32_t r = o / (uint32_t)per, w = o - r * (uint32_t)per;
        dst[(out0 + r) * per + w] = src[(int64_t)s_src[r] * per + w];
    }
}

__global__ void __launch_bounds__(kPThreads) prune_scatter_kernel(PruneIO io, int64_t n_fans, int K, float thr,
                                                                  const uint32_t *__restrict__ boff,
                                                                  const int64_t *__restrict__ n_kept) {
    __shared__ uint32_t s_warp[kPThreads / 32];
    __shared__ uint32_t s_src[kPThreads];
    const int64_t base = (int64_t)blockIdx.x * kPFans;
    const int KV = K + 1;
    const int64_t Vo = n_fans * KV, Vn = *n_kept * KV;
    uint32_t row_base = boff[blockIdx.x];
    for (int i = 0; i < kPItems; ++i) {   // rows of kPThreads consecutive fans, in order
        const int64_t f = base + i * kPThreads + threadIdx.x;
        const uint32_t faces = f < n_fans ? fan_faces(io.alpha, io.mask_in, f, K, thr) : 0u;
        uint32_t tot;
        const uint32_t rank = block_excl(faces ? 1u : 0u, s_warp, &tot);
        if (faces) {
            s_src[rank] = (uint32_t)(f - base);
            if (io.mask_o) io.mask_o[row_base + rank] = faces;
        }
        __syncthreads();
        // fan-major arrays: xyz and rgb (3 KV words a fan), alpha (KV)
        const int64_t f0 = base;   // s_src holds offsets from the block's first fan
        for (int part = 0; part < 3; ++part) {
            const int per = part == 2 ? KV : 3 * KV;
            const float *src = (part == 0 ? io.xyz : part == 1 ? io.rgb : io.alpha) + f0 * per;
            float *dst = part == 0 ? io.xyz_o : part == 1 ? io.rgb_o : io.alpha_o;
            copy_rows(src, dst, per, s_src, tot, row_base);
        }
        // moments: [xyz 3V | rgb 3V | alpha V] segments, each fan-major like the soup
        for (int mv = 0; mv < 2; ++mv) {
            const float *ms_ = mv ? io.v : io.m;
            float *mo = mv ? io.v_o : io.m_o;
            if (!ms_) continue;
            copy_rows(ms_ + f0 * 3 * KV, mo, 3 * KV, s_src, tot, row_base);
            copy_rows(ms_ + 3 * Vo + f0 * 3 * KV, mo + 3 * Vn, 3 * KV, s_src, tot, row_base);
            copy_rows(ms_ + 6 * Vo + f0 * KV, mo + 6 * Vn, KV, s_src, tot, row_base);
        }
        row_base += tot;
        __syncthreads();   // s_src is rewritten by the next row
    }
}

}  // namespace

size_t prune_scratch_bytes(int64_t n_fans) {
    const int64_t nblk = (n_fans + kPFans - 1) / kPFans;
    return (size_t)(2 * nblk + 2) * sizeof(uint32_t);
}

cudaError_t launch_prune(const float *xyz, const float *rgb, const float *alpha, const float *m, const float *v,
                         const uint32_t *mask_in, int64_t n_fans, int K, float thr, float *xyz_o, float *rgb_o,
                         float *alpha_o, float *m_o, float *v_o, uint32_t *mask_o, int64_t *n_kept, void *scratch,
                         cudaStream_t st) {
    if (n_fans == 0) return cudaMemsetAsync(n_kept, 0, sizeof(int64_t), st);
    const int64_t nblk = (n_fans + kPFans - 1) / kPFans;
    uint32_t *bsum = static_cast<uint32_t *>(scratch);
    uint32_t *boff = bsum + nblk;
    prune_count_kernel<<<(unsigned)nblk, kPThreads, 0, st>>>(alpha, mask_in, n_fans, K, thr, bsum);
    prune_scan_kernel<<<1, kPThreads, 0, st>>>(bsum, nblk, boff, n_kept);
    PruneIO io{xyz, rgb, alpha, m, v, mask_in, xyz_o, rgb_o, alpha_o, m_o, v_o, mask_o};
    prune_scatter_kernel<<<(unsigned)nblk, kPThreads, 0, st>>>(io, n_fans, K, thr, boff, n_kept);
    return cudaGetLastError();
}

}  // namespace ms
