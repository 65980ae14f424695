// LSD radix sort of the 64-bit (tile | depth | fan id) elements by their tile and depth
// bits (above the fan id's low bits), 8-bit digits.
//
// One histogram kernel reads the elements once and counts the digits of every pass; each
// pass is then a single "onesweep" kernel: a block loads its 4096 elements (all loads
// issued before any is used), ranks them with warp-cooperative multi-split
// (__match_any_sync + popc, stable), publishes its per-digit counts, and obtains its
// global per-digit offsets by decoupled look-back over the preceding blocks (bounded
// waits).  Elements are reordered through shared memory so the global stores are
// digit-contiguous.  Per pass each element is read once and written once: 2 x 8 B of HBM
// traffic per pair.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kSortThreads = 512;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // 8192 elements per block
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kHistThreads = 256;                      // histogram kernel block
// (fewer, larger tiles: the per-tile look-back and block scans, not the bytes, bound a pass)
constexpr uint32_t kLbAgg = 1u << 30, kLbPre = 2u << 30, kLbMask = (1u << 30) - 1;

__device__ __forceinline__ int64_t n_pairs(const Status *st, int64_t cap) {
    const unsigned long long p = st->pairs;
    return (int64_t)(p < (unsigned long long)cap ? p : (unsigned long long)cap);
}

__global__ void __launch_bounds__(kHistThreads) sort_hist_kernel(const unsigned long long *__restrict__ keys,
                                                                 const Status *st, int64_t cap, int passes,
                                                                 int shift0, uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += kHistThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = n_pairs(st, cap);
    const int64_t stride = (int64_t)gridDim.x * kHistThreads;
    int64_t i = (int64_t)blockIdx.x * kHistThreads + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {   // four loads in flight per thread
        unsigned long long k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k[u] = __ldg(keys + i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(k[u] >> (shift0 + 8 * p)) & 0xFF], 1u);
    }
    for (; i < n; i += stride) {
        const unsigned long long k = __ldg(keys + i);
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(k >> (shift0 + 8 * p)) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kHistThreads) {
        const uint32_t c = (&s_h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Exclusive scan of each pass's 256-digit histogram (in place), one block.
__global__ void sort_scan_kernel(uint32_t *hist, int passes) {
    __shared__ uint32_t s[256];
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = hist[p * 256 + threadIdx.x];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            const uint32_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        hist[p * 256 + threadIdx.x] = s[threadIdx.x] - v;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads, 2) sort_pass_kernel(const unsigned long long *__restrict__ kin,
                                                                 unsigned long long *__restrict__ kout, Status *st,
                                                                 int64_t cap, const uint32_t *__restrict__ digit_base,
                                                                 uint32_t *lookback, int pass, int shift) {
    extern __shared__ unsigned long long s_dyn[];
    unsigned long long *s_keys = s_dyn;                                       // kSortTile
    uint32_t *s_wh = reinterpret_cast<uint32_t *>(s_keys + kSortTile);      // kSortWarps x 256
    uint32_t *s_loc = s_wh + kSortWarps * 256;                                // 256: block-local digit offsets
    uint32_t *s_glob = s_loc + 256;                                           // 256: global digit bases
    __shared__ int s_vid;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_all = n_pairs(st, cap);
    // Persistent blocks: each takes the next tile of the pass in ticket order until none is
    // left, so the grid does not depend on the pair capacity.
    for (;;) {
    if (tid == 0) s_vid = (int)atomicAdd(&st->sort_ticket[pass], 1u);
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) s_wh[i] = 0;
    __syncthreads();
    const int64_t vid = s_vid;
    const int64_t base = vid * kSortTile;
    if (base >= n_all) return;
    const int n = (int)min64(kSortTile, n_all - base);

    // Warp w owns elements [w*512, w*512+512) of the tile, item j at j*32 + lane; all
    // loads are issued first.
    unsigned long long k[kSortItems];
    uint32_t rank[kSortItems];
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int idx = warp * (kSortItems * 32) + j * 32 + lane;
        k[j] = idx < n ? __ldg(kin + base + idx) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int idx = warp * (kSortItems * 32) + j * 32 + lane;
        const bool ok = idx < n;
        const uint32_t d = ok ? (uint32_t)((k[j] >> shift) & 0xFF) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = ok ? s_wh[warp * 256 + d] : 0u;
        __syncwarp();
        if (ok && (peers & lt_mask) == 0) s_wh[warp * 256 + d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // Threads 0..255 take one digit each: exclusive prefix over warps and block total.
    const int d = tid;
    const bool dig = tid < 256;
    uint32_t tot = 0;
    if (dig) {
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = s_wh[w * 256 + d];
            s_wh[w * 256 + d] = tot;
            tot += c;
        }
    }
    // Block-local exclusive offsets over digits (the first eight warps).
    {
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ uint32_t s_ws[8];
        if (dig && lane == 31) s_ws[warp] = x;
        __syncthreads();
        uint32_t add = 0;
        if (dig) {
            for (int w = 0; w < warp; ++w) add += s_ws[w];
            s_loc[d] = x - tot + add;
        }
    }
    // Look-back for this digit's global offset.
    if (dig) {
        uint32_t *lb = lookback + (size_t)vid * 256 + d;
        uint32_t excl = 0;
        if (vid == 0) {
            st_release_u32(lb, kLbPre | tot);
        } else {
            st_release_u32(lb, kLbAgg | tot);
            int64_t j = vid - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const uint32_t s = ld_acquire_u32(lookback + (size_t)j * 256 + d);
                const uint32_t flag = s & ~kLbMask;
                if (flag == 0) {
                    if (++spins > kSpinLimit) {
                        atomicAdd(&st->timeouts, 1u);
                        break;
                    }
                    continue;
                }
                excl += s & kLbMask;
                if (flag == kLbPre) break;
                --j;
            }
            st_release_u32(lb, kLbPre | (excl + tot));
        }
        s_glob[d] = digit_base[pass * 256 + d] + excl;
    }
    __syncthreads();
    // Reorder through shared memory by digit.
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int idx = warp * (kSortItems * 32) + j * 32 + lane;
        if (idx < n) {
            const uint32_t dd = (uint32_t)((k[j] >> shift) & 0xFF);
            s_keys[s_loc[dd] + s_wh[warp * 256 + dd] + rank[j]] = k[j];
        }
    }
    __syncthreads();
    for (int p = tid; p < n; p += kSortThreads) {
        const unsigned long long kk = s_keys[p];
        const uint32_t dd = (uint32_t)((kk >> shift) & 0xFF);
        kout[(size_t)s_glob[dd] + (p - s_loc[dd])] = kk;
    }
    __syncthreads();   // shared memory is reused by the next tile
    }
}

__global__ void tile_ranges_kernel(const unsigned long long *__restrict__ keys, const Status *st, int64_t cap,
                                   int tile_shift, uint2 *__restrict__ ranges) {
    const int64_t n = n_pairs(st, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[i] >> tile_shift);
        if (i == 0 || (uint32_t)(keys[i - 1] >> tile_shift) != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || (uint32_t)(keys[i + 1] >> tile_shift) != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

__global__ void set_pairs_kernel(Status *st, int64_t n) { st->pairs = (unsigned long long)n; }

}  // namespace

int64_t sort_tile_elems() { return kSortTile; }

size_t sort_scratch_bytes(int64_t n, int passes) {
    const int64_t blocks = (n + kSortTile - 1) / kSortTile;
    return 256 + 8 * 256 * 4 + (size_t)passes * (size_t)(blocks > 0 ? blocks : 1) * 256 * 4;
}

cudaError_t sort_u64(unsigned long long *a, unsigned long long *b, int64_t n, int shift, int passes, char *scratch,
                     cudaStream_t st, unsigned long long **result) {
    *result = a;
    if (n <= 0 || passes <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, passes), st);
    if (e != cudaSuccess) return e;
    Status *status = reinterpret_cast<Status *>(scratch);
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + 256);
    uint32_t *lookback = hist + 8 * 256;
    const int64_t blocks = (n + kSortTile - 1) / kSortTile;
    set_pairs_kernel<<<1, 1, 0, st>>>(status, n);
    const int hist_grid = (int)min64((n + kHistThreads * 8 - 1) / (kHistThreads * 8), 4 * 152);
    sort_hist_kernel<<<hist_grid, kHistThreads, 0, st>>>(a, status, n, passes, shift, hist);
    sort_scan_kernel<<<1, 256, 0, st>>>(hist, passes);
    const size_t smem = (size_t)kSortTile * 8 + (kSortWarps * 256 + 512) * 4;
    cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, n_sm = 152, per_sm = 2;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pass_kernel, kSortThreads, smem);
    const unsigned grid = (unsigned)min64(blocks, (int64_t)n_sm * (per_sm > 0 ? per_sm : 1));
    unsigned long long *kb[2] = {a, b};
    for (int p = 0; p < passes; ++p)
        sort_pass_kernel<<<grid, kSortThreads, smem, st>>>(kb[p & 1], kb[(p + 1) & 1], status, n, hist,
                                                            lookback + (size_t)p * blocks * 256, p, shift + 8 * p);
    *result = kb[passes & 1];
    count_launches(3 + passes);
    return cudaGetLastError();
}

cudaError_t launch_sort(const RenderArgs &a, cudaStream_t st) {
    const RenderLayout &L = a.L;
    if (a.n_fans == 0) return cudaSuccess;
    char *ws = a.ws;
    Status *status = reinterpret_cast<Status *>(ws + L.off_status);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.off_hist);
    unsigned long long *kb[2] = {reinterpret_cast<unsigned long long *>(ws + L.off_keys0),
                                 reinterpret_cast<unsigned long long *>(ws + L.off_keys1)};
    const int hist_grid = (int)min64((L.cap + kHistThreads * 8 - 1) / (kHistThreads * 8), 4 * 152);
    sort_hist_kernel<<<hist_grid, kHistThreads, 0, st>>>(kb[0], status, L.cap, L.passes, L.fan_bits, hist);
    sort_scan_kernel<<<1, 256, 0, st>>>(hist, L.passes);
    const size_t smem = (size_t)kSortTile * 8 + (kSortWarps * 256 + 512) * 4;
    cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, n_sm = 152, per_sm = 4;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pass_kernel, kSortThreads, smem);
    const unsigned grid = (unsigned)min64(L.sort_blocks, (int64_t)n_sm * (per_sm > 0 ? per_sm : 1));
    for (int p = 0; p < L.passes; ++p) {
        sort_pass_kernel<<<grid, kSortThreads, smem, st>>>(
            kb[p & 1], kb[(p + 1) & 1], status, L.cap, hist,
            reinterpret_cast<uint32_t *>(ws + L.off_lookback) + (size_t)p * L.sort_blocks * 256, p, L.fan_bits + 8 * p);
    }
    const unsigned long long *sorted = kb[L.passes & 1];
    const int rg = (int)min64((L.cap + 255) / 256, 8 * 152);
    tile_ranges_kernel<<<rg, 256, 0, st>>>(sorted, status, L.cap, L.fan_bits + L.depth_bits,
                                           reinterpret_cast<uint2 *>(ws + L.off_ranges));
    return cudaGetLastError();
}

}  // namespace ms
