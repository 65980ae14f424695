// Storage order of the Gaussians: a permutation that sorts them by the Morton code of their
// means, and a row gather that applies it.
//
// The render's passes reach the fans through the sorted (tile, depth) pairs and the
// fragment records, in screen order; with the Gaussians stored in input order, the fans
// that meet in one tile sit anywhere in the soup, so every pair gathers its fan from its
// own sectors, and the adjoint's per-vertex gradient sums scatter over the whole soup.
// With the soup in Morton order, fans that are near in space are near in memory: the
// gathers of one tile share sectors and L2 lines, and the chain's sums land in a few
// regions at a time.  The order changes nothing the method computes (the paper's render is
// independent of the input order except for exact depth ties, which go to the lower
// triangle index of the reordered soup).
//
// Codes: each coordinate of a mean is quantised to 10 bits over the means' bounding box,
// q = min(max(floor((m - lo) / (hi - lo) * 1024), 0), 1023) in binary32 (an axis of zero
// extent counts as extent 1), and the bits are interleaved x, y, z from the top.  Ties keep
// the input order (the index is the low word of the sorted element), so the permutation
// is unique.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kOrderBlk = 256;

// Floats as unsigned integers ordered like their values (for atomic min / max).
__device__ __forceinline__ unsigned ord_key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_val(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void box_init_kernel(unsigned *box) {
    if (threadIdx.x < 3) box[threadIdx.x] = 0xffffffffu;   // min
    else if (threadIdx.x < 6) box[threadIdx.x] = 0u;        // max
}

__global__ void __launch_bounds__(kOrderBlk) box_kernel(const float *__restrict__ means, int64_t N, unsigned *box) {
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float c = __ldg(means + 3 * i + r);
            lo[r] = fminf(lo[r], c);
            hi[r] = fmaxf(hi[r], c);
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[r] = fminf(lo[r], __shfl_xor_sync(0xffffffffu, lo[r], o));
            hi[r] = fmaxf(hi[r], __shfl_xor_sync(0xffffffffu, hi[r], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            atomicMin(&box[r], ord_key(lo[r]));
            atomicMax(&box[3 + r], ord_key(hi[r]));
        }
    }
}

// 10 bits of x moved to every third bit (bit i to bit 3 i).
__device__ __forceinline__ unsigned long long dilate3(unsigned x) {
    unsigned long long v = x & 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFull;
    v = (v | (v << 8)) & 0x0300F00Full;
    v = (v | (v << 4)) & 0x030C30C3ull;
    v = (v | (v << 2)) & 0x09249249ull;
    return v;
}

__global__ void __launch_bounds__(kOrderBlk) code_kernel(const float *__restrict__ means, int64_t N,
                                                          const unsigned *__restrict__ box,
                                                          unsigned long long *__restrict__ keys) {
    float lo[3], ext[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        lo[r] = ord_val(box[r]);
        const float e = ord_val(box[3 + r]) - lo[r];
        ext[r] = e > 0.0f ? e : 1.0f;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long code = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float q = fminf(fmaxf(floorf(__fdiv_rn(__fsub_rn(__ldg(means + 3 * i + r), lo[r]), ext[r]) * 1024.0f),
                                        0.0f), 1023.0f);
            code |= dilate3((unsigned)q) << (2 - r);
        }
        keys[i] = (code << 32) | (unsigned long long)(uint32_t)i;
    }
}

__global__ void __launch_bounds__(kOrderBlk) perm_kernel(const unsigned long long *__restrict__ sorted, int64_t N,
                                                          int32_t *__restrict__ perm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int32_t)(uint32_t)(sorted[i] & 0xffffffffull);
}

// dst row i = src row perm[i], rows of `words` 32-bit words: consecutive threads take
// consecutive words of dst, so writes are coalesced and a row's words are read together.
__global__ void __launch_bounds__(kOrderBlk) gather_kernel(const uint32_t *__restrict__ src, int64_t n, int64_t words,
                                                            const int32_t *__restrict__ perm,
                                                            uint32_t *__restrict__ dst) {
    const int64_t total = n * words;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / words, w = t - i * words;
        dst[t] = __ldg(src + (int64_t)__ldg(perm + i) * words + w);
    }
}

struct OrderLayout {
    size_t box, keys0, keys1, scratch, total;
};
OrderLayout order_layout(int64_t N) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    OrderLayout L;
    size_t o = 0;
    L.box = o;     o = al(o + 64);
    L.keys0 = o;   o = al(o + 8 * (size_t)(N > 0 ? N : 1));
    L.keys1 = o;   o = al(o + 8 * (size_t)(N > 0 ? N : 1));
    L.scratch = o; o = al(o + sort_scratch_bytes(N > 0 ? N : 1, 4));
    L.total = o;
    return L;
}

unsigned grid_for(int64_t n) { return (unsigned)min64((n + kOrderBlk - 1) / kOrderBlk, 152 * 16); }

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" MS_API size_t ms_spatial_order_workspace_size(int64_t N) {
    if (N < 0 || N >= (1ll << 31)) return 0;
    return order_layout(N).total;
}

extern "C" MS_API ms_status ms_spatial_order(const float *means, int64_t N, int32_t *perm, void *workspace,
                                             size_t ws_bytes, void *stream) {
    if (N < 0 || N >= (1ll << 31)) return set_error(MS_ERR_INVALID, "N=%lld outside 0..2^31-1", (long long)N);
    if (N == 0) return MS_OK;
    if (!means || !perm || !workspace) return set_error(MS_ERR_INVALID, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return set_error(MS_ERR_INVALID, "workspace not 256-byte aligned");
    const OrderLayout L = order_layout(N);
    if (ws_bytes < L.total)
        return set_error(MS_ERR_INVALID, "workspace %zu bytes, %zu needed", ws_bytes, L.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = static_cast<char *>(workspace);
    unsigned *box = reinterpret_cast<unsigned *>(ws + L.box);
    unsigned long long *k0 = reinterpret_cast<unsigned long long *>(ws + L.keys0);
    unsigned long long *k1 = reinterpret_cast<unsigned long long *>(ws + L.keys1);
    box_init_kernel<<<1, 32, 0, st>>>(box);
    box_kernel<<<grid_for(N), kOrderBlk, 0, st>>>(means, N, box);
    code_kernel<<<grid_for(N), kOrderBlk, 0, st>>>(means, N, box, k0);
    unsigned long long *sorted = nullptr;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = sort_u64(k0, k1, N, 32, 4, ws + L.scratch, st, &sorted);
    if (e == cudaSuccess) {
        perm_kernel<<<grid_for(N), kOrderBlk, 0, st>>>(sorted, N, perm);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "spatial order: %s", cudaGetErrorString(e));
    count_launches(4);
    return MS_OK;
}

extern "C" MS_API ms_status ms_gather_rows(const void *src, int64_t n_rows, int64_t row_bytes, const int32_t *perm,
                                           void *dst, void *stream) {
    if (n_rows < 0 || row_bytes <= 0 || (row_bytes & 3)) return set_error(MS_ERR_INVALID, "bad row size");
    if (n_rows == 0) return MS_OK;
    if (!src || !perm || !dst) return set_error(MS_ERR_INVALID, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 3)
        return set_error(MS_ERR_INVALID, "rows not 4-byte aligned");
    if (src == dst) return set_error(MS_ERR_INVALID, "src and dst must not overlap");
    const int64_t words = row_bytes / 4;
    gather_kernel<<<grid_for(n_rows * words), kOrderBlk, 0, (cudaStream_t)stream>>>(
        static_cast<const uint32_t *>(src), n_rows, words, perm, static_cast<uint32_t *>(dst));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "gather: %s", cudaGetErrorString(e));
    count_launches(1);
    return MS_OK;
}
