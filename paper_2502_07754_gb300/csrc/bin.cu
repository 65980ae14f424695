// Tile binning of fans: project, count overlapped tiles, scan and emit one 64-bit sort
// element per (tile, fan) pair, tile | quantised min depth | fan id -- one pass.
//
// The binning unit is the fan (K triangles sharing the centre), not the single
// triangle: a fan is a few pixels wide, so one record per (tile, fan) instead of per
// (tile, triangle) cuts the pairs the sort moves by about K.  Counting, the
// exclusive scan across blocks (decoupled look-back with bounded waits) and the
// emission happen in a single kernel, so fan vertices are read from HBM once.
#include "fan_geom.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kBinThreads = 256;
constexpr float kKeyMargin = 1.0f - 0x1p-20f;

struct BinArgs {
    const float *xyz;
    int64_t n_fans;
    int K, tile_shift, depth_bits, fan_bits;
    float key_scale;
    int64_t cap, fan_blocks;
    unsigned n_tiles, sort_bits;
    Status *st;
    unsigned long long *keys;
    ViewTable vt;
    float4 *dec;               // [view][vertex] decided (xr, yr, Z or -1, origin), read by the raster passes
    int64_t V;
    const uint32_t *face_mask; // per fan, bit j = face j drawn; NULL = all
    const uint32_t *zrange;    // per view: ~bits(zlo), bits(zhi) of the depth pre-pass
};

// Depth range of each view for the keys' quantisation (depth_quant): the view depths of
// every kRangeStride-th fan centre in front of the near plane and inside a frustum twice the
// image's width and height, widened by 1/32 on each side for the fans' extent (each centre
// is a sector of its own, so a sample keeps the sweep short).  Only the keys' resolution
// depends on it (depths outside clamp, which keeps every key a lower bound); eight views
// per sweep over the centres, one atomic per block and bound.
constexpr int kRangeThreads = 256, kRangeViews = 8, kRangeStride = 8;
__global__ void __launch_bounds__(kRangeThreads) depth_range_kernel(const float *__restrict__ xyz, int64_t n_fans,
                                                                    int K, const __grid_constant__ ViewTable vt,
                                                                    int v0, int nv, uint32_t *__restrict__ zr) {
    uint32_t lo_inv[kRangeViews], hi[kRangeViews];
#pragma unroll
    for (int v = 0; v < kRangeViews; ++v) lo_inv[v] = hi[v] = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kRangeStride; g < n_fans;
         g += stride * kRangeStride) {
        const float *p = xyz + g * (int64_t)(K + 1) * 3;
        const float px = __ldg(p), py = __ldg(p + 1), pz = __ldg(p + 2);
#pragma unroll
        for (int v = 0; v < kRangeViews; ++v) {
            if (v >= nv) break;
            const CamDev &c = vt.v[v0 + v].cam;
            const float dx = px - c.C[0], dy = py - c.C[1], dz = pz - c.C[2];
            const float z = fmaf(c.R[6], dx, fmaf(c.R[7], dy, c.R[8] * dz));
            if (!(z > c.znear)) continue;
            const float x = fmaf(c.R[0], dx, fmaf(c.R[1], dy, c.R[2] * dz));
            const float y = fmaf(c.R[3], dx, fmaf(c.R[4], dy, c.R[5] * dz));
            const float xs = fmaf(c.fx, x, c.cx * z), ys = fmaf(c.fy, y, c.cy * z);   // screen x, y times z
            const float W = (float)c.width, H = (float)c.height;
            if (xs < -W * z || xs > 2.0f * W * z || ys < -H * z || ys > 2.0f * H * z) continue;
            lo_inv[v] = max(lo_inv[v], ~__float_as_uint(z * (1.0f - 1.0f / 32.0f)));
            hi[v] = max(hi[v], __float_as_uint(z * (1.0f + 1.0f / 32.0f)));
        }
    }
    // warp, then block reduction: one atomic per block and bound (a few hundred in all)
    __shared__ uint32_t s_r[kRangeThreads / 32][2 * kRangeViews];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kRangeViews; ++v) {
        const uint32_t l = __reduce_max_sync(0xffffffffu, lo_inv[v]), h = __reduce_max_sync(0xffffffffu, hi[v]);
        if (lane == 0) {
            s_r[warp][2 * v] = l;
            s_r[warp][2 * v + 1] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * nv) {
        uint32_t m = 0;
        for (int w = 0; w < kRangeThreads / 32; ++w) m = max(m, s_r[w][threadIdx.x]);
        if (m) atomicMax(zr + 2 * v0 + threadIdx.x, m);
    }
}

// Blocks take virtual ids in start order; id = view * fan_blocks + fan block, so pairs
// come out view by view and, within a view, in fan order.
__global__ void __launch_bounds__(kBinThreads) bin_kernel(const __grid_constant__ BinArgs a) {
    const float *__restrict__ xyz = a.xyz;
    const int64_t n_fans = a.n_fans;
    const int K = a.K, tile_shift = a.tile_shift, depth_bits = a.depth_bits;
    const int64_t cap = a.cap;
    Status *st = a.st;
    unsigned long long *__restrict__ keys = a.keys;
    const int fan_bits = a.fan_bits;
    extern __shared__ float s_xyz[];   // kBinThreads * (K+1) * 3
    __shared__ uint32_t s_off[kBinThreads + 1];
    __shared__ uint32_t s_rect[kBinThreads][2];   // (tx0 | ty0 << 16), (w | h << 16)
    __shared__ uint32_t s_q[kBinThreads];
    __shared__ uint32_t s_warp[kBinThreads / 32];
    __shared__ unsigned long long s_excl;
    __shared__ unsigned s_culled;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int KV = K + 1;
    if (tid == 0) s_culled = 0;
    __syncthreads();
    const int64_t vid = blockIdx.x;
    const int view = (int)(vid / a.fan_blocks);
    const int64_t f0 = (vid - (int64_t)view * a.fan_blocks) * kBinThreads;
    const int nloc = (int)min64(kBinThreads, n_fans - f0);
    const CamDev &cam = a.vt.v[view].cam;
    const unsigned tiles_x = a.vt.v[view].tiles_x, tile_base = a.vt.v[view].tile_base;
    const DepthQ dq = depth_quant(a.zrange, view, depth_bits);

    // Coalesced staging of the block's vertices.
    {
        const float *src = xyz + f0 * KV * 3;
        const int n = nloc * KV * 3;
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (n & 3) == 0) {
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
            float4 *d4 = reinterpret_cast<float4 *>(s_xyz);
            for (int i = tid; i < n / 4; i += kBinThreads) d4[i] = __ldg(s4 + i);
        } else {
            for (int i = tid; i < n; i += kBinThreads) s_xyz[i] = __ldg(src + i);
        }
    }
    __syncthreads();

    uint32_t count = 0;
    if (tid < nloc) {
        const float *p = s_xyz + tid * KV * 3;
        const uint32_t all = (2u << K) - 1u;   // K+1 vertex bits
        uint32_t vmask = 0;
        float mnx = 3.0e38f, mxx = -3.0e38f, mny = 3.0e38f, mxy = -3.0e38f, zmin = 3.0e38f;
        float4 *dec = a.dec + (size_t)view * a.V + (size_t)(f0 + tid) * KV;
        // the fan's integer origin: the floor of its centre's exact screen position
        const DfVert c0 = df_project(cam, p[0], p[1], p[2]);
        const float ox = df_floor(c0.x), oy = df_floor(c0.y);
        for (int k = 0; k < KV; ++k) {
            const DVert d = decide_vertex(cam, k == 0 ? c0 : df_project(cam, p[3 * k], p[3 * k + 1], p[3 * k + 2]),
                                          ox, oy);
            // (xr, yr, Z or -1 if invalid, the origin's x / y in the first two vertices)
            dec[k] = make_float4(d.xr, d.yr, d.valid ? d.Z : -1.0f, k == 0 ? ox : (k == 1 ? oy : 0.0f));
            if (d.valid) vmask |= 1u << k;
            mnx = fminf(mnx, d.xs); mxx = fmaxf(mxx, d.xs);
            mny = fminf(mny, d.ys); mxy = fmaxf(mxy, d.ys);
            zmin = fminf(zmin, d.Z);
        }
        uint32_t tmask = tri_valid_mask(vmask, K);
        const uint32_t full = (1u << K) - 1u;
        const uint32_t drawn = a.face_mask ? (__ldg(a.face_mask + f0 + tid) & full) : full;
        const unsigned ntri_bad = K - __popc(tmask);   // culled: an invalid vertex
        tmask &= drawn;
        if ((vmask != all || drawn != full) && tmask) {   // bounds over the vertices of drawn triangles only
            mnx = 3.0e38f; mxx = -3.0e38f; mny = 3.0e38f; mxy = -3.0e38f; zmin = 3.0e38f;
            for (int k = 0; k < KV; ++k) {
                if (!vertex_used(tmask, k, K)) continue;
                const DVert d = decide_vertex(cam, df_project(cam, p[3 * k], p[3 * k + 1], p[3 * k + 2]), ox, oy);
                mnx = fminf(mnx, d.xs); mxx = fmaxf(mxx, d.xs);
                mny = fminf(mny, d.ys); mxy = fmaxf(mxy, d.ys);
                zmin = fminf(zmin, d.Z);
            }
        }
        if (ntri_bad) atomicAdd(&s_culled, ntri_bad);
        if (tmask) {
            const FanRect r = rect_from_bounds(mnx, mxx, mny, mxy, cam.width, cam.height);
            if (!r.empty) {
                const int tx0 = r.i0 >> tile_shift, tx1 = r.i1 >> tile_shift;
                const int ty0 = r.j0 >> tile_shift, ty1 = r.j1 >> tile_shift;
                const int w = tx1 - tx0 + 1, h = ty1 - ty0 + 1;
                count = (uint32_t)(w * h);
                s_rect[tid][0] = (uint32_t)tx0 | ((uint32_t)ty0 << 16);
                s_rect[tid][1] = (uint32_t)w | ((uint32_t)h << 16);
                // a lower bound of every fragment depth of the fan: the smallest rounded
                // vertex depth, lowered by 2^-20 to cover its rounding
                s_q[tid] = depth_qv(dq, zmin * (a.key_scale * kKeyMargin));
            }
        }
    }
    // Block-wide exclusive scan of the counts (fan order).
    uint32_t x = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < kBinThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kBinThreads / 32) s_warp[lane] = t;
    }
    __syncthreads();
    const uint32_t incl = x + (warp > 0 ? s_warp[warp - 1] : 0);
    s_off[tid + 1] = incl;
    if (tid == 0) s_off[0] = 0;
    const uint32_t total = s_warp[kBinThreads / 32 - 1];

    // The block's range of the pair array: one atomic reservation.  Pairs of different
    // blocks land in an arbitrary order; the sort orders them by key, and fans with equal
    // keys may then meet a pixel in any order, which the exact-order resolve absorbs.
    if (tid == 0) {
        s_excl = total ? atomicAdd(&st->pairs, (unsigned long long)total) : 0ull;
        if (vid == 0) {
            st->cap = (unsigned long long)cap;
            st->n_tiles = a.n_tiles;
            st->sort_bits = a.sort_bits;
        }
        if (s_culled) atomicAdd(&st->culled, (unsigned long long)s_culled);
    }
    __syncthreads();

    // Output-major emission: consecutive threads write consecutive pairs.
    const unsigned long long base = s_excl;
    const unsigned long long tmask = ~0ull;
    for (uint32_t o = tid; o < total; o += kBinThreads) {
        const unsigned long long idx = base + o;
        if (idx >= (unsigned long long)cap) break;
        int lo = 0, hi = nloc;   // largest f with s_off[f] <= o
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= o) lo = mid; else hi = mid;
        }
        const uint32_t k = o - s_off[lo];
        const uint32_t r0 = s_rect[lo][0], r1 = s_rect[lo][1];
        const uint32_t w = r1 & 0xFFFFu;
        const uint32_t tx = (r0 & 0xFFFFu) + k % w, ty = (r0 >> 16) + k / w;
        const unsigned long long tile = tile_base + (unsigned long long)ty * tiles_x + tx;
        keys[idx] = ((((tile << depth_bits) | s_q[lo]) << fan_bits) | (unsigned long long)(f0 + lo)) & tmask;
    }
}

}  // namespace

cudaError_t launch_bin(const RenderArgs &ra, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    if (ra.n_fans == 0) return cudaSuccess;
    const size_t smem = sizeof(float) * kBinThreads * (ra.K + 1) * 3;
    cudaFuncSetAttribute(bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    BinArgs a;
    a.xyz = ra.xyz;
    a.n_fans = ra.n_fans;
    a.K = ra.K;
    a.tile_shift = 0;
    while ((1 << a.tile_shift) < L.tile) ++a.tile_shift;
    a.depth_bits = L.depth_bits;
    a.fan_bits = L.fan_bits;
    a.key_scale = ra.key_scale;
    a.cap = L.cap;
    a.fan_blocks = L.bin_fan_blocks;
    a.n_tiles = (unsigned)L.n_tiles;
    a.sort_bits = (unsigned)(8 * L.passes);
    a.st = reinterpret_cast<Status *>(ra.ws + L.off_status);
    a.keys = reinterpret_cast<unsigned long long *>(ra.ws + L.off_keys0);
    a.vt = ra.vt;
    a.dec = reinterpret_cast<float4 *>(ra.ws + L.off_dec);
    a.V = L.V;
    a.face_mask = ra.splat ? nullptr : ra.prm.face_mask;
    a.zrange = reinterpret_cast<const uint32_t *>(ra.ws + L.off_zrange);   // zeroed with the workspace prefix
    {
        // about one centre per thread: the sweep is latency-bound, not bandwidth-bound
        const int64_t samples = (ra.n_fans + kRangeStride - 1) / kRangeStride;
        const int grid = (int)min64((samples + kRangeThreads - 1) / kRangeThreads, 16 * 152);
        for (int v0 = 0; v0 < L.n_views; v0 += kRangeViews)
            depth_range_kernel<<<grid, kRangeThreads, 0, st>>>(ra.xyz, ra.n_fans, ra.K, ra.vt, v0,
                                                               min(kRangeViews, L.n_views - v0),
                                                               reinterpret_cast<uint32_t *>(ra.ws + L.off_zrange));
        count_launches((L.n_views + kRangeViews - 1) / kRangeViews);
    }
    bin_kernel<<<(unsigned)L.bin_blocks, kBinThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ms
