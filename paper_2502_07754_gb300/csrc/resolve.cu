// Per-pixel resolve of the fragment buffer: exact depth order and front-to-back
// compositing (forward), and its adjoint (backward).
//
// One thread per pixel.  A pixel's fragment records sit contiguously in tile-list
// order, i.e. sorted by their fans' depth bounds.  The thread streams them through a
// small sorted register buffer: the front fragment is composited ("committed") once
// the next record's depth bound exceeds it -- every later fragment lies at least that
// deep, so the order is exact.  If the buffer overflows, the thread remembers the
// nearest dropped fragment and the earliest record it dropped, finishes the pass with
// everything strictly nearer, and re-reads its own records from that point, skipping
// fragments at or before the last committed one.  Order: (depth, triangle id), the depth
// a double-float value (high part in the record's first word, low part in its fourth).
// Compositing stops once the transmittance falls below T_eps.
//
// Both passes visit the pixels in orders that pixel_order_kernel builds after the pixel
// scan (by fragment count), so a warp's lanes run loops of about the same length instead
// of all waiting for the deepest pixel among 32 neighbours.
//
// The forward also records, per pixel, the record index of each committed fragment in
// commit order.  The backward walks that list (no pending buffer, no re-reads), and at
// each committed fragment f forms, from the recomputed transmittance T_f,
// dC/dc_f = T_f a_f, dC/da_f = T_f c_f - (C_out - C_{<=f}) / (1 - a_f) and
// dA/da_f = T_out / (1 - a_f).  It writes dL/dc_f and dL/da_f, with the fragment's
// triangle and pixel, as an adjoint record (the pixel's c-th composited fragment in slot
// c of its record range); the chain pass (chain.cu) takes them to the vertices record by
// record, so this pass does no atomics.
#include "raster_common.cuh"

namespace ms {

namespace {

// Pixels differ widely in their fragment counts: small blocks let an SM refill the slots
// of warps that finished early instead of holding them until the block's slowest warp.
constexpr int kResolveThreads = 64;

struct ResolveArgs {
    int K;
    int64_t npx;
    const uint32_t *counts, *offsets;
    float4 *frags;
    int64_t frag_cap;
    int depth_bits;
    float T_eps, bg0, bg1, bg2;
    Status *st;
    float *tfinal;
    uint32_t *ncommit;
    float4 *adj;               // backward: per composited fragment, in commit order within the
                               // pixel's record range: (dL/dc * T a, dL/da), (triangle, pixel, 0, 0)
    uint32_t *corder;          // per pixel: record indices in commit order (same offsets as records)
    const uint32_t *perm;      // visiting order of the pixels
    const uint32_t *zrange;    // per view depth range of the keys' quantisation (bin.cu)
    ViewTable vt;
};

// Resolve orders, built after the pixel scan.  Forward: all pixels in descending order of
// their fragment counts (a counting sort over the histogram the tile prefix gathered), so
// the 32 lanes of a warp walk lists of about the same length and the deepest pixels
// start first instead of trailing at the end of the grid.  Backward: the same sort within
// spans of kOrderSpan consecutive pixels only: that pass does little arithmetic per
// record and is bound by memory latency, and the pixels of one span (part of a row) have
// their records in the regions of the row's tiles (records are laid out tile by tile).
// The order within one count varies from run to run; no pixel's result depends on it.
constexpr int kOrderThreads = 256, kOrderItems = 4, kOrderSpan = kOrderThreads * kOrderItems;

// Exclusive prefix of v over the buckets in descending order (thread t holds bucket 255 - t).
__device__ __forceinline__ uint32_t desc_prefix(uint32_t v, uint32_t *s_warp) {
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
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    return before + x - v;
}

__global__ void __launch_bounds__(kOrderThreads) pixel_order_kernel(const uint32_t *__restrict__ counts, int64_t npx,
                                                                    const uint32_t *__restrict__ hist,
                                                                    uint32_t *__restrict__ fill,
                                                                    uint32_t *__restrict__ perm_fwd,
                                                                    uint32_t *__restrict__ perm_bwd) {
    __shared__ uint32_t s_cnt[kCountBuckets], s_span[kCountBuckets], s_glob[kCountBuckets], s_warp[kOrderThreads / 32];
    static_assert(kOrderThreads == kCountBuckets, "one thread per bucket");
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kOrderSpan;
    const int mb = kCountBuckets - 1 - tid;   // this thread's bucket in the scans
    s_cnt[tid] = 0;
    const uint32_t g0 = desc_prefix(hist[mb], s_warp);   // (its barriers also order the clear)
    int bk[kOrderItems];
    uint32_t rk[kOrderItems];
#pragma unroll
    for (int i = 0; i < kOrderItems; ++i) {
        const int64_t p = base + i * kOrderThreads + tid;
        bk[i] = -1;
        rk[i] = 0;
        if (p < npx) {
            bk[i] = count_bucket(counts[p]);
            rk[i] = atomicAdd(&s_cnt[bk[i]], 1u);
        }
    }
    __syncthreads();
    const uint32_t h = s_cnt[mb];
    s_span[mb] = desc_prefix(h, s_warp);
    s_glob[mb] = h ? g0 + atomicAdd(&fill[mb], h) : 0u;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kOrderItems; ++i)
        if (bk[i] >= 0) {
            const uint32_t p = (uint32_t)(base + i * kOrderThreads + tid);
            // both positions are < npx: the span and the histogram count each pixel once
            const int64_t ps = base + s_span[bk[i]] + rk[i];
            const int64_t pg = (int64_t)s_glob[bk[i]] + rk[i];
            if (ps < npx) perm_bwd[ps] = p;
            if (pg < npx) perm_fwd[pg] = p;
        }
}

// (depth, triangle) order of two fragments; depths are normalised double-float values,
// so comparing (high, low) lexicographically compares their values.
__device__ __forceinline__ bool frag_less(float za, float la, uint32_t ta, float zb, float lb, uint32_t tb) {
    return za < zb || (za == zb && (la < lb || (la == lb && ta < tb)));
}

template <int KB>
__global__ void __launch_bounds__(kResolveThreads) resolve_kernel(const __grid_constant__ ResolveArgs a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t pt = t < a.npx ? (int64_t)a.perm[t] : a.npx;
    const bool valid = pt < a.npx;
    const int64_t pix = valid ? pt : 0;
    const int view = view_of_pixel(a.vt, (unsigned long long)pix);
    const ViewDev &vw = a.vt.v[view];
    const int64_t lpix = pix - (int64_t)vw.pix_base;   // index within the view's image
    int n = valid ? (int)a.counts[pix] : 0;
    const int64_t off = a.offsets[pix];
    if (off + n > a.frag_cap) n = 0;   // the buffer overflowed: reported through the status block
    const DepthQ dq = depth_quant(a.zrange, view, a.depth_bits);
    constexpr int RS = kRecFwd;   // float4s per record
    float4 *rec = a.frags + (size_t)RS * off;

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    float kz[KB], kl[KB];      // pending fragments sorted by (depth, triangle): depth high, low
    uint32_t kt[KB], ki[KB];   // triangle id, record index
    float4 kc[KB];             // colour and opacity, read with the depth (one sector per record)
    int nb = 0;
    float fz = 0.0f, fl = 0.0f;   // last committed (depth, triangle); depths are > 0
    uint32_t ft = 0;
    bool has_front = false;
    float dz = 0.0f, dl = 0.0f;   // nearest dropped fragment of this pass
    uint32_t dt = 0;
    bool dropped = false;
    int restart = 0x7fffffff;
    bool done = !valid;
    uint32_t ncom = 0;

    auto commit_front = [&]() {
        // colour and opacity travel in the pending buffer: a commit waits on no load
        const float4 col = kc[0];
        const float al = col.w;
        const float c0 = col.x, c1 = col.y, c2 = col.z;
        const float w = T * al;
        C0 += w * c0;
        C1 += w * c1;
        C2 += w * c2;
        T *= (1.0f - al);
        a.corder[off + ncom] = ki[0];
        ++ncom;
        fz = kz[0];
        fl = kl[0];
        ft = kt[0];
        has_front = true;
#pragma unroll
        for (int i = 0; i + 1 < KB; ++i) {
            kz[i] = kz[i + 1]; kl[i] = kl[i + 1]; kt[i] = kt[i + 1]; ki[i] = ki[i + 1]; kc[i] = kc[i + 1];
        }
        --nb;
        if (T < a.T_eps) {
            done = true;
            nb = 0;
        }
    };

    int start = 0;
    while (!done) {
        for (int i = start; i < n && !done; ++i) {
            const float4 r0 = rec[RS * i];
            const float4 r1 = rec[RS * i + 1];
            const float z = r0.x, zl = r0.w;
            const uint32_t tri = __float_as_uint(r0.y), qk = __float_as_uint(r0.z);
            while (nb > 0 && !done && depth_qv(dq, kz[0]) < qk) commit_front();
            if (done) break;
            if (has_front && !frag_less(fz, fl, ft, z, zl, tri)) continue;   // committed in an earlier pass
            if (dropped && !frag_less(z, zl, tri, dz, dl, dt)) {
                restart = min(restart, i);
                continue;
            }
            if (nb == KB) {
                if (frag_less(z, zl, tri, kz[KB - 1], kl[KB - 1], kt[KB - 1])) {
                    dz = kz[KB - 1];   // evict the deepest pending fragment
                    dl = kl[KB - 1];
                    dt = kt[KB - 1];
                    dropped = true;
                    restart = min(restart, (int)ki[KB - 1]);
                    --nb;
                } else {
                    if (!dropped || frag_less(z, zl, tri, dz, dl, dt)) {
                        dz = z;
                        dl = zl;
                        dt = tri;
                    }
                    dropped = true;
                    restart = min(restart, i);
                    continue;
                }
            }
            bool placed = false;
#pragma unroll
            for (int s = KB - 1; s >= 1; --s) {
                if (s <= nb && !placed) {
                    if (frag_less(z, zl, tri, kz[s - 1], kl[s - 1], kt[s - 1])) {
                        kz[s] = kz[s - 1]; kl[s] = kl[s - 1]; kt[s] = kt[s - 1]; ki[s] = ki[s - 1];
                        kc[s] = kc[s - 1];
                    } else {
                        kz[s] = z; kl[s] = zl; kt[s] = tri; ki[s] = (uint32_t)i; kc[s] = r1;
                        placed = true;
                    }
                }
            }
            if (!placed) {
                kz[0] = z; kl[0] = zl; kt[0] = tri; ki[0] = (uint32_t)i; kc[0] = r1;
            }
            ++nb;
        }
        // End of pass: everything pending is nearer than anything dropped.
        while (nb > 0 && !done) commit_front();
        if (!dropped || done) break;
        atomicAdd(&a.st->extra_passes, 1ull);
        start = restart;
        dropped = false;
        restart = 0x7fffffff;
    }
    {
        if (valid) {
            reinterpret_cast<float4 *>(vw.out)[lpix] =
                make_float4(C0 + T * a.bg0, C1 + T * a.bg1, C2 + T * a.bg2, 1.0f - T);
            a.tfinal[pix] = T;
            a.ncommit[pix] = ncom;
        }
        const unsigned r = __reduce_add_sync(0xffffffffu, ncom);
        if ((threadIdx.x & 31) == 0) atomicAdd(&a.st->commits, (unsigned long long)r);
    }
}

// Backward: replay the forward's committed fragments in their recorded order.
__global__ void __launch_bounds__(kResolveThreads) resolve_bwd_kernel(const __grid_constant__ ResolveArgs a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.npx) return;
    const int64_t pix = a.perm[t];
    if (pix >= a.npx) return;
    const ViewDev &vw = a.vt.v[view_of_pixel(a.vt, (unsigned long long)pix)];
    const int64_t lpix = pix - (int64_t)vw.pix_base;
    const uint32_t n = a.ncommit[pix];
    const int64_t off = a.offsets[pix];
    const uint32_t nrec = a.counts[pix];
    if (n < nrec && off + nrec <= a.frag_cap) {
        // slots past the composited fragments carry a zero gradient (the chain pass reads
        // every slot of the pixel's range)
        for (uint32_t i = n; i < nrec; ++i) {
            a.adj[2 * (off + i)] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            a.adj[2 * (off + i) + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    if (n == 0) return;
    const float4 *rec = a.frags + (size_t)kRecFwd * off;
    const uint32_t *ord = a.corder + off;
    const float4 g = reinterpret_cast<const float4 *>(vw.dL)[lpix];
    const float4 ov = reinterpret_cast<const float4 *>(vw.out_fwd)[lpix];
    const float Tout = a.tfinal[pix];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t idx = ord[0];
    for (uint32_t c = 0; c < n; ++c) {
        const uint32_t nidx = c + 1 < n ? ord[c + 1] : 0u;   // the next index loads early
        const float4 *rc = rec + (size_t)kRecFwd * idx;
        const float4 r0 = rc[0];
        const float4 col = rc[1];
        const float al = col.w;
        const float w = T * al;
        const float nC0 = C0 + w * col.x, nC1 = C1 + w * col.y, nC2 = C2 + w * col.z;
        const float inv = 1.0f / fmaxf(1.0f - al, 1e-6f);
        const float ga = g.x * (T * col.x - (ov.x - nC0) * inv) + g.y * (T * col.y - (ov.y - nC1) * inv) +
                         g.z * (T * col.z - (ov.z - nC2) * inv) + g.w * Tout * inv;
        a.adj[2 * (off + c)] = make_float4(g.x * w, g.y * w, g.z * w, ga);
        a.adj[2 * (off + c) + 1] = make_float4(r0.y, __uint_as_float((uint32_t)pix), 0.0f, 0.0f);
        C0 = nC0; C1 = nC1; C2 = nC2;
        T *= (1.0f - al);
        idx = nidx;
    }
}

cudaError_t launch_k(const ResolveArgs &ra, bool backward, int kbuf, int64_t npx, cudaStream_t st) {
    const unsigned grid = (unsigned)((npx + kResolveThreads - 1) / kResolveThreads);
    if (npx == 0) return cudaSuccess;
    if (backward)
        resolve_bwd_kernel<<<grid, kResolveThreads, 0, st>>>(ra);
    else if (kbuf == 16)
        resolve_kernel<16><<<grid, kResolveThreads, 0, st>>>(ra);
    else
        resolve_kernel<8><<<grid, kResolveThreads, 0, st>>>(ra);
    return cudaGetLastError();
}

__global__ void grad_scatter_kernel(const float4 *__restrict__ g, int64_t V, float *__restrict__ dx,
                                    float *__restrict__ dc, float *__restrict__ da) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = g[2 * v], b = g[2 * v + 1];
        dx[3 * v] += a.x;
        dx[3 * v + 1] += a.y;
        dx[3 * v + 2] += a.z;
        da[v] += a.w;
        dc[3 * v] += b.x;
        dc[3 * v + 1] += b.y;
        dc[3 * v + 2] += b.z;
    }
}

}  // namespace

cudaError_t launch_resolve(const RenderArgs &ra, bool backward, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    ResolveArgs a;
    a.K = ra.K;
    a.npx = L.npx;
    a.counts = reinterpret_cast<const uint32_t *>(ra.ws + L.off_counts);
    a.offsets = reinterpret_cast<const uint32_t *>(ra.ws + L.off_offsets);
    a.frags = reinterpret_cast<float4 *>(ra.ws + L.off_frags);
    a.frag_cap = L.frag_cap;
    a.depth_bits = L.depth_bits;
    a.zrange = reinterpret_cast<const uint32_t *>(ra.ws + L.off_zrange);
    a.T_eps = ra.prm.T_eps;
    a.bg0 = ra.prm.bg[0];
    a.bg1 = ra.prm.bg[1];
    a.bg2 = ra.prm.bg[2];
    a.st = reinterpret_cast<Status *>(ra.ws + L.off_status);
    a.tfinal = reinterpret_cast<float *>(ra.ws + L.off_tfinal);
    a.ncommit = reinterpret_cast<uint32_t *>(ra.ws + L.off_ncommit);
    a.adj = reinterpret_cast<float4 *>(ra.ws + L.off_adj);
    a.corder = reinterpret_cast<uint32_t *>(ra.ws + L.off_corder);
    a.perm = reinterpret_cast<const uint32_t *>(ra.ws + L.off_perm) + (backward ? L.npx : 0);
    a.vt = ra.vt;
    return launch_k(a, backward, L.kbuf, L.npx, st);
}

cudaError_t launch_pixel_order(const RenderArgs &ra, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    if (L.npx == 0) return cudaSuccess;
    const uint32_t *hist = reinterpret_cast<const uint32_t *>(ra.ws + L.off_pbucket);
    uint32_t *fill = reinterpret_cast<uint32_t *>(ra.ws + L.off_pbucket) + kCountBuckets;
    uint32_t *perm = reinterpret_cast<uint32_t *>(ra.ws + L.off_perm);
    pixel_order_kernel<<<(unsigned)((L.npx + kOrderSpan - 1) / kOrderSpan), kOrderThreads, 0, st>>>(
        reinterpret_cast<const uint32_t *>(ra.ws + L.off_counts), L.npx, hist, fill, perm, perm + L.npx);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_grad_scatter(const RenderArgs &ra, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    if (L.V == 0) return cudaSuccess;
    const int grid = (int)min64((L.V + 255) / 256, 16 * 152);
    grad_scatter_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(ra.ws + L.off_grad), L.V, ra.d_xyz,
                                              ra.d_rgb, ra.d_alpha);
    return cudaGetLastError();
}

}  // namespace ms
