// Tile rasterisation into a per-pixel fragment buffer (A-buffer) in HBM.
//
// Every tile's fan list (sorted by the fans' depth bounds) is cut into work items of
// at most kItemFans fans; one warp rasterises one item, so a hot tile with thousands
// of fans spreads over many warps instead of serialising on one.  A warp projects
// a chunk of the item's fans into its own shared-memory stage (32 / chunk lanes per fan,
// sharing its vertices and triangles), then walks them in list order: for each fan its lanes enumerate exactly the pixels
// of the fan's pixel rectangle inside the tile and test the fan's K triangles at each
// with the binary32 decision formulas.  No block barriers are used.
//
// Count pass: per (item, pixel) fragment counts, the coverage mask of every (fan, pixel)
// test, and per pair its first mask index and its pixel rectangle within the tile (zero
// when the pair covers no pixel centre, so the fill skips it).  A
// per-tile prefix over the tile's items turns the counts into each item's starting slot
// within the pixel and gives the pixel totals; an exclusive scan over pixels gives record
// offsets.  Fill pass: the same walk, reading the stored masks and rectangles instead of
// staging the decisions and testing again, writes one 32-byte record per fragment at offset + item slot + running
// index -- depth (high), triangle id, the fan's depth bound, depth (low), colour, opacity -- so a
// pixel's records come out in tile-list order, which the resolve relies on.
#include "raster_common.cuh"

namespace ms {

namespace {

struct RastArgs {
    const float *xyz, *rgb, *alpha;
    int K, depth_bits, fan_bits;
    ViewTable vt;
    const unsigned long long *keys;   // sorted elements tile | depth bound | fan id
    const uint4 *items;        // (tile, start, end, index within tile)
    uint32_t *icnt;            // [item][tile pixels]: counts, then in-pixel starting slots
    const uint32_t *offsets;
    const uint32_t *counts;
    float4 *frags;
    int64_t frag_cap;
    Status *st;
    SplatSrc spl;              // source Gaussians (splat passes only)
    const float4 *dec;         // [view][vertex] decided vertices from binning
    int64_t V;
    const uint32_t *face_mask; // per fan, bit j = face j drawn; NULL = all
    uint2 *pinfo;              // per pair: index of its first coverage mask (~0 if none stored), and its
                               // pixel rectangle clipped to the tile (pair_geo; 0 if empty)
    uint16_t *masks;           // coverage masks (bit j: triangle j) of the count pass's tests
    int64_t mask_cap;
    uint32_t *mask_cursor;     // [kMaskRegions] fill levels of the mask regions (zeroed per render)
};

constexpr int kRastWarps = 2;   // warps (work items) per block: items differ widely in cost

// A pair's pixel rectangle clipped to its tile, relative to the tile's corner: x0 | y0 << 6 |
// (w - 1) << 12 | (h - 1) << 18, bit 31 set; 0 for a pair with no pixel to test.
__device__ __forceinline__ uint32_t pair_geo(int rx0, int ry0, int w, int h) {
    return 0x80000000u | (uint32_t)rx0 | (uint32_t)ry0 << 6 | (uint32_t)(w - 1) << 12 | (uint32_t)(h - 1) << 18;
}

// Pass kinds: count fragments; fill their 32-byte forward records.  The splat passes draw
// the source Gaussians themselves (count, then 32-byte records) over the tile lists of
// their circumscribing polygons.
enum RasterMode { kCount = 0, kFill = 1, kSplatCount = 3, kSplatFill = 4 };

__host__ __device__ constexpr bool mode_fills(int m) { return m == kFill || m == kSplatFill; }
__host__ __device__ constexpr bool mode_splat(int m) { return m >= kSplatCount; }
__host__ __device__ constexpr int mode_level(int m) { return mode_splat(m) ? (int)kStageDecide : m; }

template <int TILE, int STG, int MODE>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int K) {
    return (size_t)(TILE * TILE * (mode_fills(MODE) ? 2 : 1) + 32) * 4 + stage_bytes(STG, K, mode_level(MODE)) +
           (mode_splat(MODE) ? (size_t)STG * sizeof(SplatSlot) : 0);
}

template <int TILE, int STG, int KT, int MODE>
__global__ void __launch_bounds__(kRastWarps * 32) raster_kernel(const __grid_constant__ RastArgs a) {
    constexpr bool FILL = mode_fills(MODE);   // passes that address records
    constexpr bool SPLAT = mode_splat(MODE);
    constexpr int LEVEL = mode_level(MODE);
    extern __shared__ __align__(16) char smem[];
    const int K = KT > 0 ? KT : a.K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t item = blockIdx.x * kRastWarps + warp;
    if (item >= a.st->n_items) return;   // whole warp; nothing below synchronises the block
    const uint4 it = a.items[item];
    const int view = view_of_tile(a.vt, it.x);
    const ViewDev &vw = a.vt.v[view];
    SceneDev sc;
    sc.xyz = a.xyz;
    sc.rgb = a.rgb;
    sc.alpha = a.alpha;
    sc.K = K;
    sc.cam = &vw.cam;
    sc.W = vw.cam.width;
    sc.H = vw.cam.height;
    sc.dec = a.dec + (size_t)view * (size_t)a.V;
    sc.face_mask = SPLAT ? nullptr : a.face_mask;
    const int tile = (int)(it.x - vw.tile_base);
    const int tiles_x = (int)vw.tiles_x;
    const unsigned long long pix_base = vw.pix_base;
    char *mine = smem + (size_t)warp * warp_smem_bytes<TILE, STG, MODE>(K);
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(mine);   // [TILE*TILE] fragments so far
    uint32_t *s_base = s_cnt + TILE * TILE;                   // [TILE*TILE] record offsets (fill)
    uint32_t *s_nf = s_cnt + TILE * TILE * (FILL ? 2 : 1);    // [32] fragments per lane of a batch
    char *stage_base = mine + (size_t)(TILE * TILE * (FILL ? 2 : 1) + 32) * 4;
    const Stage S = stage_ptrs(stage_base, STG, K, LEVEL);
    SplatSlot *s_spl = reinterpret_cast<SplatSlot *>(stage_base + stage_bytes(STG, K, LEVEL));
    const int tx0 = (tile % tiles_x) * TILE, ty0 = (tile / tiles_x) * TILE;
    const int tx1 = min(tx0 + TILE, sc.W) - 1, ty1 = min(ty0 + TILE, sc.H) - 1;
    uint32_t *icnt = a.icnt + (size_t)item * TILE * TILE;
    for (int i = lane; i < TILE * TILE; i += 32) {
        s_cnt[i] = 0;
        if (FILL) {
            const int x = tx0 + (i % TILE), y = ty0 + (i / TILE);
            uint32_t b = 0xffffffffu;
            if (x <= tx1 && y <= ty1) {
                const size_t pix = pix_base + (size_t)y * sc.W + x;
                const int64_t o = a.offsets[pix];
                // a pixel whose records would not fit gets none (the overflow is reported)
                if (o + a.counts[pix] <= a.frag_cap) b = (uint32_t)o + icnt[i];
            }
            s_base[i] = b;
        }
    }
    uint32_t c_rect = 0, c_frag = 0;
    __syncwarp();
    for (uint32_t cb = it.y; cb < it.z; cb += STG) {
        const int cnt = (int)min((uint32_t)STG, it.z - cb);
        // The fill pass takes a chunk whose pairs all have their masks stored without the
        // decision stage: the count pass left each pair's rectangle beside its mask index.
        uint2 pinf = make_uint2(~0u, 0u);
        if (MODE == kFill && lane < cnt) pinf = __ldg(a.pinfo + cb + lane);
        const bool stored = MODE == kFill && __all_sync(0xffffffffu, lane >= cnt || pinf.x != ~0u);
        {
            constexpr int LPF = 32 / STG;   // lanes staging one fan
            const int slot = lane / LPF;
            uint32_t q = 0, fan = 0;
            if (slot < cnt) {
                const uint32_t li = cb + slot;
                const unsigned long long e = __ldg(a.keys + li);
                q = (uint32_t)((e >> a.fan_bits) & ((1ull << a.depth_bits) - 1ull));
                fan = (uint32_t)(e & ((1ull << a.fan_bits) - 1ull));
            }
            // a stored chunk skips the values of pairs that the count pass found without any
            // covered pixel centre (their rectangle word is 0)
            const uint32_t sgeo = __shfl_sync(0xffffffffu, pinf.y, slot);
            stage_fans<LPF>(sc, S, K, lane, slot < cnt && (!stored || sgeo != 0u), fan, q, LEVEL, !stored);
            if (SPLAT && lane < cnt)
                s_spl[lane] = splat_setup(a.spl, *sc.cam,
                                          (uint32_t)(__ldg(a.keys + cb + lane) & ((1ull << a.fan_bits) - 1ull)));
        }
        __syncwarp();
        // The staged fans' rectangles (clipped to the tile) form one packed (fan, pixel)
        // index space, fan-major, so every lane tests a pixel even when fans are tiny.
        int my_n = 0;
        uint32_t my_geo = 0;
        if (stored) {
            my_geo = pinf.y;
        } else if (lane < cnt) {
            const int4 r = S.rect[lane];
            const int rx0 = max(r.x, tx0), rx1 = min(r.y, tx1), ry0 = max(r.z, ty0), ry1 = min(r.w, ty1);
            if (S.flags[lane] != 0 && rx0 <= rx1 && ry0 <= ry1)
                my_geo = pair_geo(rx0 - tx0, ry0 - ty0, rx1 - rx0 + 1, ry1 - ry0 + 1);
        }
        if (my_geo) my_n = (int)((((my_geo >> 12) & 63u) + 1u) * (((my_geo >> 18) & 63u) + 1u));
        int incl = my_n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - my_n;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        // The count pass stores the coverage mask of every test of the chunk (one range per
        // chunk, reserved with one atomic) and each pair's first index; the fill pass reads
        // them instead of testing again.  Both walk a fan's rectangle in the same order.
        uint32_t mbase = ~0u, my_moff = ~0u;
        if (MODE == kCount) {
            // kMaskRegions cursors, the item picking one by its index, so that the reservations
            // of millions of chunks do not queue on one address
            if (lane == 0 && total > 0) {
                const uint32_t reg = item % kMaskRegions;
                const uint32_t rsz = (uint32_t)(a.mask_cap / kMaskRegions);
                const uint32_t b = atomicAdd(a.mask_cursor + reg, (uint32_t)total);
                if ((uint64_t)b + (uint64_t)total <= (uint64_t)rsz) mbase = reg * rsz + b;
            }
            mbase = __shfl_sync(0xffffffffu, mbase, 0);
        }
        if (MODE == kFill) my_moff = pinf.x;
        uint32_t fan_hit = 0;   // count pass: bit f set when staged fan f covers some pixel centre
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            int f = 0;   // first lane (fan) whose inclusive count exceeds idx
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, f + step - 1);
                if (v <= idx) f += step;
            }
            const int fexcl = __shfl_sync(0xffffffffu, excl, f);
            const uint32_t fmoff = __shfl_sync(0xffffffffu, my_moff, f);
            const uint32_t fgeo = __shfl_sync(0xffffffffu, my_geo, f);
            uint32_t hits = 0, flags = 0;
            int lp = -1, px = 0, py = 0;
            float sp_t = 0.0f, sp_a = 0.0f;
            if (idx < total) {
                ++c_rect;
                const int rx0 = tx0 + (int)(fgeo & 63u), ry0 = ty0 + (int)((fgeo >> 6) & 63u);
                const int w = (int)((fgeo >> 12) & 63u) + 1, local = idx - fexcl;
                // (local + 0.5) / w is at least 1/(2w) away from an integer: exact row
                const int yy = (int)(((float)local + 0.5f) * (1.0f / (float)w));
                px = rx0 + (local - yy * w);
                py = ry0 + yy;
                if (SPLAT)
                    hits = splat_hit(s_spl[f], *sc.cam, a.spl.trunc, (double)px + 0.5, (double)py + 0.5, sp_t, sp_a)
                               ? 1u : 0u;
                else if (MODE == kFill && fmoff != ~0u)
                    hits = __ldg(a.masks + fmoff + (uint32_t)local);
                else {   // decisions in the fan's relative frame (the origin is an integer)
                    flags = S.flags[f];
                    hits = cover_mask<KT>(S, STG, K, f, flags, (float)(px - (int)S.ox[f]) + 0.5f,
                                          (float)(py - (int)S.oy[f]) + 0.5f);
                }
                if (MODE == kCount && mbase != ~0u) a.masks[mbase + (uint32_t)idx] = (uint16_t)hits;
                if (hits) lp = (py - ty0) * TILE + (px - tx0);
            }
            if (MODE == kCount) fan_hit |= __reduce_or_sync(0xffffffffu, hits ? 1u << f : 0u);
            const int nf = __popc(hits);
            c_frag += nf;
            if (!FILL) {   // counting: the order of a pixel's slots does not matter yet
                if (nf) atomicAdd(&s_cnt[lp], (uint32_t)nf);
                continue;
            }
            // Lanes that hit the same pixel take consecutive slots in lane order, which is
            // fan order, so a pixel's records keep the depth-key order of the tile list.
            const unsigned grp = __match_any_sync(0xffffffffu, lp);
            if (nf) s_nf[lane] = (uint32_t)nf;
            __syncwarp();
            uint32_t slot = 0;
            if (nf) {
                uint32_t pre = 0;
                for (unsigned lower = grp & ((1u << lane) - 1u); lower; lower &= lower - 1)
                    pre += s_nf[__ffs(lower) - 1];
                slot = s_cnt[lp] + pre;
            }
            __syncwarp();
            if (nf && (grp >> lane) == 1u) s_cnt[lp] = slot + (uint32_t)nf;   // last lane of its group
            if (SPLAT && FILL && nf) {
                const uint32_t b = s_base[lp];
                if (b != 0xffffffffu) {
                    const SplatSlot &sl = s_spl[f];
                    float4 *rec = a.frags + (size_t)kRecFwd * ((size_t)b + slot);
                    rec[0] = make_float4(sp_t, __uint_as_float(S.fan[f]), __uint_as_float(S.q[f]), 0.0f);
                    rec[1] = make_float4(sl.col[0], sl.col[1], sl.col[2], sp_a);
                }
            }
            if (MODE == kFill && nf) {
                const uint32_t b = s_base[lp];
                if (b != 0xffffffffu) {
                    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
                    for (uint32_t hm = hits; hm; hm &= hm - 1, ++slot) {
                        const int j = __ffs(hm) - 1;
                        const int jn = (j + 1 == K) ? 0 : j + 1;
                        const float izc = S.viz[f];
                        const float izj = S.viz[(1 + j) * STG + f], izn = S.viz[(1 + jn) * STG + f];
                        const dfl zf = frag_depth_df(S, STG, K, f, j, pxc, pyc, *sc.cam);
                        // perspective-correct barycentrics from the accurate centre offsets
                        const float ox = __fsub_rn(S.cxh[f], pxc) + S.cxl[f];
                        const float oy = __fsub_rn(S.cyh[f], pyc) + S.cyl[f];
                        const float ujx = ox + S.du[j * STG + f], ujy = oy + S.dv[j * STG + f];
                        const float unx = ox + S.du[jn * STG + f], uny = oy + S.dv[jn * STG + f];
                        const float w0 = (ujx * uny - ujy * unx) * izc;
                        const float w1 = (unx * oy - uny * ox) * izj;
                        const float w2 = (ox * ujy - oy * ujx) * izn;
                        const float Wsum = w0 + w1 + w2;
                        const float iW = 1.0f / Wsum;
                        const float m0 = w0 * iW, m1 = w1 * iW, m2 = w2 * iW;
                        const int vc = f, vj = (1 + j) * STG + f, vn = (1 + jn) * STG + f;
                        const float al = m0 * S.ca[vc] + m1 * S.ca[vj] + m2 * S.ca[vn];
                        const float c0 = m0 * S.cr[vc] + m1 * S.cr[vj] + m2 * S.cr[vn];
                        const float c1 = m0 * S.cg[vc] + m1 * S.cg[vj] + m2 * S.cg[vn];
                        const float c2 = m0 * S.cb[vc] + m1 * S.cb[vj] + m2 * S.cb[vn];
                        const uint32_t tri = S.fan[f] * (uint32_t)K + (uint32_t)j;
                        float4 *rec = a.frags + (size_t)kRecFwd * ((size_t)b + slot);
                        rec[0] = make_float4(zf.h, __uint_as_float(tri), __uint_as_float(S.q[f]), zf.l);
                        rec[1] = make_float4(c0, c1, c2, al);
                    }
                }
            }
            __syncwarp();   // the next batch may append to the same pixels
        }
        // each pair's first mask index, and its rectangle if it covers any pixel centre
        if (MODE == kCount && lane < cnt)
            a.pinfo[cb + lane] = make_uint2(mbase == ~0u ? ~0u : mbase + (uint32_t)excl,
                                            ((fan_hit >> lane) & 1u) ? my_geo : 0u);
        __syncwarp();
    }
    if (!FILL) {
        for (int i = lane; i < TILE * TILE; i += 32) icnt[i] = s_cnt[i];
        const unsigned r0 = __reduce_add_sync(0xffffffffu, c_rect);
        const unsigned r1 = __reduce_add_sync(0xffffffffu, c_frag);
        if (lane == 0) {
            atomicAdd(&a.st->rect_tests, (unsigned long long)r0);
            atomicAdd(&a.st->fragments, (unsigned long long)r1);
        }
    }
}

// Exclusive scan of u32 counts into u32 offsets (decoupled look-back over virtual block
// ids, bounded waits); the grand total goes to *total_out.
//
// With SLOTS the scan runs over the pixels in tile order (slot s = tile * TILE^2 + row *
// TILE + column within the tile; slots outside the image count 0 and get no offset), so the
// fragment records of one screen tile are contiguous: the passes that walk the records in
// order (the adjoint chain) then find the same fans again within a few hundred records,
// and the fill's writes for a tile stay in one region of the buffer.
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPre = 2ull << 62, kValMask = (1ull << 62) - 1;

// Pixel index of slot s (tile-ordered pixels), or -1 for a slot outside its view's image.
__device__ __forceinline__ int64_t slot_pixel(const ViewTable &vt, int tile_shift, int64_t s) {
    const uint32_t t = (uint32_t)(s >> (2 * tile_shift));
    const int local = (int)(s & ((1 << (2 * tile_shift)) - 1));
    const ViewDev &vw = vt.v[view_of_tile(vt, t)];
    const int lt = (int)(t - vw.tile_base), tiles_x = (int)vw.tiles_x;
    const int x = ((lt % tiles_x) << tile_shift) + (local & ((1 << tile_shift) - 1));
    const int y = ((lt / tiles_x) << tile_shift) + (local >> tile_shift);
    if (x >= vw.cam.width || y >= vw.cam.height) return -1;
    return (int64_t)vw.pix_base + (int64_t)y * vw.cam.width + x;
}

template <bool SLOTS>
__global__ void __launch_bounds__(kScanThreads) scan_u32_kernel(const uint32_t *__restrict__ counts,
                                                                uint32_t *__restrict__ offsets, int64_t n,
                                                                int64_t nblocks, unsigned long long *state,
                                                                unsigned *ticket, unsigned long long *total_out,
                                                                Status *st, const __grid_constant__ ViewTable vt,
                                                                int tile_shift) {
    __shared__ int s_vid;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_vid = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t vid = s_vid;
    const int64_t base = vid * kScanTile + (int64_t)tid * kScanItems;
    uint32_t v[kScanItems];
    int64_t pi[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        pi[i] = base + i < n ? (SLOTS ? slot_pixel(vt, tile_shift, base + i) : base + i) : -1;
        v[i] = pi[i] >= 0 ? counts[pi[i]] : 0u;
        sum += v[i];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < kScanThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = t;
    }
    __syncthreads();
    const uint32_t total = s_warp[kScanThreads / 32 - 1];
    const uint32_t mine = x - sum + (warp > 0 ? s_warp[warp - 1] : 0);
    if (tid == 0) {
        unsigned long long excl = 0;
        if (vid == 0) {
            st_release_u64(&state[0], kFlagPre | (unsigned long long)total);
        } else {
            st_release_u64(&state[vid], kFlagAgg | (unsigned long long)total);
            int64_t j = vid - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const unsigned long long s = ld_acquire_u64(&state[j]);
                const unsigned long long flag = s & ~kValMask;
                if (flag == 0) {
                    if (++spins > kSpinLimit) {
                        atomicAdd(&st->timeouts, 1u);
                        break;
                    }
                    continue;
                }
                excl += s & kValMask;
                if (flag == kFlagPre) break;
                --j;
            }
            st_release_u64(&state[vid], kFlagPre | (excl + total));
        }
        s_excl = excl;
        if (vid == nblocks - 1) *total_out = excl + total;
    }
    __syncthreads();
    unsigned long long run = s_excl + mine;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        // offsets beyond 2^32 are clamped; such a buffer overflows its capacity anyway
        if (pi[i] >= 0) offsets[pi[i]] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
        run += v[i];
    }
}

__global__ void tile_item_count_kernel(const uint2 *__restrict__ ranges, int n_tiles, uint32_t *__restrict__ nitems) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_tiles) {
        const uint32_t len = ranges[t].y - ranges[t].x;
        nitems[t] = (len + kItemFans - 1) / kItemFans;
    }
}

__global__ void tile_item_emit_kernel(const uint2 *__restrict__ ranges, int n_tiles, const uint32_t *__restrict__ nitems,
                                      const uint32_t *__restrict__ ibase, uint4 *__restrict__ items, int64_t max_items,
                                      Status *st, unsigned long long frag_cap) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        const unsigned long long ni = st->items_total;
        st->n_items = (unsigned)(ni < (unsigned long long)max_items ? ni : (unsigned long long)max_items);
        st->frag_cap = frag_cap;
    }
    if (t >= n_tiles) return;
    const uint2 r = ranges[t];
    const uint32_t n = nitems[t], b = ibase[t];
    for (uint32_t k = 0; k < n; ++k)
        if (b + k < (uint64_t)max_items)
            items[b + k] = make_uint4((uint32_t)t, r.x + k * kItemFans, min(r.y, r.x + (k + 1) * kItemFans), k);
}

// Per tile: exclusive prefix of the (item, pixel) counts over the tile's items, the
// pixel totals, and their histogram by count_bucket (for the resolve's pixel order).  One block per tile, one thread per pixel; loads are issued four items
// at a time so a tile with many items is not latency-bound.
template <int TILE>
__global__ void __launch_bounds__(TILE *TILE) item_prefix_kernel(const uint32_t *__restrict__ nitems,
                                                                 const uint32_t *__restrict__ ibase,
                                                                 const __grid_constant__ ViewTable vt,
                                                                 uint32_t *__restrict__ icnt,
                                                                 uint32_t *__restrict__ counts,
                                                                 uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_hist[kCountBuckets];
    const int t = blockIdx.x, i = threadIdx.x;
    for (int b = i; b < kCountBuckets; b += TILE * TILE) s_hist[b] = 0;
    const uint32_t n = nitems[t], b = ibase[t];
    uint32_t *c = icnt + (size_t)b * TILE * TILE + i;
    uint32_t run = 0;
    uint32_t k = 0;
    for (; k + 4 <= n; k += 4) {
        const uint32_t v0 = c[(size_t)k * TILE * TILE], v1 = c[(size_t)(k + 1) * TILE * TILE];
        const uint32_t v2 = c[(size_t)(k + 2) * TILE * TILE], v3 = c[(size_t)(k + 3) * TILE * TILE];
        c[(size_t)k * TILE * TILE] = run;
        c[(size_t)(k + 1) * TILE * TILE] = run + v0;
        c[(size_t)(k + 2) * TILE * TILE] = run + v0 + v1;
        c[(size_t)(k + 3) * TILE * TILE] = run + v0 + v1 + v2;
        run += v0 + v1 + v2 + v3;
    }
    for (; k < n; ++k) {
        const uint32_t v = c[(size_t)k * TILE * TILE];
        c[(size_t)k * TILE * TILE] = run;
        run += v;
    }
    const ViewDev &vw = vt.v[view_of_tile(vt, (uint32_t)t)];
    const int lt = t - (int)vw.tile_base, tiles_x = (int)vw.tiles_x;
    const int x = (lt % tiles_x) * TILE + (i % TILE), y = (lt / tiles_x) * TILE + (i / TILE);
    __syncthreads();
    if (x < vw.cam.width && y < vw.cam.height) {
        counts[vw.pix_base + (size_t)y * vw.cam.width + x] = run;
        atomicAdd(&s_hist[count_bucket(run)], 1u);
    }
    __syncthreads();
    for (int b = i; b < kCountBuckets; b += TILE * TILE)
        if (s_hist[b]) atomicAdd(&hist[b], s_hist[b]);
}

template <int TILE, int KT, int MODE>
cudaError_t launch_t(const RastArgs &ra, int64_t max_items, int K, cudaStream_t st) {
    // fans staged per chunk: small enough that the shared-memory stage of a warp lets
    // many warps share an SM (the passes are latency-bound), large enough to keep the
    // packed (fan, pixel) batches full
    constexpr int STG = (MODE == kCount || MODE == kSplatCount) ? 16 : 8;
    const size_t smem = kRastWarps * warp_smem_bytes<TILE, STG, MODE>(K);
    auto fn = raster_kernel<TILE, STG, KT, MODE>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<(unsigned)((max_items + kRastWarps - 1) / kRastWarps), kRastWarps * 32, smem, st>>>(ra);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_dispatch(const RastArgs &ra, const RenderLayout &L, int K, cudaStream_t st) {
    if (mode_splat(MODE)) {   // the circumscribing polygons are K = 8 fans
        if (L.tile == 8) return launch_t<8, kSplatK, MODE>(ra, L.max_items, K, st);
        if (L.tile == 32) return launch_t<32, kSplatK, MODE>(ra, L.max_items, K, st);
        return launch_t<16, kSplatK, MODE>(ra, L.max_items, K, st);
    }
    if (L.tile == 8) {
        if (K == 8) return launch_t<8, 8, MODE>(ra, L.max_items, K, st);
        if (K == 6) return launch_t<8, 6, MODE>(ra, L.max_items, K, st);
        return launch_t<8, 0, MODE>(ra, L.max_items, K, st);
    }
    if (L.tile == 32) {
        if (K == 8) return launch_t<32, 8, MODE>(ra, L.max_items, K, st);
        if (K == 6) return launch_t<32, 6, MODE>(ra, L.max_items, K, st);
        return launch_t<32, 0, MODE>(ra, L.max_items, K, st);
    }
    if (K == 8) return launch_t<16, 8, MODE>(ra, L.max_items, K, st);
    if (K == 6) return launch_t<16, 6, MODE>(ra, L.max_items, K, st);
    return launch_t<16, 0, MODE>(ra, L.max_items, K, st);
}

RastArgs make_args(const RenderArgs &ra) {
    const RenderLayout &L = ra.L;
    RastArgs a;
    a.xyz = ra.xyz;
    a.rgb = ra.rgb;
    a.alpha = ra.alpha;
    a.K = ra.K;
    a.vt = ra.vt;
    a.depth_bits = L.depth_bits;
    a.fan_bits = L.fan_bits;
    a.keys = reinterpret_cast<const unsigned long long *>(ra.ws + (L.passes & 1 ? L.off_keys1 : L.off_keys0));
    a.items = reinterpret_cast<const uint4 *>(ra.ws + L.off_items);
    a.icnt = reinterpret_cast<uint32_t *>(ra.ws + L.off_icnt);
    a.offsets = reinterpret_cast<const uint32_t *>(ra.ws + L.off_offsets);
    a.counts = reinterpret_cast<const uint32_t *>(ra.ws + L.off_counts);
    a.frags = reinterpret_cast<float4 *>(ra.ws + L.off_frags);
    a.frag_cap = L.frag_cap;
    a.st = reinterpret_cast<Status *>(ra.ws + L.off_status);
    a.spl = ra.spl;
    a.dec = reinterpret_cast<const float4 *>(ra.ws + L.off_dec);
    a.V = L.V;
    a.face_mask = ra.prm.face_mask;
    a.pinfo = reinterpret_cast<uint2 *>(ra.ws + L.off_maskoff);
    a.masks = reinterpret_cast<uint16_t *>(ra.ws + L.off_masks);
    a.mask_cap = L.mask_cap;
    a.mask_cursor = reinterpret_cast<uint32_t *>(ra.ws + L.off_mask_cursor);
    return a;
}

}  // namespace

cudaError_t launch_raster_count(const RenderArgs &ra, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    char *ws = ra.ws;
    Status *status = reinterpret_cast<Status *>(ws + L.off_status);
    const RastArgs a = make_args(ra);
    const uint2 *ranges = reinterpret_cast<const uint2 *>(ws + L.off_ranges);
    uint32_t *nitems = reinterpret_cast<uint32_t *>(ws + L.off_tile_nitems);
    uint32_t *ibase = reinterpret_cast<uint32_t *>(ws + L.off_tile_ibase);
    const int tg = (L.n_tiles + 255) / 256;
    tile_item_count_kernel<<<tg, 256, 0, st>>>(ranges, L.n_tiles, nitems);
    scan_u32_kernel<false><<<(unsigned)L.tscan_blocks, kScanThreads, 0, st>>>(
        nitems, ibase, L.n_tiles, L.tscan_blocks, reinterpret_cast<unsigned long long *>(ws + L.off_tscan_state),
        &status->tscan_ticket, &status->items_total, status, ra.vt, 0);
    tile_item_emit_kernel<<<tg, 256, 0, st>>>(ranges, L.n_tiles, nitems, ibase,
                                              reinterpret_cast<uint4 *>(ws + L.off_items), L.max_items, status,
                                              (unsigned long long)L.frag_cap);
    cudaError_t e = ra.splat ? launch_dispatch<kSplatCount>(a, L, ra.K, st) : launch_dispatch<kCount>(a, L, ra.K, st);
    if (e != cudaSuccess) return e;
    uint32_t *cnts = reinterpret_cast<uint32_t *>(ws + L.off_counts);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.off_pbucket);
    if (L.tile == 8)
        item_prefix_kernel<8><<<L.n_tiles, 64, 0, st>>>(nitems, ibase, ra.vt, a.icnt, cnts, hist);
    else if (L.tile == 32)
        item_prefix_kernel<32><<<L.n_tiles, 1024, 0, st>>>(nitems, ibase, ra.vt, a.icnt, cnts, hist);
    else
        item_prefix_kernel<16><<<L.n_tiles, 256, 0, st>>>(nitems, ibase, ra.vt, a.icnt, cnts, hist);
    int tile_shift = 0;
    while ((1 << tile_shift) < L.tile) ++tile_shift;
    const int64_t n = (int64_t)L.n_tiles << (2 * tile_shift);   // pixel slots in tile order
    scan_u32_kernel<true><<<(unsigned)L.scan_blocks, kScanThreads, 0, st>>>(
        reinterpret_cast<const uint32_t *>(ws + L.off_counts), reinterpret_cast<uint32_t *>(ws + L.off_offsets), n,
        L.scan_blocks, reinterpret_cast<unsigned long long *>(ws + L.off_scan_state), &status->scan_ticket,
        &status->frags, status, ra.vt, tile_shift);
    e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(6);
    if (e == cudaSuccess) e = launch_pixel_order(ra, st);
    return e;
}

cudaError_t launch_raster(const RenderArgs &ra, bool fill, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    if (L.n_tiles == 0) return cudaSuccess;
    const RastArgs a = make_args(ra);
    cudaError_t e;
    if (ra.splat)
        e = fill ? launch_dispatch<kSplatFill>(a, L, ra.K, st) : launch_dispatch<kSplatCount>(a, L, ra.K, st);
    else
        e = fill ? launch_dispatch<kFill>(a, L, ra.K, st) : launch_dispatch<kCount>(a, L, ra.K, st);
    if (e == cudaSuccess) count_launches(1);
    return e;
}


}  // namespace ms
