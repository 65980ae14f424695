// Per-tile rasterisation with exact per-pixel depth order, perspective-correct
// interpolation and front-to-back compositing (forward), and its adjoint (backward).
//
// One block per screen tile, one thread per pixel.  The tile's fans arrive sorted by a
// lower bound of their fragment depths (quantised minimum vertex depth).  Fans are
// staged chunk by chunk in shared memory (decided screen vertices, edge directions,
// signed areas, pixel rectangle); every pixel tests its rectangle, then the fan's K
// triangles with the binary32 decision formulas, and inserts covered fragments into a
// small register-resident sorted buffer.  A pending fragment is composited ("committed")
// as soon as the next fan's depth bound exceeds it; that order is exact because every
// later fragment lies at least that deep.  If the buffer overflows, the pixel remembers
// the nearest dropped fragment and the earliest list position it dropped, finishes the
// pass with everything strictly nearer, and re-scans from that position; fragments at
// or before the last committed one are skipped.  The result is the full depth order
// for any buffer size.  Warps vote the pixel-rectangle test so whole warps skip fans.
//
// The backward kernel replays the identical traversal (same decisions), stops after
// the forward's committed fragment count, and at each committed fragment forms the
// adjoint from the recomputed transmittance T_f, the running colour and the forward
// output: dC/dc_f = T_f a_f, dC/da_f = T_f c_f - (C_out - C_{<=f}) / (1 - a_f),
// dA/da_f = T_out / (1 - a_f); it chains through the perspective-correct barycentrics
// and the projection to world space and accumulates per-vertex gradients with
// 16-byte vector atomics.
#include "fan_geom.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

struct CompArgs {
    const float *xyz, *rgb, *alpha;
    int K;
    CamDev cam;
    int W, H, tiles_x, depth_bits;
    float T_eps, bg0, bg1, bg2;
    const unsigned long long *keys;
    const uint32_t *vals;
    const uint2 *ranges;
    Status *st;
    float *out;
    float *tfinal;
    uint32_t *ncommit;
    const float *out_fwd, *dL;
    float4 *grad;   // V x 2 float4: (dx, dy, dz, da), (dr, dg, db, 0)
};

// Shared-memory record of a staged fan (structure of arrays, stride per field CH).
struct Stage {
    float *vx, *vy, *vz, *viz;      // [KV][CH]
    float *sdx, *sdy, *rdx, *rdy;   // [K][CH] spoke and rim directions
    float *area;                    // [K][CH] |area2|
    uint32_t *flags;                // [CH] bits 0..15 valid, 16..31 negative orientation
    int4 *rect;                     // [CH] i0, i1, j0, j1
    uint32_t *q;                    // [CH] quantised depth bound
};

template <int CH>
__device__ __forceinline__ Stage stage_ptrs(float *base, int K) {
    const int KV = K + 1;
    Stage s;
    s.vx = base;
    s.vy = s.vx + KV * CH;
    s.vz = s.vy + KV * CH;
    s.viz = s.vz + KV * CH;
    s.sdx = s.viz + KV * CH;
    s.sdy = s.sdx + K * CH;
    s.rdx = s.sdy + K * CH;
    s.rdy = s.rdx + K * CH;
    s.area = s.rdy + K * CH;
    s.flags = reinterpret_cast<uint32_t *>(s.area + K * CH);
    s.q = s.flags + CH;
    s.rect = reinterpret_cast<int4 *>(s.q + CH);
    return s;
}

template <int CH>
__host__ __device__ __forceinline__ size_t stage_bytes(int K) {
    return (size_t)CH * ((4 * (K + 1) + 5 * K + 2) * 4 + 16);
}

__device__ __forceinline__ void stage_fan(const CompArgs &a, const Stage &s, int slot, uint32_t fan, uint32_t q, int CHs) {
    const int K = a.K, KV = K + 1;
    DVert v[kMaxK + 1];
    const float *p = a.xyz + (size_t)fan * KV * 3;
    for (int k = 0; k < KV; ++k) v[k] = decide_vertex(a.cam, __ldg(p + 3 * k), __ldg(p + 3 * k + 1), __ldg(p + 3 * k + 2));
    FanRect r = fan_rect(v, K, a.W, a.H);
    for (int k = 0; k < KV; ++k) {
        s.vx[k * CHs + slot] = v[k].xs;
        s.vy[k * CHs + slot] = v[k].ys;
        s.vz[k * CHs + slot] = v[k].Z;
        s.viz[k * CHs + slot] = v[k].iz;
    }
    uint32_t flags = 0;
    for (int j = 0; j < K; ++j) {
        const int b = 1 + j, c = 1 + (j + 1 == K ? 0 : j + 1);
        s.sdx[j * CHs + slot] = __fsub_rn(v[b].xs, v[0].xs);
        s.sdy[j * CHs + slot] = __fsub_rn(v[b].ys, v[0].ys);
        // canonical rim: from the lower vertex index to the higher one
        const int lo = (j + 1 == K) ? 1 : b, hi = (j + 1 == K) ? b : c;
        s.rdx[j * CHs + slot] = __fsub_rn(v[hi].xs, v[lo].xs);
        s.rdy[j * CHs + slot] = __fsub_rn(v[hi].ys, v[lo].ys);
        const float ar = dec_area2(v[0].xs, v[0].ys, v[b].xs, v[b].ys, v[c].xs, v[c].ys);
        s.area[j * CHs + slot] = fabsf(ar);
        if (((r.valid >> j) & 1u) && ar != 0.0f) flags |= 1u << j;
        if (ar < 0.0f) flags |= 1u << (16 + j);
    }
    s.flags[slot] = r.empty ? 0u : flags;
    s.q[slot] = q;
    s.rect[slot] = make_int4(r.i0, r.i1, r.j0, r.j1);
}

// Geometry of one committed fragment, recomputed from global memory (FP32 values).
struct Frag {
    uint32_t vid[3];   // centre, b_j, b_{j+1}
    float X[3], Y[3], Z[3];
    float ux[3], uy[3];  // screen position relative to the pixel centre
    float E[3], W, mu[3];
    float c[3], a;
};

// Error-free transformations (Knuth two-sum, FMA two-product) for the double-float
// projection of the fan centre.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}
// Row r of R_cw applied to (d_hi + d_lo), as hi + lo.
__device__ __forceinline__ void df_dot(const float *R, const float dh[3], const float dl[3], float &h, float &l) {
    float p0, q0, p1, q1, p2, q2, s, e1, e2;
    two_prod(R[0], dh[0], p0, q0);
    two_prod(R[1], dh[1], p1, q1);
    two_prod(R[2], dh[2], p2, q2);
    two_sum(p0, p1, s, e1);
    two_sum(s, p2, h, e2);
    l = ((e1 + e2) + (q0 + q1 + q2)) + (R[0] * dl[0] + R[1] * dl[1] + R[2] * dl[2]);
}
// fx * (X / Z) + cx - pixel, with X, Z given as hi + lo: accurate to ~1e-6 px.
__device__ __forceinline__ float df_screen_offset(float Xh, float Xl, float Zh, float Zl, float f, float cc, float pc) {
    const float q1 = Xh / Zh;
    const float r = fmaf(-q1, Zh, Xh) + (Xl - q1 * Zl);
    const float q2 = r / Zh;
    float a1, a2, s, e;
    two_prod(f, q1, a1, a2);
    a2 = fmaf(f, q2, a2);
    two_sum(a1, cc, s, e);
    return (__fsub_rn(s, pc) + e) + a2;
}

// Value-path geometry of triangle j of a fan at a pixel centre.  The fan centre is
// projected in double-float; the other two vertices are placed by their (exact)
// world offsets from the centre, so screen positions relative to the pixel carry
// ~1e-6 px error instead of the ~1e-4 px of a plain binary32 projection.
__device__ __forceinline__ void frag_eval(const CompArgs &a, uint32_t fan, int j, float pxc, float pyc, Frag &f) {
    const int K = a.K, KV = K + 1;
    f.vid[0] = fan * KV;
    f.vid[1] = fan * KV + 1 + j;
    f.vid[2] = fan * KV + 1 + (j + 1 == K ? 0 : j + 1);
    const CamDev &c = a.cam;
    const float *pc = a.xyz + 3 * (size_t)f.vid[0];
    const float m[3] = {__ldg(pc), __ldg(pc + 1), __ldg(pc + 2)};
    float dh[3], dl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) two_sum(m[r], -c.C[r], dh[r], dl[r]);
    float Xh, Xl, Yh, Yl, Zh, Zl;
    df_dot(c.R, dh, dl, Xh, Xl);
    df_dot(c.R + 3, dh, dl, Yh, Yl);
    df_dot(c.R + 6, dh, dl, Zh, Zl);
    const float ocx = df_screen_offset(Xh, Xl, Zh, Zl, c.fx, c.cx, pxc);
    const float ocy = df_screen_offset(Yh, Yl, Zh, Zl, c.fy, c.cy, pyc);
    f.X[0] = Xh; f.Y[0] = Yh; f.Z[0] = Zh;
    f.ux[0] = ocx; f.uy[0] = ocy;
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        const float *p = a.xyz + 3 * (size_t)f.vid[k];
        const float d0 = __ldg(p) - m[0], d1 = __ldg(p + 1) - m[1], d2 = __ldg(p + 2) - m[2];
        const float dX = c.R[0] * d0 + c.R[1] * d1 + c.R[2] * d2;
        const float dY = c.R[3] * d0 + c.R[4] * d1 + c.R[5] * d2;
        const float dZ = c.R[6] * d0 + c.R[7] * d1 + c.R[8] * d2;
        f.X[k] = Xh + dX;
        f.Y[k] = Yh + dY;
        f.Z[k] = Zh + dZ;
        const float den = 1.0f / (f.Z[k] * Zh);
        f.ux[k] = ocx + c.fx * (dX * Zh - Xh * dZ) * den;
        f.uy[k] = ocy + c.fy * (dY * Zh - Yh * dZ) * den;
    }
    // E_k = cross(u_a, u_b) for the edge a -> b opposite vertex k.
    f.E[0] = f.ux[1] * f.uy[2] - f.uy[1] * f.ux[2];
    f.E[1] = f.ux[2] * f.uy[0] - f.uy[2] * f.ux[0];
    f.E[2] = f.ux[0] * f.uy[1] - f.uy[0] * f.ux[1];
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = f.E[k] / f.Z[k];
    f.W = w[0] + w[1] + w[2];
    const float iW = 1.0f / f.W;
    f.c[0] = f.c[1] = f.c[2] = 0.0f;
    f.a = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        f.mu[k] = w[k] * iW;
        const float *col = a.rgb + 3 * (size_t)f.vid[k];
        f.c[0] += f.mu[k] * __ldg(col);
        f.c[1] += f.mu[k] * __ldg(col + 1);
        f.c[2] += f.mu[k] * __ldg(col + 2);
        f.a += f.mu[k] * __ldg(a.alpha + f.vid[k]);
    }
}

// Adjoint of one fragment given dL/dc (3) and dL/da; accumulates per-vertex gradients.
__device__ __forceinline__ void frag_backward(const CompArgs &a, const Frag &f, const float gc[3], float ga) {
    const CamDev &c = a.cam;
    float gmu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *col = a.rgb + 3 * (size_t)f.vid[k];
        gmu[k] = gc[0] * __ldg(col) + gc[1] * __ldg(col + 1) + gc[2] * __ldg(col + 2) + ga * __ldg(a.alpha + f.vid[k]);
    }
    const float s = gmu[0] * f.mu[0] + gmu[1] * f.mu[1] + gmu[2] * f.mu[2];
    const float iW = 1.0f / f.W;
    float gE[3], gZ[3], gux[3] = {0, 0, 0}, guy[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gw = (gmu[k] - s) * iW;
        gE[k] = gw / f.Z[k];
        gZ[k] = -gw * f.E[k] / (f.Z[k] * f.Z[k]);
    }
    // E_k = ux_a uy_b - uy_a ux_b for (a, b) = (k+1, k+2) mod 3.
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int ia = (k + 1) % 3, ib = (k + 2) % 3;
        gux[ia] += gE[k] * f.uy[ib];
        guy[ia] -= gE[k] * f.ux[ib];
        guy[ib] += gE[k] * f.ux[ia];
        gux[ib] -= gE[k] * f.uy[ia];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float iz = 1.0f / f.Z[k];
        const float gX = gux[k] * c.fx * iz;
        const float gY = guy[k] * c.fy * iz;
        const float gZv = gZ[k] - (gux[k] * c.fx * f.X[k] + guy[k] * c.fy * f.Y[k]) * iz * iz;
        float4 g0, g1;
        g0.x = c.R[0] * gX + c.R[3] * gY + c.R[6] * gZv;
        g0.y = c.R[1] * gX + c.R[4] * gY + c.R[7] * gZv;
        g0.z = c.R[2] * gX + c.R[5] * gY + c.R[8] * gZv;
        g0.w = f.mu[k] * ga;
        g1.x = f.mu[k] * gc[0];
        g1.y = f.mu[k] * gc[1];
        g1.z = f.mu[k] * gc[2];
        g1.w = 0.0f;
        atomicAdd(a.grad + 2 * (size_t)f.vid[k], g0);
        atomicAdd(a.grad + 2 * (size_t)f.vid[k] + 1, g1);
    }
}

// Fragment order: depth, then global triangle index (fan id from the tile list).
__device__ __forceinline__ bool frag_less(const CompArgs &a, uint32_t tstart, float za, uint32_t ca, float zb,
                                          uint32_t cb) {
    if (za != zb) return za < zb;
    const uint64_t ta = (uint64_t)__ldg(a.vals + tstart + (ca >> 4)) * a.K + (ca & 15u);
    const uint64_t tb = (uint64_t)__ldg(a.vals + tstart + (cb >> 4)) * a.K + (cb & 15u);
    return ta < tb;
}

template <int TILE, int KB, int CH, bool BWD>
__global__ void __launch_bounds__(TILE *TILE) composite_kernel(CompArgs a) {
    extern __shared__ float smem[];
    const Stage S = stage_ptrs<CH>(smem, a.K);
    __shared__ int s_need, s_restart;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    constexpr int WPR = TILE / 8;   // warps per tile row; a warp covers 8 x 4 pixels
    const int wx0 = tx * TILE + (warp % WPR) * 8, wy0 = ty * TILE + (warp / WPR) * 4;
    const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
    const bool active = px < a.W && py < a.H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const uint2 rg = a.ranges[tile];
    const uint32_t tstart = rg.x;
    const int len = (int)(rg.y - rg.x);
    const int K = a.K;

    // Per-pixel state.
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    float kz[KB];
    uint32_t kc[KB];
    int n = 0;
    float fz = 0.0f;           // last committed fragment (depth, code); depth > 0 always
    uint32_t fc = 0;
    bool has_front = false;
    float dz = 0.0f;           // nearest dropped fragment of this pass
    uint32_t dc = 0;
    bool dropped = false;
    int restart = 0x7fffffff;
    bool done = !active;       // transmittance exhausted (or inactive pixel)
    bool finished = false;     // no further pass needed
    uint32_t ncom = 0;
    uint32_t ncom_limit = 0xffffffffu;
    float gR = 0, gG = 0, gB = 0, gA = 0, oR = 0, oG = 0, oB = 0, Tout = 0;
    if (BWD && active) {
        const size_t o = ((size_t)py * a.W + px);
        ncom_limit = a.ncommit[o];
        Tout = a.tfinal[o];
        const float4 g = reinterpret_cast<const float4 *>(a.dL)[o];
        const float4 ov = reinterpret_cast<const float4 *>(a.out_fwd)[o];
        gR = g.x; gG = g.y; gB = g.z; gA = g.w;
        oR = ov.x; oG = ov.y; oB = ov.z;
        if (ncom_limit == 0) done = true;
    }

    auto commit_front = [&]() {
        const uint32_t code = kc[0];
        const uint32_t fan = __ldg(a.vals + tstart + (code >> 4));
        Frag f;
        frag_eval(a, fan, (int)(code & 15u), pxc, pyc, f);
        const float w = T * f.a;
        if (BWD) {
            const float nC0 = C0 + w * f.c[0], nC1 = C1 + w * f.c[1], nC2 = C2 + w * f.c[2];
            const float inv = 1.0f / fmaxf(1.0f - f.a, 1e-6f);
            const float ga = gR * (T * f.c[0] - (oR - nC0) * inv) + gG * (T * f.c[1] - (oG - nC1) * inv) +
                             gB * (T * f.c[2] - (oB - nC2) * inv) + gA * Tout * inv;
            const float gc[3] = {gR * w, gG * w, gB * w};
            frag_backward(a, f, gc, ga);
            C0 = nC0; C1 = nC1; C2 = nC2;
        } else {
            C0 += w * f.c[0];
            C1 += w * f.c[1];
            C2 += w * f.c[2];
        }
        T *= (1.0f - f.a);
        ++ncom;
        fz = kz[0];
        fc = code;
        has_front = true;
#pragma unroll
        for (int i = 0; i + 1 < KB; ++i) {
            kz[i] = kz[i + 1];
            kc[i] = kc[i + 1];
        }
        --n;
        if (BWD ? (ncom >= ncom_limit) : (T < a.T_eps)) {
            done = true;
            n = 0;
        }
    };

    auto insert = [&](float z, uint32_t code, int lp) {
        if (has_front && !frag_less(a, tstart, fz, fc, z, code)) return;   // committed in an earlier pass
        if (dropped && !frag_less(a, tstart, z, code, dz, dc)) {
            restart = min(restart, lp);
            return;
        }
        if (n == KB) {
            if (frag_less(a, tstart, z, code, kz[KB - 1], kc[KB - 1])) {
                // evict the deepest pending fragment
                dz = kz[KB - 1];
                dc = kc[KB - 1];
                dropped = true;
                restart = min(restart, (int)(dc >> 4));
                --n;
            } else {
                if (!dropped || frag_less(a, tstart, z, code, dz, dc)) {
                    dz = z;
                    dc = code;
                }
                dropped = true;
                restart = min(restart, lp);
                return;
            }
        }
        // sorted insertion into kz[0..n)
        bool placed = false;
#pragma unroll
        for (int i = KB - 1; i >= 1; --i) {
            if (i <= n && !placed) {
                if (frag_less(a, tstart, z, code, kz[i - 1], kc[i - 1])) {
                    kz[i] = kz[i - 1];
                    kc[i] = kc[i - 1];
                } else {
                    kz[i] = z;
                    kc[i] = code;
                    placed = true;
                }
            }
        }
        if (!placed) {
            kz[0] = z;
            kc[0] = code;
        }
        ++n;
    };

    uint32_t c_rect = 0, c_frag = 0;
    int pass_start = 0;
    while (true) {
        for (int cb = pass_start; cb < len; cb += CH) {
            const int cnt = min(CH, len - cb);
            __syncthreads();
            if (tid < cnt) {
                const uint32_t li = tstart + cb + tid;
                const uint32_t q = (uint32_t)(__ldg(a.keys + li) & ((1ull << a.depth_bits) - 1ull));
                stage_fan(a, S, tid, __ldg(a.vals + li), q, CH);
            }
            __syncthreads();
            for (int f = 0; f < cnt; ++f) {
                const int4 r = S.rect[f];
                if (r.y < wx0 || r.x > wx0 + 7 || r.w < wy0 || r.z > wy0 + 3) continue;   // warp-uniform
                const uint32_t flags = S.flags[f];
                if (done || finished || px < r.x || px > r.y || py < r.z || py > r.w || flags == 0) continue;
                const uint32_t qk = S.q[f];
                ++c_rect;
                while (n > 0 && !done && depth_q(kz[0], a.depth_bits) < qk) commit_front();
                if (done) continue;
                const int lp = cb + f;
                const float xc = S.vx[f], yc = S.vy[f];
                const float qx = __fsub_rn(pxc, xc), qy = __fsub_rn(pyc, yc);
                const float S0 = __fsub_rn(__fmul_rn(S.sdx[f], qy), __fmul_rn(S.sdy[f], qx));
                float Sp = S0;
                for (int j = 0; j < K; ++j) {
                    const int jn = (j + 1 == K) ? 0 : j + 1;
                    const float Sn = jn == 0 ? S0
                                             : __fsub_rn(__fmul_rn(S.sdx[jn * CH + f], qy), __fmul_rn(S.sdy[jn * CH + f], qx));
                    if ((flags >> j) & 1u) {
                        const int lo = (j + 1 == K) ? 0 : j;
                        const float rdx = S.rdx[j * CH + f], rdy = S.rdy[j * CH + f];
                        const float Rc = dec_edge(rdx, rdy, S.vx[(1 + lo) * CH + f], S.vy[(1 + lo) * CH + f], pxc, pyc);
                        const bool wrap = (j + 1 == K);
                        const float Rf = wrap ? -Rc : Rc, rfx = wrap ? -rdx : rdx, rfy = wrap ? -rdy : rdy;
                        const float sjx = S.sdx[j * CH + f], sjy = S.sdy[j * CH + f];
                        const float snx = S.sdx[jn * CH + f], sny = S.sdy[jn * CH + f];
                        const bool neg = (flags >> (16 + j)) & 1u;
                        float E0, E1, E2;
                        bool cov;
                        if (!neg) {
                            E0 = Rf; E1 = -Sn; E2 = Sp;
                            cov = edge_pass(E0, rfx, rfy) && edge_pass(E1, -snx, -sny) && edge_pass(E2, sjx, sjy);
                        } else {
                            E0 = -Rf; E1 = -Sp; E2 = Sn;
                            cov = edge_pass(E0, -rfx, -rfy) && edge_pass(E1, -sjx, -sjy) && edge_pass(E2, snx, sny);
                        }
                        if (cov) {
                            const float iz0 = S.viz[f];
                            const float izj = S.viz[(1 + j) * CH + f], izn = S.viz[(1 + jn) * CH + f];
                            const float zf = dec_depth(S.area[j * CH + f], E0, iz0, E1, neg ? izn : izj, E2,
                                                       neg ? izj : izn, S.vz[f], S.vz[(1 + j) * CH + f],
                                                       S.vz[(1 + jn) * CH + f]);
                            ++c_frag;
                            insert(zf, ((uint32_t)lp << 4) | (uint32_t)j, lp);
                        }
                    }
                    Sp = Sn;
                }
            }
            if (__syncthreads_and(done || finished)) break;
        }
        // End of pass: everything pending is nearer than anything dropped.
        while (n > 0 && !done && !finished) commit_front();
        const bool need = dropped && !done && !finished;
        if (tid == 0) {
            s_need = 0;
            s_restart = 0x7fffffff;
        }
        __syncthreads();
        if (need) {
            atomicOr(&s_need, 1);
            atomicMin(&s_restart, restart);
            atomicAdd(&a.st->extra_passes, 1ull);
        }
        __syncthreads();
        if (!s_need) break;
        pass_start = s_restart;
        if (!need) finished = true;
        dropped = false;
        restart = 0x7fffffff;
        n = 0;
    }

    if (!BWD) {
        unsigned r0 = __reduce_add_sync(0xffffffffu, c_rect);
        unsigned r1 = __reduce_add_sync(0xffffffffu, c_frag);
        unsigned r2 = __reduce_add_sync(0xffffffffu, ncom);
        if (lane == 0) {
            atomicAdd(&a.st->rect_tests, (unsigned long long)r0);
            atomicAdd(&a.st->fragments, (unsigned long long)r1);
            atomicAdd(&a.st->commits, (unsigned long long)r2);
        }
    }
    if (!BWD && active) {
        const size_t o = (size_t)py * a.W + px;
        reinterpret_cast<float4 *>(a.out)[o] = make_float4(C0 + T * a.bg0, C1 + T * a.bg1, C2 + T * a.bg2, 1.0f - T);
        a.tfinal[o] = T;
        a.ncommit[o] = ncom;
    }
}

template <int TILE, int KB, bool BWD>
cudaError_t launch_t(const CompArgs &ca, int n_tiles, int K, cudaStream_t st) {
    constexpr int CH = TILE * TILE < 256 ? TILE * TILE : 256;
    const size_t smem = stage_bytes<CH>(K);
    auto fn = composite_kernel<TILE, KB, CH, BWD>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<n_tiles, TILE * TILE, smem, st>>>(ca);
    return cudaGetLastError();
}

template <bool BWD>
cudaError_t launch_dispatch(const CompArgs &ca, const RenderLayout &L, int K, cudaStream_t st) {
    if (L.tile == 8) return L.kbuf == 8 ? launch_t<8, 8, BWD>(ca, L.n_tiles, K, st) : launch_t<8, 16, BWD>(ca, L.n_tiles, K, st);
    if (L.tile == 32) return launch_t<32, 8, BWD>(ca, L.n_tiles, K, st);
    return L.kbuf == 8 ? launch_t<16, 8, BWD>(ca, L.n_tiles, K, st) : launch_t<16, 16, BWD>(ca, L.n_tiles, K, st);
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

cudaError_t launch_composite(const RenderArgs &ra, bool backward, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    CompArgs ca;
    ca.xyz = ra.xyz;
    ca.rgb = ra.rgb;
    ca.alpha = ra.alpha;
    ca.K = ra.K;
    ca.cam = make_cam(*ra.cam);
    ca.W = ra.cam->width;
    ca.H = ra.cam->height;
    ca.tiles_x = L.tiles_x;
    ca.depth_bits = L.depth_bits;
    ca.T_eps = ra.prm.T_eps;
    ca.bg0 = ra.prm.bg[0];
    ca.bg1 = ra.prm.bg[1];
    ca.bg2 = ra.prm.bg[2];
    ca.keys = reinterpret_cast<const unsigned long long *>(ra.ws + (L.passes & 1 ? L.off_keys1 : L.off_keys0));
    ca.vals = reinterpret_cast<const uint32_t *>(ra.ws + (L.passes & 1 ? L.off_vals1 : L.off_vals0));
    ca.ranges = reinterpret_cast<const uint2 *>(ra.ws + L.off_ranges);
    ca.st = reinterpret_cast<Status *>(ra.ws + L.off_status);
    ca.out = ra.out_rgba;
    ca.tfinal = reinterpret_cast<float *>(ra.ws + L.off_tfinal);
    ca.ncommit = reinterpret_cast<uint32_t *>(ra.ws + L.off_ncommit);
    ca.out_fwd = ra.out_fwd;
    ca.dL = ra.dL;
    ca.grad = reinterpret_cast<float4 *>(ra.ws + L.off_grad);
    if (L.n_tiles == 0) return cudaSuccess;
    return backward ? launch_dispatch<true>(ca, L, ra.K, st) : launch_dispatch<false>(ca, L, ra.K, st);
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
