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
// fragments at or before the last committed one.  Order: (depth, triangle id).
// Compositing stops once the transmittance falls below T_eps.
//
// The backward replays the same order, stops after the forward's committed count,
// and at each committed fragment f forms dC/dc_f = T_f a_f,
// dC/da_f = T_f c_f - (C_out - C_{<=f}) / (1 - a_f), dA/da_f = T_out / (1 - a_f) from
// the recomputed transmittance, then chains through the perspective-correct
// barycentrics and the projection to world space; per-vertex gradients accumulate
// with 16-byte vector atomics into a (xyz, alpha | rgb, 0) scratch, scattered to the
// caller's arrays at the end.
#include "raster_common.cuh"

namespace ms {

namespace {

struct ResolveArgs {
    SceneDev sc;
    const uint32_t *counts, *offsets;
    const float4 *frags;
    int64_t frag_cap;
    int depth_bits;
    float T_eps, bg0, bg1, bg2;
    Status *st;
    float *out;
    float *tfinal;
    uint32_t *ncommit;
    const float *out_fwd, *dL;
    float4 *grad;
};

// Geometry of a fragment recomputed from global memory (backward only).
struct Frag {
    uint32_t vid[3];     // centre, b_j, b_{j+1}
    float X[3], Y[3], Z[3];
    float ux[3], uy[3];  // screen position relative to the pixel centre
    float E[3], W, mu[3];
};

__device__ __forceinline__ void frag_geometry(const SceneDev &a, uint32_t tri, float pxc, float pyc, Frag &f) {
    const int K = a.K, KV = K + 1;
    const uint32_t fan = tri / (uint32_t)K, j = tri - fan * (uint32_t)K;
    f.vid[0] = fan * KV;
    f.vid[1] = fan * KV + 1 + j;
    f.vid[2] = fan * KV + 1 + (j + 1 == (uint32_t)K ? 0 : j + 1);
    const CamDev &c = a.cam;
    const float *pc = a.xyz + 3 * (size_t)f.vid[0];
    const float m[3] = {__ldg(pc), __ldg(pc + 1), __ldg(pc + 2)};
    const CentreProj cp = project_centre(c, m);
    const float ocx = __fsub_rn(cp.xh, pxc) + cp.xl, ocy = __fsub_rn(cp.yh, pyc) + cp.yl;
    f.X[0] = cp.Xh; f.Y[0] = cp.Yh; f.Z[0] = cp.Zh;
    f.ux[0] = ocx; f.uy[0] = ocy;
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        const float *p = a.xyz + 3 * (size_t)f.vid[k];
        const float d[3] = {__ldg(p) - m[0], __ldg(p + 1) - m[1], __ldg(p + 2) - m[2]};
        float du, dv;
        vertex_offset(c, cp, d, du, dv, f.X[k], f.Y[k], f.Z[k]);
        f.ux[k] = ocx + du;
        f.uy[k] = ocy + dv;
    }
    f.E[0] = f.ux[1] * f.uy[2] - f.uy[1] * f.ux[2];
    f.E[1] = f.ux[2] * f.uy[0] - f.uy[2] * f.ux[0];
    f.E[2] = f.ux[0] * f.uy[1] - f.uy[0] * f.ux[1];
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = f.E[k] / f.Z[k];
    f.W = w[0] + w[1] + w[2];
    const float iW = 1.0f / f.W;
#pragma unroll
    for (int k = 0; k < 3; ++k) f.mu[k] = w[k] * iW;
}

// Adjoint of one fragment given dL/dc (3) and dL/da; accumulates per-vertex gradients.
__device__ __forceinline__ void frag_backward(const SceneDev &a, float4 *grad, const Frag &f, const float gc[3],
                                              float ga) {
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
        atomicAdd(grad + 2 * (size_t)f.vid[k], g0);
        atomicAdd(grad + 2 * (size_t)f.vid[k] + 1, g1);
    }
}

__device__ __forceinline__ bool frag_less(float za, uint32_t ta, float zb, uint32_t tb) {
    return za < zb || (za == zb && ta < tb);
}

template <int KB, bool BWD>
__global__ void __launch_bounds__(256) resolve_kernel(ResolveArgs a) {
    const int64_t npx = (int64_t)a.sc.W * a.sc.H;
    const int64_t pix0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = pix0 < npx;
    const int64_t pix = valid ? pix0 : 0;
    const int px = (int)(pix % a.sc.W), py = (int)(pix / a.sc.W);
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    int n = valid ? (int)a.counts[pix] : 0;
    const int64_t off = a.offsets[pix];
    if (off + n > a.frag_cap) n = 0;   // the buffer overflowed: reported through the status block
    const float4 *rec = a.frags + 2 * off;

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    float kz[KB], kr[KB], kg[KB], kb[KB], ka[KB];
    uint32_t kt[KB], ki[KB];   // triangle id, record index
    int nb = 0;
    float fz = 0.0f;           // last committed (depth, triangle); depths are > 0
    uint32_t ft = 0;
    bool has_front = false;
    float dz = 0.0f;           // nearest dropped fragment of this pass
    uint32_t dt = 0;
    bool dropped = false;
    int restart = 0x7fffffff;
    bool done = !valid;
    uint32_t ncom = 0, ncom_limit = 0xffffffffu;
    float gR = 0, gG = 0, gB = 0, gA = 0, oR = 0, oG = 0, oB = 0, Tout = 0;
    if (BWD && valid) {
        ncom_limit = a.ncommit[pix];
        Tout = a.tfinal[pix];
        const float4 g = reinterpret_cast<const float4 *>(a.dL)[pix];
        const float4 ov = reinterpret_cast<const float4 *>(a.out_fwd)[pix];
        gR = g.x; gG = g.y; gB = g.z; gA = g.w;
        oR = ov.x; oG = ov.y; oB = ov.z;
        if (ncom_limit == 0) done = true;
    }

    auto commit_front = [&]() {
        const float al = ka[0], c0 = kr[0], c1 = kg[0], c2 = kb[0];
        const float w = T * al;
        if (BWD) {
            const float nC0 = C0 + w * c0, nC1 = C1 + w * c1, nC2 = C2 + w * c2;
            const float inv = 1.0f / fmaxf(1.0f - al, 1e-6f);
            const float ga = gR * (T * c0 - (oR - nC0) * inv) + gG * (T * c1 - (oG - nC1) * inv) +
                             gB * (T * c2 - (oB - nC2) * inv) + gA * Tout * inv;
            const float gc[3] = {gR * w, gG * w, gB * w};
            Frag f;
            frag_geometry(a.sc, kt[0], pxc, pyc, f);
            frag_backward(a.sc, a.grad, f, gc, ga);
            C0 = nC0; C1 = nC1; C2 = nC2;
        } else {
            C0 += w * c0;
            C1 += w * c1;
            C2 += w * c2;
        }
        T *= (1.0f - al);
        ++ncom;
        fz = kz[0];
        ft = kt[0];
        has_front = true;
#pragma unroll
        for (int i = 0; i + 1 < KB; ++i) {
            kz[i] = kz[i + 1]; kt[i] = kt[i + 1]; ki[i] = ki[i + 1];
            kr[i] = kr[i + 1]; kg[i] = kg[i + 1]; kb[i] = kb[i + 1]; ka[i] = ka[i + 1];
        }
        --nb;
        if (BWD ? (ncom >= ncom_limit) : (T < a.T_eps)) {
            done = true;
            nb = 0;
        }
    };

    int start = 0;
    while (!done) {
        for (int i = start; i < n && !done; ++i) {
            const float4 r0 = rec[2 * i];
            const float z = r0.x;
            const uint32_t tri = __float_as_uint(r0.y), qk = __float_as_uint(r0.z);
            while (nb > 0 && !done && depth_q(kz[0], a.depth_bits) < qk) commit_front();
            if (done) break;
            if (has_front && !frag_less(fz, ft, z, tri)) continue;   // committed in an earlier pass
            if (dropped && !frag_less(z, tri, dz, dt)) {
                restart = min(restart, i);
                continue;
            }
            if (nb == KB) {
                if (frag_less(z, tri, kz[KB - 1], kt[KB - 1])) {
                    dz = kz[KB - 1];   // evict the deepest pending fragment
                    dt = kt[KB - 1];
                    dropped = true;
                    restart = min(restart, (int)ki[KB - 1]);
                    --nb;
                } else {
                    if (!dropped || frag_less(z, tri, dz, dt)) {
                        dz = z;
                        dt = tri;
                    }
                    dropped = true;
                    restart = min(restart, i);
                    continue;
                }
            }
            const float4 r1 = rec[2 * i + 1];
            bool placed = false;
#pragma unroll
            for (int s = KB - 1; s >= 1; --s) {
                if (s <= nb && !placed) {
                    if (frag_less(z, tri, kz[s - 1], kt[s - 1])) {
                        kz[s] = kz[s - 1]; kt[s] = kt[s - 1]; ki[s] = ki[s - 1];
                        kr[s] = kr[s - 1]; kg[s] = kg[s - 1]; kb[s] = kb[s - 1]; ka[s] = ka[s - 1];
                    } else {
                        kz[s] = z; kt[s] = tri; ki[s] = (uint32_t)i;
                        kr[s] = r1.x; kg[s] = r1.y; kb[s] = r1.z; ka[s] = r0.w;
                        placed = true;
                    }
                }
            }
            if (!placed) {
                kz[0] = z; kt[0] = tri; ki[0] = (uint32_t)i;
                kr[0] = r1.x; kg[0] = r1.y; kb[0] = r1.z; ka[0] = r0.w;
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
    if (!BWD) {
        if (valid) {
            reinterpret_cast<float4 *>(a.out)[pix] =
                make_float4(C0 + T * a.bg0, C1 + T * a.bg1, C2 + T * a.bg2, 1.0f - T);
            a.tfinal[pix] = T;
            a.ncommit[pix] = ncom;
        }
        const unsigned r = __reduce_add_sync(0xffffffffu, ncom);
        if ((threadIdx.x & 31) == 0) atomicAdd(&a.st->commits, (unsigned long long)r);
    }
}

template <bool BWD>
cudaError_t launch_k(const ResolveArgs &ra, int kbuf, int64_t npx, cudaStream_t st) {
    const unsigned grid = (unsigned)((npx + 255) / 256);
    if (kbuf == 16)
        resolve_kernel<16, BWD><<<grid, 256, 0, st>>>(ra);
    else
        resolve_kernel<8, BWD><<<grid, 256, 0, st>>>(ra);
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
    const int64_t npx = (int64_t)ra.cam->width * ra.cam->height;
    ResolveArgs a;
    a.sc.xyz = ra.xyz;
    a.sc.rgb = ra.rgb;
    a.sc.alpha = ra.alpha;
    a.sc.K = ra.K;
    a.sc.cam = make_cam(*ra.cam);
    a.sc.W = ra.cam->width;
    a.sc.H = ra.cam->height;
    a.counts = reinterpret_cast<const uint32_t *>(ra.ws + L.off_counts);
    a.offsets = reinterpret_cast<const uint32_t *>(ra.ws + L.off_offsets);
    a.frags = reinterpret_cast<const float4 *>(ra.ws + L.off_frags);
    a.frag_cap = L.frag_cap;
    a.depth_bits = L.depth_bits;
    a.T_eps = ra.prm.T_eps;
    a.bg0 = ra.prm.bg[0];
    a.bg1 = ra.prm.bg[1];
    a.bg2 = ra.prm.bg[2];
    a.st = reinterpret_cast<Status *>(ra.ws + L.off_status);
    a.out = ra.out_rgba;
    a.tfinal = reinterpret_cast<float *>(ra.ws + L.off_tfinal);
    a.ncommit = reinterpret_cast<uint32_t *>(ra.ws + L.off_ncommit);
    a.out_fwd = ra.out_fwd;
    a.dL = ra.dL;
    a.grad = reinterpret_cast<float4 *>(ra.ws + L.off_grad);
    return backward ? launch_k<true>(a, L.kbuf, npx, st) : launch_k<false>(a, L.kbuf, npx, st);
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
