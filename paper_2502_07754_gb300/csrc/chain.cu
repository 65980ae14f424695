// Adjoint chain from the composited fragments to the fan vertices.
//
// The backward resolve leaves one adjoint record per composited fragment: the upstream
// gradients of its interpolated colour and opacity (dL/dc scaled by T a, and dL/da), its
// triangle (fan * K + j) and its pixel; slots past a pixel's composited fragments hold
// zeros.  Each fragment was interpolated with perspective-correct barycentrics mu over
// triangle j of its fan (centre c, boundary vertices b_j, b_{j+1}), so
//   dL/dc_k += mu_k dL/dc,  dL/da_k += mu_k dL/da,
// and mu depends on the three vertices' screen positions and view depths, through which
// the gradient reaches their world positions.  One thread takes one record, so no fan is
// rasterised again to find its fragments and the work is one uniform loop.  The fan
// geometry is recomputed from the vertices by the value-path formulas of the
// rasteriser's stage (double-float centre projection, offsets of the two boundary
// vertices from it); the view depths of the barycentric weights come from the same path.
#include "raster_common.cuh"

namespace ms {

namespace {

struct ChainArgs {
    const float *xyz, *rgb, *alpha;
    int K;
    int64_t n_fans, npx;
    const float4 *adj;          // adjoint records: (dL/dc * T a, dL/da), (triangle, pixel, 0, 0)
    int64_t frag_cap;
    float4 *grad;               // per vertex (dL/dxyz, dL/da | dL/drgb, 0) sums
    const Status *st;
    ViewTable vt;
};

// 7 warps a block and at most 73 registers (no spills), so four blocks (28 warps) share an
// SM: the chain waits on scattered loads and wants warps in flight; 8 warps at 76 registers
// fit three blocks (24 warps) and measured 5% slower on the 1M-fan step.
constexpr int kChainThreads = 224;

// One record's chain: adds its contributions to the three vertices' gradient sums.
__device__ __forceinline__ void chain_record(const ChainArgs &a, const float4 gr, const float4 id) {
    const int K = a.K;
    const uint32_t tri = __float_as_uint(id.x), pix = __float_as_uint(id.y);
    const uint32_t fan = tri / (uint32_t)K;
    const int j = (int)(tri - fan * (uint32_t)K);
    // (only the range of a pixel whose list overflowed the buffer can hold stale words;
    // the overflow is reported, and these bounds keep every access inside the arrays)
    if ((int64_t)pix >= a.npx || (int64_t)fan >= a.n_fans) return;
    const int view = view_of_pixel(a.vt, pix);
    const ViewDev &vw = a.vt.v[view];
    const CamDev &c = vw.cam;
    const int64_t lpix = (int64_t)pix - (int64_t)vw.pix_base;
    const int py = (int)(lpix / c.width), px = (int)(lpix - (int64_t)py * c.width);
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    const int jn = (j + 1 == K) ? 0 : j + 1;
    const size_t v0 = (size_t)fan * (K + 1);
    const size_t vid[3] = {v0, v0 + 1 + j, v0 + 1 + jn};
    // value-path geometry of the centre and the two boundary vertices
    const float *p = a.xyz + 3 * v0;
    const float m[3] = {__ldg(p), __ldg(p + 1), __ldg(p + 2)};
    const CentreProj cp = project_centre(c, m);
    float du[2], dv[2], vX[3], vY[3], vZ[3];
    vX[0] = cp.Xh;
    vY[0] = cp.Yh;
    vZ[0] = cp.Zh;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float *q = a.xyz + 3 * vid[1 + k];
        const float d[3] = {__ldg(q) - m[0], __ldg(q + 1) - m[1], __ldg(q + 2) - m[2]};
        vertex_offset(c, cp, d, du[k], dv[k], vX[1 + k], vY[1 + k], vZ[1 + k]);
    }
    const float iz[3] = {1.0f / vZ[0], 1.0f / vZ[1], 1.0f / vZ[2]};
    const float ox = __fsub_rn(cp.xh, pxc) + cp.xl;
    const float oy = __fsub_rn(cp.yh, pyc) + cp.yl;
    const float ujx = ox + du[0], ujy = oy + dv[0];
    const float unx = ox + du[1], uny = oy + dv[1];
    const float w0 = (ujx * uny - ujy * unx) * iz[0];
    const float w1 = (unx * oy - uny * ox) * iz[1];
    const float w2 = (ox * ujy - oy * ujx) * iz[2];
    const float iW = 1.0f / (w0 + w1 + w2);
    const float mu[3] = {w0 * iW, w1 * iW, w2 * iW};
    const float ux[3] = {ox, ujx, unx}, uy[3] = {oy, ujy, uny};
    // dL/dmu_k, then through mu_k = w_k / W, w_k = E_k / Z_k (E_k the cross product of
    // the other two offsets) to the screen offsets and view depths
    float gmu[3], sdot = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *col = a.rgb + 3 * vid[k];
        gmu[k] = gr.x * __ldg(col) + gr.y * __ldg(col + 1) + gr.z * __ldg(col + 2) + gr.w * __ldg(a.alpha + vid[k]);
        sdot += mu[k] * gmu[k];
    }
    float gux[3] = {0.0f, 0.0f, 0.0f}, guy[3] = {0.0f, 0.0f, 0.0f}, gZ[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int ia = (k + 1) % 3, ib = (k + 2) % 3;
        const float E = ux[ia] * uy[ib] - uy[ia] * ux[ib];
        const float gw = (gmu[k] - sdot) * iW;
        const float gE = gw * iz[k];
        gZ[k] = -gw * E * iz[k] * iz[k];
        gux[ia] += gE * uy[ib];
        guy[ia] -= gE * ux[ib];
        guy[ib] += gE * ux[ia];
        gux[ib] -= gE * uy[ia];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gX = gux[k] * c.fx * iz[k];
        const float gY = guy[k] * c.fy * iz[k];
        const float gZv = gZ[k] - (gux[k] * c.fx * vX[k] + guy[k] * c.fy * vY[k]) * iz[k] * iz[k];
        atomicAdd(a.grad + 2 * vid[k], make_float4(c.R[0] * gX + c.R[3] * gY + c.R[6] * gZv,
                                                   c.R[1] * gX + c.R[4] * gY + c.R[7] * gZv,
                                                   c.R[2] * gX + c.R[5] * gY + c.R[8] * gZv, mu[k] * gr.w));
        atomicAdd(a.grad + 2 * vid[k] + 1, make_float4(mu[k] * gr.x, mu[k] * gr.y, mu[k] * gr.z, 0.0f));
    }
}

// Each warp walks chunks of kChainChunk consecutive records, loading the next record's
// words while it works on the current one.  The warps of a block take consecutive chunks,
// so with the records in tile order a block works through one screen tile at a time and
// its warps find the same fans in the SM's L1 (measured on the 1M-fan 1080p step: chunks
// of 32, 64, 128, 256 and 512 records gave 1.17, 0.94, 0.91, 0.97 and 1.02 ms).
constexpr int kChainChunk = 32 * 4;

__global__ void __launch_bounds__(kChainThreads, 4) record_chain_kernel(const __grid_constant__ ChainArgs a) {
    const unsigned long long nrec_all = a.st->frags;
    const int64_t nrec = (int64_t)(nrec_all < (unsigned long long)a.frag_cap ? nrec_all : (unsigned long long)a.frag_cap);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * kChainChunk; base < nrec; base += nwarps * kChainChunk) {
        int64_t r = base + lane;
        float4 gn = make_float4(0.0f, 0.0f, 0.0f, 0.0f), in = gn;
        if (r < nrec) {
            gn = a.adj[2 * r];
            in = a.adj[2 * r + 1];
        }
#pragma unroll 1
        for (int it = 0; it < kChainChunk / 32; ++it) {
            const float4 gr = gn, id = in;
            const int64_t rn = r + 32;
            if (it + 1 < kChainChunk / 32 && rn < nrec) {
                gn = a.adj[2 * rn];
                in = a.adj[2 * rn + 1];
            }
            // (a record past the end, or one with no gradient, adds nothing)
            if (r < nrec && (gr.x != 0.0f || gr.y != 0.0f || gr.z != 0.0f || gr.w != 0.0f)) chain_record(a, gr, id);
            r = rn;
        }
    }
}

}  // namespace

cudaError_t launch_record_chain(const RenderArgs &ra, cudaStream_t st) {
    const RenderLayout &L = ra.L;
    if (L.n_tiles == 0 || L.V == 0 || L.frag_cap == 0) return cudaSuccess;
    ChainArgs a;
    a.xyz = ra.xyz;
    a.rgb = ra.rgb;
    a.alpha = ra.alpha;
    a.K = ra.K;
    a.n_fans = ra.n_fans;
    a.npx = L.npx;
    a.adj = reinterpret_cast<const float4 *>(ra.ws + L.off_adj);
    a.frag_cap = L.frag_cap;
    a.grad = reinterpret_cast<float4 *>(ra.ws + L.off_grad);
    a.st = reinterpret_cast<const Status *>(ra.ws + L.off_status);
    a.vt = ra.vt;
    // the record count is known on the device only: a grid-stride loop over a grid that
    // fills every SM several times
    const int64_t want = (L.frag_cap + kChainThreads - 1) / kChainThreads;
    const unsigned grid = (unsigned)min64(want, 152 * 8);
    record_chain_kernel<<<grid, kChainThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace ms
