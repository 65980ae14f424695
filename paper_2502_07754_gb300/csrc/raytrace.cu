// Ray tracing of the triangle soup with shadows (the paper's motivation for the mesh form,
// Sec. 1 and its discussion of ray-traced Gaussian renderers: a triangle soup is what ray
// tracers take, with secondary effects such as shadows).  The paper gives no shading
// model; the one implemented (also the oracle's):
//   * primary rays: the pixel-centre ray of the pinhole camera, x = C + t d with d of unit
//     view depth (so t is the view depth); every triangle it crosses at t > znear is a
//     fragment with the ray's barycentrics (equal to the rasteriser's perspective-correct
//     ones), ordered by t, ties by triangle index, composited front to back as the raster
//     does (C += T a c, T *= 1 - a; out = (C + T bg, 1 - T));
//   * shadows: a point light L; a fragment at p gets the transmittance S, the product of
//     (1 - a_g) over every other triangle g the segment p -> L crosses (parameter strictly
//     inside (1e-9, 1 - 1e-9)), and its colour becomes c (k + (1 - k) S), k the ambient
//     share; a shadow ray stops once S < T_eps, the primary composite's own bound.
// Intersections are decided in FP64 (Moller-Trumbore, edges closed), values in FP64.
//
// Acceleration: a linear BVH (Karras 2012, "Maximizing parallelism in the construction of
// BVHs, octrees, and k-d trees"): 30-bit Morton codes of the triangle centroids in the
// scene box, sorted (with the triangle index as the low 32 bits, so every key is unique)
// by the library's radix sort; every internal node finds its key range and split from the
// longest common prefixes of its neighbours; boxes are merged bottom-up, the second of a
// node's two children to arrive computing the node (an atomic counter per node, no waits).
// Boxes are the binary32 vertex bounds widened by a small margin so that the binary32
// slab test never rejects a box the FP64 ray meets.
//
// Tracing gathers a ray's crossings in passes: each pass walks the BVH keeping the KB
// nearest crossings beyond the last composited one (by (t, triangle)), composites them in
// order, and repeats while some crossing was left out and the transmittance is above
// T_eps.  A pass skips boxes that end before the last composited crossing and, once its
// buffer is full, boxes that start beyond the farthest kept one; a binary32 filter
// (mt_may_hit) keeps the FP64 test for triangles the ray may cross.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kBvhThreads = 256;
constexpr int kTraceThreads = 64;
constexpr int kTraceKB = 8;
constexpr int kStack = 64;
constexpr double kSegEps = 1e-9;

struct BvhNode {
    float lo[3], hi[3];
    int left, right;   // children: < n - 1 internal, >= n - 1 leaf (n - 1 + sorted position)
};

struct BvhLayout {
    size_t nodes, parent, flags, leaf_tri, keys0, keys1, bounds, status, scratch, total;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

BvhLayout bvh_layout(int64_t T) {
    BvhLayout L;
    const int64_t n = T > 0 ? T : 1;
    size_t o = 0;
    L.status = o;   o = al256(o + 256);
    L.bounds = o;   o = al256(o + 8 * sizeof(unsigned));
    L.nodes = o;    o = al256(o + (size_t)(2 * n - 1) * sizeof(BvhNode));
    L.parent = o;   o = al256(o + (size_t)(2 * n - 1) * 4);
    L.flags = o;    o = al256(o + (size_t)n * 4);
    L.leaf_tri = o; o = al256(o + (size_t)n * 4);
    L.keys0 = o;    o = al256(o + (size_t)n * 8);
    L.keys1 = o;    o = al256(o + (size_t)n * 8);
    L.scratch = o;  o = al256(o + sort_scratch_bytes(n, 4));
    L.total = o;
    return L;
}

// Vertex indices of triangle t: explicit, or the implicit fan topology of K triangles a fan.
__device__ __forceinline__ void tri_verts(const int32_t *tris, int K, int64_t t, int64_t v[3]) {
    if (tris) {
        v[0] = __ldg(tris + 3 * t);
        v[1] = __ldg(tris + 3 * t + 1);
        v[2] = __ldg(tris + 3 * t + 2);
    } else {
        const int64_t g = t / K;
        const int j = (int)(t - g * K);
        const int64_t c = g * (K + 1);
        v[0] = c;
        v[1] = c + 1 + j;
        v[2] = c + 1 + (j + 1 == K ? 0 : j + 1);
    }
}

// Floats ordered as unsigned integers (for atomic min / max of the scene box).
__device__ __forceinline__ unsigned f2o(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void bounds_init_kernel(unsigned *b) {
    if (threadIdx.x < 3) b[threadIdx.x] = 0xffffffffu;   // min
    else if (threadIdx.x < 6) b[threadIdx.x] = 0u;        // max
}

__global__ void __launch_bounds__(kBvhThreads) centroid_bounds_kernel(const float *__restrict__ xyz,
                                                                      const int32_t *__restrict__ tris, int K,
                                                                      int64_t T, unsigned *b) {
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t v[3];
        tri_verts(tris, K, t, v);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float c = (__ldg(xyz + 3 * v[0] + r) + __ldg(xyz + 3 * v[1] + r) + __ldg(xyz + 3 * v[2] + r)) *
                             (1.0f / 3.0f);
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
            atomicMin(&b[r], f2o(lo[r]));
            atomicMax(&b[3 + r], f2o(hi[r]));
        }
    }
}

// 10 bits of x spread to every third bit.
__device__ __forceinline__ unsigned long long spread3(unsigned x) {
    unsigned long long v = x & 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFull;
    v = (v | (v << 8)) & 0x0300F00Full;
    v = (v | (v << 4)) & 0x030C30C3ull;
    v = (v | (v << 2)) & 0x09249249ull;
    return v;
}

__global__ void __launch_bounds__(kBvhThreads) morton_kernel(const float *__restrict__ xyz,
                                                             const int32_t *__restrict__ tris, int K, int64_t T,
                                                             const unsigned *__restrict__ b,
                                                             unsigned long long *__restrict__ keys) {
    float lo[3], ext[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        lo[r] = o2f(b[r]);
        const float e = o2f(b[3 + r]) - lo[r];
        ext[r] = e > 0.0f ? e : 1.0f;
    }
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t v[3];
        tri_verts(tris, K, t, v);
        unsigned long long code = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float c = (__ldg(xyz + 3 * v[0] + r) + __ldg(xyz + 3 * v[1] + r) + __ldg(xyz + 3 * v[2] + r)) *
                            (1.0f / 3.0f);
            const float q = fminf(fmaxf((c - lo[r]) / ext[r] * 1024.0f, 0.0f), 1023.0f);
            code |= spread3((unsigned)q) << (2 - r);
        }
        keys[t] = (code << 32) | (unsigned long long)(uint32_t)t;
    }
}

// Common prefix length of sorted keys i and j (-1 outside [0, n)).
__device__ __forceinline__ int delta(const unsigned long long *k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    return __clzll(k[i] ^ k[j]);
}

__global__ void __launch_bounds__(kBvhThreads) radix_tree_kernel(const unsigned long long *__restrict__ keys,
                                                                 int64_t n, BvhNode *__restrict__ nodes,
                                                                 int *__restrict__ parent,
                                                                 int *__restrict__ leaf_tri) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        leaf_tri[i] = (int)(uint32_t)keys[i];
        if (i >= n - 1) continue;
        const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
        const int dmin = delta(keys, n, i, i - d);
        int64_t lmax = 2;
        while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;   // at most log2(n) + 1 doublings
        int64_t l = 0;
        for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
            if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = delta(keys, n, i, j);
        int64_t s = 0;
        for (int64_t t = (l + 1) >> 1;; t = (t + 1) >> 1) {
            if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
            if (t == 1) break;
        }
        const int64_t split = i + s * d + (d < 0 ? -1 : 0);
        const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        const int left = lo == split ? (int)(n - 1 + split) : (int)split;
        const int right = hi == split + 1 ? (int)(n - 1 + split + 1) : (int)(split + 1);
        nodes[i].left = left;
        nodes[i].right = right;
        parent[left] = (int)i;
        parent[right] = (int)i;
    }
}

__global__ void __launch_bounds__(kBvhThreads) bounds_up_kernel(const float *__restrict__ xyz,
                                                                const int32_t *__restrict__ tris, int K, int64_t n,
                                                                BvhNode *nodes, const int *__restrict__ parent,
                                                                const int *__restrict__ leaf_tri, int *flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t leaf = n - 1 + i;
        int64_t v[3];
        tri_verts(tris, K, leaf_tri[i], v);
        BvhNode &L = nodes[leaf];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float a = __ldg(xyz + 3 * v[0] + r), b = __ldg(xyz + 3 * v[1] + r), c = __ldg(xyz + 3 * v[2] + r);
            const float lo = fminf(fminf(a, b), c), hi = fmaxf(fmaxf(a, b), c);
            const float m = 1e-5f * (hi - lo) + 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f;
            L.lo[r] = lo - m;
            L.hi[r] = hi + m;
        }
        L.left = L.right = -1;
        int64_t node = leaf;
        // each internal node is completed by the second of its two children to arrive
        for (int steps = 0; node != 0 && steps < 64 + 64; ++steps) {
            const int p = parent[node];
            __threadfence();
            if (atomicAdd(&flags[p], 1) == 0) break;
            __threadfence();
            const BvhNode &a = nodes[nodes[p].left], &b = nodes[nodes[p].right];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                nodes[p].lo[r] = fminf(a.lo[r], b.lo[r]);
                nodes[p].hi[r] = fmaxf(a.hi[r], b.hi[r]);
            }
            node = p;
        }
    }
}

// ------------------------------------------------------------------------------ tracing

struct TraceArgs {
    const float *xyz, *rgb, *alpha;
    const int32_t *tris;
    int K;
    int64_t T;
    const BvhNode *nodes;
    const int *leaf_tri;
    CamDev cam;
    double L[3];
    int shadows;
    double ambient;
    double T_eps;
    float bg[3];
    float *out;
    unsigned *overflow;   // traversal stack overflows (status)
};

struct Hit {
    double t, u, v;
    int tri;
};

// Moller-Trumbore in FP64, edges closed: the crossing of o + t d with triangle (P0, P1, P2).
__device__ __forceinline__ bool mt(const double o[3], const double d[3], const double P0[3], const double P1[3],
                                   const double P2[3], double &t, double &u, double &v) {
    const double e1[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
    const double e2[3] = {P2[0] - P0[0], P2[1] - P0[1], P2[2] - P0[2]};
    const double pv[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
    const double det = (e1[0] * pv[0] + e1[1] * pv[1]) + e1[2] * pv[2];
    if (!(fabs(det) > 1e-300)) return false;
    const double inv = 1.0 / det;
    const double tv[3] = {o[0] - P0[0], o[1] - P0[1], o[2] - P0[2]};
    u = ((tv[0] * pv[0] + tv[1] * pv[1]) + tv[2] * pv[2]) * inv;
    const double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
    v = ((qv[0] * d[0] + qv[1] * d[1]) + qv[2] * d[2]) * inv;
    t = ((e2[0] * qv[0] + e2[1] * qv[1]) + e2[2] * qv[2]) * inv;
    return u >= 0.0 && v >= 0.0 && u + v <= 1.0;
}

// Binary32 filter of mt for a crossing parameter in [tmin, tmax]: false only when the
// crossing certainly fails in exact arithmetic by a margin far above the FP64 test's own
// rounding, so mt, run on what passes, decides exactly as without the filter.  Every
// binary32 quantity q below carries an error of at most a few units of 2^-24 times S_q, the
// same expression over the absolute values of its operands (with |a - b| bounded by
// |a| + |b|, which also covers the rounding of o and d to binary32); the margins are 64
// such units.  An undetermined sign of the determinant passes the triangle on to FP64.
// FP64 arithmetic runs at a small fraction of the binary32 rate on this GPU, and most
// boxes the traversal reaches hold triangles the ray misses.
struct RayF {
    float o[3], d[3], ao[3], ad[3];
};
__device__ __forceinline__ RayF ray_f(const double o[3], const double d[3]) {
    RayF r;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.o[k] = (float)o[k];
        r.d[k] = (float)d[k];
        r.ao[k] = fabsf(r.o[k]);
        r.ad[k] = fabsf(r.d[k]);
    }
    return r;
}
__device__ __forceinline__ bool mt_may_hit(const RayF &r, const float P0[3], const float P1[3], const float P2[3],
                                           float tmin, float tmax) {
    constexpr float kU = 64.0f * 0x1p-24f;
    float e1[3], e2[3], tv[3], E1[3], E2[3], TV[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e1[k] = P1[k] - P0[k];
        e2[k] = P2[k] - P0[k];
        tv[k] = r.o[k] - P0[k];
        const float a0 = fabsf(P0[k]);
        E1[k] = fabsf(P1[k]) + a0;
        E2[k] = fabsf(P2[k]) + a0;
        TV[k] = r.ao[k] + a0;
    }
    const float pv[3] = {r.d[1] * e2[2] - r.d[2] * e2[1], r.d[2] * e2[0] - r.d[0] * e2[2],
                         r.d[0] * e2[1] - r.d[1] * e2[0]};
    const float PV[3] = {r.ad[1] * E2[2] + r.ad[2] * E2[1], r.ad[2] * E2[0] + r.ad[0] * E2[2],
                         r.ad[0] * E2[1] + r.ad[1] * E2[0]};
    const float det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    const float eDet = kU * (E1[0] * PV[0] + E1[1] * PV[1] + E1[2] * PV[2]);
    if (!(fabsf(det) > eDet)) return true;
    const float sg = det > 0.0f ? 1.0f : -1.0f;
    const float U = tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2];
    const float eU = kU * (TV[0] * PV[0] + TV[1] * PV[1] + TV[2] * PV[2]);
    if (sg * U < -eU) return false;
    const float qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
    const float QV[3] = {TV[1] * E1[2] + TV[2] * E1[1], TV[2] * E1[0] + TV[0] * E1[2], TV[0] * E1[1] + TV[1] * E1[0]};
    const float V = qv[0] * r.d[0] + qv[1] * r.d[1] + qv[2] * r.d[2];
    const float eV = kU * (QV[0] * r.ad[0] + QV[1] * r.ad[1] + QV[2] * r.ad[2]);
    if (sg * V < -eV) return false;
    if (sg * (U + V - det) > eU + eV + eDet) return false;
    const float Tn = e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2];
    const float eT = kU * (E2[0] * QV[0] + E2[1] * QV[1] + E2[2] * QV[2]);
    const float t = Tn / det;
    const float dt = (eT + fabsf(t) * eDet) / (fabsf(det) - eDet) + kU * fabsf(t);
    return t + dt >= tmin && t - dt <= tmax;
}

__device__ __forceinline__ void tri_f(const TraceArgs &a, int tri, float P[3][3]) {
    int64_t v[3];
    tri_verts(a.tris, a.K, tri, v);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r) P[k][r] = __ldg(a.xyz + 3 * v[k] + r);
}

__device__ __forceinline__ void load_tri(const TraceArgs &a, int tri, int64_t v[3], double P[3][3]) {
    tri_verts(a.tris, a.K, tri, v);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r) P[k][r] = (double)__ldg(a.xyz + 3 * v[k] + r);
}

// Slab test of the ray o + t d, t in [t0, t1], against a node box (binary32, widened).
__device__ __forceinline__ bool box_hit(const BvhNode &nd, const float o[3], const float id[3], float t0, float t1) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float a = (nd.lo[r] - o[r]) * id[r], b = (nd.hi[r] - o[r]) * id[r];
        if (a > b) { const float tmp = a; a = b; b = tmp; }
        if (!(a == a)) a = -3.0e38f;   // 0 * inf
        if (!(b == b)) b = 3.0e38f;
        t0 = fmaxf(t0, a);
        t1 = fminf(t1, b);
    }
    return t0 <= t1;
}

// The same slab test returning the parameter interval [tn, tf] of the box (within t0, t1).
__device__ __forceinline__ bool box_span(const BvhNode &nd, const float o[3], const float id[3], float t0, float t1,
                                         float &tn, float &tf) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float a = (nd.lo[r] - o[r]) * id[r], b = (nd.hi[r] - o[r]) * id[r];
        if (a > b) { const float tmp = a; a = b; b = tmp; }
        if (!(a == a)) a = -3.0e38f;   // 0 * inf
        if (!(b == b)) b = 3.0e38f;
        t0 = fmaxf(t0, a);
        t1 = fminf(t1, b);
    }
    tn = t0;
    tf = t1;
    return t0 <= t1;
}

__device__ __forceinline__ bool hit_less(double ta, int ia, double tb, int ib) { return ta < tb || (ta == tb && ia < ib); }

// Transmittance of the segment p -> L through every triangle but `own`.
__device__ double shadow(const TraceArgs &a, const double p[3], int own) {
    const double d[3] = {a.L[0] - p[0], a.L[1] - p[1], a.L[2] - p[2]};
    const float of[3] = {(float)p[0], (float)p[1], (float)p[2]};
    const RayF rf = ray_f(p, d);
    float id[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) id[r] = 1.0f / (float)d[r];
    int stack[kStack];
    int sp = 0;
    stack[sp++] = 0;
    double S = 1.0;
    const int64_t n = a.T;
    while (sp > 0) {
        const int node = stack[--sp];
        const BvhNode &nd = a.nodes[node];
        if (!box_hit(nd, of, id, -1e-3f, 1.001f)) continue;
        if (node >= n - 1) {
            const int tri = a.leaf_tri[node - (n - 1)];
            if (tri == own) continue;
            {
                float Pf[3][3];
                tri_f(a, tri, Pf);
                if (!mt_may_hit(rf, Pf[0], Pf[1], Pf[2], (float)kSegEps, (float)(1.0 - kSegEps))) continue;
            }
            int64_t v[3];
            double P[3][3], t, u, w;
            load_tri(a, tri, v, P);
            if (mt(p, d, P[0], P[1], P[2], t, u, w) && t > kSegEps && t < 1.0 - kSegEps) {
                const double al = (1.0 - u - w) * __ldg(a.alpha + v[0]) + u * __ldg(a.alpha + v[1]) +
                                  w * __ldg(a.alpha + v[2]);
                S *= 1.0 - al;
                // the light is blocked to within T_eps: the colour's shadow factor moves by at
                // most (1 - ambient) T_eps, the primary composite's own termination bound
                if (S < a.T_eps) return S;
            }
            continue;
        }
        if (sp + 2 > kStack) {
            atomicAdd(a.overflow, 1u);
            continue;
        }
        stack[sp++] = nd.left;
        stack[sp++] = nd.right;
    }
    return S;
}

__global__ void __launch_bounds__(kTraceThreads) trace_kernel(const __grid_constant__ TraceArgs a) {
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = a.cam.width, H = a.cam.height;
    if (pix >= (int64_t)W * H) return;
    const int px = (int)(pix % W), py = (int)(pix / W);
    const CamDev &c = a.cam;
    // ray with unit view depth: d = R^T ((x - cx) / fx, (y - cy) / fy, 1)
    const double dc[3] = {((double)px + 0.5 - (double)c.cx) / (double)c.fx,
                          ((double)py + 0.5 - (double)c.cy) / (double)c.fy, 1.0};
    double d[3], o[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        d[r] = ((double)c.R[r] * dc[0] + (double)c.R[3 + r] * dc[1]) + (double)c.R[6 + r] * dc[2];
        o[r] = (double)c.C[r];
    }
    const float of[3] = {(float)o[0], (float)o[1], (float)o[2]};
    float id[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) id[r] = 1.0f / (float)d[r];
    const RayF rf = ray_f(o, d);
    const int64_t n = a.T;
    double T = 1.0, C0 = 0.0, C1 = 0.0, C2 = 0.0;
    double after_t = -1.0e300;
    int after_i = -1;
    for (int pass = 0; n > 0; ++pass) {
        Hit buf[kTraceKB];
        int nb = 0;
        bool more = false;
        int stack[kStack];
        int sp = 0;
        stack[sp++] = 0;
        // Boxes wholly before the last composited crossing hold nothing for this pass, and
        // boxes wholly beyond the farthest kept crossing of a full buffer only mean another
        // pass; both bounds are widened by 1e-5 relative, far above the slab test's rounding.
        const float t_after = after_t > 0.0 ? (float)after_t * (1.0f - 1e-5f) : 0.0f;
        while (sp > 0) {
            const int node = stack[--sp];
            const BvhNode &nd = a.nodes[node];
            float tn, tf;
            if (!box_span(nd, of, id, (float)c.znear * 0.999f, 3.0e38f, tn, tf)) continue;
            if (tf < t_after) continue;
            if (nb == kTraceKB && tn > (float)buf[kTraceKB - 1].t * (1.0f + 1e-5f)) {
                more = true;
                continue;
            }
            if (node >= n - 1) {
                const int tri = a.leaf_tri[node - (n - 1)];
                {
                    // crossings before the last composited one were taken in an earlier pass
                    float Pf[3][3];
                    tri_f(a, tri, Pf);
                    if (!mt_may_hit(rf, Pf[0], Pf[1], Pf[2], fmaxf(c.znear, (float)after_t), 3.0e38f)) continue;
                }
                int64_t v[3];
                double P[3][3], t, u, w;
                load_tri(a, tri, v, P);
                if (!(mt(o, d, P[0], P[1], P[2], t, u, w) && t > (double)c.znear)) continue;
                if (!hit_less(after_t, after_i, t, tri)) continue;   // composited in an earlier pass
                if (nb == kTraceKB) {
                    more = true;
                    if (!hit_less(t, tri, buf[kTraceKB - 1].t, buf[kTraceKB - 1].tri)) continue;
                    --nb;   // the farthest kept crossing waits for a later pass
                }
                int s = nb;
                while (s > 0 && hit_less(t, tri, buf[s - 1].t, buf[s - 1].tri)) {
                    buf[s] = buf[s - 1];
                    --s;
                }
                buf[s] = Hit{t, u, w, tri};
                ++nb;
                continue;
            }
            if (sp + 2 > kStack) {
                atomicAdd(a.overflow, 1u);
                continue;
            }
            stack[sp++] = nd.left;
            stack[sp++] = nd.right;
        }
        bool stop = false;
        for (int k = 0; k < nb; ++k) {
            const Hit &h = buf[k];
            int64_t v[3];
            tri_verts(a.tris, a.K, h.tri, v);
            const double w0 = 1.0 - h.u - h.v;
            const double al = w0 * __ldg(a.alpha + v[0]) + h.u * __ldg(a.alpha + v[1]) + h.v * __ldg(a.alpha + v[2]);
            double col[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                col[r] = w0 * __ldg(a.rgb + 3 * v[0] + r) + h.u * __ldg(a.rgb + 3 * v[1] + r) +
                         h.v * __ldg(a.rgb + 3 * v[2] + r);
            if (a.shadows) {
                const double p[3] = {o[0] + h.t * d[0], o[1] + h.t * d[1], o[2] + h.t * d[2]};
                const double f = a.ambient + (1.0 - a.ambient) * shadow(a, p, h.tri);
#pragma unroll
                for (int r = 0; r < 3; ++r) col[r] *= f;
            }
            C0 += T * al * col[0];
            C1 += T * al * col[1];
            C2 += T * al * col[2];
            T *= 1.0 - al;
            after_t = h.t;
            after_i = h.tri;
            if (T < a.T_eps) {
                stop = true;
                break;
            }
        }
        if (stop || !more) break;
    }
    float4 *out = reinterpret_cast<float4 *>(a.out);
    out[pix] = make_float4((float)(C0 + T * a.bg[0]), (float)(C1 + T * a.bg[1]), (float)(C2 + T * a.bg[2]),
                           (float)(1.0 - T));
}

unsigned grid_of(int64_t n, int threads) {
    return (unsigned)min64((n + threads - 1) / threads, (int64_t)32 * 152);
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" MS_API size_t ms_bvh_workspace_size(int64_t T) {
    if (T < 0) return 0;
    return bvh_layout(T).total;
}

extern "C" MS_API ms_status ms_bvh_build(const float *xyz, const int32_t *tris, int64_t T, int32_t K, void *bvh,
                                         size_t bvh_bytes, void *stream) {
    if (T < 0 || T >= (1ll << 31)) return set_error(MS_ERR_INVALID, "T outside 0 .. 2^31 - 1");
    if (!tris && (K < 3 || K > kMaxK || T % K)) return set_error(MS_ERR_INVALID, "implicit fans need K in 3..16 and T % K == 0");
    if (T > 0 && !xyz) return set_error(MS_ERR_INVALID, "xyz is NULL");
    const BvhLayout L = bvh_layout(T);
    if (!bvh || (reinterpret_cast<uintptr_t>(bvh) & 255) || bvh_bytes < L.total)
        return set_error(MS_ERR_INVALID, "BVH workspace NULL, misaligned or < %zu bytes", L.total);
    if (T == 0) return MS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char *b = static_cast<char *>(bvh);
    cudaError_t e = cudaMemsetAsync(b, 0, L.nodes, st);   // status and bounds
    if (e == cudaSuccess) e = cudaMemsetAsync(b + L.flags, 0, (size_t)T * 4, st);
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    unsigned *bounds = reinterpret_cast<unsigned *>(b + L.bounds);
    bounds_init_kernel<<<1, 32, 0, st>>>(bounds);
    centroid_bounds_kernel<<<grid_of(T, kBvhThreads), kBvhThreads, 0, st>>>(xyz, tris, K, T, bounds);
    unsigned long long *k0 = reinterpret_cast<unsigned long long *>(b + L.keys0);
    unsigned long long *k1 = reinterpret_cast<unsigned long long *>(b + L.keys1);
    morton_kernel<<<grid_of(T, kBvhThreads), kBvhThreads, 0, st>>>(xyz, tris, K, T, bounds, k0);
    unsigned long long *sorted = k0;
    e = sort_u64(k0, k1, T, 32, 4, b + L.scratch, st, &sorted);
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "BVH key sort: %s", cudaGetErrorString(e));
    BvhNode *nodes = reinterpret_cast<BvhNode *>(b + L.nodes);
    int *parent = reinterpret_cast<int *>(b + L.parent);
    int *leaf_tri = reinterpret_cast<int *>(b + L.leaf_tri);
    radix_tree_kernel<<<grid_of(T, kBvhThreads), kBvhThreads, 0, st>>>(sorted, T, nodes, parent, leaf_tri);
    bounds_up_kernel<<<grid_of(T, kBvhThreads), kBvhThreads, 0, st>>>(xyz, tris, K, T, nodes, parent, leaf_tri,
                                                                      reinterpret_cast<int *>(b + L.flags));
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "BVH build: %s", cudaGetErrorString(e));
    count_launches(5);
    return MS_OK;
}

extern "C" MS_API ms_status ms_raytrace(const float *xyz, const float *rgb, const float *alpha, const int32_t *tris,
                                        int64_t T, int32_t K, const void *bvh, const ms_camera *cam,
                                        const float *light, float ambient, float T_eps, const float *bg,
                                        float *out_rgba, void *stream) {
    if (T < 0 || T >= (1ll << 31)) return set_error(MS_ERR_INVALID, "T outside 0 .. 2^31 - 1");
    if (!tris && (K < 3 || K > kMaxK || T % K)) return set_error(MS_ERR_INVALID, "implicit fans need K in 3..16 and T % K == 0");
    if (!cam || !out_rgba || (T > 0 && (!xyz || !rgb || !alpha || !bvh)))
        return set_error(MS_ERR_INVALID, "NULL pointer");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 32768 || cam->height > 32768 || !(cam->znear > 0.0f))
        return set_error(MS_ERR_INVALID, "camera");
    if (!(ambient >= 0.0f && ambient <= 1.0f)) return set_error(MS_ERR_INVALID, "ambient outside [0, 1]");
    if (reinterpret_cast<uintptr_t>(out_rgba) & 15) return set_error(MS_ERR_INVALID, "out_rgba not 16-byte aligned");
    const BvhLayout L = bvh_layout(T);
    TraceArgs a;
    a.xyz = xyz;
    a.rgb = rgb;
    a.alpha = alpha;
    a.tris = tris;
    a.K = K;
    a.T = T;
    const char *b = static_cast<const char *>(bvh);
    a.nodes = T > 0 ? reinterpret_cast<const BvhNode *>(b + L.nodes) : nullptr;
    a.leaf_tri = T > 0 ? reinterpret_cast<const int *>(b + L.leaf_tri) : nullptr;
    a.overflow = T > 0 ? reinterpret_cast<unsigned *>(const_cast<char *>(b) + L.status) : nullptr;
    a.cam = make_cam(*cam);
    a.shadows = light != nullptr && ambient < 1.0f;
    for (int r = 0; r < 3; ++r) {
        a.L[r] = light ? (double)light[r] : 0.0;
        a.bg[r] = bg ? bg[r] : 0.0f;
    }
    a.ambient = ambient;
    a.T_eps = T_eps;
    a.out = out_rgba;
    const int64_t npx = (int64_t)cam->width * cam->height;
    trace_kernel<<<(unsigned)((npx + kTraceThreads - 1) / kTraceThreads), kTraceThreads, 0, (cudaStream_t)stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "trace_kernel: %s", cudaGetErrorString(e));
    count_launches(1);
    return MS_OK;
}

extern "C" MS_API ms_status ms_bvh_status(const void *bvh, int32_t *stack_overflows, void *stream) {
    if (!bvh || !stack_overflows) return set_error(MS_ERR_INVALID, "NULL pointer");
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, bvh, sizeof(unsigned), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "status read: %s", cudaGetErrorString(e));
    *stack_overflows = (int32_t)v;
    return v ? MS_ERR_CAPACITY : MS_OK;
}
