// Explicit triangles on the fan renderer, and the mesh-prior mode of Sec. 3.
//
// A triangle (v1, v2, v3) is drawn as a fan of K = 3 around its centroid c, whose colour
// and opacity are the means of the vertices': the three sub-triangles (c, v_i, v_i+1)
// tile the triangle (the spokes from c are shared inside the fan, so no centre is covered
// twice), and a perspective-correct interpolation of attributes that are affine on the
// triangle reproduces them on every sub-triangle.  The centroid is the binary32 value
// nearest to the exact mean of the three binary32 positions (their sum is formed exactly
// in double-float).  The adjoint of the conversion gives every vertex its own fan
// vertex's gradient plus a third of the centroid's.
//
// Mesh prior (Sec. 3, the mesh-prior paragraphs): every face (m1, m2, m3) of a geometry
// mesh carries S secondary triangles with vertices v_i = sum_k a_ik m_k, a_i on the
// simplex, kept there by the parameterisation a_ik = w_ik^2 / sum_j w_ij^2 of free weights
// w, and trainable per-vertex colour and opacity.  The builder writes the secondary
// triangles as centroid fans; the backward folds the fan gradients to the vertices and
// through v(a(w)) to the weights:
//   dL/da_ik = dL/dv_i . m_k,   dL/dw_ij = (2 w_ij / Q_i)(dL/da_ij - sum_k a_ik dL/da_ik),
//   Q_i = sum_j w_ij^2.
#include "ms_common.cuh"
#include "ms_internal.h"

namespace ms {

namespace {

constexpr int kTriThreads = 256;

// Nearest binary32 value of (a + b + c) / 3 for binary32 a, b, c.
__device__ __forceinline__ float centroid3(float a, float b, float c) {
    const dfl s = df_add_f(df_two_sum(a, b), c);
    return df_round(df_div_rcp(s, df_make(3.0f)));
}

__device__ __forceinline__ void put_fan(int64_t t, const float p[3][3], const float col[3][3], const float al[3],
                                        float *__restrict__ fx, float *__restrict__ fc, float *__restrict__ fa) {
    const int64_t v0 = 4 * t;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        fx[3 * v0 + r] = centroid3(p[0][r], p[1][r], p[2][r]);
        fc[3 * v0 + r] = centroid3(col[0][r], col[1][r], col[2][r]);
    }
    fa[v0] = centroid3(al[0], al[1], al[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            fx[3 * (v0 + 1 + k) + r] = p[k][r];
            fc[3 * (v0 + 1 + k) + r] = col[k][r];
        }
        fa[v0 + 1 + k] = al[k];
    }
}

__global__ void __launch_bounds__(kTriThreads) tris_to_fans_kernel(const float *__restrict__ xyz,
                                                                   const float *__restrict__ rgb,
                                                                   const float *__restrict__ alpha,
                                                                   const int32_t *__restrict__ tris, int64_t T,
                                                                   float *__restrict__ fx, float *__restrict__ fc,
                                                                   float *__restrict__ fa) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        float p[3][3], col[3][3], al[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int64_t v = tris ? (int64_t)__ldg(tris + 3 * t + k) : 3 * t + k;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                p[k][r] = __ldg(xyz + 3 * v + r);
                col[k][r] = __ldg(rgb + 3 * v + r);
            }
            al[k] = __ldg(alpha + v);
        }
        put_fan(t, p, col, al, fx, fc, fa);
    }
}

// Gradient of fan vertex u (0 = centroid) of triangle t: from three arrays, or from the
// render workspace's sums (two float4 per vertex: (xyz, alpha), (rgb, 0)).
struct FanGrad {
    const float *gx, *gc, *ga;
    const float4 *ws;
    __device__ __forceinline__ void get(int64_t v, float g[7]) const {
        if (ws) {
            const float4 a = ws[2 * v], b = ws[2 * v + 1];
            g[0] = a.x; g[1] = a.y; g[2] = a.z; g[6] = a.w;
            g[3] = b.x; g[4] = b.y; g[5] = b.z;
        } else {
            g[0] = gx[3 * v]; g[1] = gx[3 * v + 1]; g[2] = gx[3 * v + 2];
            g[3] = gc[3 * v]; g[4] = gc[3 * v + 1]; g[5] = gc[3 * v + 2];
            g[6] = ga[v];
        }
    }
};

// Adjoint of tris_to_fans: vertex k of triangle t receives fan vertex 1 + k's gradient and a
// third of the centroid's, added with atomics (a vertex may belong to several triangles).
__global__ void __launch_bounds__(kTriThreads) fans_to_tris_kernel(FanGrad fg, const int32_t *__restrict__ tris,
                                                                   int64_t T, float *__restrict__ dx,
                                                                   float *__restrict__ dc, float *__restrict__ da) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        float gc0[7];
        fg.get(4 * t, gc0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float g[7];
            fg.get(4 * t + 1 + k, g);
            const int64_t v = tris ? (int64_t)__ldg(tris + 3 * t + k) : 3 * t + k;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                atomicAdd(dx + 3 * v + r, g[r] + gc0[r] * (1.0f / 3.0f));
                atomicAdd(dc + 3 * v + r, g[3 + r] + gc0[3 + r] * (1.0f / 3.0f));
            }
            atomicAdd(da + v, g[6] + gc0[6] * (1.0f / 3.0f));
        }
    }
}

// Secondary triangle (face f, index s) of the mesh prior: vertex i at
// sum_k a_ik m_k with a_ik = w_ik^2 / sum_j w_ij^2.
__device__ __forceinline__ void prior_vertices(const float *__restrict__ faces, const float *__restrict__ w, int64_t f,
                                               int64_t fs, float p[3][3], float a[3][3]) {
    float m[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r) m[k][r] = __ldg(faces + 9 * f + 3 * k + r);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float q[3], Q = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float wk = __ldg(w + 9 * fs + 3 * i + k);
            q[k] = wk * wk;
            Q += q[k];
        }
        const float iQ = 1.0f / Q;
#pragma unroll
        for (int k = 0; k < 3; ++k) a[i][k] = q[k] * iQ;
#pragma unroll
        for (int r = 0; r < 3; ++r) p[i][r] = a[i][0] * m[0][r] + a[i][1] * m[1][r] + a[i][2] * m[2][r];
    }
}

__global__ void __launch_bounds__(kTriThreads) prior_build_kernel(const float *__restrict__ faces,
                                                                  const float *__restrict__ w,
                                                                  const float *__restrict__ rgb,
                                                                  const float *__restrict__ alpha, int64_t F, int S,
                                                                  float *__restrict__ fx, float *__restrict__ fc,
                                                                  float *__restrict__ fa) {
    const int64_t T = F * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        float p[3][3], a[3][3], col[3][3], al[3];
        prior_vertices(faces, w, t / S, t, p, a);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int r = 0; r < 3; ++r) col[k][r] = __ldg(rgb + 9 * t + 3 * k + r);
            al[k] = __ldg(alpha + 3 * t + k);
        }
        put_fan(t, p, col, al, fx, fc, fa);
    }
}

// Mesh-prior adjoint: fan gradients -> vertex gradients (centroid split in thirds) ->
// weight gradients; colour and opacity gradients go to the per-vertex attributes.  Each
// secondary triangle is one thread and owns its weights and attributes (no atomics).
__global__ void __launch_bounds__(kTriThreads) prior_backward_kernel(FanGrad fg, const float *__restrict__ faces,
                                                                     const float *__restrict__ w, int64_t F, int S,
                                                                     float *__restrict__ dw, float *__restrict__ drgb,
                                                                     float *__restrict__ dalpha) {
    const int64_t T = F * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / S;
        float gc0[7];
        fg.get(4 * t, gc0);
        float m[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int r = 0; r < 3; ++r) m[k][r] = __ldg(faces + 9 * f + 3 * k + r);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float g[7];
            fg.get(4 * t + 1 + i, g);
            float gv[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                gv[r] = g[r] + gc0[r] * (1.0f / 3.0f);
                drgb[9 * t + 3 * i + r] += g[3 + r] + gc0[3 + r] * (1.0f / 3.0f);
            }
            dalpha[3 * t + i] += g[6] + gc0[6] * (1.0f / 3.0f);
            float wv[3], q[3], Q = 0.0f, ga[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                wv[k] = __ldg(w + 9 * t + 3 * i + k);
                q[k] = wv[k] * wv[k];
                Q += q[k];
                ga[k] = gv[0] * m[k][0] + gv[1] * m[k][1] + gv[2] * m[k][2];
            }
            const float iQ = 1.0f / Q;
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) s += q[k] * iQ * ga[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) dw[9 * t + 3 * i + k] += 2.0f * wv[k] * iQ * (ga[k] - s);
        }
    }
}

unsigned grid_for(int64_t n) { return (unsigned)min64((n + kTriThreads - 1) / kTriThreads, 16 * 152); }

size_t fan_soup_bytes(int64_t T) { return (size_t)(4 * T) * 7 * sizeof(float); }

}  // namespace
}  // namespace ms

using namespace ms;

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

ms_status check_tris(const float *xyz, const float *rgb, const float *alpha, int64_t T, int64_t V) {
    if (T < 0 || V < 0) return set_error(MS_ERR_INVALID, "negative size");
    if (4 * T * 1 >= (1ll << 31)) return set_error(MS_ERR_INVALID, "too many triangles");
    if (T > 0 && (!xyz || !rgb || !alpha)) return set_error(MS_ERR_INVALID, "NULL vertex array");
    return MS_OK;
}

ms_status launched(const char *what, int n) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    count_launches(n);
    return MS_OK;
}

// Fan soup sections of an explicit-mesh workspace (4 T vertices): xyz, rgb, alpha, then
// the render workspace at a 256-byte boundary.
struct MeshWs {
    float *fx, *fc, *fa;
    char *rws;
    size_t rbytes;
};
MeshWs mesh_ws(void *ws, size_t bytes, int64_t T) {
    char *b = static_cast<char *>(ws);
    MeshWs m;
    m.fx = reinterpret_cast<float *>(b);
    m.fc = m.fx + 12 * T;
    m.fa = m.fc + 12 * T;
    const size_t soup = align256(fan_soup_bytes(T));
    m.rws = b + soup;
    m.rbytes = bytes > soup ? bytes - soup : 0;
    return m;
}

}  // namespace

extern "C" MS_API ms_status ms_tris_to_fans(const float *xyz, const float *rgb, const float *alpha,
                                            const int32_t *tris, int64_t T, float *fan_xyz, float *fan_rgb,
                                            float *fan_alpha, void *stream) {
    ms_status s = check_tris(xyz, rgb, alpha, T, 0);
    if (s != MS_OK) return s;
    if (T == 0) return MS_OK;
    if (!fan_xyz || !fan_rgb || !fan_alpha) return set_error(MS_ERR_INVALID, "NULL fan array");
    tris_to_fans_kernel<<<grid_for(T), kTriThreads, 0, (cudaStream_t)stream>>>(xyz, rgb, alpha, tris, T, fan_xyz,
                                                                               fan_rgb, fan_alpha);
    return launched("tris_to_fans_kernel", 1);
}

extern "C" MS_API ms_status ms_fans_to_tris_grads(const float *g_fan_xyz, const float *g_fan_rgb,
                                                  const float *g_fan_alpha, const void *grad_ws, const int32_t *tris,
                                                  int64_t T, float *d_xyz, float *d_rgb, float *d_alpha,
                                                  void *stream) {
    if (T < 0) return set_error(MS_ERR_INVALID, "T < 0");
    if (T == 0) return MS_OK;
    if (!d_xyz || !d_rgb || !d_alpha) return set_error(MS_ERR_INVALID, "NULL gradient output");
    if (!grad_ws && (!g_fan_xyz || !g_fan_rgb || !g_fan_alpha)) return set_error(MS_ERR_INVALID, "NULL fan gradient");
    if (grad_ws && (reinterpret_cast<uintptr_t>(grad_ws) & 15))
        return set_error(MS_ERR_INVALID, "grad_ws not 16-byte aligned");
    FanGrad fg{g_fan_xyz, g_fan_rgb, g_fan_alpha, static_cast<const float4 *>(grad_ws)};
    fans_to_tris_kernel<<<grid_for(T), kTriThreads, 0, (cudaStream_t)stream>>>(fg, tris, T, d_xyz, d_rgb, d_alpha);
    return launched("fans_to_tris_kernel", 1);
}

extern "C" MS_API size_t ms_mesh_workspace_size(int64_t T, const ms_camera *cam, const ms_render_params *params) {
    if (T < 0) return 0;
    const size_t r = ms_render_workspace_size(T, 3, cam, params);
    if (r == 0) return 0;
    return align256(fan_soup_bytes(T)) + r;
}

extern "C" MS_API ms_status ms_mesh_render(const float *xyz, const float *rgb, const float *alpha,
                                           const int32_t *tris, int64_t T, const ms_camera *cam,
                                           const ms_render_params *params, float *out_rgba, void *workspace,
                                           size_t ws_bytes, void *stream) {
    ms_status s = check_tris(xyz, rgb, alpha, T, 0);
    if (s != MS_OK) return s;
    const size_t need = ms_mesh_workspace_size(T, cam, params);
    if (need == 0) return set_error(MS_ERR_INVALID, "invalid render configuration");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return set_error(MS_ERR_INVALID, "workspace NULL or not 256-byte aligned");
    if (ws_bytes < need) return set_error(MS_ERR_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, need);
    const MeshWs m = mesh_ws(workspace, ws_bytes, T);
    s = ms_tris_to_fans(xyz, rgb, alpha, tris, T, m.fx, m.fc, m.fa, stream);
    if (s != MS_OK) return s;
    return ms_render(m.fx, m.fc, m.fa, T, 3, cam, params, out_rgba, m.rws, m.rbytes, stream);
}

extern "C" MS_API ms_status ms_mesh_render_backward(const float *xyz, const float *rgb, const float *alpha,
                                                    const int32_t *tris, int64_t T, const ms_camera *cam,
                                                    const ms_render_params *params, const float *out_rgba,
                                                    const float *dL_drgba, float *d_xyz, float *d_rgb, float *d_alpha,
                                                    void *workspace, size_t ws_bytes, void *stream) {
    ms_status s = check_tris(xyz, rgb, alpha, T, 0);
    if (s != MS_OK) return s;
    const size_t need = ms_mesh_workspace_size(T, cam, params);
    if (need == 0 || !workspace || ws_bytes < need) return set_error(MS_ERR_INVALID, "workspace too small or NULL");
    if (T == 0) return MS_OK;
    const MeshWs m = mesh_ws(workspace, ws_bytes, T);
    s = ms_render_backward(m.fx, m.fc, m.fa, T, 3, cam, params, out_rgba, dL_drgba, nullptr, nullptr, nullptr, m.rws,
                           m.rbytes, stream);
    if (s != MS_OK) return s;
    const size_t off = ms_render_grad_offset(T, 3, cam, 1, params);
    return ms_fans_to_tris_grads(nullptr, nullptr, nullptr, m.rws + off, tris, T, d_xyz, d_rgb, d_alpha, stream);
}

extern "C" MS_API ms_status ms_mesh_prior_build(const float *faces, const float *w, const float *rgb,
                                                const float *alpha, int64_t F, int32_t S, float *fan_xyz,
                                                float *fan_rgb, float *fan_alpha, void *stream) {
    if (F < 0 || S < 1) return set_error(MS_ERR_INVALID, "F < 0 or S < 1");
    if (F == 0) return MS_OK;
    if (!faces || !w || !rgb || !alpha || !fan_xyz || !fan_rgb || !fan_alpha)
        return set_error(MS_ERR_INVALID, "NULL pointer");
    if (4 * F * (int64_t)S >= (1ll << 31)) return set_error(MS_ERR_INVALID, "too many secondary triangles");
    prior_build_kernel<<<grid_for(F * S), kTriThreads, 0, (cudaStream_t)stream>>>(faces, w, rgb, alpha, F, S, fan_xyz,
                                                                                  fan_rgb, fan_alpha);
    return launched("prior_build_kernel", 1);
}

extern "C" MS_API ms_status ms_mesh_prior_backward(const float *faces, const float *w, const float *g_fan_xyz,
                                                   const float *g_fan_rgb, const float *g_fan_alpha,
                                                   const void *grad_ws, int64_t F, int32_t S, float *d_w,
                                                   float *d_rgb, float *d_alpha, void *stream) {
    if (F < 0 || S < 1) return set_error(MS_ERR_INVALID, "F < 0 or S < 1");
    if (F == 0) return MS_OK;
    if (!faces || !w || !d_w || !d_rgb || !d_alpha) return set_error(MS_ERR_INVALID, "NULL pointer");
    if (!grad_ws && (!g_fan_xyz || !g_fan_rgb || !g_fan_alpha)) return set_error(MS_ERR_INVALID, "NULL fan gradient");
    if (grad_ws && (reinterpret_cast<uintptr_t>(grad_ws) & 15))
        return set_error(MS_ERR_INVALID, "grad_ws not 16-byte aligned");
    FanGrad fg{g_fan_xyz, g_fan_rgb, g_fan_alpha, static_cast<const float4 *>(grad_ws)};
    prior_backward_kernel<<<grid_for(F * S), kTriThreads, 0, (cudaStream_t)stream>>>(fg, faces, w, F, S, d_w, d_rgb,
                                                                                     d_alpha);
    return launched("prior_backward_kernel", 1);
}
