// Generated by gen_gelu_poly.py: erfc(z) / 2 = t exp(-z^2) 2^G(s) for z >= 0, with
// t = 1 / (1 + z / 2.5), s = 2 t - 1 and G a polynomial of degree 8, evaluated by
// Horner's rule in binary32.
#pragma once
namespace ms {
constexpr float kGeluInvC = 4.000000000e-01f;   // 1 / 2.5
__device__ __forceinline__ float gelu_log2_g_m1(float s) {
    float q = -9.028298664e-04f;
    q = fmaf(q, s, 8.464116254e-04f);
    q = fmaf(q, s, 6.369955838e-03f);
    q = fmaf(q, s, -2.307655988e-03f);
    q = fmaf(q, s, -3.418095037e-02f);
    q = fmaf(q, s, -2.606458962e-02f);
    q = fmaf(q, s, 2.008841634e-01f);
    q = fmaf(q, s, 1.101366639e+00f);
    q = fmaf(q, s, -2.246009350e+00f);
    return q;
}
}  // namespace ms
