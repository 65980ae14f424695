// Generated by gen_gelu_poly.py: erfc(z) / 2 = t exp(-z^2) 2^G(t) for z >= 0, with
// t = 1 / (1 + z / 2) and G the polynomial of degree 7 below (coefficients of
// t^0 .. t^7), evaluated by Horner's rule in binary32.
#pragma once
namespace ms {
constexpr int kGeluDeg = 7;
constexpr float kGeluInvC = 5.000000000e-01f;   // 1 / 2
#define MS_GELU_POLY -2.825737238e+00f, 1.441846490e+00f, 5.572204590e-01f, -9.010969661e-03f, 3.942742646e-01f, -1.306002736e+00f, 9.950978160e-01f, -2.476870716e-01f
}  // namespace ms
