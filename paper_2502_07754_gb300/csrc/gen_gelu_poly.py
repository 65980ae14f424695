"""Writes gelu_poly.h: the polynomial that the tensor-core perceptron's GELU uses for
erfc on z >= 0 in the form erfc(z) = t exp(-z^2) g(t), t = 1 / (1 + z / C) in (0, 1]
(g is smooth on [0, 1] and tends to C / sqrt(pi) as z grows).

log2 g(t) - 1 (the -1 makes the result erfc(z) / 2) is fitted by Chebyshev least squares
of degree DEG in s = 2 t - 1 on [-1, 1] to values from scipy.special.erfcx
(g(t) = erfcx(z) / t), converted to monomial coefficients in s and rounded to binary32.
Run it from this directory: python gen_gelu_poly.py > gelu_poly.h
"""
import numpy as np
from numpy.polynomial import chebyshev as C
from scipy.special import erfcx

DEG = 8
C_SCALE = 2.5


def coefficients():
    t = np.linspace(1e-6, 1.0, 400001)
    z = C_SCALE * (1.0 / t - 1.0)
    c = C.chebfit(2.0 * t - 1.0, np.log2(erfcx(z) / t), DEG)
    m = C.cheb2poly(c)
    m[0] -= 1.0
    return m.astype(np.float32)


def main():
    co = coefficients()
    print("// Generated by gen_gelu_poly.py: erfc(z) / 2 = t exp(-z^2) 2^G(s) for z >= 0, with")
    print("// t = 1 / (1 + z / %g), s = 2 t - 1 and G a polynomial of degree %d, evaluated by" % (C_SCALE, DEG))
    print("// Horner's rule in binary32.")
    print("#pragma once")
    print("namespace ms {")
    print("constexpr float kGeluInvC = %.9ef;   // 1 / %g" % (1.0 / C_SCALE, C_SCALE))
    print("__device__ __forceinline__ float gelu_log2_g_m1(float s) {")
    print("    float q = %.9ef;" % co[DEG])
    for i in range(DEG - 1, -1, -1):
        print("    q = fmaf(q, s, %.9ef);" % co[i])
    print("    return q;")
    print("}")
    print("}  // namespace ms")


if __name__ == "__main__":
    main()
