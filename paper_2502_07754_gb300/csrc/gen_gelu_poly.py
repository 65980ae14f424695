"""Writes gelu_poly.h: the polynomial that the tensor-core perceptron's GELU uses for
erfc on z >= 0 in the form erfc(z) = t exp(-z^2) g(t), t = 1 / (1 + z / C) in (0, 1]
(g is smooth on [0, 1] and tends to C / sqrt(pi) as z grows).

log2 g(t) - 1 (the -1 makes the result erfc(z) / 2) is fitted by Chebyshev least squares
of degree DEG on t in [0, 1] to values from scipy.special.erfcx (g(t) = erfcx(z) / t),
converted to monomial coefficients in t and rounded to binary32.
Run it from this directory: python gen_gelu_poly.py > gelu_poly.h
"""
import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as P
from scipy.special import erfcx

DEG = 7
C_SCALE = 2.0


def coefficients():
    t = np.linspace(1e-6, 1.0, 400001)
    z = C_SCALE * (1.0 / t - 1.0)
    c = C.chebfit(2.0 * t - 1.0, np.log2(erfcx(z) / t), DEG)
    m = P.Polynomial(C.cheb2poly(c))(P.Polynomial([-1.0, 2.0])).coef   # s = 2 t - 1
    m[0] -= 1.0
    return m.astype(np.float32)


def main():
    co = coefficients()
    print("// Generated by gen_gelu_poly.py: erfc(z) / 2 = t exp(-z^2) 2^G(t) for z >= 0, with")
    print("// t = 1 / (1 + z / %g) and G the polynomial of degree %d below (coefficients of" % (C_SCALE, DEG))
    print("// t^0 .. t^%d), evaluated by Horner's rule in binary32." % DEG)
    print("#pragma once")
    print("namespace ms {")
    print("constexpr int kGeluDeg = %d;" % DEG)
    print("constexpr float kGeluInvC = %.9ef;   // 1 / %g" % (1.0 / C_SCALE, C_SCALE))
    print("#define MS_GELU_POLY %s" % ", ".join("%.9ef" % a for a in co))
    print("}  // namespace ms")


if __name__ == "__main__":
    main()
