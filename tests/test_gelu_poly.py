"""The binary32 GELU of the tensor-core perceptron (csrc/mlp.cu with the polynomial of
csrc/gelu_poly.h) against the exact x Phi(x), on the host: the header is what the
generator writes, and the formula evaluated with binary32 roundings (fused multiply-adds
rounded once, the reciprocal and the exponential's argument rounded to binary32) stays
within 4e-6 relative of the exact GELU for x >= -5.6 and within 3e-5 further out, where
|GELU| < 1e-8."""
import importlib.util
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2502_07754_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_gelu_poly", os.path.join(CSRC, "gen_gelu_poly.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _header_coefficients():
    text = open(os.path.join(CSRC, "gelu_poly.h")).read()
    body = text[text.index("gelu_log2_g_m1"):]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    # Horner order: highest degree first
    return np.array(vals[::-1], dtype=np.float32)


def test_header_is_the_generators_output():
    np.testing.assert_array_equal(_header_coefficients(), _gen().coefficients())


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_binary32_gelu_is_within_4e6_of_exact():
    co = _header_coefficients()
    f32 = np.float32
    x = np.linspace(-14.0, 12.0, 1_000_001).astype(np.float32)
    z = (np.abs(x) * f32(0.70710678118654752)).astype(np.float32)
    t = (f32(1) / _fma32(z, np.full_like(z, 0.4), np.full_like(z, 1.0))).astype(np.float32)
    sv = _fma32(t, np.full_like(t, 2.0), np.full_like(t, -1.0))
    q = np.full_like(z, co[-1])
    for a in co[-2::-1]:
        q = _fma32(q, sv, np.full_like(z, a))
    zl = (z * f32(1.4426950408889634)).astype(np.float32)
    E = (t.astype(np.float64) * np.exp2(_fma32(-zl, z, q).astype(np.float64))).astype(np.float32)
    got = np.where(x >= 0, _fma32(-x, E, x), (x * E).astype(np.float32)).astype(np.float64)
    xd = x.astype(np.float64)
    exact = 0.5 * xd * scipy_special.erfc(-xd / np.sqrt(2.0))
    nz = np.abs(exact) > 1e-37
    rel = np.abs(got[nz] - exact[nz]) / np.abs(exact[nz])
    near = x[nz] >= -5.6
    assert rel[near].max() < 4e-6, rel[near].max()
    assert rel.max() < 3e-5, rel.max()
    assert np.all(np.abs(exact[~nz & (x < 0)]) < 1e-36)
    # the positive tail rounds to x, as the exact value does
    big = x > 6
    assert np.all(np.abs(got[big] - xd[big]) <= np.spacing(x[big].astype(np.float32)))
