"""The binary32 GELU of the tensor-core perceptron (csrc/mlp.cu with the polynomial of
csrc/gelu_poly.h) against the exact x Phi(x), on the host: the header is what the
generator writes, and the formula evaluated with binary32 roundings (fused multiply-adds
rounded once, the reciprocal and the exponential's argument rounded to binary32) stays
within 3e-6 relative of the exact GELU for x >= -5.6 and within 1.2e-5 further out, where
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
    body = text[text.index("#define MS_GELU_POLY"):].splitlines()[0]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals, dtype=np.float32)   # coefficients of t^0, t^1, ...


def test_header_is_the_generators_output():
    np.testing.assert_array_equal(_header_coefficients(), _gen().coefficients())


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_binary32_gelu_is_within_3e6_of_exact():
    co = _header_coefficients()
    f32 = np.float32
    x = np.linspace(-14.0, 12.0, 1_000_001).astype(np.float32)
    t = (f32(1) / _fma32(np.abs(x), np.full_like(x, 0.35355339059327376), np.full_like(x, 1.0))).astype(np.float32)
    q = np.full_like(x, co[-1])
    for a in co[-2::-1]:
        q = _fma32(q, t, np.full_like(x, a))
    xx = (x * x).astype(np.float32)
    arg = _fma32(xx, np.full_like(x, -0.72134752044448170), q)
    E = (t * np.exp2(arg.astype(np.float64)).astype(np.float32)).astype(np.float32)
    step = (x >= 0).astype(np.float32)
    phi = _fma32(_fma32(step, np.full_like(x, -2.0), np.full_like(x, 1.0)), E, step)
    got = (x * phi).astype(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    exact = 0.5 * xd * scipy_special.erfc(-xd / np.sqrt(2.0))
    nz = np.abs(exact) > 1e-37
    rel = np.abs(got[nz] - exact[nz]) / np.abs(exact[nz])
    near = x[nz] >= -5.6
    assert rel[near].max() < 3e-6, rel[near].max()
    assert rel.max() < 1.2e-5, rel.max()
    assert np.all(np.abs(exact[~nz & (x < 0)]) < 1e-36)
    # the positive tail rounds to x, as the exact value does
    big = x > 6
    assert np.all(np.abs(got[big] - xd[big]) <= np.spacing(x[big].astype(np.float32)))
