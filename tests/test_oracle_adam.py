"""Pins of the oracle's fan optimiser step (oracle.fan_adam_step): Adam with the two
learning rates of Sec. 3 ("Optimization and Pruning": colours and opacities at lr_color,
vertex positions at exp(-3) lr_color) and the opacity kept in [0, 1].  Each expected value
is worked out by hand from Adam's moment recursions for gradients chosen so that the
bias-corrected moments come out as simple fractions; a swapped learning rate, a wrong or
missing bias correction, a wrong beta or a missing clamp fails one of them."""
import math

import numpy as np
import pytest

import oracle

LR = 5e-3
LR_XYZ = LR * math.exp(-3.0)


def _soup(V=4, seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(size=(V, 3)), rng.uniform(0.2, 0.8, (V, 3)), rng.uniform(0.2, 0.8, V)


def _run(grads_per_step, V=4):
    xyz, rgb, a = _soup(V)
    x0, c0, a0 = xyz.copy(), rgb.copy(), a.copy()
    m, v = np.zeros(7 * V), np.zeros(7 * V)
    for t, (gx, gc, ga) in enumerate(grads_per_step, start=1):
        oracle.fan_adam_step(xyz, rgb, a, gx, gc, ga, m, v, t, LR)
    return (xyz - x0, rgb - c0, a - a0)


def _signs(V=4, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = lambda *shape: np.where(rng.random(shape) < 0.5, -1.0, 1.0) * rng.uniform(0.5, 2.0, shape)
    return s(V, 3), s(V, 3), s(V)


def test_first_step_moves_each_parameter_by_its_learning_rate_against_the_gradient():
    # step 1: m_hat = g, v_hat = g^2, so the update is lr g / |g| (eps = 1e-15 is negligible)
    g = _signs()
    dx, dc, da = _run([g])
    assert np.allclose(dx, -LR_XYZ * np.sign(g[0]), rtol=1e-12, atol=0)
    assert np.allclose(dc, -LR * np.sign(g[1]), rtol=1e-12, atol=0)
    assert np.allclose(da, -LR * np.sign(g[2]), rtol=1e-12, atol=0)


def test_constant_gradient_moves_by_the_learning_rate_every_step():
    # the bias corrections 1 - b^t make m_hat = g and v_hat = g^2 at every step for a
    # constant gradient: three steps move each parameter by exactly 3 lr
    g = _signs()
    dx, dc, da = _run([g, g, g])
    assert np.allclose(dx, -3 * LR_XYZ * np.sign(g[0]), rtol=1e-12, atol=0)
    assert np.allclose(dc, -3 * LR * np.sign(g[1]), rtol=1e-12, atol=0)
    assert np.allclose(da, -3 * LR * np.sign(g[2]), rtol=1e-12, atol=0)


def test_reversed_gradient_on_step_two_gives_one_nineteenth():
    # g then -g: m_2 = 0.9 (0.1 g) - 0.1 g = -0.01 g, m_hat = -0.01 g / 0.19 = -g / 19;
    # v_2 = 0.999 (0.001 g^2) + 0.001 g^2 = 0.001999 g^2, v_hat = g^2: step 2 moves by
    # +lr / 19 along sign(g), after step 1 moved by -lr
    g = _signs()
    neg = tuple(-x for x in g)
    dx, dc, da = _run([g, neg])
    f = -1.0 + 1.0 / 19.0
    assert np.allclose(dx, f * LR_XYZ * np.sign(g[0]), rtol=1e-12, atol=0)
    assert np.allclose(dc, f * LR * np.sign(g[1]), rtol=1e-12, atol=0)
    assert np.allclose(da, f * LR * np.sign(g[2]), rtol=1e-12, atol=0)


def test_zero_gradient_on_step_two_uses_the_second_moment_decay():
    # g then 0: m_hat = 0.09 g / 0.19 = (9/19) g; v_hat = 0.000999 g^2 / 0.001999 =
    # (999/1999) g^2: step 2 moves by (9/19) / sqrt(999/1999) lr against sign(g)
    g = _signs()
    zero = tuple(np.zeros_like(x) for x in g)
    dx, dc, da = _run([g, zero])
    f = -(1.0 + (9.0 / 19.0) / math.sqrt(999.0 / 1999.0))
    assert np.allclose(dx, f * LR_XYZ * np.sign(g[0]), rtol=1e-12, atol=0)
    assert np.allclose(dc, f * LR * np.sign(g[1]), rtol=1e-12, atol=0)


def test_update_does_not_depend_on_the_gradient_scale():
    g = _signs()
    a = _run([g, tuple(0.3 * x for x in g)])
    b = _run([tuple(1e3 * x for x in g), tuple(3e2 * x for x in g)])
    for u, w in zip(a, b):
        assert np.allclose(u, w, rtol=1e-10, atol=0)


@pytest.mark.parametrize("start,grad,want", [(0.999, -1.0, 1.0), (0.001, 1.0, 0.0), (0.5, 1.0, 0.5 - LR)])
def test_opacity_is_clamped_to_the_unit_interval(start, grad, want):
    xyz, rgb = np.zeros((1, 3)), np.full((1, 3), 0.5)
    a = np.array([start])
    m, v = np.zeros(7), np.zeros(7)
    oracle.fan_adam_step(xyz, rgb, a, np.zeros((1, 3)), np.zeros((1, 3)), np.array([grad]), m, v, 1, LR)
    assert a[0] == pytest.approx(want, abs=1e-15)


def test_moments_use_the_optimiser_layout():
    # gradient only on vertex 2's y position: the first moment lands at entry 3*2+1 of the
    # xyz block and nowhere else; the opacity block starts at 6V
    V = 4
    xyz, rgb, a = _soup(V)
    m, v = np.zeros(7 * V), np.zeros(7 * V)
    gx = np.zeros((V, 3))
    gx[2, 1] = 2.0
    ga = np.zeros(V)
    ga[3] = -1.0
    oracle.fan_adam_step(xyz, rgb, a, gx, np.zeros((V, 3)), ga, m, v, 1, LR)
    want = np.zeros(7 * V)
    want[3 * 2 + 1] = 0.1 * 2.0
    want[6 * V + 3] = -0.1
    assert np.array_equal(m != 0, want != 0)
    assert np.allclose(m, want, rtol=1e-15, atol=0)
