"""Pins of the oracle's tabulated-function spline (EAM tables).

The cubic Hermite spline with 3-point knot slopes reproduces every
quadratic exactly (3-point differences are exact for quadratics, and a cubic
Hermite piece with exact values and slopes reproduces any cubic); for a
smooth function its error falls as h^3 or faster.
"""
import numpy as np
import pytest


def test_slopes_exact_for_quadratic(ora):
    h = 0.013
    xk = np.arange(200) * h
    y = 3.0 * xk ** 2 - 2.0 * xk + 0.5
    m = ora.spline_slopes(y, h)
    np.testing.assert_allclose(m, 6.0 * xk - 2.0, rtol=0, atol=1e-9)


def test_quadratic_reproduced_exactly(ora):
    rng = np.random.default_rng(5)
    h = 0.01
    n = 400
    xk = np.arange(n) * h
    y = -1.5 * xk ** 2 + 0.25 * xk + 2.0
    xs = rng.uniform(0.0, (n - 1) * h, size=2000)
    val, der = ora.spline_eval(y, h, xs)
    np.testing.assert_allclose(val, -1.5 * xs ** 2 + 0.25 * xs + 2.0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(der, -3.0 * xs + 0.25, rtol=1e-10, atol=1e-10)


def test_knots_interpolated(ora):
    rng = np.random.default_rng(6)
    y = rng.normal(size=50)
    h = 0.1
    xs = np.arange(50) * h
    val, _ = ora.spline_eval(y, h, xs)
    np.testing.assert_allclose(val, y, rtol=0, atol=1e-13)


def test_error_order_smooth_function(ora):
    """max error on exp(-x) over [0, 4] shrinks by >= 2^3 per halving of h."""
    errs = []
    for n in (101, 201, 401):
        h = 4.0 / (n - 1)
        xk = np.arange(n) * h
        xs = np.linspace(0.0, 4.0, 3001)
        val, der = ora.spline_eval(np.exp(-xk), h, xs)
        errs.append(np.max(np.abs(val - np.exp(-xs))))
    assert errs[0] / errs[1] > 7.0
    assert errs[1] / errs[2] > 7.0


def test_last_interval_used_at_right_end(ora):
    h = 0.5
    y = np.array([0.0, 1.0, 4.0, 9.0])          # x^2 at 0, .5, 1, 1.5 scaled by 4
    val, der = ora.spline_eval(y, h, np.array([1.5]))
    assert val[0] == pytest.approx(9.0, abs=1e-14)
