"""Host logic of the stationary-shock search (Sec. "Moving window
simulation"): least-squares slope of F(t) and the bisection on its sign."""
import numpy as np
import pytest

from paper_2511_22951_gb300 import shock


def test_lsq_slope_is_the_least_squares_line():
    rng = np.random.default_rng(0)
    t = np.linspace(0, 10, 30)
    f = 1.0 + 0.37 * t
    assert shock.lsq_slope(t, f) == pytest.approx(0.37, rel=1e-12)
    f2 = f + rng.normal(0, 0.1, t.size)
    assert shock.lsq_slope(t, f2) == pytest.approx(np.polyfit(t, f2, 1)[0], rel=1e-10)
    with pytest.raises(ValueError):
        shock.lsq_slope([1.0, 1.0], [0.0, 1.0])


def test_dichotomy_finds_the_root_to_1_m_per_s():
    u_star = -0.0123456
    calls = []

    def slope(u):
        calls.append(u)
        return 3.0 * (u - u_star)  # monotonic near the optimum

    u, hist = shock.dichotomy(slope, -0.03, 0.0)
    assert abs(u - u_star) < shock.M_PER_S
    assert len(hist) == len(calls)
    # the bracket halves each time: ~log2(0.03 / 1e-5) evaluations
    assert len(calls) <= 2 + int(np.ceil(np.log2(0.03 / shock.M_PER_S))) + 1


def test_dichotomy_needs_a_sign_change():
    with pytest.raises(ValueError):
        shock.dichotomy(lambda u: 1.0 + u * u, -1.0, 1.0)
