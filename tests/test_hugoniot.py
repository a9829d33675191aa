"""Host analysis of the Hugoniot from an isotherm grid (Sec. "Argon shock
Hugoniot", Eq. RH), pinned on a monatomic ideal gas: e = 3/2 k T and
P = k T / v are linear in T, so the interpolation along each volume line is
exact and the grid must return the closed-form Hugoniot
T_H = T0 (3/2 + (v0 - v) / (2 v0)) / (3/2 - (v0 - v) / (2 v)),
i.e. P_H / P0 = (4 v0 - v) / (4 v - v0) for gamma = 5/3."""
import numpy as np
import pytest

from paper_2511_22951_gb300 import hugoniot as H

K = 8.617333262e-5


def ideal_grid(v0=40.0, T0=300.0):
    V = v0 * np.array([1.0, 0.9, 0.8, 0.7, 0.6, 0.5, 0.4, 0.3])
    T = np.geomspace(T0, 1e5, 25)
    E = 1.5 * K * np.repeat(T[None, :], V.size, 0)
    P = K * T[None, :] / V[:, None]
    return V, T, E, P, v0, 1.5 * K * T0, K * T0 / v0


def test_ideal_gas_hugoniot_is_exact():
    V, T, E, P, v0, e0, p0 = ideal_grid()
    v, TH, PH, EH = H.hugoniot_from_grid(V, T, E, P, v0, e0, p0)
    assert v.size == V.size  # every line brackets its root (the v0 line at T0)
    T0 = 300.0
    want_T = T0 * (1.5 + 0.5 * (v0 - v) / v0) / (1.5 - 0.5 * (v0 - v) / v)
    np.testing.assert_allclose(TH, want_T, rtol=1e-12)
    np.testing.assert_allclose(PH / p0, (4 * v0 - v) / (4 * v - v0), rtol=1e-12)
    np.testing.assert_allclose(H.rankine_hugoniot(EH, PH, v, e0, p0, v0), 0.0, atol=1e-15)


def test_lines_without_a_root_are_skipped():
    V, T, E, P, v0, e0, p0 = ideal_grid()
    # the gamma = 5/3 gas cannot be compressed beyond v0 / 4
    V2 = np.append(V, 0.2 * v0)
    E2 = np.vstack([E, E[-1:]])
    P2 = np.vstack([P, K * T[None, :] / V2[-1]])
    v, *_ = H.hugoniot_from_grid(V2, T, E2, P2, v0, e0, p0)
    assert 0.2 * v0 not in v


def test_paper_time_step():
    assert H.paper_dt(1e5) == pytest.approx(0.1)       # 1e-2 sqrt(1e-4) ps
    assert H.paper_dt(10.0) == pytest.approx(10.0)
