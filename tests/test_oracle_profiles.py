"""Pins of the oracle's Appendix statistics (per-bin profiles).

* Uniform velocity: COM velocity equals it, temperatures are 0.
* Mass and atom counts add up to the totals.
* A single bin over a thermal system: T = 2 K / (3 k_B N) with K the kinetic
  energy in the centre-of-mass frame, i.e. the Maxwell generator's exact T
  for 3N - 3 degrees of freedom times (3N-3)/(3N).
* Pressure of a perfect lattice at rest in one bin equals W/V of the LJ
  virial, so the Appendix P_l reduces to the virial pressure.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W


def test_uniform_velocity(ora):
    x = W.fcc_lattice(4, 4, 10, 4.05)
    n = x.shape[0]
    v = np.tile([0.01, -0.002, 0.003], (n, 1))
    m = np.full(n, W.MASS_AL)
    out = ora.profiles(x, v, m, 2, 0.0, 4.05, 10, (4 * 4.05) ** 2)
    np.testing.assert_allclose(out[:, 2:5], np.tile(v[0], (10, 1)), rtol=1e-13)
    np.testing.assert_allclose(out[:, 5:8], 0.0, atol=1e-20)
    assert out[:, 0].sum() == n
    assert out[:, 1].sum() == pytest.approx(m.sum(), rel=1e-14)


def test_single_bin_temperature(ora):
    rng = np.random.default_rng(0)
    x = W.fcc_lattice(4, 4, 4, 5.26)
    n = x.shape[0]
    m = np.full(n, W.MASS_AR)
    v = W.maxwell_velocities(rng, m, 120.0)
    out = ora.profiles(x, v, m, 0, 0.0, 100.0, 1, 21.04 ** 2)
    T = out[0, 5:8].mean()
    assert T == pytest.approx(120.0 * (3 * n - 3) / (3 * n), rel=1e-12)


def test_pressure_is_virial_pressure_at_rest(ora):
    a, nc = 5.26, 4
    x = W.fcc_lattice(nc, nc, nc, a) * 0.97
    L = nc * a * 0.97
    lj = W.LJ_AR
    r = ora.lj(x, [0] * 3, [L] * 3, [1, 1, 1], lj.eps, lj.sigma, lj.rc, 1, per_atom=True)
    n = x.shape[0]
    out = ora.profiles(x, np.zeros((n, 3)), np.full(n, lj.mass), 0, 0.0, L, 1, L * L,
                       Ua=r["Ea"], Wa=r["Wa"])
    np.testing.assert_allclose(out[0, 9:15], r["W"] / L ** 3, rtol=1e-12, atol=1e-18)
    assert out[0, 8] == pytest.approx(r["E"], rel=1e-12)
