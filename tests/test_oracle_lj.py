"""Pins of the oracle's Lennard-Jones energy, force and virial.

* Perfect FCC lattice: E/N = 1/2 sum_k z_k [u(d sqrt k) - u(rc)] (shell sum),
  F = 0.
* Large cutoff, unshifted, plus the uniform-density tail: the textbook FCC
  lattice sums E/N = 2 eps [A12 (sigma/d)^12 - A6 (sigma/d)^6],
  A12 = 12.13188, A6 = 14.45392.
* Dimer: analytic u(r) and u'(r).
* -dE/dx by central differences; sum F = 0; translation invariance.
* Virial pressure of the perfect lattice equals -dU/dV of the shell sum.
* Shifted force (shift_mode 2): dimer closed form u(r) - u(rc) - (r - rc) u'(rc)
  and its force, lattice shell sum, central differences.
"""
import numpy as np
import pytest

from fcc_shells import fcc_shells
from paper_2511_22951_gb300 import workloads as W

EPS, SIG = 0.0104, 3.405
RC = 2.5 * SIG


def u_lj(r):
    s6 = (SIG / r) ** 6
    return 4 * EPS * (s6 * s6 - s6)


def du_lj(r):
    s6 = (SIG / r) ** 6
    return -24 * EPS * (2 * s6 * s6 - s6) / r


def shell_energy(a, rc, shifted=True):
    d, z = fcc_shells(a, rc)
    return 0.5 * np.sum(z * (u_lj(d) - (u_lj(rc) if shifted else 0.0)))


def lattice(a=5.26, n=4):
    x = W.fcc_lattice(n, n, n, a)
    L = n * a
    return x, np.zeros(3), np.full(3, L)


def test_perfect_lattice_energy_and_zero_force(ora):
    x, lo, hi = lattice()
    for mode, shifted in ((1, True), (0, False)):
        r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, RC, mode)
        e_ref = shell_energy(5.26, RC, shifted)
        assert r["E"] / x.shape[0] == pytest.approx(e_ref, rel=1e-12)
        assert np.max(np.abs(r["F"])) < 1e-13


def test_textbook_lattice_sums_large_cutoff(ora):
    a = 5.26
    d = a / np.sqrt(2)
    rc = 24.0
    x, lo, hi = lattice(a, 4)
    r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, rc, 0)
    rho = 4.0 / a ** 3
    tail = 0.5 * rho * 4 * np.pi * 4 * EPS * (SIG ** 12 / (9 * rc ** 9) - SIG ** 6 / (3 * rc ** 3))
    e = r["E"] / x.shape[0] + tail
    s = SIG / d
    textbook = 2 * EPS * (12.13188 * s ** 12 - 14.45392 * s ** 6)
    assert e == pytest.approx(textbook, rel=2e-4)


def test_dimer_analytic(ora):
    lo, hi = np.array([-50.0] * 3), np.array([50.0] * 3)
    for r in (3.2, 3.82, 5.0, 8.0):
        x = np.array([[0.1, 0.2, 0.3], [0.1 + r * 0.6, 0.2 + r * 0.8, 0.3]])
        res = ora.lj(x, lo, hi, [0, 0, 0], EPS, SIG, RC, 1)
        assert res["E"] == pytest.approx(u_lj(r) - u_lj(RC), rel=1e-13, abs=1e-16)
        dvec = x[1] - x[0]
        np.testing.assert_allclose(res["F"][0], du_lj(r) * dvec / r, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(res["F"][1], -res["F"][0], rtol=0, atol=1e-16)
    # beyond rc: nothing
    x = np.array([[0.0, 0.0, 0.0], [RC + 1e-9, 0.0, 0.0]])
    res = ora.lj(x, lo, hi, [0, 0, 0], EPS, SIG, RC, 1)
    assert res["E"] == 0.0 and np.all(res["F"] == 0.0)


def jittered(seed=3, n=3, a=5.26, sigma=0.15):
    rng = np.random.default_rng(seed)
    x = W.fcc_lattice(n, n, n, a) + rng.normal(0, sigma, size=(4 * n ** 3, 3))
    L = n * a
    return x, np.zeros(3), np.full(3, L)


def test_force_is_minus_gradient(ora):
    x, lo, hi = jittered()
    r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, RC, 1)
    h = 1e-5
    rng = np.random.default_rng(1)
    for i in rng.choice(x.shape[0], 6, replace=False):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            ep = ora.lj(xp, lo, hi, [1, 1, 1], EPS, SIG, RC, 1)["E"]
            em = ora.lj(xm, lo, hi, [1, 1, 1], EPS, SIG, RC, 1)["E"]
            fd = -(ep - em) / (2 * h)
            assert fd == pytest.approx(r["F"][i, k], rel=1e-6, abs=1e-9)


def test_total_force_zero_and_translation(ora):
    x, lo, hi = jittered(seed=9)
    r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, RC, 1)
    fmax = np.max(np.abs(r["F"]))
    assert np.max(np.abs(r["F"].sum(axis=0))) < 1e-12 * fmax * x.shape[0]
    shift = np.array([0.37, -1.21, 2.5])
    r2 = ora.lj(x + shift, lo, hi, [1, 1, 1], EPS, SIG, RC, 1)
    assert r2["E"] == pytest.approx(r["E"], rel=1e-12)
    np.testing.assert_allclose(r2["F"], r["F"], rtol=0, atol=1e-12 * fmax)


def test_virial_pressure_equals_minus_dU_dV(ora):
    a = 5.26
    x, lo, hi = lattice(a, 4)
    r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, RC, 0)
    V = (4 * a) ** 3
    p_vir = (r["W"][0] + r["W"][1] + r["W"][2]) / (3 * V)
    np.testing.assert_allclose(r["W"][3:], 0.0, atol=1e-12)
    # -dU/dV from the shell sum, N atoms in V = N a^3 / 4; unshifted and
    # without cutoff motion (the set of shells inside rc does not change)
    n = x.shape[0]
    da = 1e-5

    def U(aa):
        d, z = fcc_shells(aa, RC)
        return n * 0.5 * np.sum(z * u_lj(d))

    dUda = (U(a + da) - U(a - da)) / (2 * da)
    dVda = 3 * V / a
    assert p_vir == pytest.approx(-dUda / dVda, rel=1e-7)


def test_shifted_force_mode_continuous(ora):
    lo, hi = np.array([-50.0] * 3), np.array([50.0] * 3)
    x = np.array([[0.0, 0.0, 0.0], [RC - 1e-7, 0.0, 0.0]])
    res = ora.lj(x, lo, hi, [0, 0, 0], EPS, SIG, RC, 2)
    assert abs(res["E"]) < 1e-10
    assert np.max(np.abs(res["F"])) < 1e-9


def u_sf(r, rc=RC):
    """Shifted-force LJ written out: u(r) - u(rc) - (r - rc) u'(rc)."""
    return u_lj(r) - u_lj(rc) - (r - rc) * du_lj(rc)


def test_shifted_force_dimer_closed_form(ora):
    # shift_mode 2: value and slope vanish at rc; the linear term
    # -(r - rc) u'(rc) is ~10% of the dimer energy at 5 A, so a dropped or
    # mis-signed term fails the energy check, and the force carries -u'(rc)
    lo, hi = np.array([-50.0] * 3), np.array([50.0] * 3)
    for r in (3.2, 3.82, 5.0, 8.0):
        x = np.array([[0.1, 0.2, 0.3], [0.1 + r * 0.6, 0.2 + r * 0.8, 0.3]])
        res = ora.lj(x, lo, hi, [0, 0, 0], EPS, SIG, RC, 2)
        assert res["E"] == pytest.approx(u_sf(r), rel=1e-12, abs=1e-16)
        dvec = x[1] - x[0]
        fmag = du_lj(r) - du_lj(RC)
        np.testing.assert_allclose(res["F"][0], fmag * dvec / r, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(res["F"][1], -res["F"][0], rtol=0, atol=1e-16)
    # the linear term's size at 5 A (what the check above resolves)
    assert abs((5.0 - RC) * du_lj(RC)) > 0.05 * abs(u_sf(5.0))


def test_shifted_force_lattice_shell_sum(ora):
    x, lo, hi = lattice()
    r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, RC, 2)
    d, z = fcc_shells(5.26, RC)
    e_ref = 0.5 * np.sum(z * u_sf(d))
    assert r["E"] / x.shape[0] == pytest.approx(e_ref, rel=1e-12)
    assert np.max(np.abs(r["F"])) < 1e-13


def test_shifted_force_is_minus_gradient(ora):
    x, lo, hi = jittered(seed=5)
    r = ora.lj(x, lo, hi, [1, 1, 1], EPS, SIG, RC, 2)
    h = 1e-5
    rng = np.random.default_rng(2)
    for i in rng.choice(x.shape[0], 6, replace=False):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            ep = ora.lj(xp, lo, hi, [1, 1, 1], EPS, SIG, RC, 2)["E"]
            em = ora.lj(xm, lo, hi, [1, 1, 1], EPS, SIG, RC, 2)["E"]
            fd = -(ep - em) / (2 * h)
            assert fd == pytest.approx(r["F"][i, k], rel=1e-6, abs=1e-9)
