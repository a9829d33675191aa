"""Pins of the oracle's tabulated EAM (energy, force, virial, densities).

* Perfect FCC lattice: rho_i = sum_k z_k rho(d sqrt k) and
  E/N = 1/2 sum_k z_k phi(d sqrt k) + F(rho_i) in closed form (shell sums of
  the analytic functions; tables agree within the spline error), F = 0.
* Synthetic parameter sets: Al-like minimum near a = 4.05 Angstrom and
  Cu-like near 3.615 Angstrom (analytic shell sums).
* Linear embedding F = c rho reduces EAM to the pair potential phi + 2 c rho
  (checks the F'(rho_i) + F'(rho_j) force term).
* -dE/dx by central differences with a nonlinear F; sum F = 0; virial
  pressure = -dU/dV.
"""
import numpy as np
import pytest

from fcc_shells import fcc_shells
from paper_2511_22951_gb300 import workloads as W


def closed_form_energy(p, a):
    d, z = fcc_shells(a, p.rc)
    rho = np.sum(z * W.fs_rho(p, d))
    return 0.5 * np.sum(z * W.fs_phi(p, d)) + W.fs_embed(p, rho), rho


@pytest.mark.parametrize("p,n", [(W.AL_LIKE, 4), (W.CU_LIKE, 4)])
def test_perfect_lattice(ora, p, n):
    tab = W.tabulate_fs_eam(p)
    a = p.a0
    x = W.fcc_lattice(n, n, n, a)
    L = n * a
    r = ora.eam(x, [0, 0, 0], [L, L, L], [1, 1, 1], tab)
    e_ref, rho_ref = closed_form_energy(p, a)
    # table vs analytic: 5000 knots, Hermite with 3-point slopes
    assert r["E"] / x.shape[0] == pytest.approx(e_ref, rel=1e-7)
    np.testing.assert_allclose(r["rho"], rho_ref, rtol=1e-7)
    assert np.max(np.abs(r["F"])) < 1e-12


def test_parameter_sets_have_their_lattice_constant():
    for p, a_exp in ((W.AL_LIKE, 4.05), (W.CU_LIKE, 3.615)):
        aa = np.linspace(a_exp - 0.05, a_exp + 0.05, 201)
        e = np.array([closed_form_energy(p, a)[0] for a in aa])
        a_min = aa[np.argmin(e)]
        assert abs(a_min - a_exp) < 0.01
        assert -4.0 < e.min() < -3.0


def test_linear_embedding_is_a_pair_potential(ora):
    p = W.AL_LIKE
    tab = W.tabulate_fs_eam(p)
    c = -0.37
    lin = W.EAMTables(rc=tab.rc, phi=tab.phi, rho=tab.rho, rho_max=tab.rho_max,
                      F=c * np.arange(tab.nrho) * (tab.rho_max / (tab.nrho - 1)))
    pair = W.EAMTables(rc=tab.rc, phi=tab.phi + 2 * c * tab.rho, rho=np.zeros_like(tab.rho),
                       rho_max=tab.rho_max, F=np.zeros(tab.nrho))
    rng = np.random.default_rng(4)
    x = W.fcc_lattice(3, 3, 3, 4.05) + rng.normal(0, 0.1, size=(108, 3))
    L = 3 * 4.05
    a = ora.eam(x, [0] * 3, [L] * 3, [1, 1, 1], lin)
    b = ora.eam(x, [0] * 3, [L] * 3, [1, 1, 1], pair)
    assert a["E"] == pytest.approx(b["E"], rel=1e-11)
    fm = np.max(np.abs(b["F"]))
    np.testing.assert_allclose(a["F"], b["F"], rtol=0, atol=1e-11 * fm)


def test_force_is_minus_gradient(ora):
    p = W.CU_LIKE
    tab = W.tabulate_fs_eam(p)
    rng = np.random.default_rng(8)
    a = 3.4
    x = W.fcc_lattice(3, 3, 3, a) + rng.normal(0, 0.08, size=(108, 3))
    L = 3 * a
    lo, hi = [0] * 3, [L] * 3
    r = ora.eam(x, lo, hi, [1, 1, 1], tab)
    h = 1e-5
    for i in rng.choice(108, 5, replace=False):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            fd = -(ora.eam(xp, lo, hi, [1, 1, 1], tab)["E"] -
                   ora.eam(xm, lo, hi, [1, 1, 1], tab)["E"]) / (2 * h)
            assert fd == pytest.approx(r["F"][i, k], rel=1e-6, abs=1e-8)
    fmax = np.max(np.abs(r["F"]))
    assert np.max(np.abs(r["F"].sum(axis=0))) < 1e-12 * fmax * 108


def test_virial_pressure_equals_minus_dU_dV(ora):
    p = W.AL_LIKE
    tab = W.tabulate_fs_eam(p)
    a, n = 3.9, 4
    x = W.fcc_lattice(n, n, n, a)
    L = n * a
    r = ora.eam(x, [0] * 3, [L] * 3, [1, 1, 1], tab)
    V = L ** 3
    p_vir = (r["W"][0] + r["W"][1] + r["W"][2]) / (3 * V)
    da = 1e-6

    def U(aa):
        xx = W.fcc_lattice(n, n, n, aa)
        return ora.eam(xx, [0] * 3, [n * aa] * 3, [1, 1, 1], tab)["E"]

    dUdV = (U(a + da) - U(a - da)) / (2 * da) / (3 * V / a)
    assert p_vir == pytest.approx(-dUdV, rel=1e-6)


def test_rho_above_table_is_flagged(ora):
    p = W.CU_LIKE
    tab = W.tabulate_fs_eam(p)
    small = W.EAMTables(rc=tab.rc, phi=tab.phi, rho=tab.rho, rho_max=5.0, F=tab.F)
    x = W.fcc_lattice(3, 3, 3, 3.615)
    L = 3 * 3.615
    r = ora.eam(x, [0] * 3, [L] * 3, [1, 1, 1], small)
    assert r["rho_flag"]
