"""Pins of the oracle's velocity-Verlet integration and its Verlet-list MD.

* Harmonic dimer (a quadratic pair table is reproduced exactly by the
  spline): the trajectory error against the analytic cosine falls as dt^2.
* Time reversibility: n steps, negate v, n steps returns to x0.
* NVE energy conservation on the 256-atom LJ argon lattice.
* Sampled brute-force forces equal the all-pairs forces.
* Rebuild trigger: displacement rebuilds and fixed-interval rebuilds give the
  same trajectory over a short run (the list always holds every pair in rc).
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

ACC = W.EV_PER_A_U_TO_A_PER_FS2


def harmonic_tables(k, r0, rc=6.0, n=2000):
    r = np.arange(n) * (rc / (n - 1))
    phi = 0.5 * k * (r - r0) ** 2
    return W.EAMTables(rc=rc, phi=phi, rho=np.zeros(n), rho_max=10.0, F=np.zeros(n))


def test_harmonic_dimer_second_order(ora):
    k, r0, A, m = 2.0, 2.5, 0.1, 10.0
    tab = harmonic_tables(k, r0)
    mu = m / 2
    omega = np.sqrt(k / mu * ACC)
    T = 2 * np.pi / omega
    errs = []
    # a quarter period, where the cosine's slope is largest, so that the
    # O(dt^2) phase error of velocity Verlet shows up linearly
    for dt in (T / 48, T / 96, T / 192):
        nsteps = int(round(T / (4 * dt)))
        x = np.array([[0.0, 0.0, 0.0], [r0 + A, 0.0, 0.0]])
        v = np.zeros((2, 3))
        out = ora.md_run(x, v, [m, m], [-20] * 3, [20] * 3, [0, 0, 0], dt, nsteps, 0.3,
                         tables=tab)
        r = out["x"][1, 0] - out["x"][0, 0]
        errs.append(abs(r - (r0 + A * np.cos(omega * nsteps * dt))))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def test_time_reversibility(ora):
    wl = W.config0()
    s = wl.systems[0]
    out = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 40, wl.skin,
                     lj_params=wl.lj, rebuild_every=5)
    back = ora.md_run(out["x"], -out["v"], s.masses, s.lo, s.hi, s.periodic, wl.dt, 40,
                      wl.skin, lj_params=wl.lj, rebuild_every=5)
    L = s.hi - s.lo
    d = back["x"] - s.x
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-9
    np.testing.assert_allclose(-back["v"], s.v, atol=1e-12)


def test_nve_energy_conservation(ora):
    wl = W.config0()
    s = wl.systems[0]
    out = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, wl.steps, wl.skin,
                     lj_params=wl.lj)
    th = out["thermo"]
    etot = th[:, 0] + th[:, 1]
    # kinetic energy is exchanged with potential energy ...
    assert np.std(th[:, 0]) > 100 * np.std(etot)
    # ... while the total stays put: fluctuation below 2e-5 eV/atom
    assert np.max(np.abs(etot - etot[0])) / s.n < 2e-5
    assert out["n_builds"] >= 1


def test_rebuild_policies_agree(ora):
    wl = W.config0()
    s = wl.systems[0]
    a = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 30, wl.skin,
                   lj_params=wl.lj, rebuild_every=0)
    b = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 30, wl.skin,
                   lj_params=wl.lj, rebuild_every=1)
    L = s.hi - s.lo
    d = a["x"] - b["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10


def test_sampled_equals_all_pairs(ora):
    rng = np.random.default_rng(2)
    x = W.fcc_lattice(3, 3, 3, 5.26) + rng.normal(0, 0.1, size=(108, 3))
    L = 3 * 5.26
    lo, hi = [0] * 3, [L] * 3
    full = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1,
                  per_atom=True)
    sel = np.array([0, 5, 77, 107])
    s = ora.sampled("lj", x, lo, hi, [1, 1, 1], sel, lj_params=W.LJ_AR)
    np.testing.assert_allclose(s["F"], full["F"][sel], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(s["E"], full["Ea"][sel], rtol=1e-12)
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    a = 3.5
    x = W.fcc_lattice(3, 3, 3, a) + rng.normal(0, 0.1, size=(108, 3))
    L = 3 * a
    full = ora.eam(x, [0] * 3, [L] * 3, [1, 1, 1], tab, per_atom=True)
    s = ora.sampled("eam", x, [0] * 3, [L] * 3, [1, 1, 1], sel, tables=tab)
    np.testing.assert_allclose(s["F"], full["F"][sel], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s["E"], full["Ea"][sel], rtol=1e-12)


def test_piston_moves_rigidly(ora):
    wl = W.config3(ncx=12, ncyz=3)
    s = wl.systems[0]
    pis = wl.extra["piston"]
    up = wl.extra["u_p"]
    n = 20
    out = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, n, wl.skin,
                     tables=wl.tables, piston=pis, u_p=up)
    np.testing.assert_allclose(out["v"][pis], np.tile([up, 0, 0], (pis.sum(), 1)))
    L = s.hi - s.lo
    d = out["x"][pis] - s.x[pis]
    d[:, 1:] -= np.rint(d[:, 1:] / L[1:]) * L[1:]
    np.testing.assert_allclose(d[:, 0], up * wl.dt * n, rtol=1e-12)
    np.testing.assert_allclose(d[:, 1:], 0.0, atol=1e-12)
