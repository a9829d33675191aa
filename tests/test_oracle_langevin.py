"""Pins of the oracle's Langevin thermostat (Sec. "Molecular dynamics": a
Langevin force on the right-hand side of Eq. MD-system gives NVT; Sec.
"Moving window simulation": thermostats with a target temperature, a target
mean velocity and a stiffness beta, in regions along x).

* The generator is Philox4x64-10; numpy ships the same generator
  (numpy.random.Philox, which advances its counter before each block), so the
  oracle's block for counter c equals numpy's first block started at c - 1.
* Free particles (no pair inside the cutoff) make the thermostat exact to
  test: the mean velocity of a cloud relaxes by (1 - beta dt) per step (the
  half-step friction) and (1 - beta dt / 2) at the full step; the full-step
  velocities settle at mean u and temperature T (the scheme's stationary
  variance is exactly k_B T / m for a free particle).
* Atoms outside every region, and piston atoms, are untouched.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

KB = W.K_B
ACC = W.EV_PER_A_U_TO_A_PER_FS2


def test_philox_matches_numpy(ora):
    rng = np.random.default_rng(0)
    for _ in range(20):
        ctr = rng.integers(1, 2**62, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        start = ctr.copy()
        start[0] -= np.uint64(1)
        ref = np.random.Philox(counter=start, key=key).random_raw(4)
        np.testing.assert_array_equal(ora.philox4x64(ctr, key), ref)


def gas(n_side=16, spacing=10.0):
    """Simple cubic points 10 A apart: no LJ pair inside 8.5 A."""
    g = np.arange(n_side) * spacing
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 1.0
    L = n_side * spacing
    return x, [0.0] * 3, [L] * 3, [1, 1, 1]


def peculiar_T(v, m):
    dv = v - v.mean(axis=0)
    return m * np.sum(dv * dv) / (3 * v.shape[0] * KB) / ACC


def test_cloud_mean_relaxes_with_the_friction(ora):
    x, lo, hi, per = gas()
    n = x.shape[0]
    m = np.full(n, W.MASS_AR)
    v = np.zeros((n, 3))
    v[:, 0] = 0.01
    beta, dt, steps = 0.01, 2.0, 40
    r = ora.md_langevin(x, v, m, lo, hi, per, dt, steps, 0.3,
                        [(-1e9, 1e9, 300.0, (0.0, 0.0, 0.0), beta)], seed=11,
                        lj_params=W.LJ_AR)
    want = 0.01 * (1 - beta * dt) ** (steps - 1) * (1 - beta * dt / 2)
    # noise of the mean: sqrt(k_B T A / m / n) at most
    sd = np.sqrt(KB * 300.0 * ACC / W.MASS_AR / n)
    assert abs(r["v"][:, 0].mean() - want) < 5 * sd, (r["v"][:, 0].mean(), want, sd)
    assert abs(r["v"][:, 1].mean()) < 5 * sd


def test_cloud_settles_at_T_and_u(ora):
    x, lo, hi, per = gas()
    n = x.shape[0]
    m = np.full(n, W.MASS_AR)
    v = np.zeros((n, 3))
    u = (0.002, -0.001, 0.0)
    beta, dt, T = 0.02, 2.0, 300.0
    reg = [(-1e9, 1e9, T, u, beta)]
    r = ora.md_langevin(x, v, m, lo, hi, per, dt, 500, 0.3, reg, seed=5, lj_params=W.LJ_AR)
    Ts, us = [], []
    step0 = 500
    for _ in range(6):
        r = ora.md_langevin(r["x"], r["v"], m, lo, hi, per, dt, 100, 0.3, reg, seed=5,
                            lj_params=W.LJ_AR, step0=step0)
        step0 += 100
        Ts.append(peculiar_T(r["v"], W.MASS_AR))
        us.append(r["v"].mean(axis=0))
    # 6 snapshots x 3n samples: relative error of T ~ sqrt(2 / (18 n)) = 0.5%
    assert np.mean(Ts) == pytest.approx(T, rel=0.03)
    sd = np.sqrt(KB * T * ACC / W.MASS_AR / n / 6)
    np.testing.assert_allclose(np.mean(us, axis=0), u, atol=5 * sd)


def test_outside_regions_and_piston_untouched(ora):
    x, lo, hi, per = gas()
    n = x.shape[0]
    m = np.full(n, W.MASS_AR)
    rng = np.random.default_rng(3)
    v = rng.normal(0, 0.002, size=(n, 3))
    piston = (x[:, 1] < 20.0) & (x[:, 0] < 50.0)
    r = ora.md_langevin(x, v, m, lo, hi, per, 1.0, 10, 0.3,
                        [(0.0, 50.0, 300.0, (0.0, 0.0, 0.0), 0.05)], seed=2,
                        lj_params=W.LJ_AR, piston=piston, u_p=0.0)
    # free particles drift at constant velocity unless thermostatted; a
    # particle can leave [0, 50) during 10 steps only by 0.1 A, far from the
    # bounds at x = 1 + 10 k
    outside = x[:, 0] >= 50.0
    np.testing.assert_array_equal(r["v"][outside], v[outside])
    thermo = (~outside) & ~piston
    assert np.all(np.abs(r["v"][thermo] - v[thermo]).max(axis=1) > 0)
    np.testing.assert_array_equal(r["v"][piston], np.zeros((piston.sum(), 3)))


def test_noise_components_are_independent(ora):
    """Each component draws its own output of the block: after one step from
    rest the x, y and z kicks are uncorrelated across atoms."""
    x, lo, hi, per = gas()
    n = x.shape[0]
    m = np.full(n, W.MASS_AR)
    r = ora.md_langevin(x, np.zeros((n, 3)), m, lo, hi, per, 2.0, 1, 0.3,
                        [(-1e9, 1e9, 300.0, (0.0, 0.0, 0.0), 0.01)], seed=8,
                        lj_params=W.LJ_AR)
    c = np.corrcoef(r["v"].T)
    off = c[np.triu_indices(3, 1)]
    assert np.all(np.abs(off) < 5 / np.sqrt(n)), off
