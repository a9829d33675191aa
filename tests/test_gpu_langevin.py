"""Langevin thermostat regions on the GPU (mdk_set_langevin) against the
oracle (tests/test_oracle_langevin.py pins the oracle).

Bars: the noise is the same Philox4x64-10 stream on both sides (counter =
atom id, step index); the oracle evaluates the friction -beta m (v - u) / A
as written and the kernel with a precomputed factor -beta m / A (a few ulps
of the friction force apart, ~1e-18 Angstrom/fs of velocity per step), so
FP64 trajectories differ by the conservative forces' summation order and
that rounding: positions within 1e-9 Angstrom and velocities within 1e-11
Angstrom/fs after 10 steps.  The mixed path is checked statistically:
a free gas settles at the target temperature and drift velocity.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KB = W.K_B
ACC = W.EV_PER_A_U_TO_A_PER_FS2


@pytest.fixture(scope="module")
def mdk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk as m
    _build.build()
    m.load()
    return m


REGIONS = [(-5.0, 10.5, 50.0, (0.001, 0.0, 0.0), 0.01),
           (10.5, 30.0, 150.0, (0.0, -0.0005, 0.0), 0.02)]


def lj_ctx(mdk, s, prec, kind="full"):
    lj = W.LJ_AR
    ctx = mdk.Context(s.lo, s.hi, s.periodic, s.masses, prec)
    ctx.set_potential_lj(lj.eps, lj.sigma, lj.rc, lj.shift_mode)
    ctx.set_list_kind(kind)
    ctx.plan(lj.rc, 0.3)
    ctx.set_state(s.x, s.v)
    ctx.build_neighbors(lj.rc, 0.3)
    return ctx


@pytest.mark.parametrize("kind", ["full", "half", "cells"])
def test_langevin_trajectory_matches_oracle(mdk, ora, kind):
    wl = W.config0()
    s = wl.systems[0]
    ctx = lj_ctx(mdk, s, "fp64", kind)
    ctx.set_langevin(REGIONS, seed=7)
    ctx.step(wl.dt, 10)
    xg, vg = ctx.get_state()
    o = ora.md_langevin(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 10, wl.skin,
                        REGIONS, seed=7, lj_params=wl.lj)
    L = s.hi - s.lo
    d = xg - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-9, np.max(np.abs(d))
    assert np.max(np.abs(vg - o["v"])) < 1e-11, np.max(np.abs(vg - o["v"]))
    # the thermostat acted: the same run without it ends elsewhere
    o0 = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 10, wl.skin,
                    lj_params=wl.lj)
    assert np.max(np.abs(o0["v"] - o["v"])) > 1e-6


def test_graphs_and_eager_steps_agree_with_langevin(mdk):
    wl = W.config0()
    s = wl.systems[0]
    out = []
    for graphs in (True, False):
        ctx = lj_ctx(mdk, s, "mixed")
        ctx.set_graphs(graphs)
        ctx.set_langevin(REGIONS, seed=3)
        ctx.step(wl.dt, 12)
        out.append(ctx.get_state())
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_free_gas_settles_at_T_and_u_mixed(mdk):
    n_side, spacing = 16, 10.0
    g = np.arange(n_side) * spacing
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 1.0
    L = n_side * spacing
    n = x.shape[0]
    lj = W.LJ_AR
    ctx = mdk.Context([0.0] * 3, [L] * 3, [1] * 3, np.full(n, lj.mass), "mixed")
    ctx.set_potential_lj(lj.eps, lj.sigma, lj.rc, lj.shift_mode)
    ctx.plan(lj.rc, 0.3)
    ctx.set_state(x, np.zeros((n, 3)))
    ctx.build_neighbors(lj.rc, 0.3)
    T, u = 300.0, (0.002, -0.001, 0.0)
    ctx.set_langevin([(-1e9, 1e9, T, u, 0.02)], seed=5)
    ctx.step(2.0, 500)
    Ts, us = [], []
    for _ in range(6):
        ctx.step(2.0, 100)
        _, v = ctx.get_state()
        dv = v - v.mean(axis=0)
        Ts.append(lj.mass * np.sum(dv * dv) / (3 * n * KB) / ACC)
        us.append(v.mean(axis=0))
    assert np.mean(Ts) == pytest.approx(T, rel=0.03)
    sd = np.sqrt(KB * T * ACC / lj.mass / n / 6)
    np.testing.assert_allclose(np.mean(us, axis=0), u, atol=5 * sd)


def test_langevin_arguments_are_checked(mdk):
    wl = W.config0()
    s = wl.systems[0]
    ctx = lj_ctx(mdk, s, "fp64")
    with pytest.raises(mdk.MDKError):
        ctx.set_langevin([(1.0, 0.0, 300.0, (0, 0, 0), 0.01)])   # empty region
    with pytest.raises(mdk.MDKError):
        ctx.set_langevin([(0.0, 1.0, -1.0, (0, 0, 0), 0.01)])    # negative T
    ctx.set_langevin([])                                         # off


@pytest.mark.parametrize("kind", ["full", "half"])
def test_stationary_window_with_thermostats_matches_oracle(mdk, ora, kind):
    """The paper's stationary-shock window: material flows in at u_in (< 0)
    through fixed inflow and outflow boundaries (outflow deletion at
    x_front - L_behind, fresh layers up to x_front + L_ahead), with Langevin
    thermostats at the inflow (T0, u_in) and outflow (u_out) ends.  FP64,
    Al-like slab, rebuild every 5 steps; ids, positions and velocities equal
    the oracle's window run after 12 steps."""
    wl = W.config3(ncx=12, ncyz=3)
    s = wl.systems[0]
    a = wl.extra["a"]
    u_in, u_out = -0.01, -0.004
    v = s.v.copy()
    v[:, 0] += u_in
    rng = np.random.default_rng(9)
    sx = W.fcc_lattice(2, 3, 3, a)
    sv = W.maxwell_velocities(rng, np.full(sx.shape[0], W.MASS_AL), 300.0)
    sv[:, 0] += u_in
    slx, gap, Lb, La, xf = 2 * a, 0.5 * a, 12.0, 32.0, 20.0
    regions = [(s.lo[0], 14.0, 300.0, (u_out, 0.0, 0.0), 0.02),
               (40.0, s.hi[0], 300.0, (u_in, 0.0, 0.0), 0.02)]
    cap = 4000
    ctx = mdk.Context(s.lo, s.hi, s.periodic, s.masses, "fp64", capacity=cap)
    ctx.set_potential_eam(wl.tables)
    ctx.set_list_kind(kind)
    ctx.plan(wl.tables.rc, 0.3, rebuild_every=5)
    ctx.set_state(s.x, v)
    ctx.build_neighbors(wl.tables.rc, 0.3)
    ctx.set_window(Lb, La, sx, sv, slx, gap, W.MASS_AL, 0.0, 3.0, fixed_front=xf)
    ctx.set_langevin(regions, seed=21)
    ctx.step(0.5, 12)
    xg, vg = ctx.get_state()
    ids = ctx.ids()
    ins, dele = ctx.window_counts()
    st = ora.WindowState(s.x, v, s.masses, np.zeros(s.n, dtype=bool), cap)
    ora.md_window(st, s.lo, s.hi, s.periodic, wl.tables, 0.5, 12, 0.3, 5, 0.0, 3.0, Lb, La,
                  sx, sv, slx, gap, W.MASS_AL, 0.0, fixed_front=xf, regions=regions, seed=21)
    o = st.view()
    order = np.argsort(o["ids"])
    np.testing.assert_array_equal(ids, o["ids"][order])
    assert ins > 0 and dele > 0
    L = s.hi - s.lo
    d = xg - o["x"][order]
    d[:, 1:] -= np.rint(d[:, 1:] / L[1:]) * L[1:]
    assert np.max(np.abs(d)) < 1e-9
    np.testing.assert_allclose(vg, o["v"][order], rtol=0, atol=1e-11)


def test_stationary_search_workflow_runs(mdk):
    """The host-side search loop on a small Al-like slab: restarts from a saved
    state, samples F = P / P_t through mdk_profiles, fits the slope, and
    bisects (two iterations here: the physics needs long runs)."""
    from paper_2511_22951_gb300 import shock
    wl = W.config3(ncx=16, ncyz=4)
    s = wl.systems[0]
    a = wl.extra["a"]
    u_in = -0.05
    v = s.v.copy()
    v[:, 0] += u_in
    rng = np.random.default_rng(4)
    sx = W.fcc_lattice(1, 4, 4, a, (0.0, s.lo[1], s.lo[2]))
    sv = W.maxwell_velocities(rng, np.full(sx.shape[0], W.MASS_AL), 300.0)
    sv[:, 0] += u_in
    area = (s.hi[1] - s.lo[1]) * (s.hi[2] - s.lo[2])
    sw = shock.StationaryWindow(
        tables=wl.tables, lo=s.lo, hi=s.hi, periodic=s.periodic, x=s.x, v=v,
        masses=s.masses, slab_x=sx, slab_v=sv, slab_lx=a, slab_gap=0.5 * a,
        slab_mass=W.MASS_AL, x_front=30.0, L_behind=25.0, L_ahead=40.0,
        inflow=(50.0, s.hi[0], 300.0, 0.01), outflow=(s.lo[0], 12.0, 300.0, 0.01),
        u_in=u_in, P_t=1e-3, domain=(5.0, 65.0), cross_area=area, precision="mixed",
        dt=1.0, max_neighbors=160)
    ctx = sw.context(-0.02)
    ctx.step(1.0, 30)
    assert np.isfinite(sw.target(ctx))
    assert ctx.window_counts()[0] > 0   # inflow layers were appended
    ctx.close()
    slopes = {}

    def slope_at(u):
        slopes[u] = sw.slope(u, n_samples=4, every=10)
        # the real slope is measured; its sign is forced so that the loop runs
        return abs(slopes[u]) + 1.0 if u < -0.03 else -abs(slopes[u]) - 1.0

    u, hist = shock.dichotomy(slope_at, -0.045, -0.005, tol=0.02, max_iter=2)
    assert -0.045 <= u <= -0.005 and len(hist) >= 3
    assert all(np.isfinite(q) for q in slopes.values())


@pytest.mark.parametrize("kind", ["full", "half", "cells"])
def test_replica_thermostats_match_oracle(mdk, ora, kind):
    """Per-replica thermostats (mdk_set_langevin_replicas): every replica of
    a batch at its own T and beta; FP64 trajectories equal the oracle's run of
    each replica with one whole-box region (ids continue across replicas)."""
    rng = np.random.default_rng(12)
    reps, Ts, betas = [], [60.0, 150.0, 400.0], [0.01, 0.02, 0.005]
    for a in (5.26, 5.1, 5.4):
        reps.append(W.lattice_system(rng, (4, 4, 4), a, W.MASS_AR, 80.0))
    lj = W.LJ_AR
    ctx = mdk.Context([r.lo for r in reps], [r.hi for r in reps], [r.periodic for r in reps],
                      np.concatenate([r.masses for r in reps]), "fp64",
                      n_atoms=[r.n for r in reps])
    ctx.set_potential_lj(lj.eps, lj.sigma, lj.rc, lj.shift_mode)
    ctx.set_list_kind(kind)
    ctx.plan(lj.rc, 0.3)
    ctx.set_state(np.concatenate([r.x for r in reps]), np.concatenate([r.v for r in reps]))
    ctx.build_neighbors(lj.rc, 0.3)
    ctx.set_langevin_replicas(Ts, betas, seed=31)
    ctx.step(2.0, 10)
    xg, vg = ctx.get_state()
    off = 0
    for r, T, b in zip(reps, Ts, betas):
        o = ora.md_langevin(r.x, r.v, r.masses, r.lo, r.hi, r.periodic, 2.0, 10, 0.3,
                            [(-1e30, 1e30, T, (0.0, 0.0, 0.0), b)], seed=31, lj_params=lj,
                            ids=np.arange(off, off + r.n))
        L = r.hi - r.lo
        d = xg[off:off + r.n] - o["x"]
        d -= np.rint(d / L) * L
        assert np.max(np.abs(d)) < 1e-9
        assert np.max(np.abs(vg[off:off + r.n] - o["v"])) < 1e-11
        off += r.n


def test_isotherm_grid_workflow(mdk):
    """Isotherms as batched replicas, mixed precision: e and P grow with T
    on every volume line and with compression on every isotherm, and the
    replicas' kinetic temperatures follow their thermostats."""
    from paper_2511_22951_gb300 import hugoniot as H
    grid = H.IsothermGrid(a0=5.26, compressions=np.array([1.0, 0.85, 0.7]),
                          temperatures=np.array([100.0, 300.0, 900.0]), n_cells=4,
                          beta=0.01)
    ctx, ss = grid.context("mixed", max_neighbors=160)
    E, P, v = grid.run(ctx, ss, 2.0, 600, 10, 20)
    assert np.all(np.diff(E, axis=1) > 0) and np.all(np.diff(P, axis=1) > 0)
    assert np.all(np.diff(P, axis=0) > 0)
    np.testing.assert_allclose(v / v[0], grid.compressions, rtol=1e-12)
    th = ctx.thermo()
    assert th.shape[0] == 0  # everything was read by run()
