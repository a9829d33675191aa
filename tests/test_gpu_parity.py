"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (written from the arithmetic):
  * neighbour sets: bit-exact as sorted (j, image) lists, both precisions;
  * FP64 path: |dE| <= 1e-12 |E|;  max|dF| <= 1e-12 max|F| + 1e-13 eV/A;
    virial components within 1e-12 of max |W|;
  * mixed path (FP32 pair arithmetic, FP64 energy sums): ||dF||_rms /
    ||F||_rms <= 1e-5 on thermal states; |dE| <= 1e-6 (|E_pair| + |E_embed|),
    the magnitude of the terms that are summed (for LJ, |E|): EAM's pair and
    embedding energies cancel, so |E| alone is no scale for the FP32
    rounding of the terms.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk as m
    _build.build()
    m.load()
    return m


def gpu_lists(ctx):
    off, j, im = ctx.neighbors()
    out = []
    for i in range(off.shape[0] - 1):
        a, b = off[i], off[i + 1]
        rows = np.concatenate([j[a:b, None].astype(np.int64), im[a:b].astype(np.int64)], 1)
        out.append(set(map(tuple, rows.tolist())))
    return out


def oracle_lists(ora, x, lo, hi, per, rns):
    return [set(map(tuple, q.tolist())) for q in ora.neighbors(x, lo, hi, per, rns)]


def lj_ctx(mdk, x, lo, hi, per, prec, rc=W.LJ_AR.rc, skin=0.3, mode=1, v=None, masses=None):
    n = x.shape[0]
    ctx = mdk.Context(lo, hi, per, masses if masses is not None else np.full(n, W.MASS_AR), prec)
    ctx.set_potential_lj(W.LJ_AR.eps, W.LJ_AR.sigma, rc, mode)
    ctx.plan(rc, skin)
    ctx.set_state(x, v if v is not None else np.zeros((n, 3)))
    ctx.build_neighbors(rc, skin)
    return ctx


def eam_ctx(mdk, x, lo, hi, per, prec, tab, skin=0.3, v=None, mass=W.MASS_CU):
    n = x.shape[0]
    ctx = mdk.Context(lo, hi, per, np.full(n, mass), prec)
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, skin)
    ctx.set_state(x, v if v is not None else np.zeros((n, 3)))
    ctx.build_neighbors(tab.rc, skin)
    return ctx


def assert_fp64(E, F, W_, ref):
    assert abs(E - ref["E"]) <= 1e-12 * abs(ref["E"]), (E, ref["E"])
    fmax = np.max(np.abs(ref["F"])) if ref["F"].size else 0.0
    assert np.max(np.abs(F - ref["F"]), initial=0.0) <= 1e-12 * fmax + 1e-13
    wmax = np.max(np.abs(ref["W"]))
    assert np.max(np.abs(W_ - ref["W"])) <= 1e-12 * wmax + 1e-13


def energy_scale(ref):
    """|E_pair| + |E_embed| of an oracle result (|E| for a pair potential)."""
    if "E_embed" in ref:
        return abs(ref["E"] - ref["E_embed"]) + abs(ref["E_embed"])
    return abs(ref["E"])


def assert_mixed(E, F, ref):
    # energy: relative to the magnitude of the summed terms (pair and
    # embedding energies cancel in EAM, so |E| alone is ill-conditioned)
    assert abs(E - ref["E"]) <= 1e-6 * energy_scale(ref), (E, ref["E"], energy_scale(ref))
    rms = np.sqrt(np.mean((F - ref["F"]) ** 2)) / np.sqrt(np.mean(ref["F"] ** 2))
    assert rms <= 1e-5, rms


# --------------------------------------------------------------------------- lists
BOXES = [
    # (lo, L, periodic, n atoms, r_ns)
    ((0.0, 0.0, 0.0), (20.0, 20.0, 20.0), (1, 1, 1), 300, 5.8),     # several cells
    ((-1.0, 0.5, 2.0), (9.0, 9.0, 9.0), (1, 1, 1), 40, 5.8),         # 1 cell, self images
    ((0.0, 0.0, 0.0), (13.0, 12.5, 30.0), (1, 1, 1), 257, 5.8),      # 2 cells in x, y
    ((0.0, 0.0, 0.0), (30.0, 14.0, 14.0), (0, 1, 1), 251, 5.8),      # free x
    ((0.0, 0.0, 0.0), (15.0, 15.0, 15.0), (0, 0, 0), 150, 5.8),      # cluster
    ((0.0, 0.0, 0.0), (41.0, 33.0, 29.0), (1, 1, 1), 1001, 6.3),     # ragged tail
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("box", BOXES)
def test_neighbor_sets_bit_exact(mdk, ora, box, prec):
    lo, L, per, n, rns = box
    lo = np.array(lo)
    hi = lo + np.array(L)
    rng = np.random.default_rng(n)
    x = lo + rng.uniform(0, 1, size=(n, 3)) * (hi - lo)
    ctx = lj_ctx(mdk, x, lo, hi, per, prec, rc=rns - 0.3, skin=0.3)
    got = gpu_lists(ctx)
    ref = oracle_lists(ora, x, lo, hi, per, rns)
    for i in range(n):
        assert got[i] == ref[i], i
    ctx.close()


@pytest.mark.parametrize("a,ncell,rc,expect", [
    (5.26, 4, W.LJ_AR.rc, 78),
    (4.05, 3, 6.0, 54),
    (3.0, 3, 5.5, 134),
])
def test_fcc_counts_and_sets(mdk, ora, a, ncell, rc, expect):
    x = W.fcc_lattice(ncell, ncell, ncell, a)
    L = ncell * a
    ctx = lj_ctx(mdk, x, [0] * 3, [L] * 3, [1, 1, 1], "fp64", rc=rc)
    got = gpu_lists(ctx)
    assert all(len(g) == expect for g in got)
    ref = oracle_lists(ora, x, [0] * 3, [L] * 3, [1, 1, 1], rc + 0.3)
    assert got == ref


def test_cutoff_is_strict_on_gpu(mdk):
    lo, hi = np.zeros(3), np.full(3, 40.0)
    x = np.array([[10.0, 10.0, 10.0], [14.0, 10.0, 10.0],
                  [10.0, 14.0 - 4e-12, 10.0], [10.0, 10.0, 14.0 + 4e-9]])
    ctx = lj_ctx(mdk, x, lo, hi, [0, 0, 0], "mixed", rc=3.7, skin=0.3)
    got = gpu_lists(ctx)
    assert got[0] == {(2, 0, 0, 0)}


# --------------------------------------------------------------------------- LJ
def jittered_lattice(seed, n, a, sigma):
    rng = np.random.default_rng(seed)
    x = W.fcc_lattice(n, n, n, a) + rng.normal(0, sigma, size=(4 * n ** 3, 3))
    L = n * a
    x = np.mod(x, L)
    return x, np.zeros(3), np.full(3, L)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_lj_fp64_config0(mdk, ora, mode):
    wl = W.config0()
    s = wl.systems[0]
    x = s.x + np.random.default_rng(1).normal(0, 0.1, size=s.x.shape)
    ctx = lj_ctx(mdk, x, s.lo, s.hi, s.periodic, "fp64", mode=mode)
    E, F, Wv = ctx.compute()
    ref = ora.lj(x, s.lo, s.hi, s.periodic, wl.lj.eps, wl.lj.sigma, wl.lj.rc, mode)
    assert_fp64(E[0], F, Wv[0], ref)


def test_lj_fp64_per_atom(mdk, ora):
    x, lo, hi = jittered_lattice(3, 3, 5.26, 0.12)
    ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64")
    ctx.compute()
    U, Wa = ctx.per_atom()
    ref = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1, per_atom=True)
    np.testing.assert_allclose(U, ref["Ea"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Wa, ref["Wa"], rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("n,seed", [(3, 5), (5, 6)])
def test_lj_mixed(mdk, ora, n, seed):
    x, lo, hi = jittered_lattice(seed, n, 5.26, 0.15)
    ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed")
    E, F, Wv = ctx.compute()
    ref = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    assert_mixed(E[0], F, ref)


# --------------------------------------------------------------------------- EAM
@pytest.mark.parametrize("p,a,n", [(W.AL_LIKE, 4.05, 4), (W.CU_LIKE, 3.3, 3),
                                   (W.CU_LIKE, 3.0, 3)])
def test_eam_fp64(mdk, ora, p, a, n):
    tab = W.tabulate_fs_eam(p)
    x, lo, hi = jittered_lattice(11, n, a, 0.08)
    ctx = eam_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", tab, mass=p.mass)
    E, F, Wv = ctx.compute()
    ref = ora.eam(x, lo, hi, [1, 1, 1], tab)
    assert_fp64(E[0], F, Wv[0], ref)


@pytest.mark.parametrize("p,a,n", [(W.AL_LIKE, 4.05, 5), (W.CU_LIKE, 3.0, 3)])
def test_eam_mixed(mdk, ora, p, a, n):
    tab = W.tabulate_fs_eam(p)
    x, lo, hi = jittered_lattice(12, n, a, 0.08)
    ctx = eam_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed", tab, mass=p.mass)
    E, F, Wv = ctx.compute()
    ref = ora.eam(x, lo, hi, [1, 1, 1], tab)
    assert_mixed(E[0], F, ref)


def test_eam_free_surface_slab(mdk, ora):
    """x free, y/z periodic: surface atoms and clamped end cells."""
    wl = W.config3(ncx=8, ncyz=3)
    s = wl.systems[0]
    rng = np.random.default_rng(3)
    x = s.x + rng.normal(0, 0.05, size=s.x.shape)
    x[:, 1:] = np.mod(x[:, 1:] - s.lo[1:], s.hi[1:] - s.lo[1:]) + s.lo[1:]
    ctx = eam_ctx(mdk, x, s.lo, s.hi, s.periodic, "fp64", wl.tables, mass=W.MASS_AL)
    E, F, Wv = ctx.compute()
    ref = ora.eam(x, s.lo, s.hi, s.periodic, wl.tables)
    assert_fp64(E[0], F, Wv[0], ref)


# --------------------------------------------------------------------------- dynamics
def test_trajectory_fp64_lj(mdk, ora):
    wl = W.config0()
    s = wl.systems[0]
    ctx = mdk.make_context(wl)
    ctx.step(wl.dt, 10)
    x, v = ctx.get_state()
    o = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 10, wl.skin,
                   lj_params=wl.lj)
    L = s.hi - s.lo
    d = x - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10
    np.testing.assert_allclose(v, o["v"], rtol=0, atol=1e-11)


def test_trajectory_fp64_eam_and_thermo(mdk, ora):
    p = W.CU_LIKE
    tab = W.tabulate_fs_eam(p)
    x, lo, hi = jittered_lattice(2, 3, 3.615, 0.05)
    rng = np.random.default_rng(9)
    v = W.maxwell_velocities(rng, np.full(x.shape[0], p.mass), 600.0)
    ctx = eam_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", tab, v=v, mass=p.mass)
    ctx.set_thermo(1, 64)
    ctx.step(1.0, 12)
    xg, vg = ctx.get_state()
    th = ctx.thermo()
    o = ora.md_run(x, v, np.full(x.shape[0], p.mass), lo, hi, [1, 1, 1], 1.0, 12, 0.3, tables=tab)
    L = hi - lo
    d = xg - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10
    assert th.shape[0] == 12
    np.testing.assert_allclose(th[:, 0, 1], o["thermo"][:, 0], rtol=1e-11)   # K
    np.testing.assert_allclose(th[:, 0, 2], o["thermo"][:, 1], rtol=1e-11)   # U


def test_mixed_nve_drift_small(mdk):
    wl = W.config0()
    ctx = mdk.make_context(wl, precision="mixed")
    ctx.set_thermo(5, 256)
    ctx.step(wl.dt, 400)
    th = ctx.thermo()[:, 0, :]
    etot = th[:, 1] + th[:, 2]
    n = wl.systems[0].n
    assert np.max(np.abs(etot - etot[0])) / n < 5e-5
    nb, ns = ctx.counters()
    assert ns == 400 and nb >= 2


def test_piston_on_gpu(mdk, ora):
    wl = W.config3(ncx=12, ncyz=3)
    s = wl.systems[0]
    pis = wl.extra["piston"]
    ctx = eam_ctx(mdk, s.x, s.lo, s.hi, s.periodic, "fp64", wl.tables, v=s.v, mass=W.MASS_AL)
    ctx.set_piston(wl.extra["u_p"], pis)
    ctx.step(wl.dt, 20)
    xg, vg = ctx.get_state()
    o = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 20, wl.skin,
                   tables=wl.tables, piston=pis, u_p=wl.extra["u_p"])
    L = s.hi - s.lo
    d = xg - o["x"]
    d[:, 1:] -= np.rint(d[:, 1:] / L[1:]) * L[1:]
    assert np.max(np.abs(d)) < 1e-9
    np.testing.assert_allclose(vg[pis], o["v"][pis], rtol=0, atol=1e-15)


def test_empty_system(mdk):
    ctx = mdk.Context([0, 0, 0], [20.0] * 3, [1, 1, 1], np.zeros(0), "mixed")
    ctx.set_potential_lj(W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc)
    ctx.plan(W.LJ_AR.rc, 0.3)
    ctx.set_state(np.zeros((0, 3)), np.zeros((0, 3)))
    ctx.build_neighbors(W.LJ_AR.rc, 0.3)
    E, F, Wv = ctx.compute()
    assert E[0] == 0.0 and F.shape == (0, 3)
    ctx.step(1.0, 3)


# --------------------------------------------------------------------------- full size
@pytest.mark.slow
def test_config1_full_size_sampled(mdk, ora):
    """256,000-atom Al-like EAM, FP64: 54 neighbours each in the lattice, forces of
    sampled atoms after 3 steps equal the oracle's all-atom sums."""
    wl = W.config1()
    s = wl.systems[0]
    ctx = mdk.make_context(wl)
    assert np.all(ctx.neighbor_counts() == 54)
    ctx.step(wl.dt, 3)
    x, _ = ctx.get_state()
    E, F, _ = ctx.compute()
    sel = np.random.default_rng(0).choice(s.n, 24, replace=False)
    ref = ora.sampled("eam", x, s.lo, s.hi, s.periodic, sel, tables=wl.tables)
    fmax = np.max(np.abs(ref["F"]))
    assert np.max(np.abs(F[sel] - ref["F"])) <= 1e-12 * fmax + 1e-13


@pytest.mark.slow
@pytest.mark.parametrize("skin_outer", [0.0, 2.1])
def test_config2_full_size_sampled(mdk, ora, skin_outer):
    """8,388,608-atom LJ argon, mixed: 78 neighbours each in the lattice; sampled
    forces on a thermalised state (300 steps = 0.6 ps, about one vibration
    period, so that the forces are thermal and not the near-zero forces of the
    starting lattice) within the mixed-precision bar; with one-level lists and
    with the two-level lists the bench runs (outer skin 2.1 A)."""
    wl = W.config2()
    s = wl.systems[0]
    ctx = mdk.make_context(wl, skin_outer=skin_outer)
    assert np.all(ctx.neighbor_counts() == 78)
    ctx.step(wl.dt, 300)
    if skin_outer:
        nb, nf = ctx.build_counts()
        assert nb > nf >= 1, (nb, nf)
    x, _ = ctx.get_state()
    E, F, _ = ctx.compute()
    sel = np.random.default_rng(1).choice(s.n, 16, replace=False)
    ref = ora.sampled("lj", x, s.lo, s.hi, s.periodic, sel, lj_params=wl.lj)
    rms = np.sqrt(np.mean((F[sel] - ref["F"]) ** 2)) / np.sqrt(np.mean(ref["F"] ** 2))
    assert rms <= 1e-5, rms


# --------------------------------------------------------------------------- profiles
def test_profiles_match_oracle(mdk, ora):
    """Appendix per-bin statistics of a thermal slab: the GPU (FP64) against the
    oracle's direct sums over its own per-atom energies and virials."""
    wl = W.config3(ncx=16, ncyz=4)
    s = wl.systems[0]
    rng = np.random.default_rng(5)
    x = s.x + rng.normal(0, 0.05, size=s.x.shape)
    x[:, 1:] = np.mod(x[:, 1:] - s.lo[1:], s.hi[1:] - s.lo[1:]) + s.lo[1:]
    v = s.v.copy()
    v[:, 0] += np.linspace(0.0, 0.01, s.n)          # a velocity gradient along x
    ctx = eam_ctx(mdk, x, s.lo, s.hi, s.periodic, "fp64", wl.tables, v=v, mass=W.MASS_AL)
    area = (s.hi[1] - s.lo[1]) * (s.hi[2] - s.lo[2])
    nb = 16
    out = np.zeros((nb, 17))
    r = ctx.lib.mdk_profiles(ctx.h, 0, 0.0, wl.extra["a"], nb, area, mdk._ptr(out), 0)
    assert r == 0
    ref_e = ora.eam(x, s.lo, s.hi, s.periodic, wl.tables, per_atom=True)
    ref = ora.profiles(x, v, s.masses, 0, 0.0, wl.extra["a"], nb, area, Ua=ref_e["Ea"],
                       Wa=ref_e["Wa"])
    assert out[:, 0].sum() == ref[:, 0].sum() > 0
    np.testing.assert_array_equal(out[:, 0], ref[:, 0])
    scale = np.max(np.abs(ref), axis=0) + 1e-300
    np.testing.assert_allclose(out / scale, ref / scale, rtol=0, atol=1e-11)


# --------------------------------------------------------------------------- moving window
@pytest.mark.parametrize("kind", ["full", "half"])
def test_window_matches_oracle(mdk, ora, kind):
    """Piston + moving window (Al-like slab, FP64, rebuild every 5 steps): after
    12 steps the atoms present (ids), their positions and velocities equal the
    oracle's window run.  dt = 0.5 fs keeps every displacement below skin/2, so
    only the 5-step interval triggers builds, as in the oracle's run."""
    wl = W.config3(ncx=12, ncyz=3)
    s = wl.systems[0]
    a = wl.extra["a"]
    v = s.v.copy()
    v[s.x[:, 0] < 20.0, 0] = 0.015                 # shocked material behind x = 20
    pis = wl.extra["piston"]
    rng = np.random.default_rng(9)
    sx = W.fcc_lattice(2, 3, 3, a)
    sv = W.maxwell_velocities(rng, np.full(sx.shape[0], W.MASS_AL), 300.0)
    slx, gap, depth, Lb, La = 2 * a, 0.5 * a, 2 * a, 8.0, 30.0
    cap = 4000
    ctx = mdk.Context(s.lo, s.hi, s.periodic, s.masses, "fp64", capacity=cap)
    ctx.set_potential_eam(wl.tables)
    ctx.plan(wl.tables.rc, 0.3, rebuild_every=5)
    ctx.set_list_kind(kind)
    ctx.set_state(s.x, v)
    ctx.build_neighbors(wl.tables.rc, 0.3)
    ctx.set_piston(0.015, pis)
    ctx.set_window(Lb, La, sx, sv, slx, gap, W.MASS_AL, depth, 3.0)
    ctx.step(0.5, 12)
    xg, vg = ctx.get_state()
    ids = ctx.ids()
    ins, dele = ctx.window_counts()
    st = ora.WindowState(s.x, v, s.masses, pis, cap)
    ora.md_window(st, s.lo, s.hi, s.periodic, wl.tables, 0.5, 12, 0.3, 5, 0.015, 3.0, Lb, La, sx,
                  sv, slx, gap, W.MASS_AL, depth)
    o = st.view()
    order = np.argsort(o["ids"])
    np.testing.assert_array_equal(ids, o["ids"][order])
    assert ins > 0 and dele > 0 and xg.shape[0] == s.n + ins - dele
    L = s.hi - s.lo
    d = xg - o["x"][order]
    d[:, 1:] -= np.rint(d[:, 1:] / L[1:]) * L[1:]
    assert np.max(np.abs(d)) < 1e-9
    np.testing.assert_allclose(vg, o["v"][order], rtol=0, atol=1e-11)


# --------------------------------------------------------------------------- batched replicas
def small_coldcurve(n_rep=6, seed=2):
    """A handful of Cu-like cold-curve replicas of uneven size and density
    (1-cell and multi-cell boxes), jittered, as in the 64-replica workload."""
    rng = np.random.default_rng(seed)
    reps = []
    for a, n in zip(rng.uniform(3.0, 4.2, n_rep), [3, 4, 3, 5, 6, 3][:n_rep]):
        s = W.lattice_system(rng, (n, n, n), float(a), W.MASS_CU, 0.0, sigma_jitter=0.05)
        reps.append(s)
    return reps


def batch_ctx(mdk, reps, prec, tab):
    ctx = mdk.Context([r.lo for r in reps], [r.hi for r in reps], [r.periodic for r in reps],
                      np.concatenate([r.masses for r in reps]), prec, n_atoms=[r.n for r in reps])
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, 0.3)
    ctx.set_state(np.concatenate([r.x for r in reps]), np.concatenate([r.v for r in reps]))
    ctx.build_neighbors(tab.rc, 0.3)
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_replicas_match_oracle(mdk, ora, prec):
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    reps = small_coldcurve()
    ctx = batch_ctx(mdk, reps, prec, tab)
    E, F, Wv = ctx.compute()
    off = 0
    for q, r in enumerate(reps):
        ref = ora.eam(r.x, r.lo, r.hi, r.periodic, tab)
        Fq = F[off:off + r.n]
        if prec == "fp64":
            assert_fp64(E[q], Fq, Wv[q], ref)
        else:
            assert_mixed(E[q], Fq, ref)
        off += r.n


def test_launch_shapes_agree(mdk, ora):
    """Every threads-per-atom x block-size shape gives the FP64 results."""
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    reps = small_coldcurve()
    ctx = batch_ctx(mdk, reps, "fp64", tab)
    ref = [ora.eam(r.x, r.lo, r.hi, r.periodic, tab) for r in reps]
    for tpa in (1, 2, 4, 8, 32):
        for block in (128, 256, 512):
            ctx.set_launch(tpa, block)
            E, F, Wv = ctx.compute()
            off = 0
            for q, r in enumerate(reps):
                assert_fp64(E[q], F[off:off + r.n], Wv[q], ref[q])
                off += r.n
    t, b, ms = ctx.autotune()
    assert t in (1, 2, 4, 8, 32) and b in (128, 256, 512) and ms > 0.0
    xj, lo, hi = jittered_lattice(7, 4, 5.26, 0.12)
    c2 = lj_ctx(mdk, xj, lo, hi, [1, 1, 1], "mixed")
    r0 = ora.lj(xj, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    for tpa in (2, 4, 8, 32):
        c2.set_launch(tpa, 128)
        E, F, _ = c2.compute()
        assert_mixed(E[0], F, r0)
    # FP64 LJ, a warp per atom, against the oracle at the FP64 bars
    c3 = lj_ctx(mdk, xj, lo, hi, [1, 1, 1], "fp64")
    for tpa in (8, 32):
        c3.set_launch(tpa, 256)
        E, F, Wv = c3.compute()
        assert_fp64(E[0], F, Wv[0], r0)
    with pytest.raises(mdk.MDKError):
        c3.set_launch(16, 128)


def test_batched_dynamics_match_oracle(mdk, ora):
    """Ten FP64 steps of the batch equal ten oracle steps of every replica."""
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    reps = small_coldcurve(4)
    rng = np.random.default_rng(4)
    for r in reps:
        r.v = W.maxwell_velocities(rng, r.masses, 500.0)
    ctx = batch_ctx(mdk, reps, "fp64", tab)
    ctx.set_launch(2, 128)
    ctx.step(1.0, 10)
    x, v = ctx.get_state()
    off = 0
    for r in reps:
        o = ora.md_run(r.x, r.v, r.masses, r.lo, r.hi, r.periodic, 1.0, 10, 0.3, tables=tab)
        L = r.hi - r.lo
        d = x[off:off + r.n] - o["x"]
        d -= np.rint(d / L) * L
        assert np.max(np.abs(d)) < 1e-10
        np.testing.assert_allclose(v[off:off + r.n], o["v"], rtol=0, atol=1e-11)
        off += r.n


# --------------------------------------------------------------------------- CUDA graphs
def test_graph_replay_is_bit_identical(mdk):
    """Steps replayed from the captured two-step graph give exactly the state
    of the same kernels launched one by one (thermo steps interleaved, and a
    change of launch shape that forces a new capture)."""
    wl = W.config0()
    outs = []
    for graphs in (True, False):
        ctx = mdk.make_context(wl, precision="mixed")
        ctx.set_graphs(graphs)
        ctx.set_thermo(7, 64)
        ctx.step(wl.dt, 23)
        ctx.set_launch(2, 128)
        ctx.step(wl.dt, 9)
        x, v = ctx.get_state()
        outs.append((x, v, ctx.thermo()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])
