"""Half Verlet lists (each pair once, Newton's third law with accumulating
atomics) against the oracle, through the C ABI: LJ, and the EAM passes
(density to both atoms, embedding per atom, forces to both atoms); and the
list-free LJ kernel that reads the build's cells (one warp per cell).

The neighbour set of Sec. "Neighbor lists" is the oracle's full set; a half
list must hold exactly one of each mirror pair (i, j, n) / (j, i, -n).
Forces, energies and virials carry the bars of the full-list path:
  * FP64: |dE| <= 1e-12 |E|, max|dF| <= 1e-12 max|F| + 1e-13 eV/A, virial
    within 1e-12 of max |W|; per-atom energies rtol 1e-12;
  * mixed: ||dF||_rms / ||F||_rms <= 1e-5, |dE| <= 1e-6 (|E_pair| + |E_embed|).
Mixed half lists accumulate in 64-bit fixed point (unit 2^-40 eV/A), which
fixes two more properties exactly: the forces sum to zero (every pair term
is added once with each sign), and the result is bitwise reproducible.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

from test_gpu_parity import (BOXES, assert_fp64, assert_mixed, batch_ctx, eam_ctx, gpu_lists,
                             jittered_lattice, lj_ctx, oracle_lists, small_coldcurve)

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


def half_ctx(mdk, *args, **kw):
    ctx = lj_ctx(mdk, *args, **kw)
    ctx.set_list_kind("half")
    assert ctx.list_kind == "half"
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("box", BOXES)
def test_half_list_is_one_of_each_mirror_pair(mdk, ora, box, prec):
    lo, L, per, n, rns = box
    lo = np.array(lo)
    hi = lo + np.array(L)
    rng = np.random.default_rng(n)
    x = lo + rng.uniform(0, 1, size=(n, 3)) * (hi - lo)
    ctx = half_ctx(mdk, x, lo, hi, per, prec, rc=rns - 0.3, skin=0.3)
    ctx.build_neighbors(rns - 0.3, 0.3)
    half = gpu_lists(ctx)
    full = oracle_lists(ora, x, lo, hi, per, rns)
    seen = set()
    for i in range(n):
        for (j, a, b, c) in half[i]:
            assert (j, a, b, c) in full[i], (i, j)
            key = (i, j, a, b, c)
            mirror = (j, i, -a, -b, -c)
            assert key not in seen and mirror not in seen, key
            seen.add(key)
    assert len(seen) * 2 == sum(len(f) for f in full)
    ctx.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_half_lj_fp64_config0(mdk, ora, mode):
    wl = W.config0()
    s = wl.systems[0]
    x = s.x + np.random.default_rng(1).normal(0, 0.1, size=s.x.shape)
    ctx = half_ctx(mdk, x, s.lo, s.hi, s.periodic, "fp64", mode=mode)
    E, F, Wv = ctx.compute()
    ref = ora.lj(x, s.lo, s.hi, s.periodic, wl.lj.eps, wl.lj.sigma, wl.lj.rc, mode)
    assert_fp64(E[0], F, Wv[0], ref)


def test_half_lj_fp64_per_atom_and_small_boxes(mdk, ora):
    x, lo, hi = jittered_lattice(3, 3, 5.26, 0.12)
    ctx = half_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64")
    E, F, Wv = ctx.compute()
    U, Wa = ctx.per_atom()
    ref = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1, per_atom=True)
    assert_fp64(E[0], F, Wv[0], ref)
    np.testing.assert_allclose(U, ref["Ea"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Wa, ref["Wa"], rtol=1e-11, atol=1e-14)
    # one cell per dimension: pairs with the atom's own images
    x1, lo1, hi1 = jittered_lattice(8, 2, 5.26, 0.1)
    c1 = half_ctx(mdk, x1, lo1, hi1, [1, 1, 1], "fp64")
    E1, F1, W1 = c1.compute()
    r1 = ora.lj(x1, lo1, hi1, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    assert_fp64(E1[0], F1, W1[0], r1)


@pytest.mark.parametrize("n,seed", [(3, 5), (5, 6), (9, 7)])
def test_half_lj_mixed(mdk, ora, n, seed):
    x, lo, hi = jittered_lattice(seed, n, 5.26, 0.15)
    ctx = half_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed")
    E, F, Wv = ctx.compute()
    ref = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    assert_mixed(E[0], F, ref)


def test_half_mixed_third_law_exact_and_reproducible(mdk):
    x, lo, hi = jittered_lattice(11, 6, 5.26, 0.15)
    ctx = half_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed")
    _, F1, _ = ctx.compute()
    q = F1 * 2.0 ** 40
    assert np.all(q == np.rint(q))               # multiples of the unit
    tot = [sum(int(v) for v in q[:, d]) for d in range(3)]
    assert tot == [0, 0, 0], tot                 # sum of the forces: exactly 0
    ctx.build_neighbors(W.LJ_AR.rc, 0.3)
    _, F2, _ = ctx.compute()
    np.testing.assert_array_equal(F1, F2)


def test_half_trajectory_fp64_lj(mdk, ora):
    wl = W.config0()
    s = wl.systems[0]
    ctx = mdk.make_context(wl)
    ctx.set_list_kind("half")
    ctx.step(wl.dt, 10)
    x, v = ctx.get_state()
    o = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 10, wl.skin,
                   lj_params=wl.lj)
    L = s.hi - s.lo
    d = x - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10
    np.testing.assert_allclose(v, o["v"], rtol=0, atol=1e-11)


def test_half_mixed_graphs_equal_eager_and_drift(mdk):
    wl = W.config0()
    outs = []
    for graphs in (True, False):
        ctx = mdk.make_context(wl, precision="mixed")
        ctx.set_list_kind("half")
        ctx.set_graphs(graphs)
        ctx.set_thermo(5, 256)
        ctx.step(wl.dt, 400)
        x, v = ctx.get_state()
        outs.append((x, v, ctx.thermo()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    th = outs[0][2][:, 0, :]
    etot = th[:, 1] + th[:, 2]
    assert np.max(np.abs(etot - etot[0])) / wl.systems[0].n < 5e-5


def test_list_kind_arguments_and_autotune(mdk, ora):
    x, lo, hi = jittered_lattice(7, 4, 5.26, 0.12)
    ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed")
    assert ctx.list_kind == "full"
    assert ctx.lib.mdk_set_list_kind(ctx.h, 3) == mdk.MDK_ERR_BAD_ARG
    t, b, ms = ctx.autotune()
    assert ctx.list_kind in ("full", "half", "cells") and ms > 0.0
    if ctx.list_kind != "full":
        assert t == 1 and b in (128, 256)
    E, F, _ = ctx.compute()
    ref = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    assert_mixed(E[0], F, ref)
    # EAM: the autotuner times both kinds too
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    xe, loe, hie = jittered_lattice(2, 3, 3.615, 0.05)
    ce = eam_ctx(mdk, xe, loe, hie, [1, 1, 1], "mixed", tab, mass=W.CU_LIKE.mass)
    ce.autotune()
    assert ce.list_kind in ("full", "half")
    E, F, _ = ce.compute()
    assert_mixed(E[0], F, ora.eam(xe, loe, hie, [1, 1, 1], tab))


# --------------------------------------------------------------------------- EAM
def half_eam(mdk, *args, **kw):
    ctx = eam_ctx(mdk, *args, **kw)
    ctx.set_list_kind("half")
    return ctx


@pytest.mark.parametrize("p,a,n", [(W.AL_LIKE, 4.05, 4), (W.CU_LIKE, 3.3, 3),
                                   (W.CU_LIKE, 3.0, 3)])
def test_half_eam_fp64(mdk, ora, p, a, n):
    tab = W.tabulate_fs_eam(p)
    x, lo, hi = jittered_lattice(n + 10, n, a, 0.08)
    ctx = half_eam(mdk, x, lo, hi, [1, 1, 1], "fp64", tab, mass=p.mass)
    E, F, Wv = ctx.compute()
    U, Wa = ctx.per_atom()
    ref = ora.eam(x, lo, hi, [1, 1, 1], tab, per_atom=True)
    assert_fp64(E[0], F, Wv[0], ref)
    np.testing.assert_allclose(U, ref["Ea"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Wa, ref["Wa"], rtol=0, atol=1e-11 * np.abs(ref["Wa"]).max())


@pytest.mark.parametrize("p,a,n", [(W.AL_LIKE, 4.05, 5), (W.CU_LIKE, 3.615, 4)])
def test_half_eam_mixed(mdk, ora, p, a, n):
    tab = W.tabulate_fs_eam(p)
    x, lo, hi = jittered_lattice(n + 20, n, a, 0.1)
    ctx = half_eam(mdk, x, lo, hi, [1, 1, 1], "mixed", tab, mass=p.mass)
    E, F, _ = ctx.compute()
    ref = ora.eam(x, lo, hi, [1, 1, 1], tab)
    assert_mixed(E[0], F, ref)
    q = F * 2.0 ** 40
    assert [sum(int(v) for v in q[:, d]) for d in range(3)] == [0, 0, 0]
    _, F2, _ = ctx.compute()
    np.testing.assert_array_equal(F, F2)


def test_half_eam_trajectory_and_batch_fp64(mdk, ora):
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    reps = small_coldcurve(4)
    rng = np.random.default_rng(41)
    for r in reps:
        r.v = W.maxwell_velocities(rng, r.masses, 500.0)
    ctx = batch_ctx(mdk, reps, "fp64", tab)
    ctx.set_list_kind("half")
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


def test_half_eam_mixed_graphs_equal_eager_and_vjp_uses_full_lists(mdk):
    tab = W.tabulate_fs_eam(W.AL_LIKE)
    outs = []
    for graphs in (True, False):
        x, lo, hi = jittered_lattice(50, 5, 4.05, 0.05)
        v = W.maxwell_velocities(np.random.default_rng(51), np.full(x.shape[0], W.MASS_AL), 300.0)
        ctx = half_eam(mdk, x, lo, hi, [1, 1, 1], "mixed", tab, v=v, mass=W.MASS_AL)
        ctx.set_graphs(graphs)
        ctx.set_thermo(7, 64)
        ctx.step(1.0, 30)
        outs.append(ctx.get_state() + (ctx.thermo(),))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    # the adjoint walks full lists: a half-list context gives the same VJP
    x, lo, hi = jittered_lattice(52, 4, 4.05, 0.08)
    gF = np.random.default_rng(53).normal(size=(x.shape[0], 3))
    res = []
    for kind in ("full", "half"):
        c = eam_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", tab, mass=W.MASS_AL)
        c.set_list_kind(kind)
        c.compute()
        res.append(c.eam_vjp(gE=np.ones(1), gF=gF))
    for a, b in zip(res[0], res[1]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())


@pytest.mark.slow
def test_half_config2_full_size_sampled(mdk, ora):
    """8,388,608-atom LJ argon, mixed, half lists: 39 list entries per atom on
    average in the lattice; sampled forces on a thermalised state within the
    mixed-precision bar; the forces sum to exactly zero."""
    wl = W.config2()
    s = wl.systems[0]
    ctx = mdk.make_context(wl)
    ctx.set_list_kind("half")
    ctx.build_neighbors(wl.rc, wl.skin)
    assert ctx.neighbor_counts().sum() == s.n * 39
    ctx.step(wl.dt, 300)
    x, _ = ctx.get_state()
    E, F, _ = ctx.compute()
    assert np.all(np.sum(np.rint(F * 2.0 ** 40).astype(np.int64), axis=0) == 0)
    sel = np.random.default_rng(1).choice(s.n, 16, replace=False)
    ref = ora.sampled("lj", x, s.lo, s.hi, s.periodic, sel, lj_params=wl.lj)
    rms = np.sqrt(np.mean((F[sel] - ref["F"]) ** 2)) / np.sqrt(np.mean(ref["F"] ** 2))
    assert rms <= 1e-5, rms


# --------------------------------------------------------------------------- cells
def cells_ctx(mdk, *args, **kw):
    ctx = lj_ctx(mdk, *args, **kw)
    ctx.set_list_kind("cells")
    assert ctx.list_kind == "cells"
    return ctx


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cells_lj_fp64_config0(mdk, ora, mode):
    wl = W.config0()
    s = wl.systems[0]
    x = s.x + np.random.default_rng(1).normal(0, 0.1, size=s.x.shape)
    ctx = cells_ctx(mdk, x, s.lo, s.hi, s.periodic, "fp64", mode=mode)
    E, F, Wv = ctx.compute()
    ref = ora.lj(x, s.lo, s.hi, s.periodic, wl.lj.eps, wl.lj.sigma, wl.lj.rc, mode)
    assert_fp64(E[0], F, Wv[0], ref)
    with pytest.raises(mdk.MDKError):
        ctx.neighbors()


@pytest.mark.parametrize("box", BOXES)
def test_cells_lj_fp64_boxes(mdk, ora, box):
    """Random gases in the list tests' boxes: several cells, one cell per
    dimension (own images), two cells, a free dimension, a cluster, a
    ragged tail; dense enough for cells of more than 32 atoms."""
    lo, L, per, n, rns = box
    lo = np.array(lo)
    hi = lo + np.array(L)
    rng = np.random.default_rng(n + 1)
    x = lo + rng.uniform(0, 1, size=(n, 3)) * (hi - lo)
    rc = rns - 0.3
    ctx = cells_ctx(mdk, x, lo, hi, per, "fp64", rc=rc, mode=2)
    E, F, Wv = ctx.compute()
    ref = ora.lj(x, lo, hi, per, W.LJ_AR.eps, W.LJ_AR.sigma, rc, 2)
    assert_fp64(E[0], F, Wv[0], ref)
    U, Wa = ctx.per_atom()
    ra = ora.lj(x, lo, hi, per, W.LJ_AR.eps, W.LJ_AR.sigma, rc, 2, per_atom=True)
    np.testing.assert_allclose(U, ra["Ea"], rtol=1e-11, atol=1e-12 * np.abs(ra["Ea"]).max())


@pytest.mark.parametrize("n,seed", [(3, 5), (9, 7)])
def test_cells_lj_mixed(mdk, ora, n, seed):
    x, lo, hi = jittered_lattice(seed, n, 5.26, 0.15)
    ctx = cells_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed")
    E, F, _ = ctx.compute()
    ref = ora.lj(x, lo, hi, [1, 1, 1], W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    assert_mixed(E[0], F, ref)


def test_cells_trajectory_fp64_and_graphs(mdk, ora):
    wl = W.config0()
    s = wl.systems[0]
    ctx = mdk.make_context(wl)
    ctx.set_list_kind("cells")
    ctx.step(wl.dt, 10)
    x, v = ctx.get_state()
    o = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 10, wl.skin,
                   lj_params=wl.lj)
    L = s.hi - s.lo
    d = x - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10
    np.testing.assert_allclose(v, o["v"], rtol=0, atol=1e-11)
    outs = []
    for graphs in (True, False):
        c = mdk.make_context(wl, precision="mixed")
        c.set_list_kind("cells")
        c.set_graphs(graphs)
        c.set_thermo(5, 256)
        c.step(wl.dt, 200)
        outs.append(c.get_state() + (c.thermo(),))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    th = outs[0][2][:, 0, :]
    etot = th[:, 1] + th[:, 2]
    assert np.max(np.abs(etot - etot[0])) / s.n < 5e-5


def test_cells_kind_rules(mdk):
    x, lo, hi = jittered_lattice(7, 3, 5.26, 0.1)
    ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed")
    ctx.set_list_kind("cells")
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    ctx.set_potential_eam(tab)          # EAM takes full lists again
    assert ctx.list_kind == "full"
    with pytest.raises(mdk.MDKError):
        ctx.set_list_kind("cells")
