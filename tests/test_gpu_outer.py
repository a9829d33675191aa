"""Two-level lists (an outer list within rc + skin_outer; the Verlet list
filtered from it while every atom has moved less than (skin_outer - skin) / 2
since the outer list's build): the Verlet lists after filter builds equal the
definition at the current positions, and trajectories, forces and the
batched path keep the bars of the one-level lists.

Bars: neighbour sets exact (per atom, as sets of j in boxes longer than
2 (rc + skin)); FP64 trajectories as the one-level test (positions
1e-10 A, velocities 1e-11 A/fs after the same steps); FP64 forces 1e-12
relative; graphs == eager bit for bit.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

from test_gpu_parity import assert_fp64, jittered_lattice, lj_ctx

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


def gpu_jsets(ctx):
    off, j, _ = ctx.neighbors()
    return [sorted(j[off[i]:off[i + 1]].tolist()) for i in range(off.shape[0] - 1)]


def oracle_jsets(ora, x, lo, hi, rns):
    L = hi - lo
    xw = lo + np.mod(x - lo, L)
    lists = ora.neighbors(xw, lo, hi, [1, 1, 1], rns)
    return [sorted(q[:, 0].astype(int).tolist()) for q in lists]


def hot_argon(seed, n=5, T=900.0):
    rng = np.random.default_rng(seed)
    a = 5.26
    x = W.fcc_lattice(n, n, n, a) + rng.normal(0, 0.05, size=(4 * n ** 3, 3))
    L = n * a
    lo, hi = np.zeros(3), np.full(3, L)
    x = np.mod(x, L)
    v = W.maxwell_velocities(rng, np.full(x.shape[0], W.MASS_AR), T)
    return x, v, lo, hi


@pytest.mark.parametrize("prec,kind", [("fp64", "full"), ("mixed", "full"), ("mixed", "half"),
                                       ("fp64", "half")])
def test_filtered_lists_equal_the_definition(mdk, ora, prec, kind):
    """Builds every 5 steps (fixed interval), so the list of the last step
    belongs to the returned positions; the box is longer than 2 (rc + skin),
    so a pair has one image and the lists compare as sets of j."""
    x, v, lo, hi = hot_argon(1, T=300.0)
    rc, skin = W.LJ_AR.rc, 0.3
    n = x.shape[0]
    ctx = mdk.Context(lo, hi, [1, 1, 1], np.full(n, W.MASS_AR), prec)
    ctx.set_potential_lj(W.LJ_AR.eps, W.LJ_AR.sigma, rc, 1)
    ctx.plan(rc, skin, 0, 5)
    ctx.set_outer_skin(1.2)
    ctx.set_state(x, v)
    if kind == "half":
        ctx.set_list_kind("half")
    ctx.build_neighbors(rc, skin)
    compared = filtered = 0
    for _ in range(14):
        nb0, nf0 = ctx.build_counts()
        ctx.step(2.0, 5)
        nb1, nf1 = ctx.build_counts()
        if nb1 != nb0 + 1:
            continue  # the displacement trigger moved the build off the last step
        xs, _ = ctx.get_state()
        got = gpu_jsets(ctx)
        ref = oracle_jsets(ora, xs, lo, hi, rc + skin)
        if kind == "half":
            # one of each mirror pair: with the mirrors, the full sets
            full = [[] for _ in range(n)]
            for i, js in enumerate(got):
                for j in js:
                    full[i].append(j)
                    full[j].append(i)
            got = [sorted(q) for q in full]
        assert got == ref
        compared += 1
        filtered += nf1 == nf0
    assert compared >= 8 and filtered >= 4, (compared, filtered)


def test_fp64_trajectory_matches_oracle(mdk, ora):
    x, v, lo, hi = hot_argon(2, n=4, T=600.0)
    rc, skin = W.LJ_AR.rc, 0.3
    ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", rc=rc, skin=skin, v=v)
    ctx.set_outer_skin(1.2)
    ctx.build_neighbors(rc, skin)
    nsteps = 120
    ctx.step(2.0, nsteps)
    nb, nf = ctx.build_counts()
    assert nb > nf >= 1, (nb, nf)
    xg, vg = ctx.get_state()
    lj = W.LJ_AR
    o = ora.md_run(x, v, np.full(x.shape[0], W.MASS_AR), lo, hi, [1, 1, 1], 2.0, nsteps, skin,
                   lj_params=lj)
    L = hi - lo
    d = xg - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10
    np.testing.assert_allclose(vg, o["v"], rtol=0, atol=1e-11)
    E, F, Wv = ctx.compute()
    xw = lo + np.mod(xg - lo, L)
    ref = ora.lj(xw, lo, hi, [1, 1, 1], lj.eps, lj.sigma, lj.rc, lj.shift_mode)
    assert_fp64(E[0], F, Wv[0], ref)


def test_mixed_graphs_equal_eager(mdk):
    outs = []
    for graphs in (True, False):
        x, v, lo, hi = hot_argon(3)
        ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed", v=v)
        ctx.set_outer_skin(1.2)
        ctx.build_neighbors(W.LJ_AR.rc, 0.3)
        ctx.set_graphs(graphs)
        ctx.step(2.0, 150)
        xs, vs = ctx.get_state()
        outs.append((xs, vs, ctx.build_counts()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2] and outs[0][2][0] > outs[0][2][1]


def test_eam_batch_fp64_forces_after_filter_builds(mdk, ora):
    p = W.CU_LIKE
    tab = W.tabulate_fs_eam(p)
    reps = []
    for q, (n, a) in enumerate([(4, 3.615), (5, 3.55), (4, 3.7)]):
        x, lo, hi = jittered_lattice(10 + q, n, a, 0.05)
        reps.append((x, lo, hi))
    n_at = [r[0].shape[0] for r in reps]
    ctx = mdk.Context([r[1] for r in reps], [r[2] for r in reps], [[1, 1, 1]] * 3,
                      np.full(sum(n_at), p.mass), "fp64", n_atoms=n_at)
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, 0.3)
    ctx.set_outer_skin(1.0)
    rng = np.random.default_rng(5)
    x0 = np.concatenate([r[0] for r in reps])
    v0 = W.maxwell_velocities(rng, np.full(x0.shape[0], p.mass), 1200.0)
    ctx.set_state(x0, v0)
    ctx.build_neighbors(tab.rc, 0.3)
    ctx.step(1.0, 150)
    nb, nf = ctx.build_counts()
    assert nb > nf >= 1, (nb, nf)
    E, F, Wv = ctx.compute()
    xs, _ = ctx.get_state()
    off = 0
    for q, r in enumerate(reps):
        n = n_at[q]
        xq = r[1] + np.mod(xs[off:off + n] - r[1], r[2] - r[1])
        ref = ora.eam(xq, r[1], r[2], [1, 1, 1], tab)
        assert_fp64(E[q], F[off:off + n], Wv[q], ref)
        off += n


def test_outer_skin_arguments(mdk):
    x, v, lo, hi = hot_argon(4, n=4)
    n = x.shape[0]
    ctx = mdk.Context(lo, hi, [1, 1, 1], np.full(n, W.MASS_AR), "mixed")
    ctx.set_potential_lj(W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    ctx.plan(W.LJ_AR.rc, 0.3)
    # not above the skin, negative, NaN, beyond 10 (rc + skin)
    for bad in (0.3, 0.1, -1.0, float("nan"), 10.0 * (W.LJ_AR.rc + 0.3) + 1.0):
        with pytest.raises(mdk.MDKError):
            ctx.set_outer_skin(bad)
    ctx.set_outer_skin(1.2)
    ctx.set_state(x, v)
    ctx.build_neighbors(W.LJ_AR.rc, 0.3)
    ctx.step(2.0, 50)
    ctx.set_outer_skin(0.0)              # off: every build is full
    ctx.build_neighbors(W.LJ_AR.rc, 0.3)
    nb0, nf0 = ctx.build_counts()
    assert nb0 == nf0
    ctx.step(2.0, 50)
    nb1, nf1 = ctx.build_counts()
    assert nb1 == nf1 and nb1 > nb0
