"""Parity of the CUDA Behler-Parrinello path (through the C ABI) with the
oracle (Sec. "Molecular dynamics with Behler-Parrinello neural networks").

Bars:
  * FP64 path: |dE| <= 1e-12 |E|; max|dF| <= 1e-12 max|F| + 1e-13 eV/A; virial
    within 1e-12 of max |W| (+1e-13); per-atom energies and virials rtol 1e-11;
  * mixed path (FP32 descriptors, network and gradients; 64-bit fixed-point
    force sums): ||dF||_rms / ||F||_rms <= 1e-4 and |dE| / N <= 2e-6 eV/atom.
    The force bar follows from the arithmetic: a G4 value sums ~1400 FP32
    terms (relative error ~ 2^-24 sqrt(1400) ~ 2e-6 each), the network
    carries it to dE/dG, and each force is a sum of ~50 neighbour gradients
    that largely cancel (|F_i| is a few percent of the largest term), so
    relative force errors of ~1e-5 are expected; 1e-4 leaves a factor ~10.
    The forces of the mixed path sum to exactly zero (each rounded neighbour
    gradient is added once with each sign) and are bitwise reproducible.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

from test_oracle_bpnn import SMALL, model as small_model

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


def bp_ctx(mdk, x, lo, hi, per, prec, m, skin=0.3, v=None, mass=W.MASS_AL, max_neighbors=0):
    n = x.shape[0]
    ctx = mdk.Context(lo, hi, per, np.full(n, mass), prec)
    ctx.set_potential_bpnn(m)
    ctx.plan(m.rc, skin, max_neighbors)
    ctx.set_state(x, v if v is not None else np.zeros((n, 3)))
    ctx.build_neighbors(m.rc, skin)
    return ctx


def al_box(seed, n=3, a=4.05, sigma=0.08):
    rng = np.random.default_rng(seed)
    x = W.fcc_lattice(n, n, n, a) + rng.normal(0, sigma, size=(4 * n ** 3, 3))
    L = n * a
    return np.mod(x, L), np.zeros(3), np.full(3, L)


def assert_fp64(E, F, Wv, ref):
    assert abs(E - ref["E"]) <= 1e-12 * abs(ref["E"]), (E, ref["E"])
    fmax = np.max(np.abs(ref["F"]))
    assert np.max(np.abs(F - ref["F"])) <= 1e-12 * fmax + 1e-13, np.max(np.abs(F - ref["F"]))
    wmax = np.max(np.abs(ref["W"]))
    assert np.max(np.abs(Wv - ref["W"])) <= 1e-12 * wmax + 1e-13


def assert_mixed(E, F, ref):
    n = F.shape[0]
    assert abs(E - ref["E"]) / n <= 2e-6, (E, ref["E"])
    rms = np.sqrt(np.mean((F - ref["F"]) ** 2)) / np.sqrt(np.mean(ref["F"] ** 2))
    assert rms <= 1e-4, rms


def test_fp64_maise_layout_periodic(mdk, ora):
    m = W.maise_like_bpnn(0)
    x, lo, hi = al_box(1)
    ctx = bp_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", m)
    E, F, Wv = ctx.compute()
    U, Wa = ctx.per_atom()
    ref = ora.bpnn(x, lo, hi, [1, 1, 1], m, per_atom=True)
    assert_fp64(E[0], F, Wv[0], ref)
    np.testing.assert_allclose(U, ref["Ea"], rtol=1e-11)
    np.testing.assert_allclose(Wa, ref["Wa"], rtol=0, atol=1e-11 * np.abs(ref["Wa"]).max())


def test_fp64_all_kinds_small_box_and_cluster(mdk, ora):
    """G1, G2 (R_s != 0), G3, G4 and G5 with several zeta and both lambdas;
    a periodic box shorter than 2 R_c (self images) and a free cluster."""
    m = small_model(**SMALL, rc=4.0, seed=21)
    rng = np.random.default_rng(22)
    L = 7.3
    x = rng.uniform(0, L, size=(14, 3))
    ctx = bp_ctx(mdk, x, [0.0] * 3, [L] * 3, [1, 1, 1], "fp64", m)
    E, F, Wv = ctx.compute()
    ref = ora.bpnn(x, [0.0] * 3, [L] * 3, [1, 1, 1], m)
    assert_fp64(E[0], F, Wv[0], ref)
    xc = rng.normal(0, 2.5, size=(25, 3))
    lo, hi = xc.min(0) - 5, xc.max(0) + 5
    c2 = bp_ctx(mdk, xc, lo, hi, [0, 0, 0], "fp64", m)
    E, F, Wv = c2.compute()
    ref = ora.bpnn(xc, lo, hi, [0, 0, 0], m)
    assert_fp64(E[0], F, Wv[0], ref)


# zetas outside {1, 2, 4, 16}: the kernel's generic power loop (the set itself
# takes the compiled ladder of squares)
GENERIC_ZETA = dict(rad=[(2, 0.05, 0.0), (3, 0.9, 0.0)],
                    ang=[(4, 3.0, 1.0, 0.01), (4, 8.0, -1.0, 0.005), (4, 1.0, 1.0, 0.02),
                         (5, 3.0, -1.0, 0.01), (5, 64.0, 1.0, 0.03), (4, 8.0, 1.0, 0.01)],
                    H=(6, 5), w_in=0.3)


@pytest.mark.parametrize("spec", ["fixed_set", "generic"])
def test_fp64_zeta_paths(mdk, ora, spec):
    """Both ways of forming (1 +- cos)^zeta: the zeta set {1, 2, 4, 16} (all
    four, both lambdas) and zetas 1, 3, 8, 64."""
    if spec == "generic":
        m = small_model(**GENERIC_ZETA, rc=4.2, seed=41)
    else:
        ang = [(k, z, lam, 0.004 * (1 + q)) for q, (k, z, lam) in enumerate(
            [(4, 1.0, 1.0), (4, 2.0, -1.0), (4, 4.0, 1.0), (4, 16.0, -1.0),
             (5, 16.0, 1.0), (5, 4.0, -1.0), (5, 2.0, 1.0), (5, 1.0, -1.0)])]
        m = small_model(rad=[(2, 0.1, 0.0)], ang=ang, H=(6, 5), w_in=0.3, rc=4.2, seed=42)
    x, lo, hi = al_box(43, n=2, sigma=0.15)
    ctx = bp_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", m)
    E, F, Wv = ctx.compute()
    ref = ora.bpnn(x, lo, hi, [1, 1, 1], m)
    assert_fp64(E[0], F, Wv[0], ref)


def test_mixed_generic_zeta(mdk, ora):
    m = small_model(**GENERIC_ZETA, rc=4.5, seed=44)
    x, lo, hi = al_box(45, sigma=0.12)
    ctx = bp_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed", m)
    E, F, Wv = ctx.compute()
    ref = ora.bpnn(x, lo, hi, [1, 1, 1], m)
    assert_mixed(E[0], F, ref)


@pytest.mark.parametrize("seed", [3, 4])
def test_mixed_matches_oracle(mdk, ora, seed):
    m = W.maise_like_bpnn(seed)
    x, lo, hi = al_box(seed, sigma=0.12)
    ctx = bp_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed", m)
    E, F, Wv = ctx.compute()
    ref = ora.bpnn(x, lo, hi, [1, 1, 1], m)
    assert_mixed(E[0], F, ref)
    q = F * 2.0 ** 40
    assert np.all(q == np.rint(q))
    assert [sum(int(v) for v in q[:, d]) for d in range(3)] == [0, 0, 0]
    _, F2, _ = ctx.compute()
    np.testing.assert_array_equal(F, F2)


def test_fp64_trajectory_matches_oracle(mdk, ora):
    m = small_model(**SMALL, rc=4.5, seed=31)
    rng = np.random.default_rng(32)
    x, lo, hi = al_box(33, n=2, sigma=0.05)
    masses = np.full(x.shape[0], W.MASS_AL)
    v = W.maxwell_velocities(rng, masses, 600.0)
    ctx = bp_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64", m, v=v)
    ctx.step(1.0, 10)
    xg, vg = ctx.get_state()
    o = ora.md_bpnn(x, v, masses, lo, hi, [1, 1, 1], 1.0, 10, 0.3, m)
    L = hi - lo
    d = xg - o["x"]
    d -= np.rint(d / L) * L
    assert np.max(np.abs(d)) < 1e-10
    np.testing.assert_allclose(vg, o["v"], rtol=0, atol=1e-11)


def test_mixed_graphs_equal_eager(mdk):
    m = W.maise_like_bpnn(7)
    outs = []
    for graphs in (True, False):
        x, lo, hi = al_box(8, n=4, sigma=0.05)
        rng = np.random.default_rng(9)
        v = W.maxwell_velocities(rng, np.full(x.shape[0], W.MASS_AL), 300.0)
        ctx = bp_ctx(mdk, x, lo, hi, [1, 1, 1], "mixed", m, v=v)
        ctx.set_graphs(graphs)
        ctx.set_thermo(5, 64)
        ctx.step(1.0, 40)
        xg, vg = ctx.get_state()
        outs.append((xg, vg, ctx.thermo()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])


def test_bad_models_are_rejected(mdk):
    x, lo, hi = al_box(1, n=2)
    ctx = mdk.Context(lo, hi, [1, 1, 1], np.full(x.shape[0], W.MASS_AL), "mixed")
    good = W.maise_like_bpnn(0)
    bad = []
    m = W.maise_like_bpnn(0)
    m.ang_par = m.ang_par.copy()
    m.ang_par[0, 0] = 1.5            # zeta not an integer
    bad.append(m)
    m = W.maise_like_bpnn(0)
    m.ang_par = m.ang_par.copy()
    m.ang_par[1] = m.ang_par[0]      # the same function twice
    bad.append(m)
    m = W.maise_like_bpnn(0, hidden=(40, 10))   # hidden layer too wide
    bad.append(m)
    m = W.maise_like_bpnn(0)
    m.ang_par = m.ang_par.copy()
    m.ang_par[:9, 2] = np.arange(9) * 0.01 + 0.1   # 9 distinct eta
    m.ang_par[:9, 0] = 1.0
    m.ang_par[:9, 1] = 1.0
    bad.append(m)
    for b in bad:
        with pytest.raises(mdk.MDKError):
            ctx.set_potential_bpnn(b)
    ctx.set_potential_bpnn(good)
    with pytest.raises(mdk.MDKError):
        ctx.set_list_kind("half")


def cutout(x, lo, hi, k, radius):
    """Atoms (with periodic images) within `radius` of atom k, k first."""
    L = hi - lo
    d = x - x[k]
    d -= np.rint(d / L) * L
    r = np.linalg.norm(d, axis=1)
    sel = np.flatnonzero(r < radius)
    sel = np.concatenate([[k], sel[sel != k]])
    return d[sel]


@pytest.mark.slow
def test_mixed_bench_size_sampled(mdk, ora):
    """The bench workload (Al-like FCC 40^3 = 256,000 atoms, 300 K, R_c 6 A,
    8 G2 + 43 G4, 10-10 network): forces of sampled atoms against the oracle
    on a cut-out of radius 2 R_c + 0.5 A around each (every energy that
    depends on the sampled atom sees its whole neighbourhood); the forces of
    the whole system sum to exactly zero."""
    wl = W.bpnn_workload()
    s = wl.systems[0]
    m = wl.extra["bpnn"]
    ctx = mdk.make_context(wl)
    ctx.step(wl.dt, 50)
    x, _ = ctx.get_state()
    E, F, _ = ctx.compute()
    assert np.all(np.sum(np.rint(F * 2.0 ** 40).astype(np.int64), axis=0) == 0)
    rng = np.random.default_rng(5)
    errs, refs = [], []
    for k in rng.choice(s.n, 2, replace=False):
        c = cutout(x, s.lo, s.hi, k, 2 * m.rc + 0.5)
        lo, hi = c.min(0) - 1.0, c.max(0) + 1.0
        r = ora.bpnn(c, lo, hi, [0, 0, 0], m)
        errs.append(F[k] - r["F"][0])
        refs.append(r["F"][0])
    errs, refs = np.array(errs), np.array(refs)
    assert np.sqrt(np.mean(errs ** 2)) <= 1e-4 * np.sqrt(np.mean(refs ** 2)) + 1e-7
