"""Pins of the oracle's EAM adjoint (gradient of L = gE E + sum_i gF_i . F_i
with respect to the 3 x n knot values of phi, rho and F).

* E and F are linear in the phi knots and in the F knots, so L is too: central
  differences are exact up to rounding there, for any step.
* rho knots: central differences with Richardson extrapolation.
* Forward mode (dual numbers through the whole evaluation) gives the
  directional derivative along a random knot tangent v; the reverse-mode
  gradient must satisfy <grad, v> = JVP(v) (dot-product test), and the JVP is
  itself pinned to finite differences.
* Closed forms that need no chain rule: a constant shift of the phi knots
  moves E by 1/2 x (directed pairs inside rc) and leaves F; a constant shift
  of the F knots moves E by N and leaves F; phi knots on a straight line
  (phi(r) = r, reproduced exactly by the spline) give the derivative along
  that line as 1/2 gE sum r + sum_i gF_i . sum_j d^_ij; a linear embedding
  F = c rho makes the rho-knot gradient exactly 2c times the phi-knot one.
* Coverage of the spline ends: a free random cluster puts pairs in the first
  and last radial intervals and densities in the first F interval; a
  density table cut below the largest rho_i covers the linear continuation.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W


def small_tables(p, nr=300, nrho=300, rho_max=None):
    t = W.tabulate_fs_eam(p, nr=nr, nrho=nrho)
    if rho_max is None:
        return t
    r = np.arange(nrho) * (rho_max / (nrho - 1))
    return W.EAMTables(rc=t.rc, phi=t.phi, rho=t.rho, rho_max=rho_max, F=W.fs_embed(p, r))


def with_knots(t, phi=None, rho=None, F=None):
    return W.EAMTables(rc=t.rc, phi=t.phi if phi is None else phi,
                       rho=t.rho if rho is None else rho, rho_max=t.rho_max,
                       F=t.F if F is None else F)


def crystal(seed=7):
    rng = np.random.default_rng(seed)
    x = W.jitter(rng, W.fcc_lattice(3, 3, 3, 3.5), 0.08)
    L = 3 * 3.5
    return x, [0.0] * 3, [L] * 3, [1, 1, 1], rng


def cluster(seed=3, n=36, side=9.0):
    """Free random gas plus isolated dimers at chosen separations: pairs in the
    first and the last radial intervals and densities in the first F interval."""
    rng = np.random.default_rng(seed)
    x = [rng.uniform(0.0, side, size=(n, 3))]
    for q, r in enumerate((0.006, 0.025, 0.045, 5.3, 5.495)):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        a = np.array([20.0 + 10.0 * q, 20.0, 20.0])
        x.append(np.stack([a, a + r * u]))
    x = np.concatenate(x)
    return x, [-1.0] * 3, [80.0] * 3, [0, 0, 0], rng


def loss(ora, sysm, t, gE, gF):
    x, lo, hi, per, _ = sysm
    r = ora.eam(x, lo, hi, per, t)
    return gE * r["E"] + float(np.sum(gF * r["F"]))


def pair_vectors(ora, x, lo, hi, per, rc):
    """All directed pairs inside rc: (i, j, d_ij) with d = x_j - x_i + n L."""
    L = np.asarray(hi) - np.asarray(lo)
    nb = ora.neighbors(x, lo, hi, per, rc)
    rows = []
    for i, a in enumerate(nb):
        for j, nx, ny, nz in a:
            d = x[j] - x[i] + np.array([nx, ny, nz]) * L
            rows.append((i, j, d))
    return rows


def knots_to_check(g, count=12):
    """Nonzero-gradient knots, spread over the support, ends included."""
    nz = np.nonzero(g)[0]
    assert nz.size > 0
    pick = set(nz[np.linspace(0, nz.size - 1, min(count, nz.size)).astype(int)].tolist())
    return sorted(pick)


@pytest.mark.parametrize("which", ["crystal", "cluster"])
def test_linear_knots_match_central_differences(ora, which):
    sysm = crystal() if which == "crystal" else cluster()
    x, lo, hi, per, rng = sysm
    t = small_tables(W.CU_LIKE)
    gE = 0.7
    gF = rng.normal(size=x.shape)
    dphi, _, dF = ora.eam_vjp(x, lo, hi, per, t, gE, gF)
    scale_p = np.max(np.abs(dphi))
    scale_F = np.max(np.abs(dF))
    for k in knots_to_check(dphi):
        e = np.zeros(t.nr)
        e[k] = 1e-2
        fd = (loss(ora, sysm, with_knots(t, phi=t.phi + e), gE, gF) -
              loss(ora, sysm, with_knots(t, phi=t.phi - e), gE, gF)) / 2e-2
        assert abs(dphi[k] - fd) <= 1e-10 * scale_p, (k, dphi[k], fd)
    for k in knots_to_check(dF):
        e = np.zeros(t.nrho)
        e[k] = 1e-2
        fd = (loss(ora, sysm, with_knots(t, F=t.F + e), gE, gF) -
              loss(ora, sysm, with_knots(t, F=t.F - e), gE, gF)) / 2e-2
        assert abs(dF[k] - fd) <= 1e-10 * scale_F, (k, dF[k], fd)


def test_cluster_reaches_the_table_ends(ora):
    x, lo, hi, per, rng = cluster()
    t = small_tables(W.CU_LIKE)
    dphi, drho, dF = ora.eam_vjp(x, lo, hi, per, t, 1.0, rng.normal(size=x.shape))
    # first knots (one-sided slope row) and the last radial knots are reached
    assert np.all(dphi[:3] != 0) and np.all(drho[:3] != 0)
    assert np.all(dphi[-3:] != 0) and np.all(drho[-3:] != 0)
    assert np.all(dF[:3] != 0)


@pytest.mark.parametrize("which", ["crystal", "cluster"])
def test_rho_knots_match_richardson_differences(ora, which):
    sysm = crystal() if which == "crystal" else cluster()
    x, lo, hi, per, rng = sysm
    t = small_tables(W.CU_LIKE)
    gE = 0.7
    gF = rng.normal(size=x.shape)
    _, drho, _ = ora.eam_vjp(x, lo, hi, per, t, gE, gF)
    scale = np.max(np.abs(drho))

    def fd(k, h):
        e = np.zeros(t.nr)
        e[k] = h
        return (loss(ora, sysm, with_knots(t, rho=t.rho + e), gE, gF) -
                loss(ora, sysm, with_knots(t, rho=t.rho - e), gE, gF)) / (2 * h)

    for k in knots_to_check(drho, 8):
        rich = (4 * fd(k, 1e-5) - fd(k, 2e-5)) / 3
        # the F spline is C1 only: a density that crosses an F knot under the
        # perturbation leaves an O(h) term, hence 1e-7 and not 1e-10
        assert abs(drho[k] - rich) <= 1e-7 * scale, (k, drho[k], rich)


@pytest.mark.parametrize("which", ["crystal", "cluster"])
def test_reverse_mode_matches_forward_mode(ora, which):
    x, lo, hi, per, rng = crystal(11) if which == "crystal" else cluster(5)
    t = small_tables(W.CU_LIKE)
    gE = -1.3
    gF = rng.normal(size=x.shape)
    g = ora.eam_vjp(x, lo, hi, per, t, gE, gF)
    for _ in range(3):
        v = [rng.normal(size=t.nr), rng.normal(size=t.nr), rng.normal(size=t.nrho)]
        _, dL = ora.eam_jvp(x, lo, hi, per, t, v[0], v[1], v[2], gE, gF)
        dot = sum(float(a @ b) for a, b in zip(g, v))
        assert dot == pytest.approx(dL, rel=1e-12)


def test_forward_mode_matches_differences(ora):
    sysm = crystal(13)
    x, lo, hi, per, rng = sysm
    t = small_tables(W.CU_LIKE)
    gE, gF = 0.4, rng.normal(size=x.shape)
    v = [rng.normal(size=t.nr), rng.normal(size=t.nr), rng.normal(size=t.nrho)]
    L0, dL = ora.eam_jvp(x, lo, hi, per, t, v[0], v[1], v[2], gE, gF)
    assert L0 == pytest.approx(loss(ora, sysm, t, gE, gF), rel=1e-13)

    def fd(h):
        tp = with_knots(t, t.phi + h * v[0], t.rho + h * v[1], t.F + h * v[2])
        tm = with_knots(t, t.phi - h * v[0], t.rho - h * v[1], t.F - h * v[2])
        return (loss(ora, sysm, tp, gE, gF) - loss(ora, sysm, tm, gE, gF)) / (2 * h)

    rich = (4 * fd(1e-6) - fd(2e-6)) / 3
    assert dL == pytest.approx(rich, rel=1e-7)


def test_constant_shifts(ora):
    x, lo, hi, per, rng = crystal(17)
    t = small_tables(W.CU_LIKE)
    n_pairs = len(pair_vectors(ora, x, lo, hi, per, t.rc))
    dphi, _, dF = ora.eam_vjp(x, lo, hi, per, t, 1.0, None)
    # E = 1/2 sum phi + sum F: a constant c added to every knot adds c
    assert dphi.sum() == pytest.approx(0.5 * n_pairs, rel=1e-12)
    assert dF.sum() == pytest.approx(x.shape[0], rel=1e-12)
    # a constant adds nothing to a force
    gF = rng.normal(size=x.shape)
    dphi, _, dF = ora.eam_vjp(x, lo, hi, per, t, 0.0, gF)
    assert abs(dphi.sum()) <= 1e-11 * np.abs(dphi).sum()
    assert abs(dF.sum()) <= 1e-11 * np.abs(dF).sum()


@pytest.mark.parametrize("which", ["crystal", "cluster"])
def test_linear_phi_direction(ora, which):
    x, lo, hi, per, rng = crystal(19) if which == "crystal" else cluster(9)
    t = small_tables(W.CU_LIKE)
    gE = 0.9
    gF = rng.normal(size=x.shape)
    dphi, _, _ = ora.eam_vjp(x, lo, hi, per, t, gE, gF)
    r_k = np.arange(t.nr) * (t.rc / (t.nr - 1))
    want = 0.0
    for i, j, d in pair_vectors(ora, x, lo, hi, per, t.rc):
        r = np.sqrt(d @ d)
        want += 0.5 * gE * r + gF[i] @ (d / r)
    assert float(dphi @ r_k) == pytest.approx(want, rel=1e-11)


def test_linear_embedding_makes_rho_gradient_proportional(ora):
    x, lo, hi, per, rng = crystal(23)
    t = small_tables(W.CU_LIKE)
    c = -0.41
    lin = with_knots(t, F=c * np.arange(t.nrho) * (t.rho_max / (t.nrho - 1)))
    gF = rng.normal(size=x.shape)
    dphi, drho, _ = ora.eam_vjp(x, lo, hi, per, lin, 0.6, gF)
    np.testing.assert_allclose(drho, 2 * c * dphi, rtol=0, atol=1e-11 * np.abs(dphi).max())


def test_density_above_the_table(ora):
    """rho_max below the largest density: F continues linearly (F'' = 0)."""
    x, lo, hi, per, rng = crystal(29)
    t0 = small_tables(W.CU_LIKE)
    rho = ora.eam(x, lo, hi, per, t0)["rho"]
    t = small_tables(W.CU_LIKE, nrho=40, rho_max=float(np.median(rho)))
    sysm = (x, lo, hi, per, rng)
    gE, gF = 0.8, rng.normal(size=x.shape)
    r = ora.eam(x, lo, hi, per, t)
    assert r["rho_flag"]
    dphi, drho, dF = ora.eam_vjp(x, lo, hi, per, t, gE, gF)
    for k in (t.nrho - 3, t.nrho - 2, t.nrho - 1):
        e = np.zeros(t.nrho)
        e[k] = 1e-2
        fd = (loss(ora, sysm, with_knots(t, F=t.F + e), gE, gF) -
              loss(ora, sysm, with_knots(t, F=t.F - e), gE, gF)) / 2e-2
        assert abs(dF[k] - fd) <= 1e-10 * np.abs(dF).max(), (k, dF[k], fd)

    def fd_rho(k, h):
        e = np.zeros(t.nr)
        e[k] = h
        return (loss(ora, sysm, with_knots(t, rho=t.rho + e), gE, gF) -
                loss(ora, sysm, with_knots(t, rho=t.rho - e), gE, gF)) / (2 * h)

    for k in knots_to_check(drho, 5):
        rich = (4 * fd_rho(k, 1e-5) - fd_rho(k, 2e-5)) / 3
        assert abs(drho[k] - rich) <= 1e-7 * np.abs(drho).max(), (k, drho[k], rich)
