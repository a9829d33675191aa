"""Pins of the oracle's Behler-Parrinello potential (Sec. "Molecular dynamics
with Behler-Parrinello neural networks": Eqs. E_as_sum, G1-G5, AtomicNN and
force).

* Descriptors against closed forms on small geometries where every distance
  and angle is known: dimers (f_c, G1, G2 with the Gaussian's square, G3),
  an equilateral triangle, a linear trimer and a square-planar cluster
  (these fix the unordered-pair counting, the angle's vertex and the R_jk
  factor of G4 against G5).
* The network: zero weights give E_i = b3 exactly (linear output layer); a
  one-unit network gives the closed form of Eq. AtomicNN with tanh on the
  hidden layers.
* Forces equal -dE/dx by central differences (cluster, and a periodic box
  short enough that atoms see their own images); the sum of forces is zero;
  E is invariant under translation, rotation and relabelling; the virial's
  diagonal equals -L dE/dL under a homogeneous stretch; E is continuous as a
  neighbour crosses R_c; a perfect FCC lattice has equal descriptors on every
  atom and zero forces; NVE with the potential conserves energy.
"""
import math

import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

RC = 6.0


def fc(R, rc=RC):
    return 0.5 * (math.cos(math.pi * R / rc) + 1.0) if R < rc else 0.0


def model(rad=(), ang=(), H=(2, 2), seed=0, rc=RC, zero=False, w_in=0.05):
    """rad: [(kind, p0, p1)], ang: [(kind, zeta, lambda, eta)]."""
    rng = np.random.default_rng(seed)
    nr, na = len(rad), len(ang)
    G = nr + na
    H1, H2 = H
    rk = np.array([r[0] for r in rad], dtype=np.int32)
    rp = np.array([[r[1], r[2]] for r in rad], dtype=np.float64).reshape(nr, 2)
    ak = np.array([a[0] for a in ang], dtype=np.int32)
    ap = np.array([[a[1], a[2], a[3]] for a in ang], dtype=np.float64).reshape(na, 3)
    f = 0.0 if zero else 1.0
    return W.BPNNModel(rc=rc, rad_kind=rk, rad_par=rp, ang_kind=ak, ang_par=ap,
                       W01=f * rng.normal(0, w_in, (G, H1)), b1=f * rng.normal(0, 0.1, H1),
                       W12=f * rng.normal(0, 0.7, (H1, H2)), b2=f * rng.normal(0, 0.1, H2),
                       w23=f * rng.normal(0, 0.5, H2), b3=-1.0)


def big_box(x):
    lo = np.min(x, 0) - 20.0
    hi = np.max(x, 0) + 20.0
    return lo, hi, [0, 0, 0]


def desc(ora, x, m):
    lo, hi, per = big_box(x)
    return ora.bpnn(x, lo, hi, per, m, descriptors=True)["G"]


# ----------------------------------------------------------------- descriptors
@pytest.mark.parametrize("R,want", [(RC / 2, 0.5), (RC / 3, 0.75), (2 * RC / 3, 0.25),
                                    (RC + 0.1, 0.0)])
def test_cutoff_function_on_a_dimer(ora, R, want):
    m = model(rad=[(1, 0.0, 0.0)])
    G = desc(ora, np.array([[0.0, 0.0, 0.0], [R, 0.0, 0.0]]), m)
    np.testing.assert_allclose(G[:, 0], [want, want], rtol=0, atol=1e-15)


def test_radial_functions_on_a_dimer(ora):
    R = 2.5
    m = model(rad=[(2, 0.7, R), (2, 0.1, 0.0), (3, 1.3, 0.0)])
    G = desc(ora, np.array([[0.0, 0.0, 0.0], [0.0, R, 0.0]]), m)
    f = fc(R)
    # R_s = R: the Gaussian is 1 whatever eta is
    assert G[0, 0] == pytest.approx(f, abs=1e-15)
    assert G[0, 1] == pytest.approx(math.exp(-0.1 * R * R) * f, rel=1e-14)
    assert G[0, 2] == pytest.approx(math.cos(1.3 * R) * f, rel=1e-14)
    np.testing.assert_allclose(G[1], G[0], rtol=1e-15)


def test_angular_functions_on_an_equilateral_triangle(ora):
    a = 2.7
    x = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0], [a / 2, a * math.sqrt(3) / 2, 0.0]])
    ang = [(4, 1.0, 1.0, 0.01), (4, 2.0, -1.0, 0.02), (5, 4.0, 1.0, 0.005), (5, 1.0, -1.0, 0.0)]
    m = model(ang=ang)
    G = desc(ora, x, m)
    f = fc(a)
    for q, (kind, z, lam, eta) in enumerate(ang):
        base = 2.0 ** (1 - z) * (1 + lam * 0.5) ** z
        if kind == 4:
            want = base * math.exp(-eta * 3 * a * a) * f ** 3
        else:
            want = base * math.exp(-eta * 2 * a * a) * f ** 2
        np.testing.assert_allclose(G[:, q], want, rtol=1e-13)


def test_angular_functions_linear_trimer(ora):
    a = 2.2
    x = np.array([[-a, 0.0, 0.0], [0.0, 0.0, 0.0], [a, 0.0, 0.0]])
    m = model(ang=[(4, 1.0, 1.0, 0.01), (4, 3.0, -1.0, 0.01), (5, 2.0, -1.0, 0.03)])
    G = desc(ora, x, m)
    # centre atom: one pair at 180 degrees, R_jk = 2a
    assert G[1, 0] == pytest.approx(0.0, abs=1e-15)      # (1 - 1)^zeta
    want = 2.0 ** (1 - 3) * 2.0 ** 3 * math.exp(-0.01 * (2 * a * a + 4 * a * a)) * \
        fc(a) ** 2 * fc(2 * a)
    assert G[1, 1] == pytest.approx(want, rel=1e-13)
    want5 = 2.0 ** (1 - 2) * 2.0 ** 2 * math.exp(-0.03 * 2 * a * a) * fc(a) ** 2
    assert G[1, 2] == pytest.approx(want5, rel=1e-13)
    # end atom: neighbours at a and 2a on the same side (cos = 1)
    want_end = 2.0 ** 0 * 2.0 * math.exp(-0.01 * (a * a + 4 * a * a + a * a)) * \
        fc(a) * fc(2 * a) * fc(a)
    assert G[0, 0] == pytest.approx(want_end, rel=1e-13)


def test_square_planar_counts_each_angle_once(ora):
    a = 2.5
    x = np.array([[0.0, 0.0, 0.0], [a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0]])
    m = model(ang=[(5, 1.0, 1.0, 0.0), (5, 1.0, -1.0, 0.0), (4, 1.0, 1.0, 0.0)])
    G = desc(ora, x, m)
    f = fc(a)
    # 6 unordered pairs of the 4 neighbours: 4 at 90 degrees, 2 at 180
    assert G[0, 0] == pytest.approx(4 * f * f, rel=1e-13)
    assert G[0, 1] == pytest.approx(8 * f * f, rel=1e-13)
    want4 = 4 * f * f * fc(a * math.sqrt(2)) + 0.0 * 2 * f * f * fc(2 * a)
    assert G[0, 2] == pytest.approx(want4, rel=1e-13)


# ----------------------------------------------------------------- network
def test_zero_weights_give_the_output_bias(ora):
    m = model(rad=[(2, 0.1, 0.0)], ang=[(4, 1.0, 1.0, 0.01)], zero=True)
    m.b3 = 5.0
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 6, size=(9, 3))
    lo, hi, per = big_box(x)
    r = ora.bpnn(x, lo, hi, per, m, per_atom=True)
    np.testing.assert_array_equal(r["Ea"], np.full(9, 5.0))
    np.testing.assert_array_equal(r["F"], np.zeros((9, 3)))


def test_one_unit_network_closed_form(ora):
    m = model(rad=[(1, 0.0, 0.0)], H=(1, 1))
    m.W01[:] = 0.8
    m.b1[:] = 0.1
    m.W12[:] = -1.3
    m.b2[:] = 0.2
    m.w23[:] = 0.6
    m.b3 = 0.25
    R = 3.1
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    lo, hi, per = big_box(x)
    r = ora.bpnn(x, lo, hi, per, m, per_atom=True)
    Ei = 0.25 + 0.6 * math.tanh(0.2 - 1.3 * math.tanh(0.1 + 0.8 * fc(R)))
    np.testing.assert_allclose(r["Ea"], [Ei, Ei], rtol=1e-13)


# ----------------------------------------------------------------- forces
SMALL = dict(rad=[(2, 0.05, 0.0), (2, 0.4, 2.5), (3, 0.9, 0.0), (1, 0.0, 0.0)],
             ang=[(4, 1.0, 1.0, 0.01), (4, 2.0, -1.0, 0.005), (4, 16.0, 1.0, 0.02),
                  (5, 4.0, -1.0, 0.01), (5, 1.0, 1.0, 0.03)],
             H=(5, 4), w_in=0.3)


def cluster(seed, n=10, spread=3.2):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, spread, size=(n, 3))
    return x


def fd_check(ora, x, lo, hi, per, m, idx, h=1e-5, rtol=1e-7):
    r = ora.bpnn(x, lo, hi, per, m)
    F = r["F"]
    scale = np.max(np.abs(F))
    for (i, k) in idx:
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        Ep = ora.bpnn(xp, lo, hi, per, m)["E"]
        Em = ora.bpnn(xm, lo, hi, per, m)["E"]
        fd = -(Ep - Em) / (2 * h)
        assert abs(fd - F[i, k]) <= rtol * scale + 1e-12, (i, k, fd, F[i, k])
    return r


def test_forces_are_minus_the_gradient_cluster(ora):
    m = model(**SMALL)
    x = cluster(2)
    lo, hi, per = big_box(x)
    idx = [(i, k) for i in (0, 3, 7) for k in range(3)]
    r = fd_check(ora, x, lo, hi, per, m, idx)
    np.testing.assert_allclose(r["F"].sum(0), 0.0, atol=1e-13 * np.abs(r["F"]).max())


def test_forces_are_minus_the_gradient_small_periodic_box(ora):
    """L = 7.3 < 2 R_c: every atom also sees periodic images of itself."""
    m = model(**SMALL, seed=3)
    rng = np.random.default_rng(4)
    L = 7.3
    x = rng.uniform(0, L, size=(6, 3))
    idx = [(i, k) for i in (0, 5) for k in range(3)]
    r = fd_check(ora, x, [0.0] * 3, [L] * 3, [1, 1, 1], m, idx)
    np.testing.assert_allclose(r["F"].sum(0), 0.0, atol=1e-12 * np.abs(r["F"]).max())


def test_maise_layout_forces_fd(ora):
    m = W.maise_like_bpnn(5, rc=5.0)
    x = cluster(6, n=7, spread=2.0)
    lo, hi, per = big_box(x)
    fd_check(ora, x, lo, hi, per, m, [(1, 0), (1, 2), (4, 1)])


def test_invariances(ora):
    m = model(**SMALL, seed=7)
    x = cluster(8)
    lo, hi, per = big_box(x)
    r0 = ora.bpnn(x, lo, hi, per, m, per_atom=True)
    # translation
    r1 = ora.bpnn(x + np.array([0.37, -1.1, 2.9]), lo + 5, hi + 5, per, m)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-13)
    np.testing.assert_allclose(r1["F"], r0["F"], rtol=0, atol=1e-12 * np.abs(r0["F"]).max())
    # rotation: E unchanged, F rotates
    th = 0.83
    Rm = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rm = Rm @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)],
                        [0, math.sin(0.4), math.cos(0.4)]])
    xr = x @ Rm.T
    lo2, hi2, _ = big_box(xr)
    r2 = ora.bpnn(xr, lo2, hi2, per, m)
    assert r2["E"] == pytest.approx(r0["E"], rel=1e-13)
    np.testing.assert_allclose(r2["F"], r0["F"] @ Rm.T, rtol=0,
                               atol=1e-12 * np.abs(r0["F"]).max())
    # relabelling
    p = np.random.default_rng(9).permutation(x.shape[0])
    r3 = ora.bpnn(x[p], lo, hi, per, m, per_atom=True)
    assert r3["E"] == pytest.approx(r0["E"], rel=1e-13)
    np.testing.assert_allclose(r3["F"], r0["F"][p], rtol=0, atol=1e-13)
    np.testing.assert_allclose(r3["Ea"], r0["Ea"][p], rtol=1e-14)


def test_virial_diagonal_is_minus_L_dE_dL(ora):
    m = model(**SMALL, seed=11)
    rng = np.random.default_rng(12)
    L = np.array([8.1, 7.6, 9.0])
    x = rng.uniform(0, 1, size=(8, 3)) * L
    r = ora.bpnn(x, [0.0] * 3, L, [1, 1, 1], m, per_atom=True)
    np.testing.assert_allclose(r["Wa"].sum(0), r["W"], rtol=1e-13, atol=1e-14)
    h = 1e-6
    for d in range(3):
        s = np.ones(3)
        s[d] = 1 + h
        Ep = ora.bpnn(x * s, [0.0] * 3, L * s, [1, 1, 1], m)["E"]
        s[d] = 1 - h
        Em = ora.bpnn(x * s, [0.0] * 3, L * s, [1, 1, 1], m)["E"]
        want = -(Ep - Em) / (2 * h)
        assert r["W"][d] == pytest.approx(want, rel=1e-6, abs=1e-9)


def test_energy_is_continuous_at_the_cutoff(ora):
    m = model(**SMALL, seed=13)
    x = cluster(14, n=6, spread=1.5)
    lo, hi, per = big_box(x)
    far = np.array([[RC, 0, 0]]) + x[0]
    e = []
    for dR in (-1e-4, 1e-4):
        y = np.vstack([x, far + np.array([[dR, 0, 0]])])
        e.append(ora.bpnn(y, lo - 10, hi + 10, per, m)["E"])
    assert abs(e[1] - e[0]) < 1e-9


def test_perfect_lattice(ora):
    m = W.maise_like_bpnn(1, rc=5.0)
    x = W.fcc_lattice(2, 2, 2, 4.05)
    L = 2 * 4.05
    r = ora.bpnn(x, [0.0] * 3, [L] * 3, [1, 1, 1], m, per_atom=True, descriptors=True)
    np.testing.assert_allclose(r["G"], np.broadcast_to(r["G"][0], r["G"].shape), rtol=1e-12)
    assert np.abs(r["F"]).max() < 1e-12


def test_md_conserves_energy(ora):
    m = model(**SMALL, seed=15)
    rng = np.random.default_rng(16)
    x = W.fcc_lattice(2, 2, 2, 4.05) + rng.normal(0, 0.05, (32, 3))
    L = 8.1
    masses = np.full(32, W.MASS_AL)
    v = W.maxwell_velocities(rng, masses, 300.0)
    o = ora.md_bpnn(x, v, masses, [0.0] * 3, [L] * 3, [1, 1, 1], 0.5, 100, 0.3, m)
    etot = o["thermo"][:, 0] + o["thermo"][:, 1]
    assert np.ptp(etot) < 2e-3 * np.ptp(o["thermo"][:, 1]) + 1e-7
