"""Pins of the oracle's neighbour sets (Verlet list within r_ns = rc + skin).

* Perfect FCC lattices: every atom has exactly sum z_k neighbours for the
  shells inside r_ns (78 for LJ argon a=5.26, r_ns=8.8125; 54 for Al-like
  a=4.05, r_ns=6.3; 134 for Cu-like a=3.0, r_ns=5.8 in a 9 Angstrom box where
  several images of the same atom are neighbours).  The shell counts come
  from tests/fcc_shells.py, a sum over lattice vectors.
* Brute force on tiny random inputs equals a direct numpy enumeration.
* Symmetry: (j, n) in N(i)  <=>  (i, -n) in N(j).
* The paper's cell-list algorithm gives the same sets as brute force on
  random and lattice inputs, including grids with 1 and 2 cells per periodic
  dimension and a free dimension.
"""
import itertools

import numpy as np
import pytest

from fcc_shells import fcc_count
from paper_2511_22951_gb300 import workloads as W


def as_set(lst):
    return set(map(tuple, lst.tolist()))


def numpy_brute(x, lo, hi, per, rns):
    L = np.asarray(hi) - np.asarray(lo)
    out = []
    for i in range(x.shape[0]):
        s = set()
        for j in range(x.shape[0]):
            t = x[j] - x[i]
            ranges = []
            for k in range(3):
                if per[k]:
                    c = int(np.ceil(rns / L[k])) + 1
                    base = -int(np.rint(t[k] / L[k]))
                    ranges.append(range(base - c, base + c + 1))
                else:
                    ranges.append(range(0, 1))
            for n in itertools.product(*ranges):
                if j == i and n == (0, 0, 0):
                    continue
                d = t + np.array(n) * L
                r2 = d[0] * d[0] + d[1] * d[1]
                r2 = r2 + d[2] * d[2]
                if r2 < rns * rns:
                    s.add((j,) + tuple(n))
        out.append(s)
    return out


@pytest.mark.parametrize("a,ncell,rns,expect", [
    (5.26, 4, 8.5125 + 0.3, 78),     # LJ argon lattice
    (4.05, 4, 6.0 + 0.3, 54),        # Al-like
    (4.05, 3, 6.0 + 0.3, 54),        # L = 12.15 < 2 r_ns: two images of some atoms
    (3.0, 3, 5.5 + 0.3, 134),        # Cu-like compressed, L = 9 < 2 r_ns
])
def test_fcc_shell_counts(ora, a, ncell, rns, expect):
    assert fcc_count(a, rns) == expect
    x = W.fcc_lattice(ncell, ncell, ncell, a)
    L = ncell * a
    for method in ("brute", "cells"):
        nb = ora.neighbors(x, [0, 0, 0], [L, L, L], [1, 1, 1], rns, method=method)
        counts = np.array([len(q) for q in nb])
        assert np.all(counts == expect), (method, np.unique(counts))


def test_brute_matches_numpy_enumeration(ora):
    rng = np.random.default_rng(11)
    lo = np.array([0.0, -1.0, 2.0])
    hi = lo + np.array([7.0, 9.5, 13.0])
    per = [1, 1, 0]
    x = lo + rng.uniform(0, 1, size=(40, 3)) * (hi - lo)
    rns = 4.0
    ref = numpy_brute(x, lo, hi, per, rns)
    got = ora.neighbors(x, lo, hi, per, rns, method="brute")
    for i in range(x.shape[0]):
        assert as_set(got[i]) == ref[i]


def test_symmetry(ora):
    rng = np.random.default_rng(12)
    lo, hi = np.zeros(3), np.array([8.0, 8.0, 8.0])
    x = rng.uniform(0, 8.0, size=(60, 3))
    nb = ora.neighbors(x, lo, hi, [1, 1, 1], 5.0)
    sets = [as_set(q) for q in nb]
    for i, s in enumerate(sets):
        for (j, a, b, c) in s:
            assert (i, -a, -b, -c) in sets[j]


@pytest.mark.parametrize("L,per,n", [
    ((20.0, 20.0, 20.0), (1, 1, 1), 300),   # 3+ cells
    ((9.0, 9.0, 9.0), (1, 1, 1), 40),       # 1 cell per dimension
    ((13.0, 12.5, 30.0), (1, 1, 1), 200),   # 2 cells in x and y
    ((30.0, 14.0, 14.0), (0, 1, 1), 250),   # free x
    ((15.0, 15.0, 15.0), (0, 0, 0), 150),   # cluster, all free
])
def test_cells_equal_brute(ora, L, per, n):
    rng = np.random.default_rng(int(sum(L) * 10) + n)
    lo = np.array([-1.0, 0.5, 2.0])
    hi = lo + np.array(L)
    x = lo + rng.uniform(0, 1, size=(n, 3)) * (hi - lo)
    rns = 5.8
    a = ora.neighbors(x, lo, hi, per, rns, method="brute")
    b = ora.neighbors(x, lo, hi, per, rns, method="cells")
    for i in range(n):
        assert len(a[i]) == len(b[i])
        assert as_set(a[i]) == as_set(b[i])


def test_wrap_moves_by_whole_box_lengths(ora):
    lo, hi = np.array([0.0, -2.0, 1.0]), np.array([10.0, 3.0, 4.0])
    x = np.array([[10.0, -2.0, 0.999], [-0.5, 3.5, 7.0], [25.0, -9.0, 2.0]])
    w = ora.wrap(x, lo, hi, [1, 1, 0])
    assert np.all(w[:, :2] >= lo[:2]) and np.all(w[:, :2] < hi[:2])
    k = (x[:, :2] - w[:, :2]) / (hi[:2] - lo[:2])
    np.testing.assert_allclose(k, np.rint(k), atol=1e-12)
    np.testing.assert_array_equal(w[:, 2], x[:, 2])


@pytest.mark.parametrize("method", ["brute", "cells"])
def test_cutoff_is_strict(ora, method):
    """r^2 == r_ns^2 exactly (4.0^2 = 16 in binary) is not a neighbour; a pair
    one part in 1e12 inside is."""
    lo, hi = np.zeros(3), np.full(3, 40.0)
    x = np.array([[10.0, 10.0, 10.0], [14.0, 10.0, 10.0],
                  [10.0, 14.0 - 4e-12, 10.0], [10.0, 10.0, 14.0 + 4e-9]])
    nb = ora.neighbors(x, lo, hi, [0, 0, 0], 4.0, method=method)
    assert as_set(nb[0]) == {(2, 0, 0, 0)}
