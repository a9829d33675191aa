"""Oracle pins on the paper's own argon sample (tests/golden/argon_lj_mw_basic_sample.txt,
Sec. "Moving window simulation"): an FCC lattice with a = 0.462 nm under LJ with
eps = 1.0312 kJ/mol, sigma = 0.3384 nm, cut at 0.8125 nm.

* The neighbour count within the cutoff is the FCC shell count: shells at a/sqrt(2) sqrt(k)
  for k = 1..6 lie inside 8.125 Angstrom (the next shell, k = 7 with 48 atoms, is at 8.64
  Angstrom), so every atom has 12 + 6 + 24 + 12 + 24 + 8 = 86 neighbours.
* The energy per atom of the perfect lattice equals the closed-form shell sum
  1/2 sum_k z_k u(d sqrt k) (plain truncation; energy shift: minus 43 u(rc)), and the
  forces vanish.
"""
import os

import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
KJ_PER_MOL_IN_EV = 1.0 / 96.48533212331  # 1 eV = 96.485... kJ/mol


def golden():
    out = {}
    with open(os.path.join(HERE, "golden", "argon_lj_mw_basic_sample.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_paper_argon_sample(ora):
    g = golden()
    a = 10.0 * g["lattice_parameter_nm"]
    eps = g["epsilon_kJ_per_mol"] * KJ_PER_MOL_IN_EV
    sigma = 10.0 * g["sigma_nm"]
    rc = 10.0 * g["cutoff_nm"]
    n = 4
    x = W.fcc_lattice(n, n, n, a)
    L = n * a
    assert L >= 2 * rc  # one periodic image per pair
    nb = ora.neighbors(x, [0] * 3, [L] * 3, [1] * 3, rc)
    assert all(len(q) == 86 for q in nb)
    d = a / np.sqrt(2.0)
    shells = [(1, 12), (2, 6), (3, 24), (4, 12), (5, 24), (6, 8)]
    u = lambda r: 4 * eps * ((sigma / r) ** 12 - (sigma / r) ** 6)
    e_plain = 0.5 * sum(z * u(d * np.sqrt(k)) for k, z in shells)
    for mode, want in ((0, e_plain), (1, e_plain - 0.5 * 86 * u(rc))):
        r = ora.lj(x, [0] * 3, [L] * 3, [1] * 3, eps, sigma, rc, mode)
        assert r["E"] / x.shape[0] == pytest.approx(want, rel=1e-12)
        assert np.max(np.abs(r["F"])) < 1e-12
