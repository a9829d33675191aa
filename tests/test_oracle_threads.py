"""The oracle's threaded driver (ora_md_run_threads, which times the oracle
on all host cores) gives the serial cell-list run's values bit for bit: the
same per-atom helpers, totals summed in the serial order.  The serial run is
itself pinned to the O(N^2) definition (neighbour sets equal brute force,
forces equal ora.lj / ora.eam)."""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W


@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_threads_equal_serial_lj(ora, nthreads):
    wl = W.config0()                 # 256 argon atoms, 100 K, dt 2 fs
    s = wl.systems[0]
    n = 40
    a = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, n, wl.skin,
                   lj_params=wl.lj)
    b = ora.md_run_threads(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, n, wl.skin,
                           nthreads, lj_params=wl.lj)
    assert a["n_builds"] == b["n_builds"] >= 2
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["v"], b["v"])
    np.testing.assert_array_equal(a["thermo"], b["thermo"])


def test_threads_equal_serial_eam(ora):
    tab = W.tabulate_fs_eam(W.AL_LIKE)
    s = W.lattice_system(np.random.default_rng(4), (4, 4, 4), 4.05, W.MASS_AL, 600.0)
    n = 15
    a = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, 1.0, n, 0.3, tables=tab)
    b = ora.md_run_threads(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, 1.0, n, 0.3, 5,
                           tables=tab)
    assert a["n_builds"] == b["n_builds"]
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["v"], b["v"])
    np.testing.assert_array_equal(a["thermo"], b["thermo"])


def test_serial_run_matches_all_pairs_definition(ora):
    # the first force evaluation of the cell-list run equals the O(N^2) one
    wl = W.config0()
    s = wl.systems[0]
    a = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, 0, wl.skin,
                   lj_params=wl.lj)
    ref = ora.lj(s.x, s.lo, s.hi, s.periodic, wl.lj.eps, wl.lj.sigma, wl.lj.rc, 1)
    fmax = np.max(np.abs(ref["F"])) + 1e-30
    assert np.max(np.abs(a["F"] - ref["F"])) <= 1e-12 * fmax + 1e-13


def test_serial_eam_run_matches_all_pairs_definition(ora):
    # the same for the Al-like EAM of the 256,000-atom workload, on a 4^3-cell box
    tab = W.tabulate_fs_eam(W.AL_LIKE)
    s = W.lattice_system(np.random.default_rng(5), (4, 4, 4), 4.05, W.MASS_AL, 300.0,
                         sigma_jitter=0.05)
    a = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, 1.0, 0, 0.3, tables=tab)
    ref = ora.eam(s.x, s.lo, s.hi, s.periodic, tab)
    fmax = np.max(np.abs(ref["F"])) + 1e-30
    assert np.max(np.abs(a["F"] - ref["F"])) <= 1e-12 * fmax + 1e-13
