"""How the mixed path sums its forces (and its energies and virials), measured
on the 8,388,608-atom argon workload (LJ, 80 K, thermalised for 300 steps).

The mixed full-list kernels sum each atom's FP32 pair forces with a
compensated (Kahan) FP32 sum over blocks of four pairs.  The mixed half-list
kernels evaluate the same pairs -- bitwise the same pair vectors (seen from j
the vector is exactly minus the one seen from i, for the same cells, rounded
in the same order) and the same force factors V'(r)/r -- and sum the terms
in 64-bit fixed point (unit 2^-40 eV/A), exactly up to one rounding of each
term.  With both lists built at the same positions (same
cells, same FP32 offsets), the difference of the two force sets is therefore
the error of the compensated FP32 sum against an exact (FP64-quality) sum of
the same terms.  It must sit far below the mixed-path bar (RMS 1e-5): the
compensated sum's bound is ~2u |F_i| + O(n u^2) sum |f_ij|, u = 2^-24.
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


@pytest.mark.slow
def test_compensated_fp32_force_sum_equals_exact_sum(mdk, ora):
    wl = W.config2()
    s = wl.systems[0]
    ctx = mdk.make_context(wl)
    ctx.set_launch(1, 128)
    ctx.step(wl.dt, 300)
    ctx.build_neighbors(wl.rc, wl.skin)     # lists and cells of the current positions
    x, _ = ctx.get_state()
    E_kahan, F_kahan, W_kahan = ctx.compute()   # full lists: compensated FP32 sums
    ctx.set_list_kind("half")               # rebuilt at the same positions: same cells
    E_exact, F_exact, W_exact = ctx.compute()   # half lists: 64-bit fixed-point sums
    scale = np.sqrt(np.mean(F_exact ** 2))
    d = F_kahan - F_exact
    rel_rms = np.sqrt(np.mean(d ** 2)) / scale
    rel_max = np.max(np.abs(d)) / scale
    print(f"compensated FP32 vs exact sum of the same terms: rms {rel_rms:.3e}, "
          f"max {rel_max:.3e} (of the RMS force)")
    # the block sums of four pairs are plain FP32 (~u |f_ij| each, ~20 blocks),
    # the rest compensated: ~1e-7 of the RMS force expected, bar 1e-5
    assert rel_rms <= 1e-6
    assert rel_max <= 1e-5
    # energy and virial: the full-list pass sums each atom's four-pair FP32
    # block sums with compensation too (the pair energies differ from the
    # half-list ones by at most an FP32 rounding each), so the totals agree
    # far below the mixed energy bar (1e-6 of |E|)
    E_kahan, E_exact = float(np.sum(E_kahan)), float(np.sum(E_exact))
    W_kahan, W_exact = np.asarray(W_kahan, float).ravel(), np.asarray(W_exact, float).ravel()
    dE = abs(E_kahan - E_exact) / abs(E_exact)
    dW = np.max(np.abs(W_kahan - W_exact)) / np.max(np.abs(W_exact))
    print(f"energy {dE:.3e}, virial {dW:.3e} (relative)")
    assert dE <= 1e-9
    assert dW <= 1e-8
    # and both against the FP64 oracle on sampled atoms: the pair arithmetic,
    # not the summation, sets the mixed error
    sel = np.random.default_rng(3).choice(s.n, 16, replace=False)
    ref = ora.sampled("lj", x, s.lo, s.hi, s.periodic, sel, lj_params=wl.lj)
    for F in (F_kahan, F_exact):
        rms = np.sqrt(np.mean((F[sel] - ref["F"]) ** 2)) / np.sqrt(np.mean(ref["F"] ** 2))
        assert rms <= 1e-5, rms
    ctx.close()
