"""mdk_lj_compute_noalloc: the entry point for callers that cannot allocate
device memory (their memory belongs to another allocator, or their loop must
not pay for allocations).  It keeps its scratch in a fixed-size array inside
the library, so this test checks, through the C ABI, that two calls in a row
each give the oracle's energy and forces at the FP64 bars (the shared
scratch keeps the previous call's contents, which must not leak into the
next call), that a non-finite coordinate shows as NaN in that atom's forces
and in the energy while every other atom gets the forces of the system
without it, and that sizes above the fixed maximum are refused before any
GPU work.  Collected last on purpose (file name)."""
import ctypes

import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LJ = W.LJ_AR


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk
    _build.build()
    return torch, mdk, mdk.load()


def systems():
    rng = np.random.default_rng(21)
    out = []
    # 256-atom argon lattice with thermal-size jitter (one 2-cell grid)
    s = W.config0().systems[0]
    out.append((np.mod(s.x + rng.normal(0, 0.1, s.x.shape), 21.04), s.lo, s.hi, [1, 1, 1]))
    # 4000 atoms: several thread blocks, a ragged last block, 5 cells per side
    x = W.fcc_lattice(10, 10, 10, 5.26) + rng.normal(0, 0.12, (4000, 3))
    out.append((np.mod(x, 52.6), np.zeros(3), np.full(3, 52.6), [1, 1, 1]))
    # free x dimension with atoms leaving the box on both ends
    x = W.fcc_lattice(6, 4, 4, 5.26) + rng.normal(0, 0.1, (384, 3))
    x[:, 1:] = np.mod(x[:, 1:], 21.04)
    out.append((x, np.array([2.0, 0.0, 0.0]), np.array([29.0, 21.04, 21.04]), [0, 1, 1]))
    return out


def call(torch, lib, x, lo, hi, per, shift_mode=1):
    P = ctypes.c_void_p
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    Fd = torch.full(xd.shape, 7.0, dtype=torch.float64, device="cuda")
    Ed = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    lo_ = np.ascontiguousarray(lo, dtype=np.float64)
    hi_ = np.ascontiguousarray(hi, dtype=np.float64)
    per_ = np.ascontiguousarray(per, dtype=np.int32)
    st = torch.cuda.current_stream().cuda_stream
    r = lib.mdk_lj_compute_noalloc(P(xd.data_ptr()), x.shape[0], lo_.ctypes.data_as(P),
                                   hi_.ctypes.data_as(P), per_.ctypes.data_as(P), LJ.eps,
                                   LJ.sigma, LJ.rc, shift_mode, P(Fd.data_ptr()),
                                   P(Ed.data_ptr()), P(st))
    torch.cuda.synchronize()
    return r, float(Ed.item()), Fd.cpu().numpy()


def test_noalloc_matches_oracle_on_two_calls(env, ora):
    torch, mdk, lib = env
    for mode in (1, 2):
        for x, lo, hi, per in systems():
            ref = ora.lj(x, lo, hi, per, LJ.eps, LJ.sigma, LJ.rc, mode)
            fmax = np.max(np.abs(ref["F"]))
            for _ in range(2):
                r, E, F = call(torch, lib, x, lo, hi, per, mode)
                assert r == 0
                assert abs(E - ref["E"]) <= 1e-12 * abs(ref["E"])
                assert np.max(np.abs(F - ref["F"])) <= 1e-12 * fmax + 1e-13


def test_noalloc_nonfinite_coordinate_shows_as_nan(env, ora):
    torch, mdk, lib = env
    x, lo, hi, per = systems()[1]
    bad = 1234
    xb = x.copy()
    xb[bad, 1] = np.nan
    xb[bad + 1, 2] = np.inf
    keep = np.ones(x.shape[0], dtype=bool)
    keep[[bad, bad + 1]] = False
    ref = ora.lj(x[keep], lo, hi, per, LJ.eps, LJ.sigma, LJ.rc, 1)
    fmax = np.max(np.abs(ref["F"]))
    for _ in range(2):
        r, E, F = call(torch, lib, xb, lo, hi, per)
        assert r == 0
        assert np.isnan(E)
        assert np.all(np.isnan(F[~keep]))
        assert np.all(np.isfinite(F[keep]))
        assert np.max(np.abs(F[keep] - ref["F"])) <= 1e-12 * fmax + 1e-13
    # the next call with finite input is clean again
    r, E, F = call(torch, lib, x, lo, hi, per)
    ref = ora.lj(x, lo, hi, per, LJ.eps, LJ.sigma, LJ.rc, 1)
    assert r == 0 and abs(E - ref["E"]) <= 1e-12 * abs(ref["E"])


def test_noalloc_refuses_sizes_above_the_maximum(env):
    torch, mdk, lib = env
    P = ctypes.c_void_p
    lo = np.zeros(3)
    hi = np.full(3, 40.0)
    per = np.ones(3, dtype=np.int32)
    # checked on the host before any launch: the pointers are never read
    dummy = torch.zeros(3, dtype=torch.float64, device="cuda")
    r = lib.mdk_lj_compute_noalloc(P(dummy.data_ptr()), 32769,
                                   lo.ctypes.data_as(P), hi.ctypes.data_as(P),
                                   per.ctypes.data_as(P), LJ.eps, LJ.sigma, LJ.rc, 1,
                                   P(dummy.data_ptr()), P(dummy.data_ptr()), None)
    assert r == mdk.MDK_ERR_TOO_LARGE
    assert b"maximum" in lib.mdk_status_string(r)
    big = np.full(3, 2000.0)     # 234^3 cells of size >= rc: above the cell maximum
    r = lib.mdk_lj_compute_noalloc(P(dummy.data_ptr()), 1, lo.ctypes.data_as(P),
                                   big.ctypes.data_as(P), per.ctypes.data_as(P), LJ.eps,
                                   LJ.sigma, LJ.rc, 1, P(dummy.data_ptr()),
                                   P(dummy.data_ptr()), None)
    assert r == mdk.MDK_ERR_TOO_LARGE
