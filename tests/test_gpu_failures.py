"""Failure detection on the GPU, made from host-side inputs (no fault, trap
or hang is ever caused): a list capacity below the neighbour count, a
non-finite position, a moving window with no room left to append atoms.
Each case must come back as a status code, and the context must stay usable."""
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


def argon(seed=5):
    rng = np.random.default_rng(seed)
    x = W.jitter(rng, W.fcc_lattice(4, 4, 4, 5.26), 0.05)
    L = 4 * 5.26
    return x, [0.0] * 3, [L] * 3, [1, 1, 1]


def test_list_overflow_grows_the_capacity(mdk, ora):
    x, lo, hi, per = argon()
    lj = W.LJ_AR
    ctx = mdk.Context(lo, hi, per, np.full(x.shape[0], lj.mass), "fp64")
    ctx.set_potential_lj(lj.eps, lj.sigma, lj.rc, 1)
    ctx.plan(lj.rc, 0.3, max_neighbors=16)        # 78 are needed
    ctx.set_state(x)
    r = ctx.lib.mdk_build_neighbors(ctx.h, lj.rc, 0.3)
    assert r == mdk.MDK_ERR_NEIGH_OVERFLOW
    ctx.build_neighbors(lj.rc, 0.3)               # the binding grows the workspace
    assert np.all(ctx.neighbor_counts() == 78)
    E, F, _ = ctx.compute()
    ref = ora.lj(x, lo, hi, per, lj.eps, lj.sigma, lj.rc, 1)
    assert abs(E[0] - ref["E"]) <= 1e-12 * abs(ref["E"])


def test_nonfinite_position_is_reported(mdk):
    x, lo, hi, per = argon(6)
    x[17, 1] = np.nan
    lj = W.LJ_AR
    ctx = mdk.Context(lo, hi, per, np.full(x.shape[0], lj.mass), "mixed")
    ctx.set_potential_lj(lj.eps, lj.sigma, lj.rc, 1)
    ctx.plan(lj.rc, 0.3)
    ctx.set_state(x)
    r = ctx.lib.mdk_build_neighbors(ctx.h, lj.rc, 0.3)
    assert r == mdk.MDK_ERR_NONFINITE
    # the context stays usable: a finite state computes normally
    x2, *_ = argon(6)
    ctx.set_state(x2)
    ctx.build_neighbors(lj.rc, 0.3)
    E, F, _ = ctx.compute()
    assert np.isfinite(E[0]) and np.all(np.isfinite(F))


def test_window_without_room_reports_capacity(mdk):
    wl = W.config3(ncx=12, ncyz=3)
    s = wl.systems[0]
    a = wl.extra["a"]
    v = s.v.copy()
    v[s.x[:, 0] < 20.0, 0] = 0.015
    rng = np.random.default_rng(9)
    sx = W.fcc_lattice(2, 3, 3, a)
    sv = W.maxwell_velocities(rng, np.full(sx.shape[0], W.MASS_AL), 300.0)
    ctx = mdk.Context(s.lo, s.hi, s.periodic, s.masses, "fp64", capacity=s.n)  # no room
    ctx.set_potential_eam(wl.tables)
    ctx.plan(wl.tables.rc, 0.3, rebuild_every=5)
    ctx.set_state(s.x, v)
    ctx.build_neighbors(wl.tables.rc, 0.3)
    ctx.set_piston(0.015, wl.extra["piston"])
    ctx.set_window(8.0, 200.0, sx, sv, 2 * a, 0.5 * a, W.MASS_AL, 2 * a, 3.0)
    with pytest.raises(mdk.MDKError) as e:
        ctx.step(0.5, 6)
    assert e.value.code == mdk.MDK_ERR_CAPACITY
    # nothing was appended, the atoms that remain are still consistent
    ins, dele = ctx.window_counts()
    assert ins == 0 and ctx.natoms() == s.n - dele
