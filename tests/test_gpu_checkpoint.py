"""Checkpoint / resume and list overflow during stepping, on the GPU.

* A run split as 1000 steps + checkpoint + a new context + 1000 steps is
  bitwise the run of 2000 steps in one call (positions, velocities, build
  counts), with Langevin thermostats on (the noise is keyed by the permanent
  id and the step counter the checkpoint carries): mixed and FP64, full and
  half lists, one- and two-level lists (FP64 half lists sum with FP64 atomics
  in a varying order, so there the runs agree to rounding, within 1e-8 A).  Loading replays the last list
  builds at the saved build positions, so cells, order and lists are the
  saving run's.
* A list that outgrows its capacity in a build during the steps (Sec.
  "Neighbor lists construction": every pair within r_ns must be listed)
  stops the steps there; the binding grows the workspace, carries the
  mid-step state over and finishes the steps.  The result is bitwise the run
  with a capacity large enough from the start, the thermo samples are all
  there, and the FP64 run equals the oracle's velocity Verlet over the same
  steps (positions within 1e-9 A, velocities within 1e-11 A/fs).
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LJ = W.LJ_AR


@pytest.fixture(scope="module")
def mdk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk as m
    _build.build()
    m.load()
    return m


def argon(n=8, T=80.0, seed=11):
    return W.lattice_system(np.random.default_rng(seed), (n, n, n), 5.26, LJ.mass, T)


def make(mdk, s, prec, kind, outer, lang=True, max_neighbors=0):
    ctx = mdk.Context(s.lo, s.hi, s.periodic, s.masses, prec)
    ctx.set_potential_lj(LJ.eps, LJ.sigma, LJ.rc, LJ.shift_mode)
    ctx.set_list_kind(kind)
    ctx.plan(LJ.rc, 0.3, max_neighbors)
    if outer:
        ctx.set_outer_skin(outer)
    ctx.set_launch(1, 128)
    if lang:
        ctx.set_langevin([(-1e30, 1e30, 120.0, (0.0, 0.0, 0.0), 2e-3)], seed=5)
    return ctx


# FP64 half lists add pair forces with FP64 atomics, whose order varies from
# run to run: that kind is reproducible to rounding only, so its resumed run
# is compared within 1e-8 A instead of bit for bit
CASES = [("mixed", "full", 0.0), ("mixed", "half", 0.0), ("fp64", "full", 0.0),
         ("mixed", "full", 1.5), ("fp64", "full", 1.5), ("mixed", "half", 1.5),
         ("fp64", "half", 0.0)]


@pytest.mark.parametrize("prec,kind,outer", CASES)
def test_checkpoint_resume_is_bitwise(mdk, prec, kind, outer):
    s = argon()
    dt = 2.0
    a = make(mdk, s, prec, kind, outer)
    a.set_state(s.x, s.v)
    a.step(dt, 2000)
    xa, va = a.get_state()
    ba = a.counters()[0]
    a.close()

    b = make(mdk, s, prec, kind, outer)
    b.set_state(s.x, s.v)
    b.step(dt, 1000)
    ck = b.save_checkpoint()
    nb1 = b.counters()[0]
    b.close()
    c = make(mdk, s, prec, kind, outer)
    c.load_checkpoint(ck)
    assert c.counters() == (nb1, 1000)
    c.step(dt, 1000)
    xc, vc = c.get_state()
    assert c.counters() == (ba, 2000)
    assert ba > 10   # the runs crossed many displacement-triggered builds
    if prec == "fp64" and kind == "half":
        assert np.max(np.abs(xc - xa)) < 1e-8 and np.max(np.abs(vc - va)) < 1e-10
    else:
        np.testing.assert_array_equal(xc, xa)
        np.testing.assert_array_equal(vc, va)
    c.close()


def test_checkpoint_into_a_context_without_workspace_and_back(mdk):
    s = argon(n=6)
    a = make(mdk, s, "mixed", "full", 0.0)
    a.set_state(s.x, s.v)
    a.step(2.0, 50)
    ck = a.save_checkpoint()
    x0, v0 = a.get_state()
    b = make(mdk, s, "mixed", "full", 0.0)
    b.load_checkpoint(ck)           # allocates the workspace first
    x1, v1 = b.get_state()
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(v1, v0)
    # a checkpoint of another precision is refused
    c = make(mdk, s, "fp64", "full", 0.0)
    c.set_state(s.x, s.v)
    with pytest.raises(mdk.MDKError) as e:
        c.load_checkpoint(ck)
    assert e.value.code == mdk.MDK_ERR_BAD_ARG
    for q in (a, b, c):
        q.close()


def colliding_slabs(u=0.04, seed=3):
    """Argon slab, x free, y and z periodic; the two halves move towards each
    other at u (Angstrom/fs): the interface compresses and the neighbour
    counts there grow within a few steps."""
    rng = np.random.default_rng(seed)
    nx, nyz, a = 12, 4, 5.26
    x = W.fcc_lattice(nx, nyz, nyz, a) + rng.normal(0.0, 0.03, (4 * nx * nyz * nyz, 3))
    m = np.full(x.shape[0], LJ.mass)
    v = W.maxwell_velocities(rng, m, 40.0)
    mid = 0.5 * nx * a
    v[:, 0] += np.where(x[:, 0] < mid, u, -u)
    lo = np.array([-20.0, 0.0, 0.0])
    hi = np.array([nx * a + 20.0, nyz * a, nyz * a])
    x[:, 1:] = np.mod(x[:, 1:], nyz * a)
    return W.System(x=x, v=v, masses=m, lo=lo, hi=hi, periodic=np.array([0, 1, 1]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overflow_during_steps_regrows_and_finishes(mdk, ora, prec):
    s = colliding_slabs()
    dt, n = 2.0, 24
    # the capacity the initial lists need, rounded to whole groups of 8
    probe = make(mdk, s, prec, "full", 0.0, lang=False)
    probe.set_state(s.x, s.v)
    probe.build_neighbors(LJ.rc, 0.3)
    m0 = int(probe.neighbor_counts().max())
    probe.close()
    tight = make(mdk, s, prec, "full", 0.0, lang=False, max_neighbors=m0)
    tight.set_thermo(2, capacity=64)
    tight.set_state(s.x, s.v)
    tight.step(dt, n)
    assert tight.regrows >= 1          # a build during the steps overflowed
    xt, vt = tight.get_state()
    th = tight.thermo()
    np.testing.assert_array_equal(th[:, 0, 0], np.arange(2, n + 1, 2))
    assert tight.counters()[1] == n

    roomy = make(mdk, s, prec, "full", 0.0, lang=False, max_neighbors=m0 + 64)
    roomy.set_state(s.x, s.v)
    roomy.step(dt, n)
    xr, vr = roomy.get_state()
    assert roomy.regrows == 0
    assert roomy.counters() == tight.counters()
    np.testing.assert_array_equal(xt, xr)
    np.testing.assert_array_equal(vt, vr)
    if prec == "fp64":
        o = ora.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, dt, n, 0.3, lj_params=LJ)
        assert np.max(np.abs(xt - o["x"])) < 1e-9
        assert np.max(np.abs(vt - o["v"])) < 1e-11
        assert tight.counters()[0] == o["n_builds"]
    tight.close()
    roomy.close()
