"""Pins of the oracle's moving-window rules (Sec. "Moving window simulation",
read for a piston-driven shock along x).

The rules are bookkeeping, so the pins are their invariants: atom-count
balance (kept + appended), nothing left behind the cut, appended atoms exactly
at the slab positions shifted to the leading edge, ids unique and increasing
for appended atoms, the new rear layer flagged as piston, and no action when
nothing moves faster than u_p / 2.
"""
import numpy as np

from paper_2511_22951_gb300 import workloads as W

A = 4.05


def slab():
    rng = np.random.default_rng(9)
    sx = W.fcc_lattice(2, 3, 3, A)
    sv = W.maxwell_velocities(rng, np.full(sx.shape[0], W.MASS_AL), 300.0)
    return sx, sv, 2 * A


def state(ora, cap=4000):
    wl = W.config3(ncx=12, ncyz=3)
    s = wl.systems[0]
    pis = wl.extra["piston"]
    v = s.v.copy()
    # a shocked region behind x = 20: moving at u_p
    v[s.x[:, 0] < 20.0, 0] = 0.015
    return ora.WindowState(s.x, v, s.masses, pis, cap), s


def test_window_rule_invariants(ora):
    st, s = state(ora)
    sx, sv, slx = slab()
    n0 = st.n
    before = st.view()
    x_front = before["x"][before["v"][:, 0] > 0.0075, 0].max()
    x_max = before["x"][:, 0].max()
    L_behind, L_ahead, gap, depth = 8.0, 30.0, 0.5 * A, 2 * A
    ora.window_apply(st, 0.015, L_behind, L_ahead, sx, sv, slx, gap, W.MASS_AL, depth)
    after = st.view()
    cut = x_front - L_behind
    kept = before["x"][:, 0] >= cut
    copies = int(np.ceil((x_front + L_ahead - x_max) / slx))
    assert copies > 0
    assert st.n == kept.sum() + copies * sx.shape[0] <= st.cap
    assert after["x"][:, 0].min() >= cut
    np.testing.assert_array_equal(after["ids"][:kept.sum()], before["ids"][kept])
    new = after["ids"][kept.sum():]
    np.testing.assert_array_equal(new, np.arange(n0, n0 + new.shape[0]))
    for c in range(copies):
        blk = after["x"][kept.sum() + c * sx.shape[0]: kept.sum() + (c + 1) * sx.shape[0]]
        np.testing.assert_allclose(blk - sx, [[x_max + gap + c * slx, 0, 0]] * sx.shape[0],
                                   rtol=0, atol=1e-12)
    x_min = after["x"][:, 0].min()
    rear = after["x"][:, 0] < x_min + depth
    assert rear.any() and np.all(after["piston"][rear])


def test_window_needs_a_front(ora):
    st, s = state(ora)
    st.v[:, 0] = 0.0
    st.pis[:] = 0
    sx, sv, slx = slab()
    n0 = st.n
    ora.window_apply(st, 0.015, 8.0, 30.0, sx, sv, slx, 2.0, W.MASS_AL, 8.1)
    assert st.n == n0 and not st.pis[:n0].any()


def test_window_md_run_counts(ora):
    st, s = state(ora)
    sx, sv, slx = slab()
    wl = W.config3(ncx=12, ncyz=3)
    n0 = st.n
    nb = ora.md_window(st, s.lo, s.hi, s.periodic, wl.tables, 1.0, 12, 0.3, 5, 0.015, 8.0, 30.0,
                       sx, sv, slx, 0.5 * A, W.MASS_AL, 2 * A)
    assert nb == 3
    v = st.view()
    assert len(np.unique(v["ids"])) == st.n
    assert st.n != n0
    np.testing.assert_allclose(v["v"][v["piston"]], [[0.015, 0, 0]] * v["piston"].sum())
