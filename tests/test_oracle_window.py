"""Pins of the oracle's moving-window rules (Sec. "Moving window simulation",
read for a piston-driven shock along x).

The rules are bookkeeping, so the pins are their invariants: the front at
the upper edge of the last bin whose mean v_x exceeds u_p / 2 (a lattice
shocked up to a known plane, with bins that do not line up with the planes,
gives it in closed form), atom-count balance (kept + appended), nothing left
behind the cut, appended atoms exactly at the slab positions shifted to the
leading edge, ids unique and increasing for appended atoms, the new rear
layer flagged as piston, no action when no bin moves faster than u_p / 2 on
average (a single fast atom in a thermal slab is not a front), and no copy
started past the box.
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


BIN = 3.0   # front bins: edges at -2A + 3k, never on a lattice plane


def test_window_rule_invariants(ora):
    st, s = state(ora)
    sx, sv, slx = slab()
    n0 = st.n
    before = st.view()
    # planes sit at multiples of A/2 from x = 0; those below x = 20 (the last
    # at 18.225) move at u_p; the bin [15.9, 18.9) is the last shocked one
    x_front = -2 * A + 9 * BIN
    assert abs(x_front - 18.9) < 1e-12
    x_max = before["x"][:, 0].max()
    L_behind, L_ahead, gap, depth = 8.0, 30.0, 0.5 * A, 2 * A
    ora.window_apply(st, s.lo[0], s.hi[0], BIN, 0.015, L_behind, L_ahead, sx, sv, slx, gap,
                     W.MASS_AL, depth)
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
    ora.window_apply(st, s.lo[0], s.hi[0], BIN, 0.015, 8.0, 30.0, sx, sv, slx, 2.0, W.MASS_AL,
                     8.1)
    assert st.n == n0 and not st.pis[:n0].any()


def test_single_fast_atom_is_not_a_front(ora):
    st, s = state(ora)
    st.v[:st.n, 0] = s.v[:, 0]          # thermal everywhere, no shocked region
    st.pis[:] = 0
    far = int(np.argmax(s.x[:, 0]))
    st.v[far, 0] = 0.02                 # one atom faster than u_p / 2
    sx, sv, slx = slab()
    n0 = st.n
    ora.window_apply(st, s.lo[0], s.hi[0], BIN, 0.015, 8.0, 30.0, sx, sv, slx, 0.5 * A,
                     W.MASS_AL, 2 * A)
    assert st.n == n0


def test_no_copy_starts_past_the_box(ora):
    st, s = state(ora)
    sx, sv, slx = slab()
    x_max = s.x[:, 0].max()
    gap = 0.5 * A
    x_hi = x_max + gap + 1.5 * slx      # room for one copy only
    kept_before = st.n
    ora.window_apply(st, s.lo[0], x_hi, BIN, 0.015, 8.0, 500.0, sx, sv, slx, gap, W.MASS_AL,
                     2 * A)
    v = st.view()
    new = v["ids"] >= kept_before
    assert new.sum() == sx.shape[0]
    assert v["x"][new, 0].max() < x_hi


def test_window_md_run_counts(ora):
    st, s = state(ora)
    sx, sv, slx = slab()
    wl = W.config3(ncx=12, ncyz=3)
    n0 = st.n
    nb = ora.md_window(st, s.lo, s.hi, s.periodic, wl.tables, 1.0, 12, 0.3, 5, 0.015, BIN, 8.0,
                       30.0, sx, sv, slx, 0.5 * A, W.MASS_AL, 2 * A)
    assert nb == 3
    v = st.view()
    assert len(np.unique(v["ids"])) == st.n
    assert st.n != n0
    np.testing.assert_allclose(v["v"][v["piston"]], [[0.015, 0, 0]] * v["piston"].sum())


def test_fixed_front_window(ora):
    """The paper's stationary-shock window: boundaries fixed in the box, the
    same rules with the front given instead of located (velocities play no
    part)."""
    st, s = state(ora)
    st.v[:st.n] = 0.0
    st.pis[:] = 0
    sx, sv, slx = slab()
    before = st.view()
    n0 = st.n
    x_front, L_behind, L_ahead, gap = 25.0, 8.0, 40.0, 0.5 * A
    x_max = before["x"][:, 0].max()
    ora.window_apply(st, s.lo[0], s.hi[0], BIN, 0.015, L_behind, L_ahead, sx, sv, slx, gap,
                     W.MASS_AL, 0.0, fixed_front=x_front)
    after = st.view()
    kept = before["x"][:, 0] >= x_front - L_behind
    copies = int(np.ceil((x_front + L_ahead - x_max) / slx))
    assert copies > 0 and kept.sum() < n0
    assert st.n == kept.sum() + copies * sx.shape[0]
    assert after["x"][:, 0].min() >= x_front - L_behind
    assert not after["piston"].any()  # depth 0: no piston layer
