"""The rule behind two-level lists, checked with the oracle's brute-force
neighbour sets (no GPU): an outer list of every pair within R1 = rc + s1 at
positions X0 contains every pair within R0 = rc + s0 at positions X1 as long
as no atom moved more than (s1 - s0) / 2 between them, so filtering the outer
list by the exact distance test at X1 gives the Verlet list at X1.  The bound
is tight: two atoms that close in by a little more than s1 - s0 between the
builds form a pair the outer list does not hold.
"""
import numpy as np

import oracle as ora


def pairs(lists):
    return [set(tuple(r) for r in q.tolist()) for q in lists]


def filtered(outer, x, L, r0):
    """Keep the (j, image) entries of the outer list within r0 at x."""
    out = []
    for i, q in enumerate(outer):
        keep = set()
        for (j, nx, ny, nz) in q:
            d = x[j] + np.array([nx, ny, nz]) * L - x[i]
            if d @ d < r0 * r0:
                keep.add((j, nx, ny, nz))
        out.append(keep)
    return out


def random_box(seed, n=400, L=20.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, size=(n, 3)), np.zeros(3), np.full(3, L)


def moved(rng, x, dmax, lo, hi):
    """Each atom moved by at most dmax (uniform direction and length), the
    result wrapped into the box (images change with it)."""
    u = rng.normal(size=x.shape)
    u /= np.linalg.norm(u, axis=1)[:, None]
    y = x + u * (dmax * rng.uniform(0, 1, size=(x.shape[0], 1)))
    L = hi - lo
    return lo + np.mod(y - lo, L)


def test_filter_of_the_outer_list_is_the_verlet_list():
    rc, s0, s1 = 3.0, 0.3, 1.2
    r0, r1 = rc + s0, rc + s1
    budget = 0.5 * (s1 - s0)
    for seed in range(3):
        x0, lo, hi = random_box(seed)
        L = hi - lo
        outer = pairs(ora.neighbors(x0, lo, hi, [1, 1, 1], r1))
        rng = np.random.default_rng(100 + seed)
        # positions are wrapped at both builds, so an atom that crossed the box
        # edge changes its images: compare as (j, pair vector) instead
        x1 = moved(rng, x0, budget * (1 - 1e-9), lo, hi)
        ref = ora.neighbors(x1, lo, hi, [1, 1, 1], r0)
        # the outer list's images refer to x0: re-image each entry at x1
        got = []
        for i, q in enumerate(outer):
            keep = set()
            for (j, nx, ny, nz) in q:
                d = x1[j] - x1[i]
                d -= np.rint(d / L) * L          # L > 2 r1: one image per pair
                if d @ d < r0 * r0:
                    keep.add(j)
            got.append(keep)
        want = [set(q[:, 0].tolist()) for q in ref]
        assert got == want


def test_the_budget_is_tight():
    rc, s0, s1 = 3.0, 0.3, 1.2
    r0, r1 = rc + s0, rc + s1
    lo, hi = np.zeros(3), np.full(3, 30.0)
    # two atoms just outside R1, then each moves a little more than the budget
    # towards the other: they end inside R0, a pair the outer list misses
    eps = 1e-3
    x0 = np.array([[10.0, 15.0, 15.0], [10.0 + r1 + eps, 15.0, 15.0]])
    outer = pairs(ora.neighbors(x0, lo, hi, [1, 1, 1], r1))
    assert outer == [set(), set()]
    step = 0.5 * (s1 - s0) + eps
    x1 = x0 + np.array([[step, 0, 0], [-step, 0, 0]])
    ref = pairs(ora.neighbors(x1, lo, hi, [1, 1, 1], r0))
    assert ref == [{(1, 0, 0, 0)}, {(0, 0, 0, 0)}]
    assert filtered(outer, x1, hi - lo, r0) != ref
    # within the budget: a pair just inside R1 that closes in by a little less
    # than s1 - s0 ends inside R0 and is found
    x0b = np.array([[10.0, 15.0, 15.0], [10.0 + r1 - 3 * eps, 15.0, 15.0]])
    outer_b = pairs(ora.neighbors(x0b, lo, hi, [1, 1, 1], r1))
    step_b = 0.5 * (s1 - s0) - eps
    x1b = x0b + np.array([[step_b, 0, 0], [-step_b, 0, 0]])
    ref_b = pairs(ora.neighbors(x1b, lo, hi, [1, 1, 1], r0))
    assert ref_b == [{(1, 0, 0, 0)}, {(0, 0, 0, 0)}]
    assert filtered(outer_b, x1b, hi - lo, r0) == ref_b
