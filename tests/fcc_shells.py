"""Closed-form FCC lattice geometry for the oracle pins.

Lattice vectors of the FCC lattice with cubic constant a are (a/2)(i, j, k)
with integer i, j, k and i + j + k even.  Shell k (squared distance
k * d^2, d = a/sqrt(2) the nearest-neighbour distance) holds z_k sites:
12, 6, 24, 12, 24, 8, 48, 6, 36, 24, ...  These sums replace the atom loops of
the oracle by a sum over distances and are independent of its periodic-image
logic.
"""
import numpy as np


def fcc_shells(a: float, rmax: float):
    """Return (distances, multiplicities) of FCC lattice sites with 0 < r < rmax."""
    m = int(np.ceil(2.0 * rmax / a)) + 1
    r = np.arange(-m, m + 1)
    i, j, k = np.meshgrid(r, r, r, indexing="ij")
    keep = ((i + j + k) % 2 == 0)
    v = np.stack([i[keep], j[keep], k[keep]], axis=1) * (a / 2.0)
    d2 = (v * v).sum(axis=1)
    # group by integer squared half-units to avoid float grouping issues
    key = (i[keep] ** 2 + j[keep] ** 2 + k[keep] ** 2)
    out_d, out_z = [], []
    for q in np.unique(key):
        if q == 0:
            continue
        dist = np.sqrt(q) * a / 2.0
        if dist < rmax:
            out_d.append(dist)
            out_z.append(int((key == q).sum()))
    del d2
    return np.array(out_d), np.array(out_z)


def fcc_count(a: float, rmax: float) -> int:
    return int(fcc_shells(a, rmax)[1].sum())
