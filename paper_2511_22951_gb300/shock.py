"""The stationary-shock search of Sec. "Moving window simulation": find the
outflow velocity u_out at which a shock front stays put in the window.

The target function is F = P / P_t, the spatially averaged pressure of the
simulation domain (Appendix statistics, here from `mdk_profiles`) over the
pressure that puts the front at the wanted place.  Its least-squares slope
<dF/dt> over a run is monotonic in u_out near the optimum and vanishes
there, so u_out is found by bisection on the sign of the slope, each
evaluation a restart from the same saved state, until the bracket is
narrower than a tolerance (1 m/s = 1e-5 Angstrom/fs in the paper).

This module is host-side control only: every step runs in libmdk.so.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional, Sequence

import numpy as np

from . import mdk

M_PER_S = 1e-5  # 1 m/s in Angstrom/fs


def lsq_slope(t: Sequence[float], f: Sequence[float]) -> float:
    """Slope of the least-squares line through (t_m, F(t_m))."""
    t = np.asarray(t, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    tc = t - t.mean()
    den = float(tc @ tc)
    if den == 0.0:
        raise ValueError("need samples at two or more distinct times")
    return float(tc @ (f - f.mean())) / den


def dichotomy(slope_at: Callable[[float], float], u_min: float, u_max: float,
              tol: float = M_PER_S, max_iter: int = 60):
    """Bisection on the sign of <dF/dt>(u_out) between u_min and u_max, whose
    slopes must have opposite signs.  Returns (u_out, history) with history a
    list of (u_out, slope)."""
    s_lo, s_hi = slope_at(u_min), slope_at(u_max)
    hist = [(u_min, s_lo), (u_max, s_hi)]
    if s_lo == 0.0:
        return u_min, hist
    if s_hi == 0.0:
        return u_max, hist
    if (s_lo > 0) == (s_hi > 0):
        raise ValueError("the slopes at u_min and u_max have the same sign")
    lo, hi = u_min, u_max
    for _ in range(max_iter):
        if abs(hi - lo) < tol:
            break
        mid = 0.5 * (lo + hi)
        s = slope_at(mid)
        hist.append((mid, s))
        if s == 0.0:
            return mid, hist
        if (s > 0) == (s_lo > 0):
            lo, s_lo = mid, s
        else:
            hi = mid
    return 0.5 * (lo + hi), hist


@dataclasses.dataclass
class StationaryWindow:
    """A stationary-shock window set-up: EAM tables, box (x free), the saved
    state to restart from, the inflow slab, the window boundaries and the
    thermostat regions (the outflow region's target velocity is u_out)."""
    tables: object
    lo: np.ndarray
    hi: np.ndarray
    periodic: np.ndarray
    x: np.ndarray
    v: np.ndarray
    masses: np.ndarray
    slab_x: np.ndarray
    slab_v: np.ndarray
    slab_lx: float
    slab_gap: float
    slab_mass: float
    x_front: float
    L_behind: float
    L_ahead: float
    inflow: tuple          # (x_lo, x_hi, T, beta), target velocity (u_in, 0, 0)
    outflow: tuple         # (x_lo, x_hi, T, beta), target velocity (u_out, 0, 0)
    u_in: float
    P_t: float             # target pressure (eV/A^3)
    domain: tuple          # (x_lo, x_hi) over which P is averaged
    cross_area: float
    precision: str = "mixed"
    dt: float = 1.0
    capacity_factor: float = 1.5
    seed: int = 1
    max_neighbors: int = 0  # list capacity (0: from the density; shocks compress)

    def context(self, u_out: float):
        n = self.x.shape[0]
        ctx = mdk.Context(self.lo, self.hi, self.periodic, self.masses, self.precision,
                          capacity=int(n * self.capacity_factor))
        ctx.set_potential_eam(self.tables)
        ctx.plan(self.tables.rc, 0.3, self.max_neighbors)
        ctx.set_state(self.x, self.v)
        ctx.build_neighbors(self.tables.rc, 0.3)
        ctx.set_window(self.L_behind, self.L_ahead, self.slab_x, self.slab_v, self.slab_lx,
                       self.slab_gap, self.slab_mass, 0.0, self.slab_lx,
                       fixed_front=self.x_front)
        il, ih, iT, ib = self.inflow
        ol, oh, oT, ob = self.outflow
        ctx.set_langevin([(ol, oh, oT, (u_out, 0.0, 0.0), ob),
                          (il, ih, iT, (self.u_in, 0.0, 0.0), ib)], seed=self.seed)
        return ctx

    def target(self, ctx) -> float:
        """F = P / P_t with P the mean pressure of the domain (one bin)."""
        d0, d1 = self.domain
        prof = ctx.profiles(0, d0, d1 - d0, 1, self.cross_area)
        P = float(np.mean(prof[0, 9:12]))
        return P / self.P_t

    def slope(self, u_out: float, n_samples: int = 20, every: int = 50,
              on_sample: Optional[Callable[[int, float], None]] = None) -> float:
        """<dF/dt> over n_samples samples `every` steps apart, restarting from
        the saved state with the outflow thermostat at u_out."""
        ctx = self.context(u_out)
        ts, fs = [], []
        for m in range(n_samples):
            ctx.step(self.dt, every)
            f = self.target(ctx)
            ts.append((m + 1) * every * self.dt)
            fs.append(f)
            if on_sample:
                on_sample(m, f)
        ctx.close()
        return lsq_slope(ts, fs)
