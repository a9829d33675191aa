"""Shock Hugoniot from isotherms run as batched replicas (Sec. "Argon shock
Hugoniot: system of isotherms and a series MW simulations", Eq. RH).

Each point (V_i, T_j) of a volume-temperature grid is one replica of a
batched context, relaxed by its own Langevin thermostat
(`mdk_set_langevin_replicas`) and then sampled for its mean energy per atom
e(V, T) and pressure P(V, T).  The Hugoniot through the initial state
(v0, e0, P0) is the set of states with

    H(v, e, P) = e - e0 - (P + P0) (v0 - v) / 2 = 0,

found on every volume line of the grid by linear interpolation of e and P
in T between the two temperatures that bracket the root (the bilinear
interpolation of the grid, evaluated along its lines).  One time step serves
the whole batch: the paper's dt = 1e-2 sqrt(10 / T) ps at the grid's highest
temperature.

Host-side control and analysis only: every step runs in libmdk.so.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import mdk
from . import workloads as W


def rankine_hugoniot(e, p, v, e0, p0, v0):
    """H = e - e0 - (p + p0) (v0 - v) / 2 (per atom: e in eV, p in eV/A^3,
    v in A^3)."""
    return e - e0 - 0.5 * (p + p0) * (v0 - v)


def hugoniot_from_grid(V, T, E, P, v0, e0, p0):
    """V [nV] per-atom volumes, T [nT] ascending temperatures, E and P
    [nV, nT] per-atom energies and pressures.  Returns (v, T_H, P_H, e_H) on
    the volume lines where H changes sign between two grid temperatures."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    out = []
    for i, v in enumerate(V):
        h = rankine_hugoniot(E[i], P[i], v, e0, p0, v0)
        for j in range(T.size - 1):
            if h[j] == 0.0:
                out.append((v, T[j], P[i, j], E[i, j]))
                break
            if (h[j] < 0.0) != (h[j + 1] < 0.0):
                w = h[j] / (h[j] - h[j + 1])  # linear in T between the two points
                out.append((v, T[j] + w * (T[j + 1] - T[j]), P[i, j] + w * (P[i, j + 1] - P[i, j]),
                            E[i, j] + w * (E[i, j + 1] - E[i, j])))
                break
    if not out:
        return (np.zeros(0),) * 4
    a = np.array(out)
    return a[:, 0], a[:, 1], a[:, 2], a[:, 3]


def paper_dt(T_max):
    """The paper's time step 1e-2 sqrt(10 / T) ps, in fs, at the hottest point."""
    return 1e-2 * np.sqrt(10.0 / T_max) * 1e3


@dataclasses.dataclass
class IsothermGrid:
    """LJ argon isotherms: FCC n_cells^3 replicas whose lattice constant sets
    the per-atom volume, one replica per (V, T)."""
    a0: float                   # lattice constant of the initial state (A)
    compressions: np.ndarray    # v / v0 of each volume line (<= 1)
    temperatures: np.ndarray    # K, ascending
    n_cells: int = 4
    beta: float = 5e-4          # 1/fs (the paper's 0.5 1/ps)
    seed: int = 1
    lj: W.LJParams = W.LJ_AR

    def systems(self):
        rng = np.random.default_rng(self.seed)
        out = []
        for c in self.compressions:
            a = self.a0 * float(c) ** (1.0 / 3.0)
            for T in self.temperatures:
                out.append(W.lattice_system(rng, (self.n_cells,) * 3, a, self.lj.mass,
                                            float(T)))
        return out

    def context(self, precision="mixed", max_neighbors=0):
        ss = self.systems()
        ctx = mdk.Context([s.lo for s in ss], [s.hi for s in ss], [s.periodic for s in ss],
                          np.concatenate([s.masses for s in ss]), precision,
                          n_atoms=[s.n for s in ss])
        ctx.set_potential_lj(self.lj.eps, self.lj.sigma, self.lj.rc, self.lj.shift_mode)
        ctx.plan(self.lj.rc, 0.3, max_neighbors)
        ctx.set_state(np.concatenate([s.x for s in ss]), np.concatenate([s.v for s in ss]))
        ctx.build_neighbors(self.lj.rc, 0.3)
        Tr = np.repeat(self.temperatures[None, :], len(self.compressions), 0).ravel()
        ctx.set_langevin_replicas(Tr, np.full(Tr.size, self.beta), seed=self.seed)
        return ctx, ss

    def run(self, ctx, systems, dt, n_eq, n_samples, every):
        """Relax n_eq steps, then average e and P over n_samples thermo
        samples `every` steps apart.  Returns E, P [nV, nT] and the per-atom
        volumes [nV]."""
        ctx.set_thermo(every, capacity=max(n_samples, n_eq // every) + 4)
        ctx.step(dt, n_eq)
        ctx.thermo()  # drop the relaxation's samples
        ctx.step(dt, n_samples * every)
        th = ctx.thermo()[-n_samples:]             # [s, replica, 10]
        vol = np.array([np.prod(s.hi - s.lo) for s in systems])
        n = np.array([s.n for s in systems], dtype=np.float64)
        K, U, Wt = th[:, :, 1], th[:, :, 2], th[:, :, 4] + th[:, :, 5] + th[:, :, 6]
        e = ((K + U) / n).mean(axis=0)
        p = ((2.0 * K + Wt) / (3.0 * vol)).mean(axis=0)
        nV, nT = len(self.compressions), len(self.temperatures)
        return e.reshape(nV, nT), p.reshape(nV, nT), (vol / n).reshape(nV, nT)[:, 0]
