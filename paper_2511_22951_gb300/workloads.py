"""Seeded synthetic inputs for the short-range MD hot path.

This module only *makes inputs*: FCC lattices, Gaussian jitter, Maxwell
velocities, the tabulated EAM functions (knot values) and the five workload
configurations.  It holds none of the method's arithmetic (no neighbour
search, no force, no integrator, no spline construction), so both the CUDA
path and the CPU oracle can read the same arrays without sharing any of the
code that is being checked.

Units everywhere: eV, Angstrom, fs, atomic mass unit u.

Workloads follow the paper's test problems:
  * LJ argon lattice + small perturbations, periodic cube (Sec. "Performance",
    the 13 M-atom benchmark with a list rebuild every 10 steps);
  * single-element EAM metal from a tabulated file (Sec. "Comparison of
    aluminum shock Hugoniot ...", Table 1) -- the tabulated file is replaced
    by a synthetic Finnis-Sinclair-type EAM tabulated on 5000 knots;
  * shock slab with a piston and a moving window (Sec. "Moving window
    simulation");
  * cold curve E(V) of compressed FCC copper (Sec. on the Cu cold curve),
    as 64 uneven replicas.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Boltzmann constant in eV/K (CODATA 2018, exact SI definition).
K_B = 8.617333262e-5
# 1 eV/(Angstrom*u) expressed in Angstrom/fs^2:
#   1.602176634e-19 J / 1.66053906660e-27 kg / 1e-10 m  -> m/s^2, then *1e-20.
EV_PER_A_U_TO_A_PER_FS2 = 9.648533212331e-3

MASS_AR = 39.948
MASS_AL = 26.9815385
MASS_CU = 63.546


# --------------------------------------------------------------------------
# lattices, jitter, velocities
# --------------------------------------------------------------------------
def fcc_lattice(nx: int, ny: int, nz: int, a: float,
                origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """FCC positions, shape (4*nx*ny*nz, 3), x-fastest cell order."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0],
                      [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return pos + np.asarray(origin, dtype=np.float64)[None, :]


def jitter(rng: np.random.Generator, x: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian displacement of every coordinate with standard deviation sigma."""
    return x + rng.normal(0.0, sigma, size=x.shape)


def maxwell_velocities(rng: np.random.Generator, masses: np.ndarray,
                       T: float) -> np.ndarray:
    """Maxwell-Boltzmann velocities (Angstrom/fs) at temperature T (K).

    The centre-of-mass velocity is removed and the result is rescaled to an
    instantaneous temperature of exactly T with 3N-3 degrees of freedom.
    """
    m = np.asarray(masses, dtype=np.float64)
    n = m.shape[0]
    if n == 0 or T <= 0.0:
        return np.zeros((n, 3))
    sd = np.sqrt(K_B * T / m * EV_PER_A_U_TO_A_PER_FS2)
    v = rng.normal(0.0, 1.0, size=(n, 3)) * sd[:, None]
    if n > 1:
        v -= (m[:, None] * v).sum(axis=0) / m.sum()
        ke = 0.5 * (m[:, None] * v * v).sum() / EV_PER_A_U_TO_A_PER_FS2
        t_now = 2.0 * ke / ((3 * n - 3) * K_B)
        v *= math.sqrt(T / t_now)
    return v


# --------------------------------------------------------------------------
# synthetic Finnis-Sinclair-type EAM (Morse pair, exponential density,
# square-root embedding).  The paper loads single-element EAM potentials from
# tabulated files; these parameter sets stand in for those files.
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class FSEAMParams:
    D: float        # Morse well depth (eV)
    alpha: float    # Morse stiffness (1/Angstrom)
    r0: float       # Morse minimum (Angstrom)
    beta: float     # density decay (1/Angstrom)
    re: float       # density reference distance (Angstrom)
    A: float        # embedding strength: F(rho) = -A sqrt(rho)  (eV)
    rc: float       # cutoff (Angstrom)
    mass: float     # atomic mass (u)
    a0: float       # nominal FCC lattice constant (Angstrom)
    rho_max: float = 100.0


AL_LIKE = FSEAMParams(D=0.1061, alpha=1.2, r0=3.5081, beta=1.5, re=2.8638,
                      A=1.0126, rc=6.0, mass=MASS_AL, a0=4.05)
CU_LIKE = FSEAMParams(D=0.0177, alpha=1.8, r0=3.323, beta=1.75, re=2.5562,
                      A=1.2066, rc=5.5, mass=MASS_CU, a0=3.615)


def fs_phi_raw(p: FSEAMParams, r):
    e = np.exp(-p.alpha * (np.asarray(r, dtype=np.float64) - p.r0))
    return p.D * (e * e - 2.0 * e)


def fs_dphi_raw(p: FSEAMParams, r):
    e = np.exp(-p.alpha * (np.asarray(r, dtype=np.float64) - p.r0))
    return p.D * (-2.0 * p.alpha * e * e + 2.0 * p.alpha * e)


def fs_rho_raw(p: FSEAMParams, r):
    return np.exp(-p.beta * (np.asarray(r, dtype=np.float64) - p.re))


def fs_drho_raw(p: FSEAMParams, r):
    return -p.beta * fs_rho_raw(p, r)


def _shifted_force(g, dg, p, r):
    """g(r) - g(rc) - (r-rc) g'(rc): value and slope vanish at rc."""
    r = np.asarray(r, dtype=np.float64)
    return g(p, r) - g(p, p.rc) - (r - p.rc) * dg(p, p.rc)


def fs_phi(p: FSEAMParams, r):
    """Pair term, shifted-force truncated at rc (zero beyond rc)."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < p.rc, _shifted_force(fs_phi_raw, fs_dphi_raw, p, r), 0.0)


def fs_dphi(p: FSEAMParams, r):
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < p.rc, fs_dphi_raw(p, r) - fs_dphi_raw(p, p.rc), 0.0)


def fs_rho(p: FSEAMParams, r):
    """Density term, shifted-force truncated at rc (zero beyond rc)."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < p.rc, _shifted_force(fs_rho_raw, fs_drho_raw, p, r), 0.0)


def fs_drho(p: FSEAMParams, r):
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < p.rc, fs_drho_raw(p, r) - fs_drho_raw(p, p.rc), 0.0)


def fs_embed(p: FSEAMParams, rho):
    return -p.A * np.sqrt(np.maximum(np.asarray(rho, dtype=np.float64), 0.0))


def fs_dembed(p: FSEAMParams, rho):
    rho = np.asarray(rho, dtype=np.float64)
    return -0.5 * p.A / np.sqrt(rho)


@dataclasses.dataclass
class EAMTables:
    """Knot values of the three EAM functions (the 3 x n parameters theta).

    phi and rho are sampled on r_k = k * rc/(nr-1), k = 0..nr-1 (so the last
    knot sits at rc); F is sampled on rho_k = k * rho_max/(nrho-1).
    """
    rc: float
    phi: np.ndarray
    rho: np.ndarray
    rho_max: float
    F: np.ndarray

    @property
    def nr(self) -> int:
        return int(self.phi.shape[0])

    @property
    def nrho(self) -> int:
        return int(self.F.shape[0])


def tabulate_fs_eam(p: FSEAMParams, nr: int = 5000, nrho: int = 5000) -> EAMTables:
    r = np.arange(nr, dtype=np.float64) * (p.rc / (nr - 1))
    rho = np.arange(nrho, dtype=np.float64) * (p.rho_max / (nrho - 1))
    phi_k = fs_phi(p, r)
    rho_k = fs_rho(p, r)
    phi_k[-1] = 0.0
    rho_k[-1] = 0.0
    return EAMTables(rc=p.rc, phi=phi_k, rho=rho_k, rho_max=p.rho_max,
                     F=fs_embed(p, rho))


# --------------------------------------------------------------------------
# LJ argon parameters
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class LJParams:
    eps: float = 0.0104        # eV
    sigma: float = 3.405       # Angstrom
    rc: float = 2.5 * 3.405    # Angstrom
    mass: float = MASS_AR
    shift_mode: int = 1        # 0 plain truncation, 1 energy shift, 2 shifted force


LJ_AR = LJParams()


# --------------------------------------------------------------------------
# one system (or replica) with its box
# --------------------------------------------------------------------------
@dataclasses.dataclass
class System:
    x: np.ndarray                  # (N, 3) float64
    v: np.ndarray                  # (N, 3) float64
    masses: np.ndarray             # (N,)  float64
    lo: np.ndarray                 # (3,)
    hi: np.ndarray                 # (3,)
    periodic: np.ndarray           # (3,) int32

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    systems: list                  # list[System]; one entry unless batched
    potential: str                 # "lj" | "eam" | "bpnn" (model in extra["bpnn"])
    lj: Optional[LJParams]
    eam: Optional[FSEAMParams]
    tables: Optional[EAMTables]
    dt: float
    steps: int
    skin: float
    precision: str                 # "fp64" | "mixed"
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return sum(s.n for s in self.systems)

    @property
    def rc(self) -> float:
        if self.potential == "bpnn":
            return self.extra["bpnn"].rc
        return self.lj.rc if self.potential == "lj" else self.eam.rc


@dataclasses.dataclass
class BPNNModel:
    """A Behler-Parrinello potential (Sec. "Molecular dynamics with
    Behler-Parrinello neural networks"): the cutoff R_c, the symmetry-function
    parameters and the atomic network's weights.  Parameters only."""
    rc: float
    rad_kind: np.ndarray      # int32 [n_rad]: 1, 2 or 3 (G1, G2, G3)
    rad_par: np.ndarray       # [n_rad, 2]: G2 (eta, R_s), G3 (kappa, 0), G1 unused
    ang_kind: np.ndarray      # int32 [n_ang]: 4 or 5 (G4, G5)
    ang_par: np.ndarray       # [n_ang, 3]: (zeta, lambda, eta); zeta a positive integer
    W01: np.ndarray           # [G, H1], G = n_rad + n_ang
    b1: np.ndarray            # [H1]
    W12: np.ndarray           # [H1, H2]
    b2: np.ndarray            # [H2]
    w23: np.ndarray           # [H2]
    b3: float

    @property
    def n_rad(self) -> int:
        return int(self.rad_kind.shape[0])

    @property
    def n_ang(self) -> int:
        return int(self.ang_kind.shape[0])

    @property
    def n_in(self) -> int:
        return self.n_rad + self.n_ang


def maise_like_bpnn(seed: int = 0, rc: float = 6.0, hidden=(10, 10), n_rad: int = 8,
                    n_ang: int = 43, w_in: float = 0.05, e_scale: float = 0.5,
                    e0: float = -3.0) -> BPNNModel:
    """Synthetic model with the layout the paper reports for MAISE's trained
    potentials: 8 G2 functions (one R_s, different eta) and 43 G4 functions
    per element, two hidden layers of 10.  The trained weights are not
    available, so the weights are seeded Gaussians: W01 ~ N(0, w_in^2),
    W12 ~ N(0, 1/H1), w23 ~ N(0, e_scale^2 / H2), biases ~ N(0, 0.01),
    b3 = e0 (eV)."""
    rng = np.random.default_rng(seed)
    H1, H2 = hidden
    rad_kind = np.full(n_rad, 2, dtype=np.int32)
    etas = np.geomspace(0.003, 0.5, n_rad) if n_rad > 1 else np.array([0.05])
    rad_par = np.stack([etas, np.zeros(n_rad)], 1)
    combos = [(z, lam, eta) for eta in (0.0005, 0.003, 0.01, 0.02, 0.035, 0.06)
              for z in (1.0, 2.0, 4.0, 16.0) for lam in (1.0, -1.0)]
    ang_par = np.array(combos[:n_ang], dtype=np.float64).reshape(-1, 3)
    ang_kind = np.full(ang_par.shape[0], 4, dtype=np.int32)
    G = n_rad + ang_par.shape[0]
    return BPNNModel(rc=rc, rad_kind=rad_kind, rad_par=rad_par, ang_kind=ang_kind,
                     ang_par=ang_par,
                     W01=rng.normal(0.0, w_in, size=(G, H1)),
                     b1=rng.normal(0.0, 0.1, size=H1),
                     W12=rng.normal(0.0, 1.0 / np.sqrt(H1), size=(H1, H2)),
                     b2=rng.normal(0.0, 0.1, size=H2),
                     w23=rng.normal(0.0, e_scale / np.sqrt(H2), size=H2),
                     b3=float(e0))


def lattice_system(rng, n_cells, a, mass, T, periodic=(1, 1, 1), sigma_jitter=0.0,
                   origin=(0.0, 0.0, 0.0), box_pad=None) -> System:
    nx, ny, nz = n_cells
    x = fcc_lattice(nx, ny, nz, a, origin)
    if sigma_jitter > 0.0:
        x = jitter(rng, x, sigma_jitter)
    m = np.full(x.shape[0], mass)
    v = maxwell_velocities(rng, m, T)
    lo = np.asarray(origin, dtype=np.float64).copy()
    hi = lo + np.array([nx * a, ny * a, nz * a])
    if box_pad is not None:
        lo = lo - np.asarray(box_pad[0])
        hi = hi + np.asarray(box_pad[1])
    if sigma_jitter > 0.0:
        # keep periodic coordinates inside the primary box
        for d in range(3):
            if periodic[d]:
                L = hi[d] - lo[d]
                x[:, d] = lo[d] + np.mod(x[:, d] - lo[d], L)
                x[:, d] = np.where(x[:, d] >= hi[d], x[:, d] - L, x[:, d])
    return System(x=x, v=v, masses=m, lo=lo, hi=hi,
                  periodic=np.asarray(periodic, dtype=np.int32))


def config0() -> Workload:
    """LJ argon FP64: FCC 4^3 = 256 atoms, a=5.26, 100 K (seed 0), dt=2 fs, 100 steps."""
    rng = np.random.default_rng(0)
    s = lattice_system(rng, (4, 4, 4), 5.26, MASS_AR, 100.0)
    return Workload("lj_argon_256_fp64", [s], "lj", LJ_AR, None, None,
                    dt=2.0, steps=100, skin=0.3, precision="fp64")


def config1() -> Workload:
    """Al-like FS-EAM FP64: FCC 40^3 = 256,000 atoms, a=4.05, 300 K (seed 1), dt=1 fs."""
    rng = np.random.default_rng(1)
    s = lattice_system(rng, (40, 40, 40), 4.05, MASS_AL, 300.0)
    return Workload("eam_al_256000_fp64", [s], "eam", None, AL_LIKE,
                    tabulate_fs_eam(AL_LIKE), dt=1.0, steps=1000, skin=0.3,
                    precision="fp64")


def config2(n: int = 128, precision: str = "mixed") -> Workload:
    """LJ argon, FCC n^3 cells (128^3 = 8,388,608 atoms), 80 K, dt=2 fs."""
    rng = np.random.default_rng(3)
    s = lattice_system(rng, (n, n, n), 5.26, MASS_AR, 80.0)
    return Workload(f"lj_argon_{4 * n ** 3}_{precision}", [s], "lj", LJ_AR, None,
                    None, dt=2.0, steps=10000, skin=0.3, precision=precision)


def config3(ncx: int = 400, ncyz: int = 20, precision: str = "mixed") -> Workload:
    """Al-like FS-EAM shock slab: FCC 400 x 20 x 20 cells (x free; y, z periodic),
    rigid piston at x=0 moving at 1.5 km/s = 0.015 Angstrom/fs along +x."""
    rng = np.random.default_rng(4)
    a = AL_LIKE.a0
    s = lattice_system(rng, (ncx, ncyz, ncyz), a, MASS_AL, 300.0, periodic=(0, 1, 1),
                       box_pad=((2.0 * a, 0.0, 0.0), (40.0 * a, 0.0, 0.0)))
    piston = s.x[:, 0] < 2.0 * a - 1e-9
    return Workload(f"eam_al_slab_{s.n}_{precision}", [s], "eam", None, AL_LIKE,
                    tabulate_fs_eam(AL_LIKE), dt=1.0, steps=20000, skin=0.3,
                    precision=precision,
                    extra={"piston": piston, "u_p": 0.015, "a": a,
                           "L_behind": 150.0, "L_ahead": 150.0})


def config4(n_rep: int = 64, precision: str = "mixed") -> Workload:
    """Cu-like FS-EAM cold curve: 64 FCC replicas, a ~ U(3.0, 4.2), n ~ U{3..12},
    N_r = 4 n^3, Gaussian jitter sigma = 0.05 Angstrom (seed 2), 0 K velocities."""
    rng = np.random.default_rng(2)
    a_s = rng.uniform(3.0, 4.2, size=n_rep)
    n_s = rng.integers(3, 13, size=n_rep)
    systems = []
    for a, n in zip(a_s, n_s):
        s = lattice_system(rng, (int(n), int(n), int(n)), float(a), MASS_CU, 0.0,
                           sigma_jitter=0.05)
        systems.append(s)
    return Workload(f"eam_cu_coldcurve_{n_rep}rep", systems, "eam", None, CU_LIKE,
                    tabulate_fs_eam(CU_LIKE), dt=1.0, steps=1000, skin=0.3,
                    precision=precision, extra={"a": a_s, "n": n_s})


def bpnn_workload(n: int = 40, precision: str = "mixed", seed: int = 1) -> Workload:
    """Al-like FCC n^3 cells (40^3 = 256,000 atoms, a = 4.05 A, the EAM
    config's lattice), 300 K, with the synthetic MAISE-layout BPNN
    (R_c = 6 A: 54 neighbours in the lattice, 1431 neighbour pairs per atom),
    dt = 1 fs."""
    rng = np.random.default_rng(seed)
    s = lattice_system(rng, (n, n, n), 4.05, MASS_AL, 300.0)
    return Workload(f"bpnn_al_{4 * n ** 3}_{precision}", [s], "bpnn", None, None, None,
                    dt=1.0, steps=1000, skin=0.3, precision=precision,
                    extra={"bpnn": maise_like_bpnn(0, rc=6.0)})


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}
