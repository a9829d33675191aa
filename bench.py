"""Throughput of the MD hot path on GB300: atom-timesteps/s.

One bench step = one velocity-Verlet NVE timestep of the whole path: force
loop, integration, displacement check and -- whenever an atom has moved more
than skin/2 -- the cell-list Verlet-list rebuild (all in libmdk.so kernels).

Default workload: LJ argon, FCC 128^3 cells = 8,388,608 atoms, 80 K, dt = 2 fs,
skin 0.3 Angstrom, mixed precision (FP32 pair arithmetic, FP64 positions,
velocities and integration).  Inputs live in HBM and the per-step working set
(~4 GB) is larger than L2, so no L2 flush is needed between steps.  The
Verlet lists are two-level there (--outer, default 2.1 Angstrom: rebuilds
filter an outer list while the displacement budget lasts; --outer 0 for
one-level lists); the same trigger and the same lists either way.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config C] [--impl reference]

The default run also reports, outside the timed region: `e2e`, the same
metric through the C ABI from pinned host buffers (upload of x and v, a list
build, the steps, download of x and v, mdk_compute for E; timed on the host
around the second such call, the first warming the buffers); the same workload
on the FP64 path (`fp64_path`); the NVE drift of the mixed path over 10^4 steps and
of the FP64 path over 2000 steps, each with its own throughput (`drift`); a
1000-step steady-state segment with its list and full builds
(`steady_state`); and the metric's EAM half (`eam`): the Cu-like cold-curve
batch (64 uneven replicas, one context) and the Al-like bulk (256,000 atoms),
each mixed against FP64 with rooflines and both drifts, plus the adjoint of
the batch.  --no-eam, --drift-steps 0 and --steady-steps 0 skip them.

Other workloads (--config): 0 LJ argon 256 atoms FP64; 1 Al-like EAM 256,000
atoms FP64; 3 Al-like EAM shock slab (640,000 atoms, x free) with the rigid
piston and the moving window, mixed; 4 Cu-like EAM cold curve, 64 uneven
replicas in one batched context, mixed, plus --vjps adjoint calls of the loss
sum_r E_r + sum_i |F_i - F_ref,i|^2.  --drift-steps S adds an NVE drift
measurement (mixed S steps, FP64 --drift-fp64-steps steps).

--impl reference times the CPU oracle (the FP64 C program written from the
paper; cell-list Verlet MD, threaded over all host cores for LJ and EAM) on a
bounded sample of the same workload.
Multi-GPU (torchrun): replicas only -- every rank runs its own copy of the
workload on its own GPU; no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_22951_gb300 import workloads as W  # noqa: E402

METRIC = "atom-timesteps/s on 1 GB300 (LJ, EAM): mixed/batched vs FP64 at stated drift"
UNIT = "atom-timesteps/s"


def job_throughput(ms, atoms, steps, dist=None, device="cpu"):
    """Whole-job atom-timesteps/s: the atoms of every rank over the slowest
    rank's time (replicas: each rank steps its own copy of the workload).
    Returns (value, max ms)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        a = torch.tensor([float(atoms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
        ms, atoms = float(t.item()), float(a.item())
    return atoms * steps / (ms / 1e3), ms


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
def workload(cfg: int, cells: int = 128):
    if cfg == 0:
        return W.config0()
    if cfg == 1:
        return W.config1()
    if cfg == 2:
        return W.config2(n=cells)
    if cfg == 3:
        return W.config3()
    if cfg == 4:
        return W.config4()
    raise SystemExit(f"config {cfg} is not a bench workload")


def algorithmic_bytes_per_atom(wl, prec, n_list, kind="full"):
    """Bytes one force pass with the velocity-Verlet update must move per
    atom (n_list: mean entries of the list in use).  LJ, full lists (one
    kernel): own gather-copy element, list entries and count, x and v read +
    write, the reference of the displacement test (the build-time FP32
    offset in the mixed path, x_ref in FP64) and the cell word read, next
    gather-copy element written.  LJ,
    half lists: the same with half the entries, plus the per-atom force
    accumulators written and read once (the pair pass and the per-atom pass
    that finishes the step).  EAM adds the density pass: its own gather-copy
    element, list and count again, rho_i and F'(rho_i) written, F'(rho_i)
    read back.  Neighbour positions are assumed to come from cache (spatial
    order)."""
    g = 16 if prec == "mixed" else 32
    ref = 16 if prec == "mixed" else 24   # build-time offset (float4) or x_ref (FP64)
    lj = g + 4 * n_list + 4 + 48 + 48 + ref + 4 + g
    if wl.potential == "lj":
        if kind == "cells":   # no list entries and no list length
            return lj - 4
        return lj + (48 if kind == "half" else 0)
    if wl.potential == "bpnn":   # full list, force accumulators like half lists
        return lj + 48
    r = 4 if prec == "mixed" else 8
    return lj + g + 4 * n_list + 4 + 8 + r + r


# DRAM bytes per atom of one force-pass launch (dram__bytes_read.sum +
# dram__bytes_write.sum from an ncu capture, divided by the atoms of the
# captured case), valid only for the kernel sources they were taken from:
# the sha256 of those files is checked at run time and `traffic` is null
# when any of them changed since.
TRAFFIC = {
    ("lj", "mixed", "full"): {
        "bytes_per_atom": 464.4,
        "neighbors_per_atom": 78.0,
        "threads_per_atom": 1,
        "sources_sha256": "49ba2014f7f327c6495ca9ff5146e60010b11389a26d8e8d5d99d2a27f4bd60a",
        "capture": "k_lj<Mixed, kStep, T=1>, 3 launches on 2,048,000 atoms (80^3 FCC cells, "
                   "the same lattice and 78 neighbours per atom): dram__bytes_read.sum + "
                   "dram__bytes_write.sum = 951.1 MB per launch; per-atom traffic does not "
                   "depend on N, so it is scaled to the workload by its atom count"},
}
_CSRC = "paper_2511_22951_gb300/csrc/"
TRAFFIC_SOURCES = {
    "full": tuple(_CSRC + f for f in ("k_lj.cu", "lj_pair.cuh", "k_pair.cuh",
                                      "mdk_internal.cuh")),
    "half": tuple(_CSRC + f for f in ("k_lj_half.cu", "lj_pair.cuh", "k_pair.cuh",
                                      "mdk_internal.cuh")),
}


def sources_sha256(kind="full"):
    import hashlib
    h = hashlib.sha256()
    for p in TRAFFIC_SOURCES[kind]:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_per_launch(wl, prec, n_atoms, kind="full", n_avg=None, tpa=None):
    """Measured DRAM bytes per launch, when the captured kernel (same sources,
    same list length and launch shape) is the one this run uses; else None."""
    t = TRAFFIC.get((wl.potential, prec, kind))
    if t is None or t["sources_sha256"] != sources_sha256(kind):
        return None
    if n_avg is not None and abs(n_avg - t["neighbors_per_atom"]) > 1e-9:
        return None
    if tpa is not None and tpa != t["threads_per_atom"]:
        return None
    return t["bytes_per_atom"] * n_atoms


# FP64 arithmetic per unordered pair inside rc (one FMA = 2): LJ 23;
# EAM 22 (density pass: pair vector, r, spline value) + 40 (force pass:
# pair vector, r, two spline derivatives, force).  A full list evaluates every
# pair twice; that doubling is overhead, not algorithmic work.
FLOPS_PER_PAIR = {"lj": 23.0, "eam": 62.0}
FP64_PEAK_TFLOPS = 1.25   # GB300 nominal dense FP64 (no measured figure exists)
# FP32 FMA peak from unit counts: 152 SMs x 128 FP32 lanes x 2 FLOP at the
# maximum SM clock (2070 MHz); no measured FP32 figure exists
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def bpnn_flops_per_atom(m, n):
    """Algorithmic FP work of one BPNN force pass per atom with n neighbours
    within R_c (one FMA = 2, a transcendental = 1), counted from the
    arithmetic of the method: per unordered neighbour pair, the angular
    forward terms (cosine and pair geometry 21, each (eta, kind) group 7, each
    zeta group 12, each function 2) and the gradients of both neighbours from
    one evaluation (geometry 50, each group 30, each zeta group 8, each
    function 16); per neighbour, the radial functions (16 each); per atom,
    the network forward and reverse pass.  The kernel evaluates each
    pair's gradient once per ordered pair (twice), which is overhead and not
    counted."""
    ak = np.asarray(m.ang_kind)
    ap = np.asarray(m.ang_par).reshape(-1, 3)
    nY = len({(float(e), int(k)) for e, k in zip(ap[:, 2], ak)})
    nZ = len({float(z) for z in ap[:, 0]})
    nS, nR = ap.shape[0], int(np.asarray(m.rad_kind).shape[0])
    H1, H2 = m.W01.shape[1], m.W12.shape[1]
    pairs = n * (n - 1) / 2.0
    per_pair = (21 + 7 * nY + 12 * nZ + 2 * nS) + (50 + 30 * nY + 8 * nZ + 16 * nS)
    net = 2 * 2 * ((nR + nS) * H1 + H1 * H2 + H2) + 4 * (H1 + H2)
    return pairs * per_pair + n * 16 * nR + net


def pair_count_within_rc(ctx, wl, sample=20000, seed=0):
    """Mean number of neighbours inside rc per atom, every periodic image
    counted, from a random sample of atoms (host k-d tree).  Used for the
    pair-interactions/s figure only."""
    from scipy.spatial import cKDTree
    x, _ = ctx.get_state()
    rng = np.random.default_rng(seed)
    rc = wl.rc
    total, counted, off = 0.0, 0, 0
    n_all = x.shape[0]
    for s in wl.systems:
        n = s.n if len(wl.systems) > 1 else n_all
        xs = x[off:off + n] - s.lo
        off += n
        L = s.hi - s.lo
        per = np.asarray(s.periodic) > 0
        k = min(n, max(1, int(round(sample * n / n_all))))
        pick = rng.choice(n, size=k, replace=False)
        if np.all(~per | (L >= 2.0 * rc + 1e-6)):
            # periodic dims by the tree's torus; free dims shifted into a box
            # wide enough that no wrap reaches rc
            lo_free = xs.min(axis=0) - rc
            pts = np.where(per, np.mod(xs, L), xs - lo_free)
            box = np.where(per, L, (xs.max(axis=0) - lo_free) + 2.0 * rc + 1.0)
            pts = np.minimum(pts, np.nextafter(box, 0))
            tree = cKDTree(pts, boxsize=box)
            c = tree.query_ball_point(pts[pick], rc, return_length=True) - 1
        else:
            # small periodic box: tile the images explicitly
            reps = [np.arange(-int(np.ceil(rc / L[d])), int(np.ceil(rc / L[d])) + 1)
                    if per[d] else np.array([0]) for d in range(3)]
            shifts = np.array([[i, j, l] for i in reps[0] for j in reps[1] for l in reps[2]],
                              dtype=np.float64) * L
            tiled = (xs[None, :, :] + shifts[:, None, :]).reshape(-1, 3)
            tree = cKDTree(tiled)
            c = tree.query_ball_point(xs[pick], rc, return_length=True) - 1
        total += float(np.mean(c)) * n
        counted += n
    return total / max(1, counted)


def window_setup(ctx, wl):
    """Rigid piston (initial x < 2a) and the moving window of the shock slab:
    fresh one-cell FCC slabs (300 K) appended ahead of the front, atoms more
    than L_behind behind it deleted; the front is located on bins one
    lattice constant wide."""
    s = wl.systems[0]
    a = wl.extra["a"]
    ncyz = int(round((s.hi[1] - s.lo[1]) / a))
    sx = W.fcc_lattice(1, ncyz, ncyz, a, (0.0, s.lo[1], s.lo[2]))
    sv = W.maxwell_velocities(np.random.default_rng(1), np.full(sx.shape[0], wl.eam.mass), 300.0)
    ctx.set_piston(wl.extra["u_p"], wl.extra["piston"])
    ctx.set_window(wl.extra["L_behind"], wl.extra["L_ahead"], sx, sv, a, 0.5 * a, wl.eam.mass,
                   2.0 * a, a)


DRIFT_BAR = 1e-5   # eV/atom per 10^4 steps (the mixed-precision drift criterion)


def drift_run(mdk, wl, prec, steps, every=100, skin_outer=0.0):
    """NVE energy drift: E_tot / N sampled every `every` steps on the GPU, the
    slope of its least-squares line scaled to 10^4 steps (eV/atom); the same
    run's throughput (CUDA events around the steps, thermo samples included)."""
    import torch
    ctx = mdk.make_context(wl, precision=prec, skin_outer=skin_outer)
    tpa, block, _ = ctx.autotune()
    kind = ctx.list_kind
    ctx.set_thermo(every, capacity=steps // every + 4)
    ctx.build_neighbors(wl.rc, wl.skin)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    ctx.step(wl.dt, steps, check=False)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.check()
    n = ctx.natoms()
    th = ctx.thermo()
    ctx.close()
    step = th[:, 0, 0]
    e = (th[:, :, 1] + th[:, :, 2]).sum(axis=1) / th[:, :, 3].sum(axis=1)
    slope = float(np.polyfit(step, e, 1)[0]) * 1e4
    return {"precision": prec, "steps": steps, "samples": int(step.shape[0]),
            "slope_eV_per_atom_per_1e4_steps": slope, "bar": DRIFT_BAR,
            "within_bar": bool(abs(slope) <= DRIFT_BAR),
            "max_minus_min_eV_per_atom": float(e.max() - e.min()),
            "E_per_atom_first_last": [float(e[0]), float(e[-1])],
            "value": n * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "launch": {"threads_per_atom": tpa, "block": block, "list": kind,
                       "picked_by": "mdk_autotune"},
            "timing": "CUDA events around the whole run (thermo samples every "
                      f"{every} steps included)"}


def stationary_setup(ctx, wl, u_in=-0.05, u_p=0.015):
    """The paper's stationary-shock window on the slab: material flows in at
    u_in through a fixed inflow boundary (fresh 300 K layers up to the right
    end of the slab), leaves through a fixed outflow boundary, and Langevin
    thermostats hold the inflow end at (u_in, 300 K) and the outflow end at
    u_out = u_in + u_p."""
    s = wl.systems[0]
    a = wl.extra["a"]
    ncyz = int(round((s.hi[1] - s.lo[1]) / a))
    x_end = float(s.x[:, 0].max())
    sx = W.fcc_lattice(1, ncyz, ncyz, a, (0.0, s.lo[1], s.lo[2]))
    sv = W.maxwell_velocities(np.random.default_rng(1), np.full(sx.shape[0], wl.eam.mass), 300.0)
    sv[:, 0] += u_in
    x_front, L_ahead, L_behind = x_end - 150.0, 150.0 + 0.25 * a, x_end - 300.0
    ctx.set_window(L_behind, L_ahead, sx, sv, a, 0.5 * a, wl.eam.mass, 0.0, a,
                   fixed_front=x_front)
    ctx.set_langevin([(s.lo[0], 150.0, 300.0, (u_in + u_p, 0.0, 0.0), 0.01),
                      (x_front, s.hi[0], 300.0, (u_in, 0.0, 0.0), 0.01)], seed=1)
    return {"u_in_A_per_fs": u_in, "u_out_A_per_fs": u_in + u_p, "x_front_A": x_front,
            "L_behind_A": L_behind, "L_ahead_A": L_ahead}


def reference_forces(mdk, wl, x):
    """F_ref of the force-matching loss: the analytic FS-EAM, evaluated through
    tables at the largest knot count the library takes (7168), far finer than
    the 5000-knot tables being differentiated."""
    tab = W.tabulate_fs_eam(wl.eam, nr=7168, nrho=7168)
    ss = wl.systems
    c = mdk.Context([q.lo for q in ss], [q.hi for q in ss], [q.periodic for q in ss],
                    np.concatenate([q.masses for q in ss]), "fp64", n_atoms=[q.n for q in ss])
    c.set_potential_eam(tab)
    c.plan(wl.rc, wl.skin)
    c.set_state(x)
    c.build_neighbors(wl.rc, wl.skin)
    _, F, _ = c.compute()
    c.close()
    return F


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def _lattice_of(wl):
    """(a, T, mass) of the workload's lattice."""
    if wl.potential == "lj":
        return 5.26, 80.0, wl.lj.mass
    if wl.potential == "bpnn":
        return 4.05, 300.0, W.MASS_AL
    return wl.eam.a0, 300.0, wl.eam.mass


def host_cores():
    """Host threads this process may run on (the oracle's thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_md(wl, x, v, s, nsteps, threads=1):
    """The oracle's cell-list velocity Verlet on the host: LJ and EAM on
    `threads` threads (ora_md_run_threads: the serial run's values bit for
    bit), BPNN on one thread."""
    import oracle
    if wl.potential == "bpnn":
        return oracle.md_bpnn(x, v, s.masses, s.lo, s.hi, s.periodic, wl.dt, nsteps, wl.skin,
                              wl.extra["bpnn"])
    kw = {"lj_params": wl.lj} if wl.potential == "lj" else {"tables": wl.tables}
    return oracle.md_run_threads(x, v, s.masses, s.lo, s.hi, s.periodic, wl.dt, nsteps,
                                 wl.skin, threads, **kw)


def oracle_threads(wl):
    return 1 if wl.potential == "bpnn" else host_cores()


def oracle_rate(wl, n_cells, nsteps):
    """Oracle (cell-list Verlet MD, FP64, all host cores for LJ and EAM) on an
    FCC n^3-cell sub-box of the workload: atom-timesteps/s and the sample."""
    a, T, mass = _lattice_of(wl)
    rng = np.random.default_rng(100)
    s = W.lattice_system(rng, (n_cells,) * 3, a, mass, T)
    t0 = time.perf_counter()
    _oracle_md(wl, s.x, s.v, s, nsteps, oracle_threads(wl))
    t = time.perf_counter() - t0
    return s.n * nsteps / t, s.n, t


def sample_cells(wl, atom_steps_budget, small, cap=64):
    """FCC cells per side of a sub-box with about atom_steps_budget atom-steps
    of oracle work per timed step, sized from timing runs that grow the box
    until a run is long enough to time (the threads' start-up costs dominate
    tiny boxes)."""
    n_cells = small
    while True:
        rate, n, t = oracle_rate(wl, n_cells, 2 if wl.potential == "bpnn" else 4)
        want = int(round((rate * atom_steps_budget / 4) ** (1 / 3)))
        if t > 0.5 or n_cells >= cap or want <= n_cells:
            return int(max(small, min(cap, want)))
        n_cells = min(cap, max(2 * n_cells, want // 2))


def cpu_baseline(wl, budget_s=15.0):
    # size the sample for ~budget_s of work, then time it
    small = 3 if wl.potential == "bpnn" else 8   # BPNN: ~25 ms per atom-step
    steps = 4 if wl.potential == "bpnn" else 20
    n_cells = sample_cells(wl, budget_s / steps, small)
    rate, n, t = oracle_rate(wl, n_cells, steps)
    nt = oracle_threads(wl)
    return {"value": rate, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"{n} atoms ({n_cells}^3 FCC cells of the same lattice, potential, "
                      f"temperature and dt), {steps} velocity-Verlet steps with Verlet-list "
                      f"rebuilds, FP64, cell-list oracle on {nt} host thread(s) "
                      f"(ora_md_run_threads, bitwise the serial run), {t:.1f} s"}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    nt = oracle_threads(wl)
    # size each step so that warmup + steps end within ~90 s
    small = 3 if wl.potential == "bpnn" else 8
    n_cells = sample_cells(wl, 90.0 / max(1, args.steps + args.warmup), small)
    a, T, mass = _lattice_of(wl)
    s = W.lattice_system(np.random.default_rng(100), (n_cells,) * 3, a, mass, T)
    out = _oracle_md(wl, s.x, s.v, s, args.warmup, nt)
    t0 = time.perf_counter()
    _oracle_md(wl, out["x"], out["v"], s, args.steps, nt)
    t = time.perf_counter() - t0
    val = s.n * args.steps / t
    sample = (f"{s.n} atoms ({n_cells}^3 FCC cells of the workload's lattice, potential, "
              f"temperature and dt) per step, FP64 cell-list Verlet MD on {nt} host "
              f"thread(s)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "atoms_per_step_sample": s.n},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fma_peaks(mdk):
    """FMA pipe peaks measured on this device (the ALU rooflines' denominators)."""
    try:
        return {"fp64": mdk.fma_peak("fp64"), "mixed": mdk.fma_peak("mixed")}
    except mdk.MDKError:
        return None


def roofline_for(wl, prec, kind, n_now, n_list, n_avg, n_rc, tpa, prof, ms, prof_steps, steps,
                 hbm, peak_kind, fma_pk):
    """The force pass's roofline record: algorithmic bytes (mixed) or FLOPs
    (FP64, BPNN) over its CUDA-event time from the profiled segment."""
    force_ms = prof["force_ms"] / max(1.0, prof["force_passes"])
    bpa = algorithmic_bytes_per_atom(wl, prec, n_list, kind)
    gbs = n_now * bpa / (force_ms / 1e3) / 1e9
    if kind == "cells":
        kdesc = (f"k_lj_cells<{prec}> (one warp per cell, neighbour cells tiled in shared "
                 "memory, no list) with the fused velocity-Verlet update")
    elif kind == "half":
        kdesc = ((f"k_lj_half<{prec}> pair pass" if wl.potential == "lj" else
                  f"k_rho_half + k_embed + k_eam_half<{prec}> passes") +
                 " (half lists, accumulating atomics) + k_half_fin per-atom velocity-Verlet pass")
    else:
        kdesc = (("k_lj" if wl.potential == "lj" else "k_rho + k_eam") +
                 f"<{prec}> force pass with the fused velocity-Verlet update")
    common = {"kernel": kdesc, "force_ms": force_ms,
              "force_share_of_step": prof["force_ms"] / (ms * prof_steps / steps),
              "rebuild_share_of_step": prof["rebuild_ms"] / (ms * prof_steps / steps),
              "timed_from": f"CUDA events around each of {int(prof['force_passes'])} force "
                            f"passes of a {prof_steps}-step profiled segment"}
    if wl.potential == "bpnn":
        fpa = bpnn_flops_per_atom(wl.extra["bpnn"], n_rc)
        tflops = n_now * fpa / (force_ms / 1e3) / 1e12
        nominal = FP32_PEAK_TFLOPS if prec == "mixed" else FP64_PEAK_TFLOPS
        pk = fma_pk[prec] if fma_pk else nominal
        common["kernel"] = (f"k_bpnn<{prec}> (descriptors, network, gradients; one warp per "
                            "atom) + k_half_fin per-atom velocity-Verlet pass")
        return {"bound": "alu", "achieved": tflops, "peak": pk, "unit": "TFLOP/s",
                "frac": tflops / pk, "traffic": None, "flops_per_atom": fpa,
                "peak_kind": (("measured: FP32" if prec == "mixed" else "measured: FP64") +
                              " FMA probe (mdk_fma_peak)") if fma_pk else "nominal",
                "peak_nominal": nominal, **common}
    if prec == "mixed":
        tr = traffic_per_launch(wl, prec, n_now, kind, n_avg, tpa)
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "traffic": tr, "bytes_per_atom": bpa,
                "traffic_unit": "bytes per launch", "peak_kind": peak_kind, **common}
    tflops = n_now * 0.5 * n_rc * FLOPS_PER_PAIR[wl.potential] / (force_ms / 1e3) / 1e12
    pk = fma_pk["fp64"] if fma_pk else FP64_PEAK_TFLOPS
    return {"bound": "alu", "achieved": tflops, "peak": pk,
            "unit": "TFLOP/s", "frac": tflops / pk, "traffic": None,
            "flops_per_pair": FLOPS_PER_PAIR[wl.potential],
            "peak_kind": ("measured: FP64 FMA probe (mdk_fma_peak)" if fma_pk
                          else "GB300 nominal dense FP64"),
            "peak_nominal": FP64_PEAK_TFLOPS,
            "hbm": {"achieved": gbs, "peak": hbm, "frac": gbs / hbm,
                    "bytes_per_atom": bpa}, **common}


def vjp_timing(mdk, ctx, wl, vjps, barrier):
    """The adjoint of the cold-curve batch: forward pass, loss gradient and
    mdk_eam_vjp, timed with CUDA events over `vjps` repetitions."""
    import torch as _t
    n_atoms = ctx.natoms()
    stream = ctx.stream
    x_now, _ = ctx.get_state()
    Fref = _t.tensor(reference_forces(mdk, wl, x_now), device="cuda")
    R = ctx.n_rep
    Ed = _t.empty(R, dtype=_t.float64, device="cuda")
    Fd = _t.empty((n_atoms, 3), dtype=_t.float64, device="cuda")
    Wd = _t.empty((R, 6), dtype=_t.float64, device="cuda")
    gE = _t.ones(R, dtype=_t.float64, device="cuda")
    nk = 2 * wl.tables.nr + wl.tables.nrho
    dth = _t.empty(nk, dtype=_t.float64, device="cuda")

    def one():
        ctx.compute_device(Ed, Fd, Wd)
        gF = 2.0 * (Fd - Fref)          # d/dF of sum |F - F_ref|^2
        ctx.eam_vjp_device(gE, gF, dth)

    for _ in range(3):
        one()
    barrier()
    ctx.profile(False)
    v0 = _t.cuda.Event(enable_timing=True)
    v1 = _t.cuda.Event(enable_timing=True)
    v0.record(stream)
    for _ in range(vjps):
        one()
    v1.record(stream)
    barrier()
    vms = v0.elapsed_time(v1) / vjps
    n_rc = pair_count_within_rc(ctx, wl)
    out = {"loss": "sum_r E_r + sum_i |F_i - F_ref,i|^2",
           "F_ref": "analytic FS-EAM through 7168-knot tables",
           "knots": nk, "ms_per_vjp": vms, "vjps": vjps,
           "vjp_per_s": 1e3 / vms, "atoms": n_atoms,
           "pair_evaluations_per_s": n_atoms * 0.5 * n_rc / (vms / 1e3),
           "includes": "forward force pass + loss gradient + mdk_eam_vjp",
           "gpu_launches": int(ctx.get_profile()["kernels"])}
    ctx.check()
    return out


def measure(mdk, wl, prec, steps, warmup, barrier, hbm, peak_kind, fma_pk, outer_skin=0.0,
            n_rc=None):
    """One workload in one precision: autotuned launch, `warmup` untimed steps,
    `steps` timed with CUDA events on the context's stream (inputs in HBM),
    then a profiled segment for the force pass's roofline.  Returns the
    record and the context."""
    import torch
    ctx = mdk.make_context(wl, precision=prec, skin_outer=outer_skin)
    tpa, block, _ = ctx.autotune()
    kind = ctx.list_kind
    n_avg = float(ctx.neighbor_counts().mean()) if kind != "cells" else float("nan")
    if n_rc is None:
        n_rc = pair_count_within_rc(ctx, wl)
    n_list = {"full": n_avg, "half": 0.5 * n_avg, "cells": 0.0}[kind]
    ctx.step(wl.dt, warmup, check=True)
    barrier()
    b0 = ctx.build_counts()
    ctx.profile(False)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    ctx.step(wl.dt, steps, check=False)
    e1.record(ctx.stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = int(ctx.get_profile()["kernels"])
    b1 = ctx.build_counts()
    ctx.check()
    prof_steps = max(20, min(steps, 200))
    ctx.profile(True)
    ctx.step(wl.dt, prof_steps, check=False)
    prof = ctx.get_profile()
    ctx.profile(False)
    ctx.check()
    n = ctx.natoms()
    roof = roofline_for(wl, prec, kind, n, n_list, n_avg, n_rc, tpa, prof, ms, prof_steps, steps,
                        hbm, peak_kind, fma_pk)
    rec = {"workload": wl.name, "precision": prec, "atoms": n, "replicas": len(wl.systems),
           "value": n * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup, "gpu_launches": launches,
           "pair_interactions_per_s": n * steps / (ms / 1e3) * n_rc / 2.0,
           "list_builds": b1[0] - b0[0], "full_builds": b1[1] - b0[1],
           "launch": {"threads_per_atom": tpa, "block": block, "list": kind,
                      "picked_by": "mdk_autotune"},
           "roofline": roof}
    return rec, ctx


def eam_record(mdk, barrier, hbm, peak_kind, fma_pk, drift_steps, drift_fp64_steps, vjps):
    """The metric's EAM half on one GPU: the Cu-like cold-curve batch (64
    uneven replicas in one context, the batched path) and the Al-like bulk
    (256,000 atoms), each mixed against FP64 with both NVE drifts, plus the
    adjoint of the batch."""
    import torch
    out = {}
    for key, wl, steps, fsteps in (("cu_coldcurve_batched", W.config4(), 500, 200),
                                   ("al_bulk", W.config1(), 200, 100)):
        mixed, ctx = measure(mdk, wl, "mixed", steps, 10, barrier, hbm, peak_kind, fma_pk)
        rec = {"mixed": mixed}
        if key == "cu_coldcurve_batched" and vjps > 0:
            rec["vjp"] = vjp_timing(mdk, ctx, wl, vjps, barrier)
        del ctx
        torch.cuda.empty_cache()
        fp64, ctx = measure(mdk, wl, "fp64", fsteps, 5, barrier, hbm, peak_kind, fma_pk)
        del ctx
        torch.cuda.empty_cache()
        rec["fp64"] = fp64
        rec["mixed_over_fp64"] = mixed["value"] / fp64["value"]
        if drift_steps > 0:
            rec["drift"] = [drift_run(mdk, wl, "mixed", drift_steps)]
            if drift_fp64_steps > 0:
                rec["drift"].append(drift_run(mdk, wl, "fp64", drift_fp64_steps))
        torch.cuda.empty_cache()
        out[key] = rec
    return out


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--cells", type=int, default=128, help="FCC cells per side (config 2)")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--impl", default="mdk")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--vjps", type=int, default=100, help="adjoint calls timed (config 4)")
    ap.add_argument("--hugoniot", action="store_true",
                    help="the isotherm grid of the Hugoniot runs: 8 x 8 argon replicas")
    ap.add_argument("--stationary", action="store_true",
                    help="config 3 as the paper's stationary-shock window (inflow/outflow)")
    ap.add_argument("--langevin", default=None,
                    help="T,beta: a Langevin thermostat on the whole system (K, 1/fs)")
    ap.add_argument("--bpnn", action="store_true",
                    help="Behler-Parrinello workload: Al-like FCC 40^3 = 256,000 atoms, "
                         "synthetic 8 G2 + 43 G4 model, 10-10 network")
    ap.add_argument("--launch", default=None,
                    help="threads-per-atom x block (e.g. 1x128) instead of the autotuner")
    ap.add_argument("--outer", type=float, default=None,
                    help="outer-list skin in Angstrom (two-level lists; 0 = off; default: "
                         "7 x skin = 2.1 A for the 8.4M-atom LJ argon config, where it "
                         "measured fastest of 1.5, 1.8 and 2.1 A, else off)")
    ap.add_argument("--list", default=None, choices=("full", "half", "cells"),
                    help="with --launch: the Verlet-list kind (LJ; default full)")
    ap.add_argument("--drift-steps", type=int, default=None,
                    help="NVE drift measurement of this many mixed steps (default: 10000 "
                         "for the 8.4M-atom argon headline, else 0)")
    ap.add_argument("--drift-fp64-steps", type=int, default=2000)
    ap.add_argument("--no-eam", action="store_true",
                    help="skip the EAM record (Cu cold-curve batch and Al bulk, mixed "
                         "against FP64, drifts, adjoint) of the default headline run")
    ap.add_argument("--steady-steps", type=int, default=1000,
                    help="headline: when --steps is shorter, also time this many steps "
                         "(full builds of the two-level lists included)")
    args = ap.parse_args()
    if args.list and not args.launch:
        ap.error("--list goes with --launch (the autotuner picks the list kind)")
    args.warmup = max(3, args.warmup)
    wl = workload(args.config, args.cells)
    if args.bpnn:
        wl = W.bpnn_workload()
    grid = None
    if args.hugoniot:
        from paper_2511_22951_gb300 import hugoniot as H
        # the paper's isotherm grid: 6912-atom argon replicas, v/v0 from 1 to 0.3,
        # T from 300 K to 1e5 K, one dt for the batch (the hottest replica's)
        grid = H.IsothermGrid(a0=5.26, compressions=np.linspace(1.0, 0.3, 8),
                              temperatures=np.geomspace(300.0, 1e5, 8), n_cells=12,
                              beta=5e-4)
        ss = grid.systems()
        wl = W.Workload("lj_argon_isotherms_64x6912", ss, "lj", W.LJ_AR, None, None,
                        dt=float(H.paper_dt(grid.temperatures.max())), steps=1000, skin=0.3,
                        precision="mixed")
    if args.impl == "reference":
        return run_reference(args, wl)
    # the default run is the headline: LJ argon 8.4M atoms (config 2), which
    # also reports the NVE drift of both paths and the EAM record
    headline = (args.config == 2 and not args.hugoniot and not args.bpnn and
                not args.langevin and args.cells == 128)
    if args.drift_steps is None:
        args.drift_steps = 10000 if headline else 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2511_22951_gb300 import _build, mdk
    _build.build()
    prec = args.precision or wl.precision
    if prec != wl.precision and wl.name.endswith("_" + wl.precision):
        wl.name = wl.name[:-len(wl.precision)] + prec   # the workload as run
    n_atoms = wl.n_atoms
    windowed = args.config == 3
    # two-level lists: outer skin (0: off); a moving window rebuilds fully anyway
    if args.outer is not None:
        outer_skin = float(args.outer)
    else:
        outer_skin = 7.0 * wl.skin if (args.config == 2 and not args.hugoniot and
                                       not args.bpnn) else 0.0
    outer_skin = 0.0 if windowed else outer_skin
    if args.stationary:
        if not windowed:
            raise SystemExit("--stationary applies to the slab (--config 3)")
        for q in wl.systems:
            q.v[:, 0] += -0.05           # the material flows in at u_in
    ctx = mdk.make_context(wl, precision=prec,
                           capacity=int(n_atoms * 1.1) if windowed else None,
                           max_neighbors=(120 if args.stationary else
                                          (320 if grid is not None else 0)),
                           skin_outer=outer_skin)
    if grid is not None:
        Tr = np.repeat(grid.temperatures[None, :], len(grid.compressions), 0).ravel()
        ctx.set_langevin_replicas(Tr, np.full(Tr.size, grid.beta), seed=1)
    stream = ctx.stream
    n_avg = float(ctx.neighbor_counts().mean())
    n_rc = pair_count_within_rc(ctx, wl) if rank == 0 else 0.0
    stationary = None
    if args.stationary:
        stationary = stationary_setup(ctx, wl)
    elif windowed:
        window_setup(ctx, wl)
    lang = None
    if args.langevin:
        T_l, beta_l = (float(q) for q in args.langevin.split(","))
        lang = [(-1e30, 1e30, T_l, (0.0, 0.0, 0.0), beta_l)]
        ctx.set_langevin(lang, seed=1)
    if args.launch:
        tpa, block = (int(q) for q in args.launch.split("x"))
        ctx.set_launch(tpa, block)
        if args.list:
            ctx.set_list_kind(args.list)
            ctx.build_neighbors(wl.rc, wl.skin)
        picked = "--launch"
    else:
        tpa, block, _ = ctx.autotune()
        picked = "mdk_autotune"
    kind = ctx.list_kind
    # a half list holds each pair once; the cell kernel reads no list
    n_list = {"full": n_avg, "half": 0.5 * n_avg, "cells": 0.0}[kind]

    # warm-up (untimed; also captures the step graphs)
    ctx.step(wl.dt, args.warmup, check=True)
    barrier()
    clocks = Clocks()
    clocks.start()
    builds_before = ctx.counters()[0]
    full_before = ctx.build_counts()[1]
    n_start = ctx.natoms()      # the moving window changes N between builds
    ctx.profile(False)          # clears the counters; kernels are still counted
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(wl.dt, args.steps, check=False)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = int(ctx.get_profile()["kernels"])
    builds0 = ctx.counters()[0]
    full_builds = ctx.build_counts()[1] - full_before
    ck = clocks.stop()
    ctx.check()
    # per-kernel times: a separate segment with CUDA events around every force
    # pass and rebuild chain (graphs off there, events on the same stream)
    prof_steps = max(20, min(args.steps, 200))
    ctx.profile(True)
    ctx.step(wl.dt, prof_steps, check=False)
    prof = ctx.get_profile()
    ctx.profile(False)
    ctx.check()
    n_mean = 0.5 * (n_start + ctx.natoms())
    value, ms = job_throughput(ms, n_mean, args.steps, dist, "cuda")
    # a longer segment at the same settings: a short timed region may hold no
    # full build of the two-level lists; this one shows the steady state
    steady = None
    if rank == 0 and world == 1 and headline and args.steady_steps > args.steps:
        sb0 = ctx.build_counts()
        barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        ctx.step(wl.dt, args.steady_steps, check=False)
        s1.record(stream)
        barrier()
        sms = s0.elapsed_time(s1)
        sb1 = ctx.build_counts()
        ctx.check()
        steady = {"steps": args.steady_steps, "value": n_atoms * args.steady_steps / (sms / 1e3),
                  "ms_per_step": sms / args.steady_steps, "list_builds": sb1[0] - sb0[0],
                  "full_builds": sb1[1] - sb0[1],
                  "note": "same context and settings as the timed region, right after it"}

    # dominant kernel: the fused force + integration pass
    hbm, peak_kind = peaks()
    n_now = ctx.natoms()
    fma_pk = fma_peaks(mdk)
    roof = roofline_for(wl, prec, kind, n_now, n_list, n_avg, n_rc, tpa, prof, ms, prof_steps,
                        args.steps, hbm, peak_kind, fma_pk)

    # the adjoint of the cold-curve batch: forward pass, loss gradient and VJP
    vjp = None
    if args.config == 4 and args.vjps > 0:
        vjp = vjp_timing(mdk, ctx, wl, args.vjps, barrier)

    # end to end through the C ABI with host buffers: upload the state from
    # pinned memory, run the steps, read positions, velocities and energy back
    e2e = None
    if not args.no_e2e and not windowed:
        xs = torch.empty((n_atoms, 3), dtype=torch.float64, pin_memory=True)
        vs = torch.empty((n_atoms, 3), dtype=torch.float64, pin_memory=True)
        xg, vg = ctx.get_state()
        xs.numpy()[:] = xg
        vs.numpy()[:] = vg
        E = np.zeros(len(wl.systems))  # mdk_compute writes one energy per replica

        def e2e_call():
            ctx.lib.mdk_set_state(ctx.h, mdk._P(xs.data_ptr()), mdk._P(vs.data_ptr()), 0)
            ctx.lib.mdk_build_neighbors(ctx.h, wl.rc, wl.skin)
            ctx.lib.mdk_step(ctx.h, wl.dt, args.steps)
            ctx.lib.mdk_get_state(ctx.h, mdk._P(xs.data_ptr()), mdk._P(vs.data_ptr()), 0)
            ctx.lib.mdk_compute(ctx.h, mdk._ptr(E), None, None, 0)

        # one untimed call first: the first transfers from freshly pinned
        # buffers pay one-time mapping costs (~15 ms on 400 MB)
        e2e_call()
        xs.numpy()[:] = xg
        vs.numpy()[:] = vg
        barrier()
        t0 = time.perf_counter()
        e2e_call()
        barrier()
        t = time.perf_counter() - t0
        ctx.check()
        e2e = {"value": n_atoms * args.steps * world / t, "unit": UNIT,
               "h2d_bytes_per_step": 48 * n_atoms / args.steps,
               "d2h_bytes_per_step": (48 * n_atoms + 8 * E.size) / args.steps}

    # the plain FP64 GPU path on the same workload, for comparison
    fp64 = None
    if prec != "fp64" and args.fp64_steps > 0 and rank == 0:
        del ctx
        torch.cuda.empty_cache()
        c64 = mdk.make_context(wl, precision="fp64",
                               capacity=int(n_atoms * 1.1) if windowed else None,
                               max_neighbors=(120 if args.stationary else
                                              (320 if grid is not None else 0)),
                               skin_outer=outer_skin)
        if args.stationary:
            stationary_setup(c64, wl)
        elif windowed:
            window_setup(c64, wl)
        if lang:
            c64.set_langevin(lang, seed=1)
        if grid is not None:
            c64.set_langevin_replicas(Tr, np.full(Tr.size, grid.beta), seed=1)
        t64, b64, _ = c64.autotune()
        c64.step(wl.dt, 3)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(c64.stream)
        c64.step(wl.dt, args.fp64_steps, check=False)
        f1.record(c64.stream)
        torch.cuda.synchronize()
        c64.check()
        fms = f0.elapsed_time(f1)
        fp64 = {"value": n_atoms * args.fp64_steps / (fms / 1e3), "unit": UNIT,
                "ms_per_step": fms / args.fp64_steps, "steps": args.fp64_steps,
                "launch": {"threads_per_atom": t64, "block": b64, "list": c64.list_kind,
                           "picked_by": "mdk_autotune"}}
        del c64

    drift = None
    if rank == 0 and world == 1 and args.drift_steps > 0:
        torch.cuda.empty_cache()
        drift = [drift_run(mdk, wl, prec, args.drift_steps, skin_outer=outer_skin)]
        if prec != "fp64" and args.drift_fp64_steps > 0:
            torch.cuda.empty_cache()
            drift.append(drift_run(mdk, wl, "fp64", args.drift_fp64_steps,
                                   skin_outer=outer_skin))
    eam = None
    if rank == 0 and world == 1 and headline and not args.no_eam:
        torch.cuda.empty_cache()
        eam = eam_record(mdk, barrier, hbm, peak_kind, fma_pk, 10000, args.drift_fp64_steps,
                         args.vjps)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(wl)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "atoms": n_atoms, "potential": wl.potential,
                       "precision": prec, "dt_fs": wl.dt, "skin_A": wl.skin,
                       "replicas": len(wl.systems),
                       "neighbors_per_atom": n_avg, "neighbors_within_rc": n_rc,
                       "launch": {"threads_per_atom": tpa, "block": block,
                                  "list": kind, "list_entries_per_atom": n_list,
                                  "picked_by": picked},
                       "rebuild": "when an atom moved > skin/2 since the last build",
                       "outer_list": ({"skin_A": outer_skin, "full_builds": full_builds}
                                      if outer_skin else None),
                       "list_builds_in_timed_region": builds0 - builds_before,
                       "step_graphs": "two-step CUDA graphs replayed by mdk_step",
                       "l2": "inputs larger than L2 (~4 GB touched per step); no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "pair_interactions_per_s": value * n_rc / 2.0,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": ck,
            "fp64_path": fp64,
            "vjp": vjp,
            "drift": drift,
            "steady_state": steady,
            "eam": eam,
        }
        if lang:
            line["config"]["langevin"] = {"T_K": lang[0][2], "beta_per_fs": lang[0][4],
                                          "regions": "whole system"}
        if grid is not None:
            line["config"]["isotherms"] = {
                "v_over_v0": [round(float(c), 4) for c in grid.compressions],
                "T_K": [round(float(t), 1) for t in grid.temperatures],
                "thermostat": "per replica, beta 5e-4 1/fs", "dt_fs": wl.dt}
        if stationary:
            line["config"]["stationary_window"] = dict(stationary, atoms_at_end=n_now)
        elif windowed:
            line["config"]["piston_u_p_A_per_fs"] = wl.extra["u_p"]
            line["config"]["window"] = {"L_behind": wl.extra["L_behind"],
                                        "L_ahead": wl.extra["L_ahead"],
                                        "atoms_at_end": n_now}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
