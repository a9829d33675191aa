"""Throughput of the MD hot path on GB300: atom-timesteps/s.

One bench step = one velocity-Verlet NVE timestep of the whole path: force
loop, integration, displacement check and -- whenever an atom has moved more
than skin/2 -- the cell-list Verlet-list rebuild (all in libmdk.so kernels).

Default workload: LJ argon, FCC 128^3 cells = 8,388,608 atoms, 80 K, dt = 2 fs,
skin 0.3 Angstrom, mixed precision (FP32 pair arithmetic, FP64 positions,
velocities and integration).  Inputs live in HBM and the per-step working set
(~4 GB) is larger than L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config C] [--impl reference]

--impl reference times the CPU oracle (the FP64 C program written from the
paper) on a bounded sample of the same workload on the host cores.
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
    raise SystemExit(f"config {cfg} is not a bench workload")


def algorithmic_bytes_per_atom(wl, prec, n_avg):
    """Bytes one fused force+integration launch must move per atom:
    own gather-copy element, list entries + count, x and v read+write, x_ref
    and cell word read, next gather-copy element written.  Neighbour
    positions are assumed to come from cache (spatial order)."""
    g = 16 if prec == "mixed" else 32
    return g + 4 * n_avg + 4 + 48 + 48 + 24 + 4 + g


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
def oracle_rate(wl, n_cells, nsteps):
    """Oracle (cell-list Verlet MD, FP64, one host thread) on an FCC n^3-cell
    sub-box of the workload: returns atom-timesteps/s and the sample size."""
    import oracle
    a = 5.26 if wl.potential == "lj" else wl.eam.a0
    T = 80.0 if wl.potential == "lj" else 300.0
    rng = np.random.default_rng(100)
    mass = wl.lj.mass if wl.potential == "lj" else wl.eam.mass
    s = W.lattice_system(rng, (n_cells,) * 3, a, mass, T)
    kw = {"lj_params": wl.lj} if wl.potential == "lj" else {"tables": wl.tables}
    t0 = time.perf_counter()
    oracle.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, nsteps, wl.skin, **kw)
    t = time.perf_counter() - t0
    return s.n * nsteps / t, s.n, t


def cpu_baseline(wl, budget_s=15.0):
    # calibrate on a small box, then size the sample for ~budget_s of work
    rate0, _, _ = oracle_rate(wl, 6, 4)
    steps = 20
    target_atoms = rate0 * budget_s / steps
    n_cells = int(max(6, min(40, round((target_atoms / 4) ** (1 / 3)))))
    rate, n, t = oracle_rate(wl, n_cells, steps)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} atoms ({n_cells}^3 FCC cells of the same lattice, potential, "
                      f"temperature and dt), {steps} velocity-Verlet steps with Verlet-list "
                      f"rebuilds, FP64, one host thread, {t:.1f} s"}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    # size each step so that warmup + steps end within ~90 s
    rate0, _, _ = oracle_rate(wl, 6, 4)
    per_step_atoms = rate0 * 90.0 / max(1, args.steps + args.warmup)
    n_cells = int(max(3, min(40, round((per_step_atoms / 4) ** (1 / 3)))))
    a = 5.26 if wl.potential == "lj" else wl.eam.a0
    T = 80.0 if wl.potential == "lj" else 300.0
    mass = wl.lj.mass if wl.potential == "lj" else wl.eam.mass
    s = W.lattice_system(np.random.default_rng(100), (n_cells,) * 3, a, mass, T)
    kw = {"lj_params": wl.lj} if wl.potential == "lj" else {"tables": wl.tables}
    out = oracle.md_run(s.x, s.v, s.masses, s.lo, s.hi, s.periodic, wl.dt, args.warmup,
                        wl.skin, **kw)
    t0 = time.perf_counter()
    oracle.md_run(out["x"], out["v"], s.masses, s.lo, s.hi, s.periodic, wl.dt, args.steps,
                  wl.skin, **kw)
    t = time.perf_counter() - t0
    val = s.n * args.steps / t
    sample = (f"{s.n} atoms ({n_cells}^3 FCC cells of the workload's lattice, potential, "
              f"temperature and dt) per step, FP64 cell-list Verlet MD, one host thread")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "atoms_per_step_sample": s.n},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    wl = workload(args.config, args.cells)
    if args.impl == "reference":
        return run_reference(args, wl)

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
    n_atoms = wl.n_atoms
    ctx = mdk.make_context(wl, precision=prec)
    stream = ctx.stream
    n_avg = float(ctx.neighbor_counts().mean())
    tpa, block, _ = ctx.autotune()

    # warm-up (untimed; also captures the step graphs)
    ctx.step(wl.dt, args.warmup, check=True)
    barrier()
    clocks = Clocks()
    clocks.start()
    builds_before = ctx.counters()[0]
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
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n_atoms * args.steps * world / (ms / 1e3)

    # dominant kernel: the fused force + integration pass
    hbm, peak_kind = peaks()
    force_ms = prof["force_ms"] / max(1.0, prof["force_passes"])
    bpa = algorithmic_bytes_per_atom(wl, prec, n_avg)
    achieved = n_atoms * bpa / (force_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None,
            "kernel": f"k_lj<{prec}> fused force + velocity Verlet",
            "bytes_per_atom": bpa, "peak_kind": peak_kind,
            "force_share_of_step": prof["force_ms"] / (ms * prof_steps / args.steps),
            "rebuild_share_of_step": prof["rebuild_ms"] / (ms * prof_steps / args.steps),
            "timed_from": f"CUDA events around each of {int(prof['force_passes'])} force "
                          f"passes of a {prof_steps}-step profiled segment"}

    # end to end through the C ABI with host buffers: upload the state from
    # pinned memory, run the steps, read positions, velocities and energy back
    e2e = None
    if not args.no_e2e:
        xs = torch.empty((n_atoms, 3), dtype=torch.float64, pin_memory=True)
        vs = torch.empty((n_atoms, 3), dtype=torch.float64, pin_memory=True)
        xg, vg = ctx.get_state()
        xs.numpy()[:] = xg
        vs.numpy()[:] = vg
        E = np.zeros(1)
        barrier()
        t0 = time.perf_counter()
        ctx.lib.mdk_set_state(ctx.h, mdk._P(xs.data_ptr()), mdk._P(vs.data_ptr()), 0)
        ctx.lib.mdk_build_neighbors(ctx.h, wl.rc, wl.skin)
        ctx.lib.mdk_step(ctx.h, wl.dt, args.steps)
        ctx.lib.mdk_get_state(ctx.h, mdk._P(xs.data_ptr()), mdk._P(vs.data_ptr()), 0)
        ctx.lib.mdk_compute(ctx.h, mdk._ptr(E), None, None, 0)
        barrier()
        t = time.perf_counter() - t0
        ctx.check()
        e2e = {"value": n_atoms * args.steps * world / t, "unit": UNIT,
               "h2d_bytes_per_step": 48 * n_atoms / args.steps,
               "d2h_bytes_per_step": (48 * n_atoms + 8) / args.steps}

    # the plain FP64 GPU path on the same workload, for comparison
    fp64 = None
    if prec != "fp64" and args.fp64_steps > 0 and rank == 0:
        del ctx
        torch.cuda.empty_cache()
        c64 = mdk.make_context(wl, precision="fp64")
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
                "ms_per_step": fms / args.fp64_steps, "steps": args.fp64_steps}
        del c64

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
                       "neighbors_per_atom": n_avg,
                       "launch": {"threads_per_atom": tpa, "block": block,
                                  "picked_by": "mdk_autotune"},
                       "rebuild": "when an atom moved > skin/2 since the last build",
                       "list_builds_in_timed_region": builds0 - builds_before,
                       "step_graphs": "two-step CUDA graphs replayed by mdk_step",
                       "l2": "inputs larger than L2 (~4 GB touched per step); no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "pair_interactions_per_s": value * n_avg / 2.0,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": ck,
            "fp64_path": fp64,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
