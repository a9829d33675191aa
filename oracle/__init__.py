"""CPU oracle for the short-range MD hot path -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C implementation (``oracle.c``) of what the hot path computes,
written from the paper: brute-force neighbour sets over all periodic images,
the paper's cell-list Verlet-list algorithm, LJ and tabulated-EAM energies,
forces and virials, velocity-Verlet NVE integration, the Appendix per-bin
statistics, the moving window, Langevin thermostats, the EAM adjoint and the
Behler-Parrinello potential.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import this package; the CUDA product path never does.

Parity pins (what fixes the oracle independently of itself) live in
``tests/test_oracle_*.py``; every function here is pinned there.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
           "-pthread"]


def _fingerprint() -> str:
    """sha256 of the source, the flags and the compiler's version (the
    library is rebuilt whenever the stamp beside it differs)."""
    h = hashlib.sha256()
    with open(_SRC, "rb") as f:
        h.update(f.read())
    h.update(" ".join(_CFLAGS).encode())
    try:
        h.update(subprocess.run(["gcc", "--version"], capture_output=True, text=True).stdout.encode())
    except OSError:
        h.update(b"no gcc")
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction) into liboracle.so."""
    stamp_path = _LIB + ".stamp"
    fp = _fingerprint()
    fresh = os.path.exists(_LIB) and os.path.exists(stamp_path) and \
        open(stamp_path).read().strip() == fp
    if force or not fresh:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
        with open(stamp_path + f".tmp{os.getpid()}", "w") as f:
            f.write(fp + "\n")
        os.replace(stamp_path + f".tmp{os.getpid()}", stamp_path)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        L.ora_neighbors_brute.argtypes = [I64, P, P, P, P, D, P, P, P, I64]
        L.ora_neighbors_brute.restype = I64
        L.ora_neighbors_cells.argtypes = [I64, P, P, P, P, D, P, P, P, I64]
        L.ora_neighbors_cells.restype = I64
        L.ora_wrap.argtypes = [I64, P, P, P, P]
        L.ora_wrap.restype = None
        L.ora_spline_eval_many.argtypes = [P, I, D, I64, P, P, P]
        L.ora_spline_eval_many.restype = None
        L.ora_spline_slopes.argtypes = [P, I, D, P]
        L.ora_spline_slopes.restype = None
        L.ora_lj.argtypes = [I64, P, P, P, P, D, D, D, I, P, P, P, P, P]
        L.ora_lj.restype = I
        L.ora_eam.argtypes = [I64, P, P, P, P, I, D, P, P, I, D, P, P, P, P, P, P, P, P]
        L.ora_eam.restype = I
        L.ora_sampled.argtypes = [I, I64, P, P, P, P, P, I, D, P, P, I, D, P, I64, P, P, P]
        L.ora_sampled.restype = I
        L.ora_md_run.argtypes = [I64, P, P, P, P, P, P, I, P, I, D, P, P, I, D, P, D, D,
                                 I64, I, P, D, P, P]
        L.ora_md_run.restype = I64
        L.ora_md_run_threads.argtypes = [I64, P, P, P, P, P, P, I, P, I, D, P, P, I, D, P, D,
                                         D, I64, I, P]
        L.ora_md_run_threads.restype = I64
        L.ora_bpnn_set_model.argtypes = [D, I, P, P, I, P, P, I, I, P, P, P, P, P, D]
        L.ora_bpnn_set_model.restype = I
        L.ora_bpnn.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P]
        L.ora_bpnn.restype = I
        L.ora_profiles.argtypes = [I64, P, P, P, P, P, I, D, D, I, D, P]
        L.ora_profiles.restype = None
        L.ora_window_apply.argtypes = [I64, I64, P, P, P, P, P, P, D, D, D, D, D, D, D, P,
                                       P, I64, D, D, D, D]
        L.ora_window_apply.restype = I64
        L.ora_md_window.argtypes = [P, I64, P, P, P, P, P, P, P, P, P, I, D, P, P, I, D, P, D,
                                    D, I64, I, D, D, D, D, D, P, P, I64, D, D, D, D, P,
                                    ctypes.c_uint64]
        L.ora_md_window.restype = I64
        L.ora_philox4x64.argtypes = [P, P, P]
        L.ora_philox4x64.restype = None
        L.ora_md_langevin.argtypes = [I64, P, P, P, P, P, P, I, P, I, D, P, P, I, D, P, D, D,
                                      I64, I, P, D, P, P, P, P, ctypes.c_uint64, I64]
        L.ora_md_langevin.restype = I64
        L.ora_eam_vjp.argtypes = [I64, P, P, P, P, I, D, P, P, I, D, P, D, P, P]
        L.ora_eam_vjp.restype = I
        L.ora_eam_jvp.argtypes = [I64, P, P, P, P, I, D, P, P, I, D, P, P, P, P, D, P, P]
        L.ora_eam_jvp.restype = I
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _box(lo, hi, periodic):
    return (_f64(lo, (3,)), _f64(hi, (3,)),
            np.ascontiguousarray(periodic, dtype=np.int32).reshape(3))


# ---------------------------------------------------------------------------
def neighbors(x, lo, hi, periodic, rns, method="brute"):
    """Neighbour set: list over atoms of int64 arrays of shape (k, 4) with
    rows (j, nx, ny, nz), in the order the oracle produces them."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    off = np.zeros(n + 1, dtype=np.int64)
    fn = lib().ora_neighbors_brute if method == "brute" else lib().ora_neighbors_cells
    tot = fn(n, _p(x), _p(lo), _p(hi), _p(per), rns, _p(off), None, None, 0)
    if tot < 0:
        raise ValueError(f"oracle neighbour search failed ({tot})")
    j = np.zeros(max(tot, 1), dtype=np.int32)
    im = np.zeros((max(tot, 1), 3), dtype=np.int32)
    fn(n, _p(x), _p(lo), _p(hi), _p(per), rns, _p(off), _p(j), _p(im), tot)
    out = []
    for i in range(n):
        a, b = off[i], off[i + 1]
        out.append(np.concatenate([j[a:b, None].astype(np.int64),
                                   im[a:b].astype(np.int64)], axis=1))
    return out


def wrap(x, lo, hi, periodic):
    x = _f64(x, (-1, 3)).copy()
    lo, hi, per = _box(lo, hi, periodic)
    lib().ora_wrap(x.shape[0], _p(x), _p(lo), _p(hi), _p(per))
    return x


def spline_eval(y, h, xs):
    y = _f64(y)
    xs = _f64(xs)
    val = np.zeros_like(xs)
    der = np.zeros_like(xs)
    lib().ora_spline_eval_many(_p(y), y.shape[0], h, xs.shape[0], _p(xs), _p(val), _p(der))
    return val, der


def spline_slopes(y, h):
    y = _f64(y)
    m = np.zeros_like(y)
    lib().ora_spline_slopes(_p(y), y.shape[0], h, _p(m))
    return m


def lj(x, lo, hi, periodic, eps, sigma, rc, shift_mode=1, per_atom=False):
    """LJ by brute force: returns dict(E, F, W[6], Ea?, Wa?)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    E = np.zeros(1)
    F = np.zeros((n, 3))
    W = np.zeros(6)
    Ea = np.zeros(n) if per_atom else None
    Wa = np.zeros((n, 6)) if per_atom else None
    rc_ = lib().ora_lj(n, _p(x), _p(lo), _p(hi), _p(per), eps, sigma, rc, shift_mode,
                       _p(E), _p(F), _p(W), _p(Ea), _p(Wa))
    if rc_ < 0:
        raise RuntimeError("oracle lj failed")
    out = {"E": float(E[0]), "F": F, "W": W}
    if per_atom:
        out["Ea"] = Ea
        out["Wa"] = Wa
    return out


def eam(x, lo, hi, periodic, tables, per_atom=False):
    """EAM by brute force from knot tables (workloads.EAMTables-like)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
    E = np.zeros(1)
    F = np.zeros((n, 3))
    W = np.zeros(6)
    Ea = np.zeros(n) if per_atom else None
    Wa = np.zeros((n, 6)) if per_atom else None
    rho_o = np.zeros(n)
    fp_o = np.zeros(n)
    flag = lib().ora_eam(n, _p(x), _p(lo), _p(hi), _p(per), phi.shape[0], tables.rc,
                         _p(phi), _p(rho), Ft.shape[0], tables.rho_max, _p(Ft),
                         _p(E), _p(F), _p(W), _p(Ea), _p(Wa), _p(rho_o), _p(fp_o))
    if flag < 0:
        raise RuntimeError("oracle eam failed")
    out = {"E": float(E[0]), "F": F, "W": W, "rho": rho_o, "Fp": fp_o,
           "rho_flag": bool(flag & 1)}
    # the embedding part sum_i F(rho_i) of E, through the same spline (its
    # pair part is E minus this); inside the table only
    if not out["rho_flag"]:
        out["E_embed"] = float(np.sum(spline_eval(Ft, tables.rho_max / (Ft.shape[0] - 1),
                                                  rho_o)[0]))
    if per_atom:
        out["Ea"] = Ea
        out["Wa"] = Wa
    return out


def eam_vjp(x, lo, hi, periodic, tables, gE=0.0, gF=None):
    """Reverse-mode gradient of L = gE * E + sum_i gF_i . F_i with respect to
    the knot values: returns (d_phi, d_rho, d_F), the three knot arrays."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
    gF = np.zeros((n, 3)) if gF is None else _f64(gF, (n, 3))
    nr, nrho = phi.shape[0], Ft.shape[0]
    out = np.zeros(2 * nr + nrho)
    rc = lib().ora_eam_vjp(n, _p(x), _p(lo), _p(hi), _p(per), nr, tables.rc, _p(phi),
                           _p(rho), nrho, tables.rho_max, _p(Ft), float(gE), _p(gF), _p(out))
    if rc < 0:
        raise RuntimeError("oracle eam_vjp failed")
    return out[:nr].copy(), out[nr:2 * nr].copy(), out[2 * nr:].copy()


def eam_jvp(x, lo, hi, periodic, tables, dphi, drho, dF, gE=0.0, gF=None):
    """Forward-mode (dual-number) value and directional derivative of
    L = gE * E + sum_i gF_i . F_i along the knot tangent (dphi, drho, dF)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
    dphi, drho, dF = _f64(dphi), _f64(drho), _f64(dF)
    gF = np.zeros((n, 3)) if gF is None else _f64(gF, (n, 3))
    out = np.zeros(2)
    rc = lib().ora_eam_jvp(n, _p(x), _p(lo), _p(hi), _p(per), phi.shape[0], tables.rc,
                           _p(phi), _p(rho), Ft.shape[0], tables.rho_max, _p(Ft), _p(dphi),
                           _p(drho), _p(dF), float(gE), _p(gF), _p(out))
    if rc == -2:
        raise ValueError("a density lies above the F table (forward mode needs rho <= rho_max)")
    if rc < 0:
        raise RuntimeError("oracle eam_jvp failed")
    return float(out[0]), float(out[1])


def sampled(kind, x, lo, hi, periodic, sel, lj_params=None, tables=None):
    """Force (and per-atom energy) of the atoms in `sel`, by brute force."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    Fs = np.zeros((sel.shape[0], 3))
    Es = np.zeros(sel.shape[0])
    if kind == "lj":
        par = _f64([lj_params.eps, lj_params.sigma, lj_params.rc, lj_params.shift_mode])
        flag = lib().ora_sampled(0, n, _p(x), _p(lo), _p(hi), _p(per), _p(par), 0, 0.0,
                                 None, None, 0, 0.0, None, sel.shape[0], _p(sel),
                                 _p(Fs), _p(Es))
    else:
        phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
        flag = lib().ora_sampled(1, n, _p(x), _p(lo), _p(hi), _p(per), None,
                                 phi.shape[0], tables.rc, _p(phi), _p(rho), Ft.shape[0],
                                 tables.rho_max, _p(Ft), sel.shape[0], _p(sel),
                                 _p(Fs), _p(Es))
    return {"F": Fs, "E": Es, "rho_flag": bool(flag & 1)}


def md_run(x, v, masses, lo, hi, periodic, dt, nsteps, skin, lj_params=None,
           tables=None, rebuild_every=0, piston=None, u_p=0.0):
    """Velocity-Verlet NVE with Verlet lists (the paper's algorithm).

    Returns dict(x, v, F, thermo (nsteps, 3): K, U, W-trace, n_builds)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    m = _f64(masses, (n,))
    lo, hi, per = _box(lo, hi, periodic)
    thermo = np.zeros((max(nsteps, 1), 3))
    F = np.zeros((n, 3))
    pis = None if piston is None else np.ascontiguousarray(piston, dtype=np.uint8)
    if lj_params is not None:
        par = _f64([lj_params.eps, lj_params.sigma, lj_params.rc, lj_params.shift_mode])
        nb = lib().ora_md_run(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 0, _p(par),
                              0, 0.0, None, None, 0, 0.0, None, skin, dt, nsteps,
                              rebuild_every, _p(pis), u_p, _p(thermo), _p(F))
    else:
        phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
        nb = lib().ora_md_run(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 1, None,
                              phi.shape[0], tables.rc, _p(phi), _p(rho), Ft.shape[0],
                              tables.rho_max, _p(Ft), skin, dt, nsteps, rebuild_every,
                              _p(pis), u_p, _p(thermo), _p(F))
    if nb < 0:
        raise RuntimeError(f"oracle md_run failed ({nb})")
    return {"x": x, "v": v, "F": F, "thermo": thermo[:nsteps], "n_builds": int(nb)}


def md_run_threads(x, v, masses, lo, hi, periodic, dt, nsteps, skin, nthreads,
                   lj_params=None, tables=None):
    """md_run (LJ or EAM, no piston) with the per-atom work on nthreads host
    threads: the same values bit for bit, for timing the oracle on all
    cores."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    m = _f64(masses, (n,))
    lo, hi, per = _box(lo, hi, periodic)
    thermo = np.zeros((max(nsteps, 1), 3))
    if lj_params is not None:
        par = _f64([lj_params.eps, lj_params.sigma, lj_params.rc, lj_params.shift_mode])
        nb = lib().ora_md_run_threads(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 0,
                                      _p(par), 0, 0.0, None, None, 0, 0.0, None, skin, dt,
                                      nsteps, int(nthreads), _p(thermo))
    else:
        phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
        nb = lib().ora_md_run_threads(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 1,
                                      None, phi.shape[0], tables.rc, _p(phi), _p(rho),
                                      Ft.shape[0], tables.rho_max, _p(Ft), skin, dt, nsteps,
                                      int(nthreads), _p(thermo))
    if nb < 0:
        raise RuntimeError(f"oracle md_run_threads failed ({nb})")
    return {"x": x, "v": v, "thermo": thermo[:nsteps], "n_builds": int(nb)}


def _bpnn_set(model):
    """Hand the model to the oracle (it keeps one model at a time)."""
    rk = np.ascontiguousarray(model.rad_kind, dtype=np.int32)
    ak = np.ascontiguousarray(model.ang_kind, dtype=np.int32)
    rp = _f64(model.rad_par).reshape(-1)
    ap = _f64(model.ang_par).reshape(-1)
    H1, H2 = model.W01.shape[1], model.W12.shape[1]
    r = lib().ora_bpnn_set_model(model.rc, rk.shape[0], _p(rk), _p(rp), ak.shape[0], _p(ak),
                                 _p(ap), H1, H2, _p(_f64(model.W01)), _p(_f64(model.b1)),
                                 _p(_f64(model.W12)), _p(_f64(model.b2)), _p(_f64(model.w23)),
                                 float(model.b3))
    if r != 0:
        raise ValueError("oracle rejected the BPNN model")


def bpnn(x, lo, hi, periodic, model, per_atom=False, descriptors=False):
    """BPNN by brute force over all atoms and images within R_c: returns
    dict(E, F, W[6]) plus Ea, Wa [N, 6] (per_atom) and G, dEdG [N, n_in]
    (descriptors)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    lo, hi, per = _box(lo, hi, periodic)
    _bpnn_set(model)
    E = np.zeros(1)
    F = np.zeros((n, 3))
    W = np.zeros(6)
    Ea = np.zeros(n) if per_atom else None
    Wa = np.zeros((n, 6)) if per_atom else None
    G = np.zeros((n, model.n_in)) if descriptors else None
    dG = np.zeros((n, model.n_in)) if descriptors else None
    r = lib().ora_bpnn(n, _p(x), _p(lo), _p(hi), _p(per), _p(E), _p(F), _p(W), _p(Ea), _p(Wa),
                       _p(G), _p(dG))
    if r < 0:
        raise RuntimeError("oracle bpnn failed")
    out = {"E": float(E[0]), "F": F, "W": W}
    if per_atom:
        out["Ea"] = Ea
        out["Wa"] = Wa
    if descriptors:
        out["G"] = G
        out["dEdG"] = dG
    return out


def md_bpnn(x, v, masses, lo, hi, periodic, dt, nsteps, skin, model, rebuild_every=0):
    """Velocity-Verlet NVE with Verlet lists and the BPNN model."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    m = _f64(masses, (n,))
    lo, hi, per = _box(lo, hi, periodic)
    _bpnn_set(model)
    thermo = np.zeros((max(nsteps, 1), 3))
    F = np.zeros((n, 3))
    nb = lib().ora_md_run(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 2, None, 0, 0.0,
                          None, None, 0, 0.0, None, skin, dt, nsteps, rebuild_every, None, 0.0,
                          _p(thermo), _p(F))
    if nb < 0:
        raise RuntimeError(f"oracle md_bpnn failed ({nb})")
    return {"x": x, "v": v, "F": F, "thermo": thermo[:nsteps], "n_builds": int(nb)}


def philox4x64(ctr, key):
    """Philox4x64-10 block for a 4-word counter and a 2-word key (uint64)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().ora_philox4x64(_p(c), _p(k), _p(out))
    return out


def md_langevin(x, v, masses, lo, hi, periodic, dt, nsteps, skin, regions, seed,
                lj_params=None, tables=None, ids=None, step0=0, rebuild_every=0,
                piston=None, u_p=0.0):
    """md_run with Langevin thermostat regions: regions = [(x_lo, x_hi, T,
    (u_x, u_y, u_z), beta), ...] (at most 8); ids = permanent atom ids
    (default 0..N-1); step0 = steps done before this run."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    m = _f64(masses, (n,))
    lo, hi, per = _box(lo, hi, periodic)
    thermo = np.zeros((max(nsteps, 1), 3))
    F = np.zeros((n, 3))
    pis = None if piston is None else np.ascontiguousarray(piston, dtype=np.uint8)
    lp = [float(len(regions))]
    for (xl, xh, T, u, beta) in regions:
        lp += [xl, xh, T, u[0], u[1], u[2], beta]
    lp = _f64(lp)
    idv = np.arange(n, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, np.int64)
    if lj_params is not None:
        par = _f64([lj_params.eps, lj_params.sigma, lj_params.rc, lj_params.shift_mode])
        nb = lib().ora_md_langevin(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 0,
                                   _p(par), 0, 0.0, None, None, 0, 0.0, None, skin, dt, nsteps,
                                   rebuild_every, _p(pis), u_p, _p(thermo), _p(F), _p(lp),
                                   _p(idv), int(seed), int(step0))
    else:
        phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
        nb = lib().ora_md_langevin(n, _p(x), _p(v), _p(m), _p(lo), _p(hi), _p(per), 1, None,
                                   phi.shape[0], tables.rc, _p(phi), _p(rho), Ft.shape[0],
                                   tables.rho_max, _p(Ft), skin, dt, nsteps, rebuild_every,
                                   _p(pis), u_p, _p(thermo), _p(F), _p(lp), _p(idv),
                                   int(seed), int(step0))
    if nb < 0:
        raise RuntimeError(f"oracle md_langevin failed ({nb})")
    return {"x": x, "v": v, "F": F, "thermo": thermo[:nsteps], "n_builds": int(nb)}


def profiles(x, v, masses, axis, origin, width, nbins, cross_area, Ua=None, Wa=None):
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    n = x.shape[0]
    m = _f64(masses, (n,))
    Ua = None if Ua is None else _f64(Ua, (n,))
    Wa = None if Wa is None else _f64(Wa, (n, 6))
    out = np.zeros((nbins, 17))
    lib().ora_profiles(n, _p(x), _p(v), _p(m), _p(Ua), _p(Wa), axis, origin, width,
                       nbins, cross_area, _p(out))
    return out


class WindowState:
    """Atoms of a window run with room for `cap` atoms (ids, piston flags)."""

    def __init__(self, x, v, masses, piston, cap):
        n = x.shape[0]
        self.cap = cap
        self.x = np.zeros((cap, 3))
        self.v = np.zeros((cap, 3))
        self.m = np.zeros(cap)
        self.pis = np.zeros(cap, dtype=np.uint8)
        self.ids = np.zeros(cap, dtype=np.int64)
        self.x[:n] = x
        self.v[:n] = v
        self.m[:n] = masses
        self.pis[:n] = np.asarray(piston, dtype=np.uint8)
        self.ids[:n] = np.arange(n)
        self.n = n
        self.next_id = np.array([n], dtype=np.int64)

    def view(self):
        n = self.n
        return {"x": self.x[:n].copy(), "v": self.v[:n].copy(), "m": self.m[:n].copy(),
                "piston": self.pis[:n].astype(bool), "ids": self.ids[:n].copy()}


def window_apply(st, x_lo, x_hi, front_bin, u_p, L_behind, L_ahead, slab_x, slab_v, slab_lx,
                 slab_gap, slab_mass, piston_depth, fixed_front=float("nan")):
    """One application of the window rules (x_lo, x_hi: the box along x;
    front_bin: width of the bins that locate the shock front; a finite
    fixed_front replaces the located front)."""
    sx = _f64(slab_x, (-1, 3))
    sv = _f64(slab_v, (-1, 3))
    st.n = int(lib().ora_window_apply(st.n, st.cap, _p(st.x), _p(st.v), _p(st.m), _p(st.pis),
                                      _p(st.ids), _p(st.next_id), x_lo, x_hi, front_bin,
                                      fixed_front, u_p, L_behind, L_ahead, _p(sx), _p(sv),
                                      sx.shape[0], slab_lx, slab_gap, slab_mass, piston_depth))
    return st


def md_window(st, lo, hi, periodic, tables, dt, nsteps, skin, rebuild_every, u_p, front_bin,
              L_behind, L_ahead, slab_x, slab_v, slab_lx, slab_gap, slab_mass, piston_depth,
              fixed_front=float("nan"), regions=None, seed=0):
    lo, hi, per = _box(lo, hi, periodic)
    phi, rho, Ft = _f64(tables.phi), _f64(tables.rho), _f64(tables.F)
    sx = _f64(slab_x, (-1, 3))
    sv = _f64(slab_v, (-1, 3))
    lp = None
    if regions is not None:
        lp = [float(len(regions))]
        for (xl, xh, T, u, beta) in regions:
            lp += [xl, xh, T, u[0], u[1], u[2], beta]
        lp = _f64(lp)
    n = np.array([st.n], dtype=np.int64)
    nb = lib().ora_md_window(_p(n), st.cap, _p(st.x), _p(st.v), _p(st.m), _p(st.pis),
                             _p(st.ids), _p(st.next_id), _p(lo), _p(hi), _p(per), phi.shape[0],
                             tables.rc, _p(phi), _p(rho), Ft.shape[0], tables.rho_max, _p(Ft),
                             skin, dt, nsteps, rebuild_every, u_p, front_bin, fixed_front,
                             L_behind, L_ahead, _p(sx), _p(sv), sx.shape[0], slab_lx, slab_gap,
                             slab_mass, piston_depth, _p(lp), int(seed))
    if nb < 0:
        raise RuntimeError(f"oracle md_window failed ({nb})")
    st.n = int(n[0])
    return int(nb)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
