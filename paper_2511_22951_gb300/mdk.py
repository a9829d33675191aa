"""Python binding of libmdk.so: the C-ABI functions under their own names,
plus a small `Context` class that does the argument marshalling.

Only marshalling happens here: device memory comes from torch (one uint8
workspace tensor per context), streams from torch.cuda, and every step of the
MD path runs in the library's CUDA kernels.  There is no CPU fallback: if the
extension is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdk.so")
# MDK_DEBUG=1 in the environment: load the debug build (index checks in the
# kernels, MDK_ERR_BOUNDS), built on first use
DEBUG_LIB_PATH = os.path.join(_HERE, "libmdk_debug.so")

MDK_OK = 0
MDK_ERR_BAD_ARG = -1
MDK_ERR_BOX_TOO_SMALL = -2
MDK_ERR_NEIGH_OVERFLOW = -3
MDK_ERR_ATOM_LOST = -4
MDK_ERR_NONFINITE = -5
MDK_ERR_TIMEOUT = -6
MDK_ERR_CUDA = -7
MDK_ERR_WORKSPACE = -8
MDK_ERR_ORDER = -9
MDK_ERR_RHO_RANGE = -10
MDK_ERR_TOO_LARGE = -11
MDK_ERR_CAPACITY = -12
MDK_ERR_BOUNDS = -13
MDK_FP64 = 0
MDK_MIXED = 1
MDK_LIST_FULL = 0
MDK_LIST_HALF = 1
MDK_LIST_CELLS = 2
_KINDS = {"full": MDK_LIST_FULL, "half": MDK_LIST_HALF, "cells": MDK_LIST_CELLS}

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SZ = ctypes.c_size_t

# name -> argtypes (restype int unless noted)
SIGNATURES = {
    "mdk_create": [ctypes.POINTER(_P), _P, _P, _P, _I64, _P, _I, _P],
    "mdk_create_batch": [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P, _I, _P],
    "mdk_destroy": [_P],
    "mdk_set_capacity": [_P, _I64],
    "mdk_set_potential_lj": [_P, _D, _D, _D, _I],
    "mdk_set_potential_eam": [_P, _I, _D, _P, _P, _I, _D, _P],
    "mdk_set_potential_bpnn": [_P, _D, _I, _P, _P, _I, _P, _P, _I, _I, _P, _P, _P, _P, _P, _D],
    "mdk_workspace_size": [_P, ctypes.POINTER(_SZ)],
    "mdk_set_workspace": [_P, _P, _SZ],
    "mdk_set_state": [_P, _P, _P, _I],
    "mdk_get_state": [_P, _P, _P, _I],
    "mdk_get_natoms": [_P, ctypes.POINTER(_I64)],
    "mdk_checkpoint_size": [_P, ctypes.POINTER(_SZ)],
    "mdk_save_checkpoint": [_P, _P, _SZ],
    "mdk_load_checkpoint": [_P, _P, _SZ],
    "mdk_plan_neighbors": [_P, _D, _D, _I, _I],
    "mdk_build_neighbors": [_P, _D, _D],
    "mdk_neighbor_count": [_P, ctypes.POINTER(_I64)],
    "mdk_get_neighbors": [_P, _P, _P, _P],
    "mdk_compute": [_P, _P, _P, _P, _I],
    "mdk_get_per_atom": [_P, _P, _P],
    "mdk_step": [_P, _D, _I64],
    "mdk_set_thermo": [_P, _I, _I],
    "mdk_get_thermo": [_P, _P, _I, ctypes.POINTER(_I)],
    "mdk_get_counters": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "mdk_set_outer_skin": [_P, _D],
    "mdk_get_build_counts": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "mdk_set_piston": [_P, _D, _P],
    "mdk_set_window": [_P, _D, _D, _P, _P, _I64, _D, _D, _D, _D, _D, _D],
    "mdk_get_ids": [_P, _P],
    "mdk_window_counts": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "mdk_profiles": [_P, _I, _D, _D, _I, _D, _P, _I],
    "mdk_status_string": [_I],
    "mdk_last_device_status": [_P, ctypes.POINTER(_I)],
    "mdk_autotune": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)],
    "mdk_set_launch": [_P, _I, _I],
    "mdk_set_list_kind": [_P, _I],
    "mdk_fma_peak": [_I, ctypes.POINTER(_D)],
    "mdk_get_list_kind": [_P, ctypes.POINTER(_I)],
    "mdk_set_graphs": [_P, _I],
    "mdk_profile": [_P, _I],
    "mdk_get_profile": [_P, _P],
    "mdk_lj_compute_noalloc": [_P, _I64, _P, _P, _P, _D, _D, _D, _I, _P, _P, _P],
    "mdk_eam_vjp": [_P, _P, _P, _P, _I],
    "mdk_set_langevin": [_P, _I, _P, _P, _P, _P, _P, ctypes.c_uint64],
    "mdk_set_langevin_replicas": [_P, _P, _P, ctypes.c_uint64],
}

_lib = None


def load(path: str = None):
    """Load libmdk.so (libmdk_debug.so when MDK_DEBUG=1) and declare every
    C-ABI function.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        if os.environ.get("MDK_DEBUG", "0") not in ("", "0"):
            from . import _build
            path = _build.build(debug=True)
        else:
            path = LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"libmdk.so not found at {path}: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "mdk_status_string" else _I
    _lib = lib
    return lib


class MDKError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load().mdk_status_string(code).decode()
        super().__init__(f"{what}: {msg} ({code})")


def _check(code: int, what: str):
    if code != MDK_OK:
        raise MDKError(code, what)


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(_P)
    return _P(a.data_ptr())


def _host_f64(a, shape):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(shape)


class Context:
    """One MD system (or a batch of replicas) on the current CUDA device.

    Device memory: a single torch uint8 tensor (the workspace) that the
    library lays out; it is reallocated when a call reports that it is too
    small (list capacity growth, new potential table sizes).
    """

    def __init__(self, lo, hi, periodic, masses, precision="fp64", stream=None,
                 device=None, n_atoms=None, capacity=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        self.prec = MDK_FP64 if precision in ("fp64", MDK_FP64) else MDK_MIXED
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        masses = np.ascontiguousarray(masses, dtype=np.float64).ravel()
        h = _P()
        if n_atoms is None:
            lo_ = _host_f64(lo, (3,))
            hi_ = _host_f64(hi, (3,))
            per = np.ascontiguousarray(periodic, dtype=np.int32).reshape(3)
            _check(self.lib.mdk_create(ctypes.byref(h), _ptr(lo_), _ptr(hi_), _ptr(per),
                                       masses.shape[0], _ptr(masses), self.prec,
                                       _P(self.stream.cuda_stream)), "mdk_create")
            self.n_rep = 1
        else:
            n_atoms = np.ascontiguousarray(n_atoms, dtype=np.int64).ravel()
            R = n_atoms.shape[0]
            lo_ = _host_f64(lo, (R, 3))
            hi_ = _host_f64(hi, (R, 3))
            per = np.ascontiguousarray(periodic, dtype=np.int32).reshape(R, 3)
            _check(self.lib.mdk_create_batch(ctypes.byref(h), R, _ptr(lo_), _ptr(hi_),
                                             _ptr(per), _ptr(n_atoms), _ptr(masses),
                                             self.prec, _P(self.stream.cuda_stream)),
                   "mdk_create_batch")
            self.n_rep = R
        self.h = h
        self.n = masses.shape[0]
        self.ws = None
        self._state = None
        self._has_state = False
        self._eam_sizes = None
        self.version = 0  # bumped by every call that changes positions or tables
        self.regrows = 0  # workspaces grown after a list overflow during steps
        self._thermo_every = 0
        self._thermo_stash = []
        if capacity is not None:
            _check(self.lib.mdk_set_capacity(self.h, int(capacity)), "mdk_set_capacity")

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if self.h:
            self.lib.mdk_destroy(self.h)
            self.h = _P()
        self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup ----------------------------------------------------------------
    def set_potential_lj(self, eps, sigma, rc, shift_mode=1):
        self.version += 1
        _check(self.lib.mdk_set_potential_lj(self.h, eps, sigma, rc, shift_mode),
               "mdk_set_potential_lj")

    def set_potential_eam(self, tables):
        phi = _host_f64(tables.phi, (-1,))
        rho = _host_f64(tables.rho, (-1,))
        F = _host_f64(tables.F, (-1,))
        _check(self.lib.mdk_set_potential_eam(self.h, phi.shape[0], tables.rc, _ptr(phi),
                                              _ptr(rho), F.shape[0], tables.rho_max, _ptr(F)),
               "mdk_set_potential_eam")
        self._eam_sizes = (phi.shape[0], F.shape[0])
        self.version += 1

    def set_potential_bpnn(self, model):
        """Behler-Parrinello model (workloads.BPNNModel-like: rc, rad_kind,
        rad_par [n_rad, 2], ang_kind, ang_par [n_ang, 3], W01, b1, W12, b2,
        w23, b3)."""
        rk = np.ascontiguousarray(model.rad_kind, dtype=np.int32)
        ak = np.ascontiguousarray(model.ang_kind, dtype=np.int32)
        rp = _host_f64(model.rad_par, (-1,))
        ap = _host_f64(model.ang_par, (-1,))
        W01 = _host_f64(model.W01, (-1,))
        W12 = _host_f64(model.W12, (-1,))
        H1, H2 = model.W01.shape[1], model.W12.shape[1]
        _check(self.lib.mdk_set_potential_bpnn(
            self.h, float(model.rc), rk.shape[0], _ptr(rk), _ptr(rp), ak.shape[0], _ptr(ak),
            _ptr(ap), H1, H2, _ptr(W01), _ptr(_host_f64(model.b1, (-1,))), _ptr(W12),
            _ptr(_host_f64(model.b2, (-1,))), _ptr(_host_f64(model.w23, (-1,))),
            float(model.b3)), "mdk_set_potential_bpnn")
        self.version += 1

    def plan(self, rc, skin, max_neighbors=0, rebuild_every=0):
        _check(self.lib.mdk_plan_neighbors(self.h, rc, skin, max_neighbors, rebuild_every),
               "mdk_plan_neighbors")

    def workspace_bytes(self) -> int:
        b = _SZ()
        _check(self.lib.mdk_workspace_size(self.h, ctypes.byref(b)), "mdk_workspace_size")
        return int(b.value)

    def alloc_workspace(self):
        """(Re)allocate the workspace.  A state already in the context is
        carried over whole by a checkpoint (ids, step counter, a step
        pending after a list overflow, the lists' build positions)."""
        ck = None
        if self.ws is not None and self._thermo_every > 0:
            try:  # samples not read yet live in the old workspace's ring
                self._thermo_stash.append(self._read_thermo())
            except MDKError:
                pass
        if self.ws is not None and self._has_state:
            try:
                ck = self.save_checkpoint()
            except MDKError:
                ck = None
        for _ in range(4):
            nbytes = self.workspace_bytes()
            self.ws = None
            self.ws = self.torch.empty(nbytes + 256, dtype=self.torch.uint8, device=self.device)
            base = self.ws.data_ptr()
            off = (-base) % 256
            _check(self.lib.mdk_set_workspace(self.h, _P(base + off), nbytes),
                   "mdk_set_workspace")
            if ck is not None:
                r = self.lib.mdk_load_checkpoint(self.h, _ptr(ck), ck.nbytes)
                if r == MDK_ERR_NEIGH_OVERFLOW:   # the replayed lists need more room
                    continue
                _check(r, "mdk_load_checkpoint")
            elif self._state is not None:
                x, v, on_dev = self._state
                _check(self.lib.mdk_set_state(self.h, _ptr(x), _ptr(v), on_dev),
                       "mdk_set_state")
            return
        raise MDKError(MDK_ERR_NEIGH_OVERFLOW, "mdk_load_checkpoint")

    def save_checkpoint(self):
        """The context's whole dynamic state as a numpy uint8 buffer."""
        n = _SZ()
        _check(self.lib.mdk_checkpoint_size(self.h, ctypes.byref(n)), "mdk_checkpoint_size")
        buf = np.zeros(int(n.value), dtype=np.uint8)
        _check(self.lib.mdk_save_checkpoint(self.h, _ptr(buf), buf.nbytes),
               "mdk_save_checkpoint")
        return buf

    def load_checkpoint(self, buf):
        """Restore a state saved by save_checkpoint (this context configured
        like the saving one); continues bitwise like the saving run."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        if self.ws is None:
            self.alloc_workspace()
        for _ in range(4):
            r = self.lib.mdk_load_checkpoint(self.h, _ptr(buf), buf.nbytes)
            if r in (MDK_ERR_NEIGH_OVERFLOW, MDK_ERR_WORKSPACE):
                nbytes = self.workspace_bytes()
                self.ws = None
                self.ws = self.torch.empty(nbytes + 256, dtype=self.torch.uint8,
                                           device=self.device)
                base = self.ws.data_ptr()
                _check(self.lib.mdk_set_workspace(self.h, _P(base + (-base) % 256), nbytes),
                       "mdk_set_workspace")
                continue
            _check(r, "mdk_load_checkpoint")
            self._has_state = True
            self._state = None
            self.version += 1
            return
        raise MDKError(MDK_ERR_NEIGH_OVERFLOW, "mdk_load_checkpoint")

    def set_thermo(self, every, capacity=1024):
        self._thermo_every = int(every)
        self._thermo_stash = []
        r = self.lib.mdk_set_thermo(self.h, every, capacity)
        if r == MDK_ERR_WORKSPACE:
            if self.ws is not None:
                self.alloc_workspace()
        else:
            _check(r, "mdk_set_thermo")

    # -- state ----------------------------------------------------------------
    def set_state(self, x, v=None):
        """x, v: numpy (host) or torch CUDA tensors, shape [N, 3] float64."""
        if self.ws is None:
            self.alloc_workspace()
        if isinstance(x, np.ndarray):
            x = _host_f64(x, (self.n, 3))
            v = None if v is None else _host_f64(v, (self.n, 3))
            on_dev = 0
        else:
            on_dev = 1
        self._state = (x, v, on_dev)
        self._has_state = True
        self.version += 1
        _check(self.lib.mdk_set_state(self.h, _ptr(x), _ptr(v), on_dev), "mdk_set_state")

    def _save_state(self):
        x, v = self.get_state()
        self._state = (x, v, 0)

    def get_state(self):
        n = self.natoms()
        x = np.zeros((n, 3))
        v = np.zeros((n, 3))
        _check(self.lib.mdk_get_state(self.h, _ptr(x), _ptr(v), 0), "mdk_get_state")
        return x, v

    def natoms(self) -> int:
        n = _I64()
        _check(self.lib.mdk_get_natoms(self.h, ctypes.byref(n)), "mdk_get_natoms")
        return int(n.value)

    # -- neighbours -------------------------------------------------------------
    def build_neighbors(self, rc, skin):
        for _ in range(4):
            r = self.lib.mdk_build_neighbors(self.h, rc, skin)
            if r in (MDK_ERR_NEIGH_OVERFLOW, MDK_ERR_WORKSPACE):
                # capacity raised or new plan: resize the workspace, restore the state
                self.alloc_workspace()
                continue
            _check(r, "mdk_build_neighbors")
            return
        raise MDKError(MDK_ERR_NEIGH_OVERFLOW, "mdk_build_neighbors")

    def neighbor_counts(self):
        """Number of list entries of every atom (caller's order)."""
        n = self.natoms()
        off = np.zeros(n + 1, dtype=np.int64)
        _check(self.lib.mdk_get_neighbors(self.h, _ptr(off), None, None), "mdk_get_neighbors")
        return np.diff(off)

    def neighbors(self):
        """(offsets[N+1], j[total], image[total,3]) in the caller's atom order."""
        n = self.natoms()
        tot = _I64()
        _check(self.lib.mdk_neighbor_count(self.h, ctypes.byref(tot)), "mdk_neighbor_count")
        off = np.zeros(n + 1, dtype=np.int64)
        j = np.zeros(max(tot.value, 1), dtype=np.int32)
        im = np.zeros((max(tot.value, 1), 3), dtype=np.int32)
        _check(self.lib.mdk_get_neighbors(self.h, _ptr(off), _ptr(j), _ptr(im)),
               "mdk_get_neighbors")
        return off, j[:tot.value], im[:tot.value]

    # -- compute / step -----------------------------------------------------------
    def compute(self):
        """Host results: (E [n_rep], F [N,3], virial [n_rep,6])."""
        n = self.natoms()
        E = np.zeros(self.n_rep)
        F = np.zeros((n, 3))
        W = np.zeros((self.n_rep, 6))
        r = self.lib.mdk_compute(self.h, _ptr(E), _ptr(F), _ptr(W), 0)
        if r in (MDK_ERR_NEIGH_OVERFLOW, MDK_ERR_WORKSPACE):
            self.alloc_workspace()
            r = self.lib.mdk_compute(self.h, _ptr(E), _ptr(F), _ptr(W), 0)
        _check(r, "mdk_compute")
        return E, F, W

    def compute_device(self, E, F, W):
        _check(self.lib.mdk_compute(self.h, _ptr(E), _ptr(F), _ptr(W), 1), "mdk_compute")

    def eam_vjp(self, gE=None, gF=None):
        """Host gradient of sum_r gE[r] E_r + sum_i gF_i . F_i with respect to the
        EAM knots: returns (d_phi [nr], d_rho [nr], d_F [nrho])."""
        nr, nrho = self._eam_sizes
        gE = None if gE is None else _host_f64(gE, (self.n_rep,))
        gF = None if gF is None else _host_f64(gF, (self.natoms(), 3))
        out = np.zeros(2 * nr + nrho)
        r = self.lib.mdk_eam_vjp(self.h, _ptr(gE), _ptr(gF), _ptr(out), 0)
        if r in (MDK_ERR_NEIGH_OVERFLOW, MDK_ERR_WORKSPACE):
            self.alloc_workspace()
            r = self.lib.mdk_eam_vjp(self.h, _ptr(gE), _ptr(gF), _ptr(out), 0)
        _check(r, "mdk_eam_vjp")
        return out[:nr], out[nr:2 * nr], out[2 * nr:]

    def eam_vjp_device(self, gE, gF, out):
        """Device variant: gE [n_rep], gF [N,3] (either may be None), out
        [2 nr + nrho] float64 CUDA tensors; returns after enqueueing."""
        _check(self.lib.mdk_eam_vjp(self.h, _ptr(gE), _ptr(gF), _ptr(out), 1), "mdk_eam_vjp")

    def per_atom(self):
        n = self.natoms()
        U = np.zeros(n)
        Wa = np.zeros((n, 6))
        _check(self.lib.mdk_get_per_atom(self.h, _ptr(U), _ptr(Wa)), "mdk_get_per_atom")
        return U, Wa

    def step(self, dt, nsteps, check=True):
        """nsteps velocity-Verlet steps.  check=True: read the device status
        afterwards; a list that outgrew its capacity during the steps (which
        stops them at that build) is handled by growing the workspace,
        carrying the mid-step state over by a checkpoint and running the
        remaining steps (each overflow once; `regrows` counts them)."""
        self.version += 1
        if not check:
            _check(self.lib.mdk_step(self.h, dt, int(nsteps)), "mdk_step")
            return
        left = int(nsteps)
        for _ in range(16):
            s0 = self.counters()[1]
            _check(self.lib.mdk_step(self.h, dt, left), "mdk_step")
            try:
                self.check()
                return
            except MDKError as e:
                if e.code != MDK_ERR_NEIGH_OVERFLOW:
                    raise
            done = self.counters()[1] - s0
            if not 0 <= done < left:
                raise MDKError(MDK_ERR_NEIGH_OVERFLOW, "mdk_step")
            left -= done
            self.regrows += 1
            self.alloc_workspace()
        raise MDKError(MDK_ERR_NEIGH_OVERFLOW, "mdk_step: the lists kept outgrowing them")

    def check(self):
        bits = _I()
        _check(self.lib.mdk_last_device_status(self.h, ctypes.byref(bits)),
               "device status")

    def _read_thermo(self, max_samples=100000):
        out = np.zeros((max_samples, self.n_rep, 10))
        n = _I()
        _check(self.lib.mdk_get_thermo(self.h, _ptr(out), max_samples, ctypes.byref(n)),
               "mdk_get_thermo")
        return out[:n.value]

    def thermo(self, max_samples=100000):
        """Samples taken since the last call: [n, n_rep, 10] = step, E_kin,
        E_pot, n_atoms, virial[6] (including samples kept across a workspace
        that grew after a list overflow)."""
        out = self._read_thermo(max_samples)
        if self._thermo_stash:
            out = np.concatenate(self._thermo_stash + [out])
            self._thermo_stash = []
        return out

    def counters(self):
        b, s = _I64(), _I64()
        _check(self.lib.mdk_get_counters(self.h, ctypes.byref(b), ctypes.byref(s)),
               "mdk_get_counters")
        return int(b.value), int(s.value)

    def set_outer_skin(self, skin_outer):
        """Two-level lists: an outer list within rc + skin_outer from which
        the Verlet list is filtered while the displacement budget lasts (0:
        off).  Call after plan(); the workspace is re-allocated on next use."""
        _check(self.lib.mdk_set_outer_skin(self.h, float(skin_outer)), "mdk_set_outer_skin")
        if self.ws is not None:
            self.alloc_workspace()

    def build_counts(self):
        """(list builds, full builds) so far."""
        b, f = _I64(), _I64()
        _check(self.lib.mdk_get_build_counts(self.h, ctypes.byref(b), ctypes.byref(f)),
               "mdk_get_build_counts")
        return int(b.value), int(f.value)

    def autotune(self, reps=3, key=None):
        """Pick threads-per-atom and block size by timing every shape (LJ:
        full and half lists; `list_kind` tells which won).  With the
        environment variable MDK_AUTOTUNE_CACHE naming a JSON file and a `key`
        describing the workload (any string), a shape found before for that
        key and device is reused instead of timed again (ms is then NaN)."""
        path = os.environ.get("MDK_AUTOTUNE_CACHE", "")
        ck = None
        if path and key is not None:
            ck = autotune_cache_key(key, self.prec, self.torch.cuda.get_device_name(self.device))
            hit = autotune_cache_get(path, ck)
            if hit is not None:
                self.set_launch(hit["tpa"], hit["block"])
                if self.list_kind != hit["list"]:
                    self.set_list_kind(hit["list"])
                return hit["tpa"], hit["block"], float("nan")
        t, b, ms = _I(), _I(), _D()
        _check(self.lib.mdk_autotune(self.h, reps, ctypes.byref(t), ctypes.byref(b),
                                     ctypes.byref(ms)), "mdk_autotune")
        if ck is not None:
            autotune_cache_put(path, ck, {"tpa": int(t.value), "block": int(b.value),
                                          "list": self.list_kind, "ms": float(ms.value)})
        return int(t.value), int(b.value), float(ms.value)

    def set_graphs(self, enable=True):
        _check(self.lib.mdk_set_graphs(self.h, 1 if enable else 0), "mdk_set_graphs")

    def set_launch(self, tpa, block):
        _check(self.lib.mdk_set_launch(self.h, tpa, block), "mdk_set_launch")

    def set_list_kind(self, kind):
        """'full' (every atom lists all its neighbours), 'half' (each pair
        once, Newton's third law with accumulating atomics; LJ and EAM) or
        'cells' (no list: LJ forces from the cells, one warp per cell)."""
        _check(self.lib.mdk_set_list_kind(self.h, _KINDS[kind]), "mdk_set_list_kind")

    @property
    def list_kind(self):
        k = _I()
        _check(self.lib.mdk_get_list_kind(self.h, ctypes.byref(k)), "mdk_get_list_kind")
        return {v: n for n, v in _KINDS.items()}[k.value]

    def profile(self, enable=True):
        _check(self.lib.mdk_profile(self.h, 1 if enable else 0), "mdk_profile")

    def get_profile(self):
        out = np.zeros(8)
        _check(self.lib.mdk_get_profile(self.h, _ptr(out)), "mdk_get_profile")
        keys = ("force_ms", "force_passes", "rebuild_ms", "rebuild_chains", "kernels",
                "builds", "kick_ms", "kicks")
        return dict(zip(keys, out.tolist()))

    def set_window(self, L_behind, L_ahead, slab_x, slab_v, slab_lx, slab_gap, slab_mass,
                   piston_depth, front_bin, fixed_front=float("nan")):
        sx = _host_f64(slab_x, (-1, 3))
        sv = _host_f64(slab_v, (-1, 3))
        args = (L_behind, L_ahead, _ptr(sx), _ptr(sv), sx.shape[0], slab_lx, slab_gap,
                slab_mass, piston_depth, front_bin, fixed_front)
        r = self.lib.mdk_set_window(self.h, *args)
        if r == MDK_ERR_WORKSPACE:
            self.alloc_workspace()
            r = self.lib.mdk_set_window(self.h, *args)
        _check(r, "mdk_set_window")
        self.version += 1

    def ids(self):
        n = self.natoms()
        out = np.zeros(n, dtype=np.int64)
        _check(self.lib.mdk_get_ids(self.h, _ptr(out)), "mdk_get_ids")
        return out

    def window_counts(self):
        a, b = _I64(), _I64()
        _check(self.lib.mdk_window_counts(self.h, ctypes.byref(a), ctypes.byref(b)),
               "mdk_window_counts")
        return int(a.value), int(b.value)

    def profiles(self, axis, origin, bin_w, nbins, cross_area):
        """Appendix statistics per bin (host [nbins, 17]): N, M, u[3], T[3],
        E_pot, P[xx, yy, zz, xy, xz, yz], E_kin, V."""
        out = np.zeros((nbins, 17))
        _check(self.lib.mdk_profiles(self.h, int(axis), float(origin), float(bin_w), int(nbins),
                                     float(cross_area), _ptr(out), 0), "mdk_profiles")
        return out

    def set_langevin(self, regions, seed=0):
        """regions = [(x_lo, x_hi, T, (u_x, u_y, u_z), beta), ...] (<= 8; [] = off)."""
        n = len(regions)
        xl = np.array([r[0] for r in regions], dtype=np.float64)
        xh = np.array([r[1] for r in regions], dtype=np.float64)
        T = np.array([r[2] for r in regions], dtype=np.float64)
        u = np.array([r[3] for r in regions], dtype=np.float64).reshape(n, 3)
        b = np.array([r[4] for r in regions], dtype=np.float64)
        _check(self.lib.mdk_set_langevin(self.h, n, _ptr(xl), _ptr(xh), _ptr(T), _ptr(u),
                                         _ptr(b), int(seed)), "mdk_set_langevin")
        self.version += 1

    def set_langevin_replicas(self, T, beta, seed=0):
        """Whole-replica thermostats: T [n_rep] (K), beta [n_rep] (1/fs); T=None: off."""
        if T is None:
            _check(self.lib.mdk_set_langevin_replicas(self.h, None, None, int(seed)),
                   "mdk_set_langevin_replicas")
        else:
            Tv = _host_f64(T, (self.n_rep,))
            bv = _host_f64(np.broadcast_to(beta, (self.n_rep,)), (self.n_rep,))
            _check(self.lib.mdk_set_langevin_replicas(self.h, _ptr(Tv), _ptr(bv), int(seed)),
                   "mdk_set_langevin_replicas")
        self.version += 1

    def set_piston(self, u_p, flags):
        f = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
        _check(self.lib.mdk_set_piston(self.h, u_p, _ptr(f)), "mdk_set_piston")


def autotune_cache_key(key, precision, device_name):
    """The cache entry of a workload key on a device model and precision."""
    return f"{device_name}|{'fp64' if precision in (MDK_FP64, 'fp64') else 'mixed'}|{key}"


def autotune_cache_get(path, ck):
    """The stored launch shape of cache key ck, or None."""
    import json
    try:
        with open(path) as f:
            e = json.load(f).get(ck)
    except (OSError, ValueError):
        return None
    if not isinstance(e, dict) or e.get("list") not in _KINDS or \
            e.get("tpa") not in (1, 2, 4, 8, 32) or e.get("block") not in (128, 256, 512):
        return None
    return e


def autotune_cache_put(path, ck, entry):
    """Store a launch shape under key ck (the file is rewritten atomically)."""
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        if not isinstance(d, dict):
            d = {}
    except (OSError, ValueError):
        d = {}
    d[ck] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def fma_peak(precision="fp64"):
    """Measured FMA throughput (TFLOP/s) of the current device: "fp64" or
    "mixed" (FP32)."""
    lib = load()
    v = _D()
    _check(lib.mdk_fma_peak(MDK_FP64 if precision == "fp64" else MDK_MIXED, ctypes.byref(v)),
           "mdk_fma_peak")
    return float(v.value)


def make_context(wl, precision=None, stream=None, rebuild_every=0, max_neighbors=0,
                 capacity=None, skin_outer=0.0):
    """Context for a workloads.Workload: potential, plan, workspace, state, lists
    (skin_outer > 0: two-level lists, see Context.set_outer_skin)."""
    prec = precision or wl.precision
    if len(wl.systems) == 1:
        s = wl.systems[0]
        ctx = Context(s.lo, s.hi, s.periodic, s.masses, prec, stream, capacity=capacity)
    else:
        ss = wl.systems
        ctx = Context([q.lo for q in ss], [q.hi for q in ss], [q.periodic for q in ss],
                      np.concatenate([q.masses for q in ss]), prec, stream,
                      n_atoms=[q.n for q in ss])
    if wl.potential == "lj":
        ctx.set_potential_lj(wl.lj.eps, wl.lj.sigma, wl.lj.rc, wl.lj.shift_mode)
    elif wl.potential == "bpnn":
        ctx.set_potential_bpnn(wl.extra["bpnn"])
    else:
        ctx.set_potential_eam(wl.tables)
    ctx.plan(wl.rc, wl.skin, max_neighbors, rebuild_every)
    if skin_outer:
        ctx.set_outer_skin(skin_outer)
    x = np.concatenate([q.x for q in wl.systems])
    v = np.concatenate([q.v for q in wl.systems])
    ctx.set_state(x, v)
    ctx.build_neighbors(wl.rc, wl.skin)
    return ctx
