"""The debug build (libmdk_debug.so: every kernel's index checks compiled in,
MDK_DEBUG=1 selects it) on the GPU: the small parity cases -- LJ and EAM,
FP64 and mixed, full and half lists, a few velocity-Verlet steps with list
rebuilds -- run without a single check firing and give the oracle's results
at the usual bars.  Run in a child process, since a process loads one
library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, sys
sys.path.insert(0, ROOT)
import oracle
from paper_2511_22951_gb300 import mdk, workloads as W
lib = mdk.load()
assert mdk.load() is lib
import ctypes
rng = np.random.default_rng(4)
lj = W.LJ_AR
x = W.fcc_lattice(4, 4, 4, 5.26) + rng.normal(0, 0.1, (256, 3))
L = 4 * 5.26
x = np.mod(x, L)
ref = oracle.lj(x, [0] * 3, [L] * 3, [1, 1, 1], lj.eps, lj.sigma, lj.rc, 1)
for prec in ("fp64", "mixed"):
    for kind in ("full", "half"):
        c = mdk.Context([0] * 3, [L] * 3, [1, 1, 1], np.full(256, lj.mass), prec)
        c.set_potential_lj(lj.eps, lj.sigma, lj.rc, 1)
        c.set_list_kind(kind)
        c.plan(lj.rc, 0.3)
        c.set_state(x, np.zeros_like(x))
        E, F, _ = c.compute()
        tol = 1e-12 if prec == "fp64" else 1e-5
        rms = np.sqrt(np.mean((F - ref["F"]) ** 2)) / np.sqrt(np.mean(ref["F"] ** 2))
        assert rms <= tol, (prec, kind, rms)
        v = W.maxwell_velocities(rng, np.full(256, lj.mass), 300.0)
        c.set_state(x, v)
        c.step(2.0, 40)           # check=True: any debug check raises MDK_ERR_BOUNDS
        assert c.counters()[0] > 1
        c.close()
tab = W.tabulate_fs_eam(W.CU_LIKE)
xe = W.fcc_lattice(3, 3, 3, 3.3) + rng.normal(0, 0.05, (108, 3))
Le = 3 * 3.3
re_ = oracle.eam(xe, [0] * 3, [Le] * 3, [1, 1, 1], tab)
for prec in ("fp64", "mixed"):
    for kind in ("full", "half"):
        c = mdk.Context([0] * 3, [Le] * 3, [1, 1, 1], np.full(108, W.MASS_CU), prec)
        c.set_potential_eam(tab)
        c.set_list_kind(kind)
        c.plan(tab.rc, 0.3)
        c.set_state(xe, np.zeros_like(xe))
        E, F, _ = c.compute()
        tol = 1e-12 if prec == "fp64" else 1e-5
        rms = np.sqrt(np.mean((F - re_["F"]) ** 2)) / np.sqrt(np.mean(re_["F"] ** 2))
        assert rms <= tol, (prec, kind, rms)
        c.step(1.0, 20)
        c.close()
print("debug build clean")
'''


def test_debug_build_runs_the_parity_cases_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, MDK_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build clean" in r.stdout
    assert os.path.exists(os.path.join(ROOT, "paper_2511_22951_gb300", "libmdk_debug.so"))
