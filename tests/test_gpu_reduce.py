"""The per-replica sums behind mdk_compute and the thermo samples.

A first pass sums chunks of 8192 atoms of each replica (one block per chunk),
a second pass sums each replica's chunk partials in chunk order.  Checked
against host sums of the per-atom energies and virials that the same force
pass stored (FP64 path: the per-atom values are plain FP64 results, so the two
totals differ only by the order of the additions: 1e-12 of the summed
magnitudes), on a single replica whose last chunk is ragged and on a batch
whose replicas take one chunk or several.  The sums are also deterministic:
the same state gives bitwise the same totals.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

from test_gpu_parity import lj_ctx

pytestmark = pytest.mark.gpu

CHUNK = 8192


@pytest.fixture(scope="module")
def mdk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk as m
    _build.build()
    m.load()
    return m


def check_totals(E, Wv, U, Wa, bounds):
    for q, (a, b) in enumerate(bounds):
        u, w = U[a:b], Wa[a:b]
        assert abs(E[q] - u.sum()) <= 1e-12 * np.abs(u).sum(), (q, E[q], u.sum())
        np.testing.assert_allclose(Wv[q], w.sum(axis=0), rtol=0,
                                   atol=1e-12 * np.abs(w).sum() + 1e-300)


def test_single_replica_several_chunks(mdk):
    rng = np.random.default_rng(5)
    n = 19                                  # 27,436 atoms: 3 full chunks + 2,860
    a = 5.26
    x = W.fcc_lattice(n, n, n, a) + rng.normal(0, 0.05, size=(4 * n ** 3, 3))
    L = n * a
    lo, hi = np.zeros(3), np.full(3, L)
    x = np.mod(x, L)
    assert x.shape[0] > 3 * CHUNK and x.shape[0] % CHUNK
    ctx = lj_ctx(mdk, x, lo, hi, [1, 1, 1], "fp64")
    E, F, Wv = ctx.compute()
    U, Wa = ctx.per_atom()
    check_totals(E, Wv, U, Wa, [(0, x.shape[0])])
    E2, _, W2 = ctx.compute()
    assert E2[0] == E[0] and np.array_equal(W2, Wv)
    ctx.close()


def test_batched_replicas_one_or_several_chunks(mdk):
    rng = np.random.default_rng(6)
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    reps = [W.lattice_system(rng, (k, k, k), float(a), W.MASS_CU, 0.0, sigma_jitter=0.05)
            for k, a in ((3, 3.6), (14, 3.61), (5, 3.9), (17, 3.55))]
    sizes = [r.n for r in reps]
    assert max(sizes) > 2 * CHUNK and min(sizes) < CHUNK
    ctx = mdk.Context([r.lo for r in reps], [r.hi for r in reps], [r.periodic for r in reps],
                      np.concatenate([r.masses for r in reps]), "fp64", n_atoms=sizes)
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, 0.3)
    ctx.set_state(np.concatenate([r.x for r in reps]), np.concatenate([r.v for r in reps]))
    ctx.build_neighbors(tab.rc, 0.3)
    E, F, Wv = ctx.compute()
    U, Wa = ctx.per_atom()
    ends = np.cumsum(sizes)
    check_totals(E, Wv, U, Wa, list(zip(np.r_[0, ends[:-1]], ends)))
    ctx.close()
