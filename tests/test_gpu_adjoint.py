"""Parity of the GPU EAM adjoint (mdk_eam_vjp, through the C ABI) with the
oracle's gradient, and with finite differences of the GPU forward pass.

Bars (from the arithmetic):
  * FP64 path: every knot gradient within 1e-10 of the largest one of its
    table.  The GPU takes r = r^2 rsqrt(r^2) and sums in another order, so
    u = r / h moves by a few ulp (5000 * 2^-52 ~ 1e-12) and each weight by
    ~1e-11 relative; 1e-10 leaves a margin of ten.
  * mixed path (FP32 pair arithmetic): r carries a relative rounding of
    2^-24, so u = r / h is off by up to 5000 * 6e-8 = 3e-4 and a pair's
    weight moves between the two knots of its interval by that much.  The
    physical content is the derivative along a smooth knot direction, which
    such shifts barely touch: |<g_gpu - g_oracle, v>| <= 1e-5 sum_k |g_k v_k|
    (the size of the terms of the sum, since a projection may cancel) for
    smooth v; knot by knot the bar is 2e-3 of the table's largest entry.
"""
import numpy as np
import pytest

from paper_2511_22951_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk as m
    _build.build()
    m.load()
    return m


def eam_ctx(mdk, x, lo, hi, per, prec, tab, mass=W.MASS_CU):
    n = x.shape[0]
    ctx = mdk.Context(lo, hi, per, np.full(n, mass), prec)
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, 0.3)
    ctx.set_state(x, np.zeros((n, 3)))
    ctx.build_neighbors(tab.rc, 0.3)
    return ctx


def crystal(seed, n=3, a=3.5, sigma=0.08):
    rng = np.random.default_rng(seed)
    x = W.jitter(rng, W.fcc_lattice(n, n, n, a), sigma)
    L = n * a
    return x, [0.0] * 3, [L] * 3, [1, 1, 1], rng


def smooth_directions(n, count, rng):
    k = np.arange(n) / (n - 1)
    return [sum(rng.normal() * np.sin(np.pi * (m + 1) * k + rng.uniform(0, 6.3))
                for m in range(4)) for _ in range(count)]


def assert_fp64_grad(g, o):
    for a, b in zip(g, o):
        scale = np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= 1e-10 * scale, np.max(np.abs(a - b)) / scale


def assert_mixed_grad(g, o, rng):
    for a, b in zip(g, o):
        scale = np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= 2e-3 * scale, np.max(np.abs(a - b)) / scale
        for v in smooth_directions(b.shape[0], 3, rng):
            ref = float(b @ v)
            size = float(np.abs(b) @ np.abs(v))
            assert abs(float(a @ v) - ref) <= 1e-5 * size, (a @ v, ref, size)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vjp_matches_oracle(mdk, ora, prec):
    x, lo, hi, per, rng = crystal(7)
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    gE = 0.7
    gF = rng.normal(size=x.shape)
    ctx = eam_ctx(mdk, x, lo, hi, per, prec, tab)
    g = ctx.eam_vjp([gE], gF)
    o = ora.eam_vjp(x, lo, hi, per, tab, gE, gF)
    if prec == "fp64":
        assert_fp64_grad(g, o)
    else:
        assert_mixed_grad(g, o, rng)


def test_vjp_energy_only_and_forces_only(mdk, ora):
    """gE or gF left out (NULL) counts as zero."""
    x, lo, hi, per, rng = crystal(8)
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    ctx = eam_ctx(mdk, x, lo, hi, per, "fp64", tab)
    assert_fp64_grad(ctx.eam_vjp([1.0], None), ora.eam_vjp(x, lo, hi, per, tab, 1.0, None))
    gF = rng.normal(size=x.shape)
    assert_fp64_grad(ctx.eam_vjp(None, gF), ora.eam_vjp(x, lo, hi, per, tab, 0.0, gF))


def test_vjp_small_tables_and_ends(mdk, ora):
    """Few knots: pairs reach the first and last intervals, densities sit in
    the first F interval and above rho_max (linear continuation)."""
    rng = np.random.default_rng(3)
    gas = rng.uniform(0.0, 9.0, size=(36, 3))
    dimers = []
    for q, r in enumerate((0.006, 0.025, 0.045, 5.3, 5.495)):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        a = np.array([20.0 + 10.0 * q, 20.0, 20.0])
        dimers.append(np.stack([a, a + r * u]))
    x = np.concatenate([gas] + dimers)
    lo, hi, per = [-1.0] * 3, [80.0] * 3, [0, 0, 0]
    p = W.CU_LIKE
    t0 = W.tabulate_fs_eam(p, nr=300, nrho=300)
    rho = ora.eam(x, lo, hi, per, t0)["rho"]
    rmax = float(np.quantile(rho, 0.9))
    tab = W.EAMTables(rc=t0.rc, phi=t0.phi, rho=t0.rho, rho_max=rmax,
                      F=W.fs_embed(p, np.arange(40) * (rmax / 39)))
    gE, gF = 0.8, rng.normal(size=x.shape)
    ctx = eam_ctx(mdk, x, lo, hi, per, "fp64", tab)
    from paper_2511_22951_gb300.mdk import MDKError, MDK_ERR_RHO_RANGE
    with pytest.raises(MDKError) as e:
        ctx.eam_vjp([gE], gF)
    assert e.value.code == MDK_ERR_RHO_RANGE
    out = np.zeros(2 * tab.nr + tab.nrho)
    gE_h = np.array([gE])
    gF_h = np.ascontiguousarray(gF)
    rc = ctx.lib.mdk_eam_vjp(ctx.h, gE_h.ctypes.data, gF_h.ctypes.data, out.ctypes.data, 0)
    assert rc == MDK_ERR_RHO_RANGE  # flagged, gradient still written
    g = (out[:tab.nr], out[tab.nr:2 * tab.nr], out[2 * tab.nr:])
    o = ora.eam_vjp(x, lo, hi, per, tab, gE, gF)
    assert np.all(o[0][:3] != 0) and np.all(o[2][-1] != 0)
    assert_fp64_grad(g, o)


def test_vjp_matches_gpu_finite_differences(mdk):
    """E and F are linear in the phi and F knots: central differences of the
    GPU's own FP64 forward pass are exact up to rounding; rho knots by
    Richardson differences along a random direction."""
    x, lo, hi, per, rng = crystal(9)
    tab = W.tabulate_fs_eam(W.CU_LIKE, nr=600, nrho=600)
    gE = 0.3
    gF = rng.normal(size=x.shape)
    ctx = eam_ctx(mdk, x, lo, hi, per, "fp64", tab)
    dphi, drho, dF = ctx.eam_vjp([gE], gF)

    def loss(phi=tab.phi, rho=tab.rho, F=tab.F):
        ctx.set_potential_eam(W.EAMTables(rc=tab.rc, phi=phi, rho=rho, rho_max=tab.rho_max, F=F))
        E, Fo, _ = ctx.compute()
        return gE * E[0] + float(np.sum(gF * Fo))

    for g, name, n in ((dphi, "phi", tab.nr), (dF, "F", tab.nrho)):
        base = getattr(tab, name)
        for k in np.nonzero(g)[0][::37]:
            e = np.zeros(n)
            e[k] = 1e-2
            fd = (loss(**{name: base + e}) - loss(**{name: base - e})) / 2e-2
            assert abs(g[k] - fd) <= 1e-9 * np.max(np.abs(g)), (name, k, g[k], fd)
    v = rng.normal(size=tab.nr)

    def fd_rho(h):
        return (loss(rho=tab.rho + h * v) - loss(rho=tab.rho - h * v)) / (2 * h)

    rich = (4 * fd_rho(1e-6) - fd_rho(2e-6)) / 3
    assert float(drho @ v) == pytest.approx(rich, rel=1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_vjp_matches_oracle(mdk, ora, prec):
    """Replicas share the tables: the batch gradient is the sum over replicas
    of each replica's gradient with its own energy weight."""
    rng = np.random.default_rng(2)
    reps = []
    for a, n in zip(rng.uniform(3.0, 4.2, 5), [3, 4, 3, 5, 3]):
        reps.append(W.lattice_system(rng, (n, n, n), float(a), W.MASS_CU, 0.0,
                                     sigma_jitter=0.05))
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    ctx = mdk.Context([r.lo for r in reps], [r.hi for r in reps], [r.periodic for r in reps],
                      np.concatenate([r.masses for r in reps]), prec,
                      n_atoms=[r.n for r in reps])
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, 0.3)
    ctx.set_state(np.concatenate([r.x for r in reps]))
    ctx.build_neighbors(tab.rc, 0.3)
    gE = rng.uniform(0.5, 1.5, len(reps))
    gF = rng.normal(size=(sum(r.n for r in reps), 3))
    g = ctx.eam_vjp(gE, gF)
    o = [np.zeros(tab.nr), np.zeros(tab.nr), np.zeros(tab.nrho)]
    off = 0
    for q, r in enumerate(reps):
        oq = ora.eam_vjp(r.x, r.lo, r.hi, r.periodic, tab, gE[q], gF[off:off + r.n])
        for a, b in zip(o, oq):
            a += b
        off += r.n
    if prec == "fp64":
        assert_fp64_grad(g, o)
    else:
        assert_mixed_grad(g, o, rng)


def test_device_and_host_calls_agree(mdk):
    import torch
    x, lo, hi, per, rng = crystal(12)
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    ctx = eam_ctx(mdk, x, lo, hi, per, "fp64", tab)
    gF = rng.normal(size=x.shape)
    h = np.concatenate(ctx.eam_vjp([0.5], gF))
    out = torch.empty(2 * tab.nr + tab.nrho, dtype=torch.float64, device="cuda")
    ctx.eam_vjp_device(torch.tensor([0.5], dtype=torch.float64, device="cuda"),
                       torch.tensor(gF, device="cuda"), out)
    torch.cuda.synchronize()
    d = out.cpu().numpy()
    assert np.max(np.abs(d - h)) <= 1e-12 * np.max(np.abs(h))


def test_empty_system_gradient_is_zero(mdk):
    tab = W.tabulate_fs_eam(W.CU_LIKE, nr=100, nrho=100)
    ctx = mdk.Context([0, 0, 0], [20, 20, 20], [1, 1, 1], np.zeros(0), "fp64")
    ctx.set_potential_eam(tab)
    ctx.plan(tab.rc, 0.3)
    ctx.set_state(np.zeros((0, 3)))
    g = ctx.eam_vjp([1.0], np.zeros((0, 3)))
    assert all(np.all(a == 0) for a in g)


def test_vjp_needs_eam(mdk):
    from paper_2511_22951_gb300.mdk import MDKError, MDK_ERR_ORDER
    rng = np.random.default_rng(1)
    x = W.jitter(rng, W.fcc_lattice(3, 3, 3, 5.26), 0.05)
    L = 3 * 5.26
    ctx = mdk.Context([0] * 3, [L] * 3, [1] * 3, np.full(x.shape[0], W.MASS_AR), "fp64")
    ctx.set_potential_lj(W.LJ_AR.eps, W.LJ_AR.sigma, W.LJ_AR.rc, 1)
    ctx.plan(W.LJ_AR.rc, 0.3)
    ctx.set_state(x)
    ctx._eam_sizes = (3, 3)
    with pytest.raises(MDKError) as e:
        ctx.eam_vjp([1.0], None)
    assert e.value.code == MDK_ERR_ORDER


def test_autograd_function_matches_oracle(mdk, ora):
    """loss = sum_r E_r + sum_i |F_i - F_ref,i|^2 through torch.autograd."""
    import torch
    from paper_2511_22951_gb300.adjoint import eam_energy_forces
    x, lo, hi, per, rng = crystal(14)
    tab = W.tabulate_fs_eam(W.CU_LIKE)
    ctx = eam_ctx(mdk, x, lo, hi, per, "fp64", tab)
    F_ref = torch.tensor(rng.normal(scale=0.3, size=x.shape), device="cuda")
    phi = torch.tensor(tab.phi, requires_grad=True)
    rho = torch.tensor(tab.rho, requires_grad=True)
    Fk = torch.tensor(tab.F, requires_grad=True)
    E, F = eam_energy_forces(ctx, phi, rho, Fk, tab.rc, tab.rho_max)
    loss = E.sum() + ((F - F_ref) ** 2).sum()
    loss.backward()
    ref = ora.eam(x, lo, hi, per, tab)
    assert float(E[0].detach()) == pytest.approx(ref["E"], rel=1e-12)
    gF = 2.0 * (ref["F"] - F_ref.cpu().numpy())
    o = ora.eam_vjp(x, lo, hi, per, tab, 1.0, gF)
    assert_fp64_grad((phi.grad.numpy(), rho.grad.numpy(), Fk.grad.numpy()), o)
    # the context moved on: a second backward through the old graph refuses
    E, F = eam_energy_forces(ctx, phi, rho, Fk, tab.rc, tab.rho_max)
    ctx.step(1.0, 1)
    with pytest.raises(RuntimeError):
        E.sum().backward()


@pytest.mark.slow
def test_coldcurve_64_replicas_vjp(mdk, ora):
    """The 64-replica Cu cold curve at full size, mixed precision, loss
    sum_r E_r + sum_i |F_i - F_ref,i|^2 with seeded F_ref."""
    wl = W.config4()
    ctx = mdk.make_context(wl, precision="mixed")
    rng = np.random.default_rng(40)
    n = sum(s.n for s in wl.systems)
    F_ref = rng.normal(scale=0.2, size=(n, 3))
    E, F, _ = ctx.compute()
    gF = 2.0 * (F - F_ref)
    gE = np.ones(len(wl.systems))
    g = ctx.eam_vjp(gE, gF)
    tab = wl.tables
    o = [np.zeros(tab.nr), np.zeros(tab.nr), np.zeros(tab.nrho)]
    off = 0
    for q, s in enumerate(wl.systems):
        oq = ora.eam_vjp(s.x, s.lo, s.hi, s.periodic, tab, 1.0, gF[off:off + s.n])
        for a, b in zip(o, oq):
            a += b
        off += s.n
    assert_mixed_grad(g, o, rng)
