"""Differentiable EAM energies and forces: a torch.autograd.Function over the
library's force loop (mdk_compute) and its adjoint kernels (mdk_eam_vjp).

    E, F = eam_energy_forces(context, phi, rho, F_knots, rc, rho_max)

gives the per-replica potential energies E [n_rep] and the forces F [N, 3]
(caller's atom order) at the context's current positions as functions of the
three knot tensors; ``backward`` asks the library for the gradient of
sum_r gE_r E_r + sum_i gF_i . F_i with respect to the knots.  Pair distances
are recomputed on the GPU (none are stored).  This module only marshals
arguments and orders streams; all arithmetic runs in libmdk.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mdk
from .workloads import EAMTables


def _knots(t: torch.Tensor) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


class EAMForceField(torch.autograd.Function):
    @staticmethod
    def forward(fctx, phi, rho, F, context, rc, rho_max):
        dev = context.device
        cur = torch.cuda.current_stream(dev)
        context.set_potential_eam(EAMTables(rc=float(rc), phi=_knots(phi), rho=_knots(rho),
                                            rho_max=float(rho_max), F=_knots(F)))
        n = context.natoms()
        E = torch.empty(context.n_rep, dtype=torch.float64, device=dev)
        Fo = torch.empty((n, 3), dtype=torch.float64, device=dev)
        W = torch.empty((context.n_rep, 6), dtype=torch.float64, device=dev)
        context.stream.wait_stream(cur)
        try:
            context.compute_device(E, Fo, W)
        except mdk.MDKError as e:
            if e.code not in (mdk.MDK_ERR_WORKSPACE, mdk.MDK_ERR_NEIGH_OVERFLOW):
                raise
            context.alloc_workspace()  # new table sizes or list capacity
            context.compute_device(E, Fo, W)
        cur.wait_stream(context.stream)
        fctx.context = context
        fctx.version = context.version
        fctx.sizes = context._eam_sizes
        fctx.devices = (phi.device, rho.device, F.device)
        return E, Fo

    @staticmethod
    def backward(fctx, gE, gF):
        context = fctx.context
        if context.version != fctx.version:
            raise RuntimeError("the context's positions or tables changed between the "
                               "forward and the backward pass")
        nr, nrho = fctx.sizes
        dev = context.device
        cur = torch.cuda.current_stream(dev)
        gE = None if gE is None else gE.detach().to(dev, torch.float64).contiguous()
        gF = None if gF is None else gF.detach().to(dev, torch.float64).contiguous()
        out = torch.empty(2 * nr + nrho, dtype=torch.float64, device=dev)
        context.stream.wait_stream(cur)
        context.eam_vjp_device(gE, gF, out)
        cur.wait_stream(context.stream)
        d_phi, d_rho, d_F = out[:nr], out[nr:2 * nr], out[2 * nr:]
        return (d_phi.to(fctx.devices[0]), d_rho.to(fctx.devices[1]), d_F.to(fctx.devices[2]),
                None, None, None)


def eam_energy_forces(context, phi, rho, F, rc, rho_max):
    """(E [n_rep], F [N, 3]) of the context's current positions; differentiable
    with respect to the knot tensors phi [nr], rho [nr] and F [nrho]."""
    return EAMForceField.apply(phi, rho, F, context, rc, rho_max)
