"""Differentiable LOD runs: ``torch.autograd.Function`` over libbiofvm's forward and adjoint.

Forward: ``n_steps`` graph-launched steps, keeping the field every ``checkpoint_every`` steps.
Backward: for each checkpoint segment, last first, the segment is recomputed from its
checkpoint with ``biofvm_step_save`` (which keeps the states each adjoint step needs) and then
walked in reverse with ``biofvm_adjoint_step``.  Memory: one field per checkpoint plus four
fields per step of one segment.  Gradients: the initial field, every agent's secretion rate,
and the per-substrate D and lambda (accumulated in FP64 on the device, reproducibly).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class LODSteps(torch.autograd.Function):
    """out = LOD^n(rho0; secretion, D, lambda) with the agents' positions, targets, uptake
    rates and weights held fixed (``agents``: dict of numpy arrays voxel, target, uptake,
    weight)."""

    @staticmethod
    def forward(ctx, rho0, secretion, D, lam, sim, agents, n_steps, checkpoint_every):
        sim.set_params(D.detach().double().cpu().numpy(), lam.detach().double().cpu().numpy())
        sim.set_sources(agents["voxel"], secretion.detach().double().cpu().numpy(),
                        agents.get("target"), agents.get("uptake"), agents.get("weight"))
        sim.set_density(rho0.detach().reshape(sim.shape))
        ckpts = []
        for k in range(n_steps):
            if k % checkpoint_every == 0:
                ckpts.append(sim.field_tensor().clone())
            sim.step(1)
        out = sim.field_tensor().clone()
        ctx.sim, ctx.ckpts = sim, ckpts
        ctx.n_steps, ctx.K = n_steps, checkpoint_every
        ctx.meta = (rho0.shape, rho0.dtype, rho0.device, secretion.shape, secretion.dtype,
                    secretion.device, D.dtype, D.device, lam.dtype, lam.device)
        return out

    @staticmethod
    def backward(ctx, gout):
        sim = ctx.sim
        fd = sim._field_dtype()
        ns = sim.shape[3]
        (r_shape, r_dtype, r_dev, s_shape, s_dtype, s_dev, d_dtype, d_dev, l_dtype,
         l_dev) = ctx.meta
        dev = gout.device
        g = gout.detach().to(dtype=fd).contiguous().clone()
        dD = torch.zeros(ns, dtype=torch.float64, device=dev)
        dl = torch.zeros(ns, dtype=torch.float64, device=dev)
        dsec = torch.zeros(int(np.prod(s_shape)), dtype=torch.float64, device=dev)
        nel = sim.n_elem
        for seg in range(len(ctx.ckpts) - 1, -1, -1):
            k0 = seg * ctx.K
            k1 = min(ctx.n_steps, k0 + ctx.K)
            sim.set_density(ctx.ckpts[seg])
            saved = torch.empty((k1 - k0, 4 * nel), dtype=fd, device=dev)
            for j in range(k1 - k0):
                sim.step_save(saved[j])
            for j in range(k1 - k0 - 1, -1, -1):
                sim.adjoint_step(g, g, dD, dl, dsec, saved[j])
        sim.sync()
        return (g.reshape(r_shape).to(dtype=r_dtype, device=r_dev),
                dsec.reshape(s_shape).to(dtype=s_dtype, device=s_dev),
                dD.to(dtype=d_dtype, device=d_dev), dl.to(dtype=l_dtype, device=l_dev),
                None, None, None, None)


def lod_steps(rho0, secretion, D, lam, sim, agents, n_steps, checkpoint_every=20):
    """Differentiable ``n_steps`` LOD steps on the GPU (see LODSteps)."""
    return LODSteps.apply(rho0, secretion, D, lam, sim, agents, n_steps, checkpoint_every)
