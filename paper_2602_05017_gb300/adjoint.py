"""Differentiable LOD runs: ``torch.autograd.Function`` over libbiofvm's forward and adjoint.

Forward: ``n_steps`` graph-launched steps, keeping the field every ``checkpoint_every`` steps.
Backward: for each checkpoint segment, last first, the segment is recomputed from its
checkpoint with ``biofvm_step_save`` (which keeps the states each adjoint step needs) and then
walked in reverse with ``biofvm_adjoint_step_rates``.  Memory: one field per checkpoint plus
four fields per step of one segment.  Gradients: the initial field, every agent's secretion
and uptake rates, and the per-substrate D and lambda (accumulated in FP64 on the device,
reproducibly).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class LODSteps(torch.autograd.Function):
    """out = LOD^n(rho0; secretion, uptake, D, lambda) with the agents' positions, targets and
    weights held fixed (``agents``: dict of numpy arrays voxel, target, weight)."""

    @staticmethod
    def forward(ctx, rho0, secretion, uptake, D, lam, sim, agents, n_steps, checkpoint_every):
        sim.set_params(D.detach().double().cpu().numpy(), lam.detach().double().cpu().numpy())
        sim.set_sources(agents["voxel"], secretion.detach().double().cpu().numpy(),
                        agents.get("target"), uptake.detach().double().cpu().numpy(),
                        agents.get("weight"))
        sim.set_density(rho0.detach().reshape(sim.shape))
        ckpts = []
        for k in range(n_steps):
            if k % checkpoint_every == 0:
                ckpts.append(sim.field_tensor().clone())
            sim.step(1)
        out = sim.field_tensor().clone()
        ctx.sim, ctx.ckpts = sim, ckpts
        ctx.n_steps, ctx.K = n_steps, checkpoint_every
        ctx.meta = [(t.shape, t.dtype, t.device) for t in (rho0, secretion, uptake, D, lam)]
        return out

    @staticmethod
    def backward(ctx, gout):
        sim = ctx.sim
        fd = sim._field_dtype()
        ns = sim.shape[3]
        r_meta, s_meta, u_meta, d_meta, l_meta = ctx.meta
        dev = gout.device
        g = gout.detach().to(dtype=fd).contiguous().clone()
        dD = torch.zeros(ns, dtype=torch.float64, device=dev)
        dl = torch.zeros(ns, dtype=torch.float64, device=dev)
        dsec = torch.zeros(int(np.prod(s_meta[0])), dtype=torch.float64, device=dev)
        dupt = torch.zeros(int(np.prod(u_meta[0])), dtype=torch.float64, device=dev)
        nel = sim.n_elem
        for seg in range(len(ctx.ckpts) - 1, -1, -1):
            k0 = seg * ctx.K
            k1 = min(ctx.n_steps, k0 + ctx.K)
            sim.set_density(ctx.ckpts[seg])
            saved = torch.empty((k1 - k0, 4 * nel), dtype=fd, device=dev)
            for j in range(k1 - k0):
                sim.step_save(saved[j])
            for j in range(k1 - k0 - 1, -1, -1):
                sim.adjoint_step(g, g, dD, dl, dsec, saved[j], dupt=dupt)
        sim.sync()

        def back(t, meta):
            return t.reshape(meta[0]).to(dtype=meta[1], device=meta[2])
        return (back(g, r_meta), back(dsec, s_meta), back(dupt, u_meta), back(dD, d_meta),
                back(dl, l_meta), None, None, None, None)


def lod_steps(rho0, secretion, D, lam, sim, agents, n_steps, checkpoint_every=20, uptake=None):
    """Differentiable ``n_steps`` LOD steps on the GPU (see LODSteps).  ``uptake``: a tensor of
    the agents' uptake rates [n_agents, n_sub] to differentiate through, else
    ``agents["uptake"]`` (or zero) held fixed."""
    if uptake is None:
        u = agents.get("uptake")
        uptake = torch.as_tensor(np.zeros(tuple(secretion.shape)) if u is None else
                                 np.asarray(u, dtype=np.float64), device=secretion.device)
    return LODSteps.apply(rho0, secretion, uptake, D, lam, sim, agents, n_steps,
                          checkpoint_every)
