"""Differentiable ETD2RK-DS time integration for PyTorch.

``solve(u0, kappa, rx_params, ...)`` advances u0 by n_steps and is
differentiable with respect to u0, the per-component diffusivities and the
reaction parameters. The forward pass keeps a checkpoint of the state every
``checkpoint_every`` steps; the backward pass runs the library's adjoint step
(etd_step_adjoint) segment by segment, newest first, each segment recomputing
its own forward states on the device. Argument handling only: all arithmetic
runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import etd


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, kappa, rx_params, cfg):
        d, n, q, dt, pade, precision, reaction, n_steps, every = cfg
        kap = [float(k) for k in kappa.detach().cpu()]
        rp = [float(v) for v in rx_params.detach().cpu()]
        plan = etd.Plan(d, n, kap[0], q, dt, pade=pade, precision=precision, reaction=reaction, rx_params=rp,
                        n_comp=len(kap), kappa_comp=kap)
        u = u0.detach().clone().contiguous()
        ckpts, done = [], 0
        while done < n_steps:
            seg = min(every, n_steps - done)
            ckpts.append((u.clone(), seg))
            plan.step(u, seg)
            done += seg
        plan.sync()
        ctx.plan, ctx.ckpts = plan, ckpts
        ctx.kappa_shape, ctx.rx_shape = kappa.shape, rx_params.shape
        ctx.kappa_dtype, ctx.rx_dtype = kappa.dtype, rx_params.dtype
        return u

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        lam = grad_out.detach().to(plan.dtype).contiguous().clone()
        gk = [0.0, 0.0]
        gr = [0.0] * 4
        for ck, seg in reversed(ctx.ckpts):
            k, r = plan.adjoint(ck, lam, seg)
            gk = [a + b for a, b in zip(gk, k)]
            gr = [a + b for a, b in zip(gr, r)]
        ncomp = ctx.kappa_shape[0]
        g_kappa = torch.tensor(gk[:ncomp], dtype=ctx.kappa_dtype)
        g_rx = torch.tensor(gr[:ctx.rx_shape[0]], dtype=ctx.rx_dtype)
        plan.close()
        return lam, g_kappa, g_rx, None


def solve(u0, kappa, rx_params, *, d, n, q, dt, n_steps, pade=2, precision="fp64split", reaction="fhn",
          checkpoint_every=20):
    """u(n_steps * dt) from u0 (CUDA tensor, shape (n_comp, n, ..)); kappa a CPU
    tensor of per-component diffusivities, rx_params a CPU tensor of reaction
    parameters (both may require grad)."""
    cfg = (d, n, q, dt, pade, precision, reaction, n_steps, checkpoint_every)
    return _Solve.apply(u0, kappa, rx_params, cfg)
