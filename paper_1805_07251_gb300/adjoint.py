"""Differentiable rollouts: ``LBRollout`` is a ``torch.autograd.Function`` whose forward
advances a run on the GPU (checkpointing every ``ckpt_every`` steps; ``spec["precision"]``
"fp64" by default, or "fp32_mixed" / "fp32_dfmu" for FP32 storage with an FP32 adjoint)
and whose backward calls the library's hand-written adjoint of the fused timestep
(``lb_rollout_backward``).  Gradients flow to a_12 (the shared value of the symmetric
pair a_12 = a_21), to kappa (one value for every pair, as in the workloads), to b and to
the initial densities.  The torch tensors are plumbing: every step of the rollout and of
its adjoint runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Simulation, capi


class LBRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a12, kappa, b, rho0, spec):
        """a12, kappa: 0-d tensors; b: [N]; rho0: [N, ny, nx] (float64); spec: dict with
        lattice, ncomp, tau, kT, gamma_mu, a (N x N, a12 overridden), lam, steps, ckpt_every
        and optional device.  Returns the densities after ``steps`` timesteps."""
        N = int(spec["ncomp"])
        a = np.array(spec["a"], dtype=np.float64).reshape(N, N).copy()
        a[0, 1] = a[1, 0] = float(a12)
        kap = np.full((N, N), float(kappa))
        bb = b.detach().cpu().numpy().astype(np.float64)
        r0 = rho0.detach().cpu().numpy().astype(np.float64)
        sim = Simulation(lattice=spec["lattice"], nx=r0.shape[2], ny=r0.shape[1], ncomp=N, tau=spec["tau"],
                         kT=spec["kT"], gamma_mu=spec["gamma_mu"], a=a, kappa=kap, lam=spec["lam"], b=bb,
                         precision=spec.get("precision", "fp64"), device=spec.get("device", 0))
        sim.init(r0)
        capi.lb_rollout_forward(sim.ctx, spec["steps"], spec.get("ckpt_every", 100))
        rho_T, _ = sim.moments()
        ctx.sim = sim
        ctx.N = N
        ctx.device = rho0.device
        return torch.from_numpy(rho_T).to(rho0.device)

    @staticmethod
    def backward(ctx, grad_rho_T):
        N = ctx.N
        rb0, g = capi.lb_rollout_backward(ctx.sim.ctx, grad_rho_T.detach().cpu().numpy(), N)
        ctx.sim.close()
        ga = g[: N * N].reshape(N, N)
        gk = g[N * N: 2 * N * N]
        gb = g[2 * N * N:]
        dev = ctx.device
        return (torch.tensor(ga[0, 1] + ga[1, 0], dtype=torch.float64, device=dev),
                torch.tensor(gk.sum(), dtype=torch.float64, device=dev),
                torch.from_numpy(gb.copy()).to(dev), torch.from_numpy(rb0).to(dev), None)


def rollout(a12, kappa, b, rho0, spec):
    return LBRollout.apply(a12, kappa, b, rho0, spec)
