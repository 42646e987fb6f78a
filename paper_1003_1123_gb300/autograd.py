"""torch.autograd wrapper of the reverse-time adjoint (ld_backward).

``langevin_energy(system, n_steps, K_per, gamma, kT)`` returns the
trajectory-averaged total energy L = (1/S) sum_t E(t) of a run of the system
under the fixed noise of its generator, as a differentiable function of the
per-oscillator spring constants and of gamma and kT.  The caller's system is
left untouched: the forward pass runs on a copy (rng_clone + copies of x, v),
the backward pass on a second copy of the same starting state, so the noise
of both passes is the same bit for bit.  Both passes run in libgbrng.so.
"""
from __future__ import annotations

import torch

from . import gbrng as G


def _copy_system(system: "G.LdSystem", K_per, gamma: float, kT: float) -> "G.LdSystem":
    return G.LdSystem(G.rng_clone(system.rng), system.x.clone(), system.v.clone(), K=system.K,
                      m=system.m, gamma=gamma, kT=kT, dt=system.dt, K_per=K_per)


class LangevinEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, K_per, gamma, kT, system, n_steps, ckpt_every):
        Kp = K_per.detach().contiguous()
        g, t = float(gamma), float(kT)
        run = _copy_system(system, Kp, g, t)
        st = G.ld_run(run, n_steps)
        ctx.system, ctx.n_steps, ctx.ckpt = system, n_steps, ckpt_every
        ctx.save_for_backward(Kp)
        ctx.gamma, ctx.kT = g, t
        ctx.start = (G.rng_clone(system.rng), system.x.clone(), system.v.clone())
        return torch.tensor(st["energy_time_avg"], dtype=torch.float64, device=K_per.device)

    @staticmethod
    def backward(ctx, grad_out):
        (Kp,) = ctx.saved_tensors
        rng, x, v = ctx.start
        s = ctx.system
        sysb = G.LdSystem(rng, x, v, K=s.K, m=s.m, gamma=ctx.gamma, kT=ctx.kT, dt=s.dt, K_per=Kp)
        r = G.ld_backward(sysb, ctx.n_steps, ctx.ckpt)
        go = grad_out.to(torch.float64)
        dK = (r["dK"].to(torch.float64) * go).to(Kp.dtype)
        dg = torch.tensor(r["dgamma"], dtype=torch.float64, device=Kp.device) * go
        dT = torch.tensor(r["dkT"], dtype=torch.float64, device=Kp.device) * go
        return dK, dg, dT, None, None, None


def langevin_energy(system: "G.LdSystem", n_steps: int, K_per: torch.Tensor,
                    gamma: torch.Tensor, kT: torch.Tensor, ckpt_every: int = 100):
    """Differentiable trajectory-averaged energy (see module docstring)."""
    return LangevinEnergy.apply(K_per, gamma, kT, system, n_steps, ckpt_every)
