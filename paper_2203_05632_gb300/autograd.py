"""torch.autograd interface to the library's hand-written adjoint.

``mcmp2_energy(eps, C, engine, r, tau)`` returns the replay estimate
E = (1/n) sum_n I'_n of the MP2 energy for fixed samples (positions r
[n][m][2][3], times tau [n][n_tau]) as a differentiable function of the
orbital energies eps (float64 [n_orb]) and the spinor coefficients C
(complex128 [4 n_L][n_orb]).  The forward pass runs the library's replay
(mcmp2_eval_fixed); the backward pass runs its adjoint (mcmp2_backward) under
the same samples (common random numbers), with lambda, eps_HOMO and eps_LUMO
held at the values of the system the engine was created with.  Complex
gradients follow torch's convention dE/dRe C + i dE/dIm C.

``engine`` is a ``paper_2203_05632_gb300.Context`` in the FP64 form.
"""
from __future__ import annotations

import numpy as np
import torch


class MCMP2Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, C, engine, r, tau):
        eps_np = eps.detach().cpu().numpy().astype(np.float64)
        C_np = C.detach().cpu().numpy().astype(np.complex128)
        engine.load(eps=eps_np, C=C_np)
        r_np = np.ascontiguousarray(r, dtype=np.float64)
        tau_np = np.ascontiguousarray(tau, dtype=np.float64)
        e = float(engine.eval_fixed(r_np, tau_np).mean())
        ctx.engine = engine
        ctx.samples = (r_np, tau_np)
        ctx.params = (eps_np, C_np)
        ctx.devices = (eps.device, C.device)
        return torch.tensor(e, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_e):
        engine = ctx.engine
        eps_np, C_np = ctx.params
        engine.load(eps=eps_np, C=C_np)
        _, d_eps, d_C = engine.backward(*ctx.samples)
        g = grad_e.detach().to("cpu", torch.float64)
        d_eps_t = (g * torch.from_numpy(d_eps)).to(ctx.devices[0])
        d_C_t = (g.to(torch.complex128) * torch.from_numpy(d_C)).to(ctx.devices[1])
        return d_eps_t, d_C_t, None, None, None


def mcmp2_energy(eps, C, engine, r, tau):
    return MCMP2Energy.apply(eps, C, engine, r, tau)
