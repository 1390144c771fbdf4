"""torch.autograd interface to the library's adjoint of the coupled LB + chain step.

``chain_displacement(x0, zeta, ...)`` returns O = sum_b |x_b(T) - x_b(0)|^2 after T coupled
steps started from bead positions x0 (fluid at rest) with friction zeta; its backward pass
gives dO/dx0 and dO/dzeta from the CUDA adjoint (noise held fixed, checkpoints every K
steps).  The forward and the adjoint run in the library; this module only marshals tensors.
When neither input needs a gradient, the forward runs the T steps alone (no adjoint).
"""
from __future__ import annotations

import numpy as np
import torch

from . import lb


class ChainDisplacement(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, zeta, params: dict, T: int, K: int):
        p = dict(params)
        N = x0.shape[0]
        X0 = x0.detach().cpu().numpy().astype(np.float64)
        sim = lb.Simulation(L=p["L"], rho=p.get("rho", 1.0), eta=p.get("eta", 3.0), eta_b=p.get("eta_b", 3.0),
                            kT=p.get("kT", 1.0), h=p.get("h", 0.01), a=p.get("a", 1.0), seed=p.get("seed", 7),
                            precision=p.get("precision", lb.LB_FP32))
        try:
            sim.add_chain(N, m=p.get("m", 1.0), zeta=float(zeta), k_fene=p.get("k_fene", 30.0), R0=p.get("R0", 1.5),
                          eps=p.get("eps", 1.0), sigma=p.get("sigma", 1.0), x0=X0)
            if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
                sim._bind()
                O, gx, gz = lb.lb_adjoint_displacement(sim.ctx, T, K, N)
                ctx.save_for_backward(torch.as_tensor(gx, dtype=x0.dtype, device=x0.device),
                                      torch.as_tensor(gz, dtype=zeta.dtype, device=zeta.device))
            else:
                sim.step(T)
                x, _ = sim.beads()
                O = float(((x - X0) ** 2).sum())
        finally:
            sim.close()
        return torch.as_tensor(O, dtype=x0.dtype, device=x0.device)

    @staticmethod
    def backward(ctx, gO):
        gx, gz = ctx.saved_tensors
        return gO * gx, gO * gz, None, None, None


def chain_displacement(x0: torch.Tensor, zeta: torch.Tensor, params: dict, T: int = 100, K: int = 10):
    return ChainDisplacement.apply(x0, zeta, params, T, K)
