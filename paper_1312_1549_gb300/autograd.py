"""torch.autograd.Function over the OMM solve: E(H, S) with dE/dH and dE/dS.

The forward runs omm_create + omm_solve; the backward runs omm_backward, whose
CUDA kernels form dE/dH = D = 2 C (2I - S_W) C^T and
dE/dS = -EDM = -(2 C H~_W C^T + eta D) at the converged minimum (exact there
by the envelope theorem on the OMM functional, Eq. 8 of the paper, with
H~ = H - eta S). The upstream scalar gradient is applied by the chain rule.

The two m x m gradients are formed once, on the first backward call, and kept
on the autograd context, so a second backward through the same graph
(retain_graph=True) reuses them; the solver context and its device buffers are
released as soon as they exist, or with the graph if no backward ever runs.
"""
from __future__ import annotations

import torch

from .solver import OMMSolver


class OMMEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, S, T, C0, n, eta, tau, precision, tol_grad):
        solver = OMMSolver(H.detach().contiguous(), S.detach().contiguous(), T.detach().contiguous(),
                           int(n), float(eta), float(tau), precision=precision, tol_grad=tol_grad)
        C, E, _, info = solver.solve(C0.detach().contiguous())
        ctx.solver = solver
        ctx.device = H.device
        ctx.mark_non_differentiable(C)
        return torch.tensor(E, dtype=torch.float64, device=H.device), C

    @staticmethod
    def backward(ctx, gE, gC):
        if getattr(ctx, "grads", None) is None:
            solver = ctx.solver
            if solver is None:
                raise RuntimeError("OMMEnergy.backward: the solver of this forward has been released")
            ctx.grads = solver.backward(device=ctx.device)
            solver.close()
            ctx.solver = None
        dH, dS = ctx.grads
        gH = dH * gE if ctx.needs_input_grad[0] else None
        gS = dS * gE if ctx.needs_input_grad[1] else None
        return gH, gS, None, None, None, None, None, None, None


def omm_energy(H, S, T, C0, n, eta, tau, precision="fp64", tol_grad=1e-9):
    """Band energy E = 2 sum_{i<=n} eps_i of H x = eps S x by the OMM, differentiable in H and S.

    Returns (E, C): E a 0-dim float64 tensor, C the converged n x m coefficients.
    """
    return OMMEnergy.apply(H, S, T, C0, n, eta, tau, precision, tol_grad)
