"""torch.autograd.Function around the library's hand-written adjoint.

    J = final_field_energy(x0, v0, sim, n_steps, weights=(0, 0, 1))
    J.backward()          # x0.grad, v0.grad from pic_adjoint_backward

The forward pass loads (x0, v0) into the Simulation and runs n_steps steps
with checkpoints (pic_adjoint_forward); the backward pass is the reverse
sweep with segment recomputation (pic_adjoint_backward).  Both run in the
CUDA library; this module only moves tensors across the C ABI.
"""
from __future__ import annotations

import torch


class FinalFieldEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, sim, n_steps, weights, checkpoint_every):
        if x0.dtype != torch.float64 or v0.dtype != torch.float64:
            raise TypeError("x0 and v0 must be float64 (N, 3) tensors")
        sim.load(x0.detach().contiguous(), v0.detach().contiguous())
        J = sim.adjoint_forward(int(n_steps), tuple(weights), int(checkpoint_every))
        ctx.sim = sim
        ctx.device = x0.device
        return torch.tensor(J, dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(ctx, grad_J):
        gx, gv = ctx.sim.adjoint_backward(scale=float(grad_J), device=True)
        return gx.to(ctx.device), gv.to(ctx.device), None, None, None, None


def final_field_energy(x0, v0, sim, n_steps, weights=(1.0, 1.0, 1.0), checkpoint_every=20):
    """Weighted field energy sum_d w_d h^3 sum_g E_d^2 of the last step's field."""
    return FinalFieldEnergy.apply(x0, v0, sim, n_steps, weights, checkpoint_every)
