"""Differentiable forward map calF[m] whose backward is the adjoint (RTM) kernel.

For J[m] = 1/2 ||d - calF[m]||^2 (Sec. 1.1) the gradient is
dJ/dm = -F*[m] (d - calF[m]) = F*[m] (calF[m] - d): the backward pass of
``ForwardMap`` maps the incoming data-space gradient g_d to F*[m] g_d with the
Born operator linearised at the current model m -- one incident sweep from
sqrt(nt)-spaced checkpoints, the segment-wise recomputation and the adjoint
sweep with the imaging condition, all in the CUDA library (probe_gradient).
The sponge keeps the values of the background model given at set-up, so the
derivative is with respect to the interior model only.
"""
from __future__ import annotations

import torch

from .binding import Probe


class ForwardMap(torch.autograd.Function):
    """d = calF[m]: receiver traces [ns, nt, nr] of m u_tt - Lap u = f_s."""

    @staticmethod
    def forward(ctx, m: torch.Tensor, probe: Probe) -> torch.Tensor:
        m = m.detach().contiguous()
        ctx.probe = probe
        ctx.save_for_backward(m)
        return probe.forward_nonlinear(m)

    @staticmethod
    def backward(ctx, grad_d: torch.Tensor):
        (m,) = ctx.saved_tensors
        g = ctx.probe.gradient(m, grad_d.detach().contiguous().to(torch.float32))
        return g, None


def forward_map(m: torch.Tensor, probe: Probe) -> torch.Tensor:
    """Apply calF with autograd support (m: interior model, CUDA float32)."""
    return ForwardMap.apply(m, probe)


def misfit(m: torch.Tensor, d_obs: torch.Tensor, probe: Probe) -> torch.Tensor:
    """J[m] = 1/2 ||d_obs - calF[m]||^2, accumulated in float64."""
    r = forward_map(m, probe).double() - d_obs.double()
    return 0.5 * torch.sum(r * r)
