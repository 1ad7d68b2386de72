"""torch.autograd.Function around the adjoint entry point ddrw_force.

``Exponents.apply(omega, m2, ctx, nhit, seed, hit_offset)`` returns the exponents
e_j = eta_j^dag (Mh^dag Mh - 1) eta_j of the configuration loaded in ``ctx``.  ``omega``
([V, 4, 8] float64, requires_grad) are tangent coordinates of the links at that configuration,
U_mu(x) -> exp(i sum_a omega[x, mu, a] lambda_a / 2) U_mu(x); the function is evaluated at
omega = 0 (the loaded links) and its backward pass returns d(sum_j g_j e_j)/d omega from one call of
ddrw_force with weights g_j, which recomputes the solves instead of storing Krylov iterates.
``m2`` (0-dim float64 tensor, requires_grad) is the target mass; its gradient is sum_j g_j de_j/dm2.
All arithmetic runs in the CUDA library; this module only marshals tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class Exponents(torch.autograd.Function):
    @staticmethod
    def forward(fctx, omega, m2, ctx, nhit, seed, hit_offset):
        if bool((omega != 0).any()):
            raise ValueError("Exponents is evaluated at the loaded links: omega must be zero")
        ctx.set_params(ctx._csw, ctx._m1, float(m2))
        e, _, _, _ = ctx.estimate(nhit, seed=seed, hit_offset=hit_offset)
        fctx.ddrw = (ctx, nhit, seed, hit_offset)
        fctx.omega_shape = omega.shape
        fctx.omega_device = omega.device
        return torch.as_tensor(e, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(fctx, grad_e):
        ctx, nhit, seed, hit_offset = fctx.ddrw
        w = grad_e.detach().to("cpu", torch.float64).contiguous().numpy()
        dU = torch.zeros(fctx.omega_shape, dtype=torch.float64, device=fctx.omega_device)
        _, dm2, _ = ctx.force(nhit, seed=seed, hit_offset=hit_offset, weights=w, dU=dU)
        g_m2 = torch.tensor(float(np.dot(w, dm2)), dtype=torch.float64, device=fctx.omega_device)
        return dU, g_m2, None, None, None, None


def exponents(ctx: "binding.Context", omega, m2, nhit, seed=2, hit_offset=0):
    """Differentiable exponents at the loaded configuration (see Exponents)."""
    return Exponents.apply(omega, m2, ctx, nhit, seed, hit_offset)
