"""IPSA as differentiation: raw VUP moments as a differentiable function of
each density's location and width (Sec. 5.2 sensitivity of output statistics
to input measurement uncertainty).

``VUPMoments.apply(mu, sigma, grid, kind, lo, hi, precision)`` returns the raw
moments M[k, j] = sum_i W[k, i] y_i^j.  Its backward pass calls the library's
adjoint kernels (``vup_ipsa_sensitivity`` with the incoming gradient as the
vector-Jacobian seed), which recompute W rather than storing it.  Only
argument marshalling happens here.
"""
from __future__ import annotations

import torch

from . import vup


class VUPMoments(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, sigma, grid, kind, lo, hi, precision="fp32"):
        dev = dict(kind=kind, mu=mu.detach().contiguous(), sigma=sigma.detach().contiguous(), lo=lo, hi=hi)
        raw, _, _ = grid.propagate(dev, precision, moments=True, central=False, hist=False)
        ctx.grid, ctx.precision = grid, precision
        ctx.save_for_backward(dev["mu"], dev["sigma"], kind, lo, hi)
        return raw

    @staticmethod
    def backward(ctx, grad_raw):
        mu, sigma, kind, lo, hi = ctx.saved_tensors
        dev = dict(kind=kind, mu=mu, sigma=sigma, lo=lo, hi=hi)
        g = grad_raw.detach().to(torch.float64).contiguous()
        dmu, dsg = ctx.grid.ipsa(dev, ctx.precision, grad=g)
        return dmu.to(mu.dtype), dsg.to(sigma.dtype), None, None, None, None, None


def vup_moments(grid, dens_dev, precision="fp32"):
    """Differentiable raw moments; ``dens_dev['mu']`` / ``['sigma']`` may require grad."""
    return VUPMoments.apply(dens_dev["mu"], dens_dev["sigma"], grid, dens_dev["kind"], dens_dev["lo"],
                            dens_dev["hi"], precision)
