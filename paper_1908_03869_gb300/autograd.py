"""torch.autograd glue over the C ABI.

``integrate_final(integrator, params, x0)`` returns X^K and, on backward,
calls ``sdeb_grad`` (the discrete adjoint with checkpointed recompute and
regenerated noise).  ``order_parameter(theta)`` is Eq. 7 through
``sdeb_order_param`` with its analytic gradient.  Both only marshal tensors;
the arithmetic runs in libsdeb.so.
"""
import ctypes

import torch

from . import SDEB_FP64, sdeb_order_param


class _IntegrateFinal(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, x0, integrator):
        integrator.set_params(params.detach().contiguous(), x0.detach().contiguous())
        integrator.integrate()
        ctx.integrator = integrator
        return integrator.final()

    @staticmethod
    def backward(ctx, grad_xK):
        dp, dx0 = ctx.integrator.grad(grad_xK.contiguous(), want_dx0=ctx.needs_input_grad[1])
        return dp, dx0, None


def integrate_final(integrator, params, x0):
    """X^K of every orbit, differentiable in params and x0.  The integrator's
    problem must have ckpt_every > 0 and be a Kuramoto model."""
    return _IntegrateFinal.apply(params, x0, integrator)


class _OrderParameter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta):
        theta = theta.detach().contiguous()
        orbits, n = theta.shape
        precision = SDEB_FP64 if theta.dtype == torch.float64 else 0
        r = torch.empty(orbits, dtype=theta.dtype, device=theta.device)
        dr = torch.empty_like(theta)
        sdeb_order_param(ctypes.c_void_p(theta.data_ptr()), orbits, n, precision, ctypes.c_void_p(r.data_ptr()),
                         ctypes.c_void_p(dr.data_ptr()), torch.cuda.current_stream().cuda_stream)
        ctx.save_for_backward(dr)
        return r

    @staticmethod
    def backward(ctx, grad_r):
        (dr,) = ctx.saved_tensors
        return grad_r.unsqueeze(1) * dr


def order_parameter(theta):
    """Eq. 7: r per orbit of phases theta [orbits][n] (device tensor)."""
    return _OrderParameter.apply(theta)
