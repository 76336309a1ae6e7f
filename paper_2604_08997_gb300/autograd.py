"""torch.autograd wrappers of the projector pair with a PSF-sigma gradient.

`SipoProject` is A p = P_mu K p; its backward is the hand-written
backprojection A^T g = K P_mu^T g, and dL/dsigma_a = < P_mu^T g, dK/dsigma_a p >
(P_mu^T g is recomputed by the library, the blurred volume K p is never
stored).  `SipoBackproject` is A^T y = K P_mu^T y with backward A g and
dL/dsigma_a = < P_mu^T y, dK/dsigma_a g >.  Both call only the C ABI.

The context's PSF radii are frozen at creation; `sigma` is written into the
context on every forward call, and the backward writes the forward's sigma
back before it runs (the context may have been used with other sigmas in
between).
"""
from __future__ import annotations

import torch

from . import _abi


def _sigma_list(sigma):
    if sigma is None:
        return None
    return [float(x) for x in sigma.detach().cpu().tolist()]


class SipoProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, sigma, handle):
        if sigma is not None:
            _abi.sipo_set_psf_sigma(handle, _sigma_list(sigma))
        p = p.contiguous()
        out = torch.empty(handle.sino_shape, dtype=p.dtype, device=p.device)
        _abi.sipo_project(handle, p, out)
        ctx.save_for_backward(p)
        ctx.handle = handle
        ctx.sigma_dtype = None if sigma is None else sigma.dtype
        ctx.sigma_vals = _sigma_list(sigma)
        return out

    @staticmethod
    def backward(ctx, g):
        (p,) = ctx.saved_tensors
        h = ctx.handle
        if ctx.sigma_vals is not None:
            _abi.sipo_set_psf_sigma(h, ctx.sigma_vals)
        g = g.contiguous()
        grad_p = grad_s = None
        if ctx.needs_input_grad[0]:
            grad_p = torch.empty(h.vol_shape, dtype=g.dtype, device=g.device)
            _abi.sipo_backproject(h, g, grad_p)
        if ctx.sigma_dtype is not None and ctx.needs_input_grad[1]:
            grad_s = torch.tensor(_abi.sipo_psf_grad(h, g, p), dtype=ctx.sigma_dtype)
        return grad_p, grad_s, None


class SipoBackproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, sigma, handle):
        if sigma is not None:
            _abi.sipo_set_psf_sigma(handle, _sigma_list(sigma))
        y = y.contiguous()
        out = torch.empty(handle.vol_shape, dtype=y.dtype, device=y.device)
        _abi.sipo_backproject(handle, y, out)
        ctx.save_for_backward(y)
        ctx.handle = handle
        ctx.sigma_dtype = None if sigma is None else sigma.dtype
        ctx.sigma_vals = _sigma_list(sigma)
        return out

    @staticmethod
    def backward(ctx, g):
        (y,) = ctx.saved_tensors
        h = ctx.handle
        if ctx.sigma_vals is not None:
            _abi.sipo_set_psf_sigma(h, ctx.sigma_vals)
        g = g.contiguous()
        grad_y = grad_s = None
        if ctx.needs_input_grad[0]:
            grad_y = torch.empty(h.sino_shape, dtype=g.dtype, device=g.device)
            _abi.sipo_project(h, g, grad_y)
        if ctx.sigma_dtype is not None and ctx.needs_input_grad[1]:
            grad_s = torch.tensor(_abi.sipo_psf_grad(h, y, g), dtype=ctx.sigma_dtype)
        return grad_y, grad_s, None


def project(handle, p, sigma=None):
    """A p with autograd (sigma: optional 3-vector tensor of PSF sigmas)."""
    return SipoProject.apply(p, sigma, handle)


def backproject(handle, y, sigma=None):
    """A^T y with autograd."""
    return SipoBackproject.apply(y, sigma, handle)
