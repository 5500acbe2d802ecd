"""Differentiable Richardson-Lucy deconvolution (torch.autograd.Function).

``RLDeconvolve.apply(d, sigma_xy, sigma_z, amp, n_iter, eps, ckpt_every)`` runs
``n_iter`` Richardson-Lucy iterations (the paper's Section 4 step: blur by the
PSF, quotient of the image by the blur, correlation of the quotient with the
PSF, product with the estimate) on every volume of ``d`` ([B, Z, Y, X] or
[Z, Y, X] float32 CUDA) with the normalised anisotropic Gaussian PSF
``amp * g / sum(g)`` of the given parameters, and returns the estimates.  Its
backward returns dL/dd and dL/d(sigma_xy, sigma_z, amp).

Every step runs in the library's kernels: the PSF (``cubic_psf_gaussian``), the
checkpointed forward (``cubic_rl_deconvolve_ckpt``), the reverse sweep
(``cubic_rl_backward``, which also accumulates the PSF gradient across the
batch) and the parameter reduction (``cubic_psf_gaussian_backward``).  torch
supplies memory and the stream.
"""
from __future__ import annotations

import math

import torch

from . import (cubic_psf_gaussian, cubic_psf_gaussian_backward, cubic_rl_backward, cubic_rl_deconvolve_ckpt,
               cubic_rl_plan, n_checkpoints)


def _as_float(x) -> float:
    return float(x.detach().item()) if isinstance(x, torch.Tensor) else float(x)


class RLDeconvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, sigma_xy, sigma_z, amp, n_iter: int, eps: float = 1e-6, ckpt_every=None):
        if d.dim() == 3:
            d = d.unsqueeze(0)
            ctx.squeeze = True
        else:
            ctx.squeeze = False
        if d.dim() != 4 or not d.is_cuda or d.dtype != torch.float32:
            raise ValueError("d must be a float32 CUDA tensor [B, Z, Y, X] or [Z, Y, X]")
        d = d.contiguous()
        n_iter = int(n_iter)
        c = int(ckpt_every) if ckpt_every else max(1, int(round(math.sqrt(n_iter))))
        sxy, sz, a = _as_float(sigma_xy), _as_float(sigma_z), _as_float(amp)
        shape = tuple(d.shape[1:])
        psf = torch.empty(shape, dtype=torch.float32, device=d.device)
        cubic_psf_gaussian(shape, sxy, sz, a, psf)
        plan = cubic_rl_plan(shape, psf)
        nck = n_checkpoints(n_iter, c)
        ckpts = torch.empty((d.shape[0], nck) + shape, dtype=torch.float32, device=d.device)
        out = torch.empty_like(d)
        for b in range(d.shape[0]):
            cubic_rl_deconvolve_ckpt(plan, d[b], n_iter, eps, c, ckpts[b], out[b])
        ctx.save_for_backward(d, ckpts)
        ctx.plan = plan
        ctx.cfg = (sxy, sz, a, n_iter, float(eps), c)
        ctx.param_like = tuple(p if isinstance(p, torch.Tensor) else None for p in (sigma_xy, sigma_z, amp))
        return out.squeeze(0) if ctx.squeeze else out

    @staticmethod
    def backward(ctx, grad_out):
        d, ckpts = ctx.saved_tensors
        sxy, sz, a, n_iter, eps, c = ctx.cfg
        g = grad_out.unsqueeze(0) if ctx.squeeze else grad_out
        g = g.contiguous().to(torch.float32)
        shape = tuple(d.shape[1:])
        want_d = ctx.needs_input_grad[0]
        want_p = any(ctx.needs_input_grad[1:4])
        grad_d = torch.empty_like(d) if want_d else None
        grad_psf = torch.empty(shape, dtype=torch.float32, device=d.device) if want_p else None
        for b in range(d.shape[0]):
            cubic_rl_backward(ctx.plan, d[b], n_iter, eps, c, ckpts[b], g[b],
                              grad_d[b] if want_d else None, grad_psf, accumulate_psf=b > 0)
        grads = [None, None, None]
        if want_p:
            gp = torch.empty(3, dtype=torch.float32, device=d.device)
            cubic_psf_gaussian_backward(shape, sxy, sz, a, grad_psf, gp)
            for i, like in enumerate(ctx.param_like):
                if like is not None:
                    grads[i] = gp[i].reshape(like.shape).to(like.dtype).to(like.device)
        if want_d and ctx.squeeze:
            grad_d = grad_d.squeeze(0)
        return grad_d, grads[0], grads[1], grads[2], None, None, None


def rl_deconvolve_differentiable(d, sigma_xy, sigma_z, amp, n_iter: int, eps: float = 1e-6, ckpt_every=None):
    return RLDeconvolve.apply(d, sigma_xy, sigma_z, amp, n_iter, eps, ckpt_every)
