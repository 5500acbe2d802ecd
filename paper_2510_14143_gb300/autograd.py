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
supplies memory and the streams: the volumes of a batch spread over up to
``MAX_STREAMS`` streams with a plan each, and the few parameter gradients of
the streams are added at the end.
"""
from __future__ import annotations

import math

import torch

from . import (cubic_psf_gaussian, cubic_psf_gaussian_backward, cubic_rl_backward, cubic_rl_deconvolve_ckpt,
               cubic_rl_plan, cubic_rl_plan_update_psf, n_checkpoints)


def _as_float(x) -> float:
    return float(x.detach().item()) if isinstance(x, torch.Tensor) else float(x)


#: volumes of a batch run on up to this many CUDA streams, one plan (and workspace) each, so
#: that the passes of small volumes overlap instead of leaving most of the GPU idle
MAX_STREAMS = 4
_side = {}


def _streams(n: int, device):
    key = (torch.device(device).index, n)
    if key not in _side:
        _side[key] = [torch.cuda.Stream(device=device) for _ in range(n)]
    return _side[key]


# Plans by (device, shape), reused across calls: a forward takes free plans and loads its
# PSF into them (cubic_rl_plan_update_psf), the backward returns them.  New plans and
# their first backward allocate device memory, which synchronises the whole device.
_pool = {}
_POOL_CAP = 2 * MAX_STREAMS


def _take_plans(shape, device, n: int, psf):
    free = _pool.setdefault((torch.device(device).index, shape), [])
    plans = []
    for _ in range(n):
        if free:
            plan = free.pop()
            cubic_rl_plan_update_psf(plan, psf)
        else:
            plan = cubic_rl_plan(shape, psf)
        plans.append(plan)
    return plans


class _Lease:
    """Holds a call's plans; returns them to the pool when the autograd context that owns
    it is freed (after its last backward).  Work queued on them is ordered before any
    later use: the streams joined the current stream, on which the next PSF load runs."""

    def __init__(self, shape, device, plans):
        self.key = (torch.device(device).index, shape)
        self.plans = plans

    def __del__(self):
        try:
            free = _pool.setdefault(self.key, [])
            free.extend(self.plans[:max(0, _POOL_CAP - len(free))])
        except Exception:
            pass


def _fan_out(streams, tensors):
    """Side streams start after the current stream's work; the allocator keeps `tensors`."""
    main = torch.cuda.current_stream()
    for st in streams:
        st.wait_stream(main)
        for t in tensors:
            if t is not None:
                t.record_stream(st)


def _fan_in(streams):
    main = torch.cuda.current_stream()
    for st in streams:
        main.wait_stream(st)


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
        ns = min(d.shape[0], MAX_STREAMS)
        plans = _take_plans(shape, d.device, ns, psf)
        nck = n_checkpoints(n_iter, c)
        ckpts = torch.empty((d.shape[0], nck) + shape, dtype=torch.float32, device=d.device)
        out = torch.empty_like(d)
        streams = _streams(ns, d.device)
        _fan_out(streams, (d, ckpts, out))
        for b in range(d.shape[0]):
            with torch.cuda.stream(streams[b % ns]):
                cubic_rl_deconvolve_ckpt(plans[b % ns], d[b], n_iter, eps, c, ckpts[b], out[b])
        _fan_in(streams)
        ctx.save_for_backward(d, ckpts)
        ctx.plans = plans
        ctx.lease = _Lease(shape, d.device, plans)
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
        ns = len(ctx.plans)
        # one PSF-gradient volume per stream (the parameter gradient is linear in it)
        grad_psf = [torch.empty(shape, dtype=torch.float32, device=d.device) for _ in range(ns)] if want_p else None
        streams = _streams(ns, d.device)
        _fan_out(streams, (d, ckpts, g, grad_d) + tuple(grad_psf or ()))
        for b in range(d.shape[0]):
            i = b % ns
            with torch.cuda.stream(streams[i]):
                cubic_rl_backward(ctx.plans[i], d[b], n_iter, eps, c, ckpts[b], g[b],
                                  grad_d[b] if want_d else None, grad_psf[i] if want_p else None,
                                  accumulate_psf=b >= ns)
        _fan_in(streams)
        grads = [None, None, None]
        if want_p:
            parts = torch.empty((ns, 3), dtype=torch.float32, device=d.device)
            for i in range(ns):
                cubic_psf_gaussian_backward(shape, sxy, sz, a, grad_psf[i], parts[i])
            gp = parts.sum(0)
            for i, like in enumerate(ctx.param_like):
                if like is not None:
                    grads[i] = gp[i].reshape(like.shape).to(like.dtype).to(like.device)
        if want_d and ctx.squeeze:
            grad_d = grad_d.squeeze(0)
        return grad_d, grads[0], grads[1], grads[2], None, None, None


def rl_deconvolve_differentiable(d, sigma_xy, sigma_z, amp, n_iter: int, eps: float = 1e-6, ckpt_every=None):
    return RLDeconvolve.apply(d, sigma_xy, sigma_z, amp, n_iter, eps, ckpt_every)
