"""Differentiable unrolled PnP-MS2G (torch.autograd) on the library's kernels.

Sec. 2 of the paper notes that the sketched iterations can be unrolled and
trained end to end.  ``UnrolledStep`` is one iteration of Algorithm 1 as an
autograd Function of (y_{i-1}, x_{i-1}, lambda): its forward is
``pnp_unrolled_step_save`` (or ``pnp_unrolled_step``) and its backward
``pnp_unrolled_step_vjp_saved``, which starts from the iteration's stored
gradient step z (or ``pnp_unrolled_step_vjp``, which recomputes it from the
saved input y_{i-1}).  So an unrolled run keeps one image per iteration
(per-iteration checkpointing) and every numerical step, forward and backward,
runs in the CUDA kernels.
The data b is a constant of the unrolled map.
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import _native


class Project(torch.autograd.Function):
    """A_s^{(p)} v (Eq. 1, Eq. 4) as a differentiable operation on the level-s
    image v [batch, n/s, n/s]: the backward pass is the matched backprojector
    A_s^{(p)T} (pnp_backproject), so autograd gradients of any loss of A v are
    exact for the discrete operator."""

    @staticmethod
    def forward(ctx, img, plan, factor, subset, n_subsets):
        g = plan.g
        sino = torch.empty(g.batch, _native.subset_views(g, subset, n_subsets), g.n_det, device=img.device)
        plan.project(factor, img.contiguous(), sino, None, subset, n_subsets)
        ctx.args = (plan, factor, subset, n_subsets)
        return sino

    @staticmethod
    def backward(ctx, gsino):
        plan, factor, subset, n_subsets = ctx.args
        ns = plan.g.n // factor
        gimg = torch.empty(plan.g.batch, ns, ns, device=gsino.device)
        plan.backproject(factor, gsino.contiguous(), gimg, subset, n_subsets)
        return gimg, None, None, None, None


class Backproject(torch.autograd.Function):
    """A_s^{(p)T} r as a differentiable operation; its backward is A_s^{(p)}."""

    @staticmethod
    def forward(ctx, sino, plan, factor, subset, n_subsets):
        ns = plan.g.n // factor
        img = torch.empty(plan.g.batch, ns, ns, device=sino.device)
        plan.backproject(factor, sino.contiguous(), img, subset, n_subsets)
        ctx.args = (plan, factor, subset, n_subsets)
        return img

    @staticmethod
    def backward(ctx, gimg):
        plan, factor, subset, n_subsets = ctx.args
        g = plan.g
        gsino = torch.empty(g.batch, _native.subset_views(g, subset, n_subsets), g.n_det, device=gimg.device)
        plan.project(factor, gimg.contiguous(), gsino, None, subset, n_subsets)
        return gsino, None, None, None, None


def project(plan, img, factor: int = 1, subset: int = 0, n_subsets: int = 1):
    """Differentiable forward projection of the level-`factor` image."""
    return Project.apply(img, plan, factor, subset, n_subsets)


def backproject(plan, sino, factor: int = 1, subset: int = 0, n_subsets: int = 1):
    """Differentiable backprojection of a subset sinogram."""
    return Backproject.apply(sino, plan, factor, subset, n_subsets)


class UnrolledStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, xprev, lam, plan, b, factor, subset, n_subsets, eta, alpha, tv_iters, amom, vjp_ws,
                keep_z=True):
        g = plan.g
        xout = torch.empty_like(y)
        yout = torch.empty_like(y)
        if keep_z:      # keep the gradient step z too: the backward then skips one projector pair
            z = torch.empty_like(y)
            _native.unrolled_step_save(g, factor, subset, n_subsets, eta, alpha, float(lam), tv_iters, amom,
                                       y.contiguous(), xprev.contiguous(), b, xout, yout, z, plan.ws)
            ctx.save_for_backward(z)
        else:           # keep y only and recompute z in the backward
            _native.unrolled_step(g, factor, subset, n_subsets, eta, alpha, float(lam), tv_iters, amom,
                                  y.contiguous(), xprev.contiguous(), b, xout, yout, plan.ws)
            ctx.save_for_backward(y)
        ctx.keep_z = keep_z
        ctx.args = (plan, b, factor, subset, n_subsets, eta, alpha, float(lam), tv_iters, amom, vjp_ws)
        ctx.lam_meta = (lam.dtype, lam.device) if torch.is_tensor(lam) else None
        return xout, yout

    @staticmethod
    def backward(ctx, xbar, ybar):
        (saved,) = ctx.saved_tensors
        plan, b, factor, subset, n_subsets, eta, alpha, lam, tv_iters, amom, vjp_ws = ctx.args
        xbar = torch.zeros_like(saved) if xbar is None else xbar.contiguous()
        ybar = torch.zeros_like(saved) if ybar is None else ybar.contiguous()
        ybar_in = torch.empty_like(saved)
        xpbar = torch.empty_like(saved)
        if ctx.keep_z:
            lb = _native.unrolled_step_vjp_saved(plan.g, factor, subset, n_subsets, eta, alpha, lam, tv_iters,
                                                 amom, saved, xbar, ybar, ybar_in, xpbar, plan.ws, vjp_ws)
        else:
            lb = _native.unrolled_step_vjp(plan.g, factor, subset, n_subsets, eta, alpha, lam, tv_iters, amom,
                                           saved.contiguous(), b, xbar, ybar, ybar_in, xpbar, plan.ws, vjp_ws)
        lam_grad = None
        if ctx.lam_meta is not None:
            lam_grad = torch.tensor(float(lb.sum()), dtype=ctx.lam_meta[0], device=ctx.lam_meta[1])
        return (ybar_in, xpbar, lam_grad) + (None,) * 11


def unrolled_pnp(plan, stages: Sequence, eta, seq, b, x0, lam, *, alpha: float = 1.0,
                 tv_iters: int = 20, momentum: bool = True, keep_z: bool = True, subset_seed: int = 0):
    """x_T of Algorithm 1 as a differentiable function of x0 (float32 CUDA
    tensor [batch, n, n]) and lam (a float64 scalar tensor, may require grad).
    eta: step size per stage, or None for the library's eta_k = 1/L_k
    (pnp_step_sizes).  seq: the subset id of every iteration, or None for the
    library's order drawn from subset_seed (pnp_subset_sequence, as pnp_run
    draws it).  The walk over iterations (stage, subset, momentum a_i)
    comes from pnp_schedule.  keep_z: keep each iteration's gradient step z for
    the backward pass (one projector pair fewer per iteration); False keeps only
    y and recomputes z."""
    g = plan.g
    if eta is None:
        eta = plan.step_sizes(stages)
    st = _native._stages(stages)
    if seq is None:
        seq = _native.subset_sequence(stages, subset_seed)
    stage_of, subset_of, amom_of = _native.schedule(stages, seq, momentum)
    vjp_ws = torch.empty(_native.vjp_workspace_size(g, tv_iters), dtype=torch.uint8, device=x0.device)
    y = x0
    x = x0
    for k, p, a in zip(stage_of.tolist(), subset_of.tolist(), amom_of.tolist()):
        s_k = st[k]
        x, y = UnrolledStep.apply(y, x, lam, plan, b, s_k.factor, p, s_k.n_subsets, float(eta[k]), alpha, tv_iters,
                                  a, vjp_ws, keep_z)
    return x
