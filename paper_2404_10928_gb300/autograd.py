"""Differentiable forms of the time-of-flight operator for PyTorch.

``ForwardOp`` (p = A(x; c)) and ``AdjointOp`` (g = A^T(r; c)) are
``torch.autograd.Function``s whose backward passes are the library's own
kernels: the backward of A is A^T, the backward of A^T is A, and the derivative
with respect to the speed of sound c (the c of Eq. 1 and Eq. 6) is ``pa_dc``:

    d/dc <g, A(x; c)>   = pa_dc(x, g)
    <v, (dA^T/dc) r>    = <(dA/dc) v, r> = pa_dc(v, r).

``TVOp`` is the smoothed TV term of Eq. 8 (``pa_tv``).  ``UnrolledLandweber``
chains projected Landweber steps x <- max(0, x - omega A^T(A(x; c) - y)) and
checkpoints every step (only x_k is kept; A x_k is recomputed in backward).

Images are ``[..., N]`` float32 CUDA tensors and traces ``[..., S, K]``; leading
dimensions are a batch of frames sharing the plan's geometry and c.  c is a
0-d tensor; changing it rebuilds the plan's reference table (a blocking call).
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint


def _set_c(plan, c) -> None:
    cv = float(c)
    if cv != plan.c:
        plan.set_sound_speed(cv)


def _frames(t: torch.Tensor, n: int) -> torch.Tensor:
    return t.reshape(-1, n).contiguous()


class ForwardOp(torch.autograd.Function):
    """p = A(x; c) with gradients for x (A^T) and c (pa_dc)."""

    @staticmethod
    def forward(ctx, x, c, plan):
        _set_c(plan, c)
        xb = _frames(x, plan.n_pixels)
        out = torch.empty((xb.shape[0], plan.n_sensors, plan.n_samples), device=x.device,
                          dtype=torch.float32)
        for b in range(xb.shape[0]):
            plan.forward(xb[b], out=out[b])
        ctx.plan = plan
        ctx.xshape = x.shape
        ctx.save_for_backward(xb, c)
        return out.reshape(*x.shape[:-1], plan.n_sensors, plan.n_samples)

    @staticmethod
    def backward(ctx, gp):
        xb, c = ctx.saved_tensors
        plan = ctx.plan
        _set_c(plan, c)
        gb = _frames(gp, plan.n_sensors * plan.n_samples)
        gx = gc = None
        if ctx.needs_input_grad[0]:
            gx = torch.empty_like(xb)
            for b in range(xb.shape[0]):
                plan.adjoint(gb[b], out=gx[b])
            gx = gx.reshape(ctx.xshape)
        if ctx.needs_input_grad[1]:
            tot = torch.zeros((), dtype=torch.float64, device=xb.device)
            for b in range(xb.shape[0]):
                tot = tot + plan.dc(xb[b], gb[b])
            gc = tot.to(c.dtype)
        return gx, gc, None


class AdjointOp(torch.autograd.Function):
    """g = A^T(r; c) with gradients for r (A) and c (pa_dc)."""

    @staticmethod
    def forward(ctx, r, c, plan):
        _set_c(plan, c)
        rb = _frames(r, plan.n_sensors * plan.n_samples)
        out = torch.empty((rb.shape[0], plan.n_pixels), device=r.device, dtype=torch.float32)
        for b in range(rb.shape[0]):
            plan.adjoint(rb[b], out=out[b])
        ctx.plan = plan
        ctx.rshape = r.shape
        ctx.save_for_backward(rb, c)
        return out.reshape(*r.shape[:-2], plan.n_pixels)

    @staticmethod
    def backward(ctx, gg):
        rb, c = ctx.saved_tensors
        plan = ctx.plan
        _set_c(plan, c)
        gb = _frames(gg, plan.n_pixels)
        gr = gc = None
        if ctx.needs_input_grad[0]:
            gr = torch.empty_like(rb)
            for b in range(rb.shape[0]):
                plan.forward(gb[b], out=gr[b])
            gr = gr.reshape(ctx.rshape)
        if ctx.needs_input_grad[1]:
            tot = torch.zeros((), dtype=torch.float64, device=rb.device)
            for b in range(rb.shape[0]):
                tot = tot + plan.dc(gb[b], rb[b])
            gc = tot.to(c.dtype)
        return gr, gc, None


class TVOp(torch.autograd.Function):
    """Sum over frames of the smoothed TV (float64 scalar); backward uses pa_tv's gradient."""

    @staticmethod
    def forward(ctx, x, plan, eps):
        xb = _frames(x, plan.n_pixels)
        grads = torch.empty_like(xb)
        tot = torch.zeros((), dtype=torch.float64, device=x.device)
        for b in range(xb.shape[0]):
            val, _ = plan.tv(xb[b], eps, grad=grads[b])
            tot = tot + val
        ctx.save_for_backward(grads)
        ctx.xshape = x.shape
        return tot

    @staticmethod
    def backward(ctx, gv):
        (grads,) = ctx.saved_tensors
        return (gv.to(torch.float32) * grads).reshape(ctx.xshape), None, None


def data_tv_loss(plan, x, c, p, tv_weight: float = 1e-3, eps: float = 1e-4):
    """||A(x; c) - p||^2 + tv_weight * TV(x), summed over frames (float64 scalar)."""
    r = ForwardOp.apply(x, c, plan) - p
    return (r.double() ** 2).sum() + tv_weight * TVOp.apply(x, plan, eps)


class UnrolledLandweber(torch.nn.Module):
    """n steps of x <- max(0, x - omega A^T(A(x; c) - y)), differentiable in x0, y
    and c; with ``checkpointing`` only the iterates are kept and each step is
    recomputed in backward."""

    def __init__(self, plan, n_iter: int, omega: float, checkpointing: bool = True):
        super().__init__()
        self.plan = plan
        self.n_iter = int(n_iter)
        self.omega = float(omega)
        self.checkpointing = checkpointing

    def step(self, x, y, c):
        r = ForwardOp.apply(x, c, self.plan) - y
        return torch.relu(x - self.omega * AdjointOp.apply(r, c, self.plan))

    def forward(self, x0, y, c):
        x = x0
        for _ in range(self.n_iter):
            if self.checkpointing:
                x = checkpoint(self.step, x, y, c, use_reentrant=False)
            else:
                x = self.step(x, y, c)
        return x
