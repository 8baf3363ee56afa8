"""Differentiable forms of the time-of-flight operator for PyTorch.

Every function here is marshalling: the arithmetic of each forward and
backward pass runs in the library's kernels, one launch per operator for all
frames of a batch (images ``[..., N]``, traces ``[..., S, K]``; the leading
dimensions are frames sharing the plan's geometry and c).

* ``ForwardOp`` (p = A(x; c)) and ``AdjointOp`` (g = A^T(r; c)): the backward
  of A is A^T and vice versa; the derivative with respect to the speed of sound
  c (the c of Eq. 1 and Eq. 6) is the library's speed-of-sound derivative
  summed over the frames:
      d/dc <g, A(x; c)>   = pa_dc_frames(x, g)
      <v, (dA^T/dc) r>    = <(dA/dc) v, r> = pa_dc_frames(v, r).
* ``TVOp``: the smoothed TV term of Eq. 8 per frame (``pa_tv_frames``).
* ``DataTVLoss`` / ``data_tv_loss``: sum over frames of ||A(x; c) - p||^2 +
  tv_weight TV(x), the data and TV terms of Eq. 8, with residual, norms, TV and
  the loss total computed by ``pa_data_tv_loss_frames`` and the gradients in x
  and c by ``pa_data_tv_loss_vjp_frames``.
* ``LandweberStep`` / ``UnrolledLandweber``: projected Landweber steps
  x <- max(0, x + omega A^T(y - A(x; c))) (``pa_landweber_step_frames``), whose
  backward (``pa_landweber_step_vjp_frames``) gives the gradients in x, y and
  c; the unrolled loop checkpoints every step (only x_k is kept and each step
  is recomputed in backward).

c is a 0-d tensor; changing it rebuilds the plan's reference table (a
blocking call).
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint


def _set_c(plan, c) -> None:
    cv = float(c)
    if cv != plan.c:
        plan.set_sound_speed(cv)


def _img(t: torch.Tensor, plan) -> torch.Tensor:
    return t.reshape(-1, plan.n_pixels).contiguous()


def _trace(t: torch.Tensor, plan) -> torch.Tensor:
    return t.reshape(-1, plan.n_sensors, plan.n_samples).contiguous()


def _upstream(g: torch.Tensor) -> float:
    """The incoming gradient of a scalar output, as the factor the library
    applies to the gradients it forms."""
    return float(g)


class ForwardOp(torch.autograd.Function):
    """p = A(x; c) with gradients for x (A^T) and c (speed-of-sound derivative)."""

    @staticmethod
    def forward(ctx, x, c, plan):
        _set_c(plan, c)
        xb = _img(x, plan)
        out = plan.forward_frames(xb)
        ctx.plan = plan
        ctx.xshape = x.shape
        ctx.save_for_backward(xb, c)
        return out.reshape(*x.shape[:-1], plan.n_sensors, plan.n_samples)

    @staticmethod
    def backward(ctx, gp):
        xb, c = ctx.saved_tensors
        plan = ctx.plan
        _set_c(plan, c)
        gb = _trace(gp.to(torch.float32), plan)
        gx = gc = None
        if ctx.needs_input_grad[0]:
            gx = plan.adjoint_frames(gb).reshape(ctx.xshape)
        if ctx.needs_input_grad[1]:
            gc = plan.dc_frames(xb, gb).to(c.dtype)
        return gx, gc, None


class AdjointOp(torch.autograd.Function):
    """g = A^T(r; c) with gradients for r (A) and c (speed-of-sound derivative)."""

    @staticmethod
    def forward(ctx, r, c, plan):
        _set_c(plan, c)
        rb = _trace(r, plan)
        out = plan.adjoint_frames(rb)
        ctx.plan = plan
        ctx.rshape = r.shape
        ctx.save_for_backward(rb, c)
        return out.reshape(*r.shape[:-2], plan.n_pixels)

    @staticmethod
    def backward(ctx, gg):
        rb, c = ctx.saved_tensors
        plan = ctx.plan
        _set_c(plan, c)
        gb = _img(gg.to(torch.float32), plan)
        gr = gc = None
        if ctx.needs_input_grad[0]:
            gr = plan.forward_frames(gb).reshape(ctx.rshape)
        if ctx.needs_input_grad[1]:
            gc = plan.dc_frames(gb, rb).to(c.dtype)
        return gr, gc, None


class TVOp(torch.autograd.Function):
    """Per-frame smoothed TV (float64 [frames]); backward uses the gradients
    pa_tv_frames returns with the values."""

    @staticmethod
    def forward(ctx, x, plan, eps):
        xb = _img(x, plan)
        vals, grads = plan.tv_frames(xb, eps)
        ctx.save_for_backward(grads)
        ctx.xshape = x.shape
        return vals

    @staticmethod
    def backward(ctx, gv):
        (grads,) = ctx.saved_tensors
        return (gv.to(torch.float32)[:, None] * grads).reshape(ctx.xshape), None, None


class DataTVLoss(torch.autograd.Function):
    """sum over frames of ||A(x; c) - p||^2 + tv_weight TV_eps(x) (float64
    scalar), with gradients in x and c; p (the measured traces) gets none."""

    @staticmethod
    def forward(ctx, x, c, p, plan, tv_weight, eps):
        _set_c(plan, c)
        xb = _img(x, plan)
        loss, r, tg = plan.data_tv_loss_frames(xb, _trace(p.to(torch.float32), plan),
                                               float(tv_weight), float(eps))
        ctx.plan = plan
        ctx.xshape = x.shape
        ctx.tv_weight = float(tv_weight)
        ctx.save_for_backward(xb, r, tg if tg is not None else xb, c)
        ctx.has_tv = tg is not None
        return loss

    @staticmethod
    def backward(ctx, g):
        xb, r, tg, c = ctx.saved_tensors
        plan = ctx.plan
        _set_c(plan, c)
        gx, gc = plan.data_tv_loss_vjp_frames(xb, r, tg if ctx.has_tv else None, ctx.tv_weight,
                                              _upstream(g), need_x=ctx.needs_input_grad[0],
                                              need_c=ctx.needs_input_grad[1])
        if gx is not None:
            gx = gx.reshape(ctx.xshape)
        if gc is not None:
            gc = gc.to(c.dtype)
        return gx, gc, None, None, None, None


def data_tv_loss(plan, x, c, p, tv_weight: float = 1e-3, eps: float = 1e-4):
    """||A(x; c) - p||^2 + tv_weight * TV(x), summed over frames (float64 scalar)."""
    return DataTVLoss.apply(x, c, p, plan, tv_weight, eps)


class LandweberStep(torch.autograd.Function):
    """x_out = max(0, x + omega A^T (y - A(x; c))) (the projection only with
    nonneg), with gradients in x, y and c."""

    @staticmethod
    def forward(ctx, x, y, c, plan, omega, nonneg):
        _set_c(plan, c)
        xb = _img(x, plan)
        yb = _trace(y, plan)
        out = plan.landweber_step_frames(xb, yb, float(omega), bool(nonneg))
        ctx.plan = plan
        ctx.shapes = (x.shape, y.shape)
        ctx.omega, ctx.nonneg = float(omega), bool(nonneg)
        ctx.save_for_backward(xb, yb, out, c)
        return out.reshape(x.shape)

    @staticmethod
    def backward(ctx, g):
        xb, yb, out, c = ctx.saved_tensors
        plan = ctx.plan
        _set_c(plan, c)
        gx, gy, gc = plan.landweber_step_vjp_frames(
            xb, yb, out, _img(g.to(torch.float32), plan), ctx.omega, ctx.nonneg,
            need_y=ctx.needs_input_grad[1], need_c=ctx.needs_input_grad[2])
        gx = gx.reshape(ctx.shapes[0])
        if gy is not None:
            gy = gy.reshape(ctx.shapes[1])
        if gc is not None:
            gc = gc.to(c.dtype)
        return gx, gy, gc, None, None, None


class UnrolledLandweber(torch.nn.Module):
    """n steps of x <- max(0, x + omega A^T(y - A(x; c))), differentiable in x0, y
    and c; with ``checkpointing`` only the iterates are kept and each step is
    recomputed in backward."""

    def __init__(self, plan, n_iter: int, omega: float, checkpointing: bool = True,
                 nonneg: bool = True):
        super().__init__()
        self.plan = plan
        self.n_iter = int(n_iter)
        self.omega = float(omega)
        self.checkpointing = checkpointing
        self.nonneg = bool(nonneg)

    def step(self, x, y, c):
        return LandweberStep.apply(x, y, c, self.plan, self.omega, self.nonneg)

    def forward(self, x0, y, c):
        x = x0
        for _ in range(self.n_iter):
            if self.checkpointing:
                x = checkpoint(self.step, x, y, c, use_reentrant=False)
            else:
                x = self.step(x, y, c)
        return x
