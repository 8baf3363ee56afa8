"""Sensor-sharded CGLS for one large frame.

The rows of A (Eq. 6 at every sensor and sample) split by sensor: A = [A_1;
...; A_R], and ||A x - y||^2 (the data term of Eq. 8) is the sum of the
shards' ||A_r x - y_r||^2.  Each shard is a plan over its own sensors and the
whole image grid.  Per CGLS iteration every shard applies A_r and A_r^T to its
own sensors in the library's kernels (``pa_shard_cgls_*``); the only exchange
is two sums over all shards:

* the partial images A_r^T r_r (N floats) after every A^T, and
* the scalars ||A_r p||^2 (FP64) after every A, for alpha.

Shards held by one process add into one buffer in turn (the library's
accumulate mode, in shard order); ranks of a ``torch.distributed`` group then
all-reduce that buffer (NCCL between GPUs).  gamma = ||A^T r||^2, alpha, beta
and x then agree on every rank without further exchange.

``sharded_cgls`` drives any objects with the ``shard_cgls_*`` methods of
``api.Plan`` (the library's plans in the product); it holds no arithmetic of
the method itself.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch


def sensor_ranges(n_sensors: int, n_shards: int) -> list[tuple[int, int]]:
    """Contiguous, near-equal split of sensors 0..n_sensors-1 into n_shards
    ranges [begin, end) (the first n_sensors % n_shards ranges one longer)."""
    if n_shards < 1 or n_sensors < n_shards:
        raise ValueError("need 1 <= n_shards <= n_sensors")
    base, extra = divmod(n_sensors, n_shards)
    out, b = [], 0
    for r in range(n_shards):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def shard_plans(prob, ranges, **plan_kw):
    """One ``api.Plan`` per sensor range of the problem (same grid, c, f_s, t0
    and amplitude), for the shards this process holds."""
    from .api import Plan
    kw = dict(plan_kw)
    ydt = kw.pop("y_dtype", prob.extra.get("y_dtype", "f32"))
    return [Plan(np.asarray(prob.sensors)[b:e], prob.shape, prob.spacing, prob.origin, prob.c,
                 prob.fs, prob.n_samples, t0=prob.t0, amp_scale=prob.amp_scale, y_dtype=ydt,
                 dim=prob.dim, **kw)
            for b, e in ranges]


def sharded_cgls(shards: Sequence, ys: Sequence[torch.Tensor], n_iter: int,
                 x0: Optional[torch.Tensor] = None, nonneg: bool = True,
                 process_group=None, history: bool = False):
    """CGLS on ||A x - y||^2 with A split by sensors over ``shards`` (this
    process's) and, with ``process_group``, over the shards of every rank of
    that group (each rank calls this with its own shards and traces).

    ys[i]: the traces of shards[i]'s sensors.  Returns x (the same on every
    rank; clamped to x >= 0 at the end with ``nonneg``, as ``pa_reconstruct``'s
    CGLS) and, with ``history``, ||y - A x_n||^2 over all shards, n = 0..n_iter.
    """
    if len(shards) == 0 or len(shards) != len(ys):
        raise ValueError("one trace tensor per shard, at least one shard")
    n = shards[0].n_pixels
    if any(sh.n_pixels != n for sh in shards):
        raise ValueError("every shard must cover the same image grid")
    dev = shards[0].device
    dtype = getattr(shards[0], "image_dtype", torch.float32)

    def total(t: torch.Tensor) -> None:
        if process_group is not None:
            torch.distributed.all_reduce(t, group=process_group)

    x = (x0.to(device=dev, dtype=dtype).clone() if x0 is not None
         else torch.zeros(n, device=dev, dtype=dtype))
    s = torch.empty(n, device=dev, dtype=dtype)          # sum of the partial images
    delta = torch.empty(1, device=dev, dtype=torch.float64)  # sum of ||A_r p||^2
    for i, (sh, y) in enumerate(zip(shards, ys)):
        sh.shard_cgls_begin(n_iter, y, x, s, accumulate=i > 0)
    total(s)
    for it in range(n_iter):
        for i, sh in enumerate(shards):
            sh.shard_cgls_direction(it, s, delta, accumulate=i > 0)
        total(delta)
        for i, sh in enumerate(shards):
            # one shard per process updates x; every shard updates its residual
            sh.shard_cgls_update(it, delta, x if i == 0 else None, s, accumulate=i > 0)
        total(s)
    hist = torch.empty(n_iter + 1, device=dev, dtype=torch.float64) if history else None
    for i, sh in enumerate(shards):
        sh.shard_cgls_finish(x if i == 0 else None, nonneg and i == 0, hist, accumulate=i > 0)
    if hist is None:
        return x
    total(hist)
    return x, hist.cpu().numpy()
