"""Autotuner for the gathers' work decomposition ("tile shapes" at run time).

Four plan options change how the work of A and A^T is cut into CTAs without
changing what is computed:

* ``adj_cluster``: how many CTAs (a thread-block cluster) split one pixel
  tile's sensors in the adjoint;
* ``adj_warps``: how many compute warps share an adjoint CTA's 1024 pixels
  (4 or 8: 8 or 4 pixels per thread);
* ``fwd_sensors_per_cta``: how many sensors one forward tile work item covers;
* ``fwd_threads``: how many threads share a forward work item's 1024 pixels
  (64, 128 or 256: 16, 8 or 4 pixels each).

For a size class (GPU, dimension, and the pixel / sensor / sample counts
rounded up to powers of two) the tuner builds a plan per candidate, times a
short graph-captured CGLS reconstruction (the forward with its direction
update, the combine, the vector step and the adjoint, as a reconstruction runs
them) with CUDA events and keeps the fastest.
Results are cached in a JSON file (``PA_TUNE_CACHE``, default
``~/.cache/pa_gb300/autotune.json``).
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, Iterable, Optional, Tuple

ADJ_CLUSTERS = (1, 2, 4, 8)
FWD_SENSORS = (8, 12, 16, 20, 24, 32, 48, 64, 96, 128)
FWD_THREADS = (64, 128, 256)
ADJ_WARPS = (4, 8)
# (adj_cluster, fwd_sensors_per_cta, fwd_threads, adj_warps) held fixed while
# the other operator's options vary
DEFAULT = (1, 32, 128, 8)


def _pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


def size_key(gpu: str, dim: int, n_pixels: int, n_sensors: int, n_samples: int,
             y_dtype: str = "f32") -> str:
    return (f"{gpu}|{dim}d|N{_pow2(n_pixels)}|S{_pow2(n_sensors)}|K{_pow2(n_samples)}|"
            f"y{y_dtype}")


def candidates(n_sensors: int) -> Iterable[Tuple[int, int, int, int]]:
    """(adj_cluster, fwd_sensors_per_cta, fwd_threads, adj_warps).  The
    cluster and warps only change the adjoint, the other two only the forward,
    so the forward pair is searched jointly with the adjoint at its defaults,
    and the adjoint pair with the forward at its defaults."""
    for nt in FWD_THREADS:
        for spc in FWD_SENSORS:
            yield DEFAULT[0], spc, nt, DEFAULT[3]
    for c in ADJ_CLUSTERS:
        for aw in ADJ_WARPS:
            if (c, aw) != (DEFAULT[0], DEFAULT[3]) and (c == 1 or 2 * c <= n_sensors):
                yield c, DEFAULT[1], DEFAULT[2], aw


def default_cache_path() -> str:
    return os.environ.get("PA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pa_gb300",
                                       "autotune.json"))


class Autotuner:
    """Pick (adj_cluster, fwd_sensors_per_cta, fwd_threads, adj_warps) per
    size class.

    ``measure(prob, adj_cluster, spc, fwd_threads, adj_warps) -> seconds``
    defaults to timing real plans on the current GPU; tests inject their own."""

    def __init__(self, cache_path: Optional[str] = None,
                 measure: Optional[Callable] = None, gpu_name: Optional[str] = None):
        self.cache_path = cache_path or default_cache_path()
        self.measure = measure or _measure_gpu
        self._gpu = gpu_name
        self.cache: Dict[str, dict] = {}
        if os.path.exists(self.cache_path):
            try:
                with open(self.cache_path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    @property
    def gpu(self) -> str:
        if self._gpu is None:
            import torch
            self._gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        return self._gpu

    def key(self, prob) -> str:
        return size_key(self.gpu, prob.dim, prob.n_pixels, prob.n_sensors, prob.n_samples,
                        prob.extra.get("y_dtype", "f32"))

    @staticmethod
    def plan_options(entry: dict) -> dict:
        """The plan keyword arguments of a tuning entry."""
        return {"adj_cluster": entry["adj_cluster"],
                "fwd_sensors_per_cta": entry["fwd_sensors_per_cta"],
                "fwd_threads": entry.get("fwd_threads", 0),
                "adj_warps": entry.get("adj_warps", 0)}

    def best(self, prob, force: bool = False) -> dict:
        k = self.key(prob)
        if not force and k in self.cache:
            return self.cache[k]
        timings = {}
        for cand in candidates(prob.n_sensors):
            timings[cand] = float(self.measure(prob, *cand))
        # the forward pair with the adjoint at its defaults (ties to fewer
        # threads, then fewer sensors); the adjoint pair with the forward at
        # its defaults (ties to the smaller cluster, then fewer warps)
        fwd = {(spc, nt): t for (c, spc, nt, aw), t in timings.items()
               if (c, aw) == (DEFAULT[0], DEFAULT[3])}
        spc, nt = min(fwd, key=lambda v: (fwd[v], v[1], v[0]))
        adj = {(c, aw): t for (c, spc_, nt_, aw), t in timings.items()
               if (spc_, nt_) == DEFAULT[1:3]}
        c, aw = min(adj, key=lambda v: (adj[v], v))
        entry = {"adj_cluster": c, "fwd_sensors_per_cta": spc, "fwd_threads": nt,
                 "adj_warps": aw,
                 "timings_s": {",".join(map(str, k)): t for k, t in timings.items()}}
        self.cache[k] = entry
        self._save()
        return entry

    def _save(self) -> None:
        os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)


def _measure_gpu(prob, adj_cluster: int, spc: int, fwd_threads: int, adj_warps: int,
                 reps: int = 5, n_iter: int = 4) -> float:
    """Median time (s) of one CGLS iteration on the GPU: the mix a reconstruction
    runs (the forward gather with its direction update, the combine, the vector
    step, the adjoint with its norm), from an n_iter-iteration graph-captured
    reconstruction of random traces, each sample timing enough back-to-back
    reconstructions (at least ~2 ms) that launch and event overheads do not
    decide between close candidates."""
    import torch

    from .api import Plan

    with Plan.from_problem(prob, adj_cluster=adj_cluster, fwd_sensors_per_cta=spc,
                           fwd_threads=fwd_threads, adj_warps=adj_warps) as plan:
        g = torch.Generator(device="cuda").manual_seed(0)
        ydt = torch.float16 if plan.y_dtype == "f16" else torch.float32
        y = torch.randn(prob.n_sensors * prob.n_samples, device="cuda", generator=g).to(ydt)
        x = torch.zeros(prob.n_pixels, device="cuda")

        def run(n: int) -> float:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(n):
                plan.reconstruct(y, "cgls", n_iter, out=x)
            b.record()
            b.synchronize()
            return a.elapsed_time(b) * 1e-3 / (n * n_iter)

        run(2)
        inner = max(1, min(100, int(2e-3 / max(run(1) * n_iter, 1e-6))))
        return statistics.median(run(inner) for _ in range(reps))
