"""Autotuner for the gathers' work decomposition ("tile shapes" at run time).

Three plan options change how the work of A and A^T is cut into CTAs without
changing what is computed:

* ``adj_cluster``: how many CTAs (a thread-block cluster) split one pixel
  tile's sensors in the adjoint;
* ``fwd_sensors_per_cta``: how many sensors one forward tile work item covers;
* ``fwd_threads``: how many threads share a forward work item's 1024 pixels
  (64, 128 or 256: 16, 8 or 4 pixels each).

For a size class (GPU, dimension, and the pixel / sensor / sample counts
rounded up to powers of two) the tuner builds a plan per candidate, times a
few forward + adjoint applications with CUDA events and keeps the fastest.
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
DEFAULT = (1, 32, 128)  # (adj_cluster, fwd_sensors_per_cta, fwd_threads) held fixed while another varies


def _pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


def size_key(gpu: str, dim: int, n_pixels: int, n_sensors: int, n_samples: int,
             y_dtype: str = "f32") -> str:
    return (f"{gpu}|{dim}d|N{_pow2(n_pixels)}|S{_pow2(n_sensors)}|K{_pow2(n_samples)}|"
            f"y{y_dtype}")


def candidates(n_sensors: int) -> Iterable[Tuple[int, int, int]]:
    """(adj_cluster, fwd_sensors_per_cta, fwd_threads) triples.  adj_cluster
    only changes the adjoint and the other two only the forward, so the forward
    pair is searched jointly with the cluster at its default, and the cluster
    with the forward pair at its default."""
    for nt in FWD_THREADS:
        for spc in FWD_SENSORS:
            yield 1, spc, nt
    for c in ADJ_CLUSTERS[1:]:
        if 2 * c <= n_sensors:
            yield c, DEFAULT[1], DEFAULT[2]


def default_cache_path() -> str:
    return os.environ.get("PA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pa_gb300",
                                       "autotune.json"))


class Autotuner:
    """Pick (adj_cluster, fwd_sensors_per_cta, fwd_threads) per size class.

    ``measure(prob, adj_cluster, spc, fwd_threads) -> seconds`` defaults to
    timing real plans on the current GPU; tests inject their own."""

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
                "fwd_threads": entry.get("fwd_threads", 0)}

    def best(self, prob, force: bool = False) -> dict:
        k = self.key(prob)
        if not force and k in self.cache:
            return self.cache[k]
        timings = {}
        for c, spc, nt in candidates(prob.n_sensors):
            timings[(c, spc, nt)] = float(self.measure(prob, c, spc, nt))
        # the forward pair at the default cluster; ties to fewer threads, then
        # fewer sensors
        fwd = {(spc, nt): t for (c, spc, nt), t in timings.items() if c == DEFAULT[0]}
        spc, nt = min(fwd, key=lambda v: (fwd[v], v[1], v[0]))
        adj = {c: t for (c, s, n), t in timings.items() if (s, n) == DEFAULT[1:]}
        c = min(adj, key=lambda v: (adj[v], v))
        entry = {"adj_cluster": c, "fwd_sensors_per_cta": spc, "fwd_threads": nt,
                 "timings_s": {f"{a},{b},{d}": t for (a, b, d), t in timings.items()}}
        self.cache[k] = entry
        self._save()
        return entry

    def _save(self) -> None:
        os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)


def _measure_gpu(prob, adj_cluster: int, spc: int, fwd_threads: int, reps: int = 5) -> float:
    """Median time (s) of one forward + one adjoint application on the GPU."""
    import torch

    from .api import Plan

    with Plan.from_problem(prob, adj_cluster=adj_cluster, fwd_sensors_per_cta=spc,
                           fwd_threads=fwd_threads) as plan:
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.rand(prob.n_pixels, device="cuda", generator=g)
        y = torch.randn(prob.n_sensors, prob.n_samples, device="cuda", generator=g)
        p = torch.empty_like(y)
        z = torch.empty_like(x)
        for _ in range(2):
            plan.forward(x, out=p)
            plan.adjoint(y, out=z)
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.forward(x, out=p)
            plan.adjoint(y, out=z)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b) * 1e-3)
        return statistics.median(times)
