"""Benchmark: iterative photoacoustic reconstruction on one or more GB300s.

A step is one full reconstruction of one frame of the 2D ring workload
(256x256 pixels at 0.1 mm, 256-sensor ring of radius 20 mm, 2048 samples at
40 MHz, Bezier vessel phantom, 1% noise, 50 CGLS iterations with FP64
reductions), with the measured traces already resident in device memory.
``value`` is pixel-sensor updates per second (one update = one (pixel, sensor)
pair evaluated by A or A^T) summed over all ranks; every rank reconstructs its
own frame (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
reference arm), on a bounded sample of the same workload per step.

Besides the contract keys (``roofline`` for the dominant gather, ``cpu_baseline``,
``e2e`` through the host-buffer entry point, ``clocks``, ``gpu_launches``), the
line carries the other workloads, each timed with CUDA events outside the timed
region (``--no-extras`` skips them): ``bp_vs_ir`` (back-projection against
CGLS and FISTA), ``batched`` (64 ragged frames, persistent launch against the
per-frame loop), ``differentiable`` (loss and gradients in x and c),
``volume3d`` (the 128^3 planar workload), ``dense_paper_size`` (the 6144 x 16384
matrix) and ``frequency_domain``.  ``--profile-case 2d|3d|dense|freq|batch|dc|cgls``
runs only a small fixed workload for ncu captures.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel·sensor updates/s for A and Aᵀ; recon frames/s batched vs plain, % FP32 peak"
UNIT = "pixel·sensor updates/s"
WORKLOAD = "2D 256x256 0.1mm, 256-sensor ring R=20mm, 2048 samples @40MHz, c=1500, vessel phantom + 1% noise, 50 CGLS (FP64 reductions)"
N_ITER = 50
FLOPS_PER_PAIR = 18  # 9 FP32 instructions per pair (FFMA-equivalent, 2 flop each)
MUFU_PER_PAIR = 2    # rsqrt (1/d) and rcp (the difference form of the arrival) per pair
SFU_PER_SM_CLK = 16  # MUFU results per SM per clock
L2_FLUSH_BYTES = 256 << 20


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cgls_launches(n_iter: int) -> int:
    """Kernels of one CGLS reconstruction (A = tile gather + combine; every norm
    is summed by the kernel that consumes it): setup (A, pack, A^T) = 4, per
    iteration (A with the fused direction update, alpha + x/r update, A^T) = 4,
    then the residual history and the final clamp = 2."""
    return 4 + 4 * n_iter + 2


def max_over_ranks(dist, device, value: float) -> float:
    """The largest of every rank's `value` (the job's clock is its slowest
    rank); the value itself when not distributed."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed per second of the job's clock (weak scaling:
    every rank processes units_per_rank)."""
    return units_per_rank * world / seconds


def frame_noise(shape, rank: int) -> np.ndarray:
    """Each rank reconstructs its own frame: the benchmark geometry with its own
    noise draw (frames are independent, so they shard across ranks with no
    exchange)."""
    return np.random.default_rng(2003 + rank).standard_normal(shape)


def cgls_applications(n_iter: int) -> int:
    return 2 + 2 * n_iter


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.environ.get("PA_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), f"pa_bench_clocks_{os.getpid()}_{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
            # the tool takes a while to start: let its first sample land before
            # the timed region begins, so the samples fall under load
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        if len(lines) > 2:
            lines = lines[1:]  # the first sample predates the timed region
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle (CPU) timing: the cpu_baseline leg and the reference arm
# ---------------------------------------------------------------------------
def oracle_sample(prob, y, target_s: float = 15.0):
    """Time the FP64 oracle's CGLS on the workload: as many iterations as fit in
    about target_s seconds of host time.  Returns (pairs/s, seconds, iterations)."""
    os.environ.setdefault("OMP_NUM_THREADS", str(cores()))
    from oracle import oracle as orc
    geo = orc.Geometry.of(prob)
    t = time.perf_counter()
    orc.cgls(geo, y, 1)  # 4 applications
    per_app = (time.perf_counter() - t) / 4.0
    n_it = max(1, int((target_s / per_app - 2) / 2))
    t = time.perf_counter()
    orc.cgls(geo, y, n_it)
    dt = time.perf_counter() - t
    apps = cgls_applications(n_it)
    return prob.pairs * apps / dt, dt, n_it


def oracle_detail(c2_prob, c2_y) -> dict:
    """The rest of the CPU-baseline plan, on the machine's host cores: the benchmark
    frame's CGLS on one core, the linear-array disk workload in full (power
    iteration and 10 Landweber steps), and one application of A and of A^T on
    the 3D planar workload (128^3, dense random image) and on the ragged time
    series (all 64 frames) -- per-application figures for the workloads whose
    full reconstruction on the CPU would take far longer."""
    from oracle import oracle as orc
    from paper_2404_10928_gb300 import phantoms as ph
    n_all = cores()
    out = {"cores_all": n_all}
    orc.set_threads(1)
    rate1, secs1, it1 = oracle_sample(c2_prob, c2_y, target_s=5.0)
    out["ring256_cgls_1core"] = {"pairs_per_s": rate1, "seconds": secs1, "cgls_iterations": it1}
    orc.set_threads(n_all)
    out["ring256_cgls_all_cores_vs_1core"] = None
    d = ph.linear_array_disks()
    geo = orc.Geometry.of(d)
    y = orc.forward(geo, d.x_true)
    t = time.perf_counter()
    lam = orc.power_iteration(geo, ph.power_start(d.n_pixels), 50)
    orc.landweber(geo, y, 10, omega=1.0 / lam)
    dt = time.perf_counter() - t
    out["disks64_landweber10_full"] = {"seconds": dt, "pairs_per_s": d.pairs * (100 + 21) / dt,
                                       "includes": "50 power steps + 10 Landweber steps"}
    v = ph.planar_vessel_tree()
    geo = orc.Geometry.of(v)
    xr = np.random.default_rng(0).uniform(0.0, 1.0, v.n_pixels)
    t = time.perf_counter()
    pv = orc.forward(geo, xr)
    tf = time.perf_counter() - t
    t = time.perf_counter()
    orc.adjoint(geo, pv)
    ta = time.perf_counter() - t
    out["planar128_per_application"] = {"forward_s": tf, "adjoint_s": ta,
                                        "pairs_per_s": 2 * v.pairs / (tf + ta),
                                        "cgls30_extrapolated_s": 31 * (tf + ta)}
    frames = ph.ragged_time_series()
    t = time.perf_counter()
    pairs = 0
    for f in frames:
        g = orc.Geometry.of(f)
        orc.adjoint(g, orc.forward(g, f.x_true))
        pairs += 2 * f.pairs
    tr = time.perf_counter() - t
    out["ragged64_per_application"] = {"seconds_all_frames_A_and_AT": tr, "pairs_per_s": pairs / tr,
                                       "landweber20_extrapolated_s": 20.5 * tr}
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_2404_10928_gb300 import phantoms as ph
    from oracle import oracle as orc
    prob = ph.ring_vessels()
    geo = orc.Geometry.of(prob)
    y = ph.add_noise(orc.forward(geo, prob.x_true), prob.noise_unit, prob.noise_level)
    y = y.astype(np.float32).astype(np.float64)
    os.environ.setdefault("OMP_NUM_THREADS", str(cores()))
    n_it = 2  # bounded sample per step: 2 CGLS iterations = 6 operator applications
    for _ in range(args.warmup):
        orc.cgls(geo, y, 0)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        orc.cgls(geo, y, n_it)
        times.append(time.perf_counter() - t)
    apps = cgls_applications(n_it)
    total = sum(times)
    value = prob.pairs * apps * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{n_it} CGLS iterations per step "
                   f"({apps} operator applications of {prob.pairs} pairs)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle", "sample": f"{n_it} CGLS iterations per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def read_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 2 and parts[0] == kernel and not line.startswith("#"):
            try:
                return float(parts[1])
            except ValueError:
                return None
    return None


def read_per_pair(kernel: str):
    """(thread instructions, shared-memory wavefronts) per pixel-sensor pair of
    `kernel` from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", "ncu_per_pair.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and not line.startswith("#"):
            try:
                return float(parts[1]), float(parts[2])
            except ValueError:
                return None
    return None


def _events_time(torch, fn, reps: int) -> float:
    """Median seconds of fn() measured with CUDA events on the current stream."""
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(times)


def bench_batched(torch, tuner, n_iter: int = 20, reps: int = 3) -> dict:
    """Ragged time series: 64 frames (grids 128^2..512^2, 128-512 ring sensors,
    1024-4096 samples at 40 MHz, FP16 traces), 20 projected Landweber iterations
    each: one persistent batched launch vs a loop of per-frame reconstructions."""
    from paper_2404_10928_gb300 import phantoms as ph
    from paper_2404_10928_gb300.api import Batch, Plan
    frames = ph.ragged_time_series()
    plans, ys, xs, omegas = [], [], [], []
    for prob in frames:
        t = tuner.best(prob)
        plan = Plan.from_problem(prob, adj_cluster=1, fwd_sensors_per_cta=t["fwd_sensors_per_cta"])
        x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
        ys.append(plan.forward(x_true).to(torch.float16))
        omegas.append(1.0 / plan.power_iteration(20))
        xs.append(torch.zeros(prob.n_pixels, dtype=torch.float32, device="cuda"))
        plans.append(plan)
    pairs = sum(p.pairs for p in frames) * (2 * n_iter + 1)

    def plain():
        for plan, y, x, om in zip(plans, ys, xs, omegas):
            x.zero_()
            plan.reconstruct(y, "landweber", n_iter, omega=om, out=x)

    batch = Batch(plans)

    def batched():
        for x in xs:
            x.zero_()
        batch.landweber(ys, xs, omegas, n_iter)

    def plain_cgls():
        for plan, y, x in zip(plans, ys, xs):
            x.zero_()
            plan.reconstruct(y, "cgls", n_iter, out=x)

    def batched_cgls():
        for x in xs:
            x.zero_()
        batch.reconstruct(ys, xs, "cgls", n_iter)

    plain()
    batched()
    t_plain = _events_time(torch, plain, reps)
    t_batch = _events_time(torch, batched, reps)
    plain_cgls()
    batched_cgls()
    t_plain_c = _events_time(torch, plain_cgls, reps)
    t_batch_c = _events_time(torch, batched_cgls, reps)
    batch.close()
    for p in plans:
        p.close()
    pairs_c = sum(p.pairs for p in frames) * (2 + 2 * n_iter)
    return {"workload": f"{len(frames)} ragged frames (grids 128^2..512^2, 128-512 ring sensors, "
                        f"1024-4096 samples, FP16 y), {n_iter} projected Landweber iterations; "
                        f"the same frames by {n_iter} CGLS iterations",
            "frames_per_s_batched": len(frames) / t_batch,
            "frames_per_s_plain": len(frames) / t_plain,
            "speedup": t_plain / t_batch,
            "pairs_per_s_batched": pairs / t_batch,
            "launches_batched": 2, "launches_plain": len(frames),
            "cgls": {"frames_per_s_batched": len(frames) / t_batch_c,
                     "frames_per_s_plain": len(frames) / t_plain_c,
                     "speedup": t_plain_c / t_batch_c,
                     "pairs_per_s_batched": pairs_c / t_batch_c},
            "timing": f"median of {reps}, CUDA events"}


def bench_differentiable(torch, reps: int = 3) -> dict:
    """Speed-of-sound calibration workload: batch of 8 vessel frames (256^2,
    128-sensor ring, 2048 samples); loss ||A(x;c) - p||^2 + 1e-3 TV(x) and its
    gradients in x and c; and a 10-step unrolled Landweber with per-step
    checkpointing, differentiated end to end."""
    from paper_2404_10928_gb300 import phantoms as ph
    from paper_2404_10928_gb300.api import Plan
    from paper_2404_10928_gb300.autograd import UnrolledLandweber, data_tv_loss
    frames = ph.ring_vessels_batch()
    prob = frames[0]
    plan = Plan.from_problem(prob, c=1500.0)
    xs = torch.tensor(np.stack([f.x_true for f in frames]), dtype=torch.float32, device="cuda")
    plan.set_sound_speed(1540.0)
    ps = torch.stack([plan.forward(x) for x in xs])
    plan.set_sound_speed(1500.0)
    omega = 1.0 / plan.power_iteration(20)

    def loss_grad():
        x = xs.clone().requires_grad_(True)
        c = torch.tensor(1500.0, dtype=torch.float64, device="cuda", requires_grad=True)
        data_tv_loss(plan, x, c, ps, 1e-3).backward()

    net = UnrolledLandweber(plan, 10, omega, checkpointing=True)

    def unrolled():
        c = torch.tensor(1500.0, dtype=torch.float64, device="cuda", requires_grad=True)
        x0 = torch.zeros_like(xs, requires_grad=True)
        (net(x0, ps, c).double() ** 2).sum().backward()

    loss_grad()
    unrolled()
    t_lg = _events_time(torch, loss_grad, reps)
    t_un = _events_time(torch, unrolled, reps)
    plan.close()
    apps_lg = len(frames) * 3           # A; backward A^T and d/dc, per frame
    # per step and frame: A, A^T; recomputed in backward A, A^T; the step's vector-Jacobian
    # product A, A^T, A (residual) and two d/dc gathers
    apps_un = len(frames) * 10 * 9
    return {"workload": "batch of 8 vessel frames, 256^2, 128-sensor ring, 2048 samples, c=1500",
            "loss_grad_ms": t_lg * 1e3, "loss_grad_frames_per_s": len(frames) / t_lg,
            "unrolled10_grad_ms": t_un * 1e3,
            "operator_applications": {"loss_grad": apps_lg, "unrolled10_grad": apps_un},
            "timing": f"median of {reps}, CUDA events"}


def bench_bp_vs_ir(torch, plan, prob, y, x_ir, ir_ms: float, reps: int = 20) -> dict:
    """Back-projection against iterative reconstruction on the benchmark frame
    (the comparison of Sec. 4, Experiment 1, Table 2): the time of one filtered
    back-projection (universal back-projection filter + A^T) against the time of
    the 50-iteration CGLS step measured above, and the error of each image
    against the phantom (the back-projection after its best scalar fit, its
    scale being arbitrary)."""
    out = torch.empty(prob.n_pixels, dtype=torch.float32, device=y.device)
    for _ in range(3):
        plan.backproject(y, "ubp", out=out)
    bp_ms = 1e3 * _events_time(torch, lambda: plan.backproject(y, "ubp", out=out), reps)
    truth = prob.x_true.astype(np.float64)

    def fitted_error(img):
        img = img.cpu().numpy().astype(np.float64)
        scale = float(np.dot(img, truth) / max(np.dot(img, img), 1e-300))
        return float(np.linalg.norm(scale * img - truth) / np.linalg.norm(truth))

    err_bp = fitted_error(out)
    err_das = fitted_error(plan.backproject(y, "none"))
    err_ir = float(np.linalg.norm(x_ir.cpu().numpy().astype(np.float64) - truth)
                   / np.linalg.norm(truth))
    # the full objective of Eq. 8 (L1 and TV terms) by FISTA on the same frame
    sigma2 = plan.power_iteration(50)
    eps = 1e-2
    alpha = 1e-3 * float(plan.adjoint(y).abs().max())
    beta = 0.01 * sigma2 * eps
    tau = 1.0 / (2.0 * sigma2 + 8.0 * beta / eps)
    xf = torch.zeros(prob.n_pixels, dtype=torch.float32, device=y.device)

    def fista():
        xf.zero_()
        plan.reconstruct(y, "fista", 50, out=xf, omega=tau, l1=alpha, tv=beta, tv_eps=eps)

    fista()
    fista_ms = 1e3 * _events_time(torch, fista, 5)
    err_fista = float(np.linalg.norm(xf.cpu().numpy().astype(np.float64) - truth)
                      / np.linalg.norm(truth))
    return {"workload": WORKLOAD.replace("50 CGLS (FP64 reductions)", "BP vs 50 CGLS"),
            "bp_ms": bp_ms, "ir_ms": ir_ms, "ir_over_bp": ir_ms / bp_ms,
            "fista50_l1_tv_ms": fista_ms,
            "rel_error_vs_phantom": {"bp_ubp_best_scaled": err_bp,
                                     "bp_unfiltered_best_scaled": err_das, "ir_cgls50": err_ir,
                                     "fista50_l1_tv": err_fista},
            "paper": "IR/BP time ratio up to ~50x on a Xeon E5-2620 v2 in MATLAB FP64, "
                     "127x127 murine frames (Table 2)",
            "timing": f"median of {reps}, CUDA events (warm L2)"}


def bench_dense(torch, hbm_gbs: float, reps: int = 10) -> dict:
    """The paper's own method at the paper's size (Sec. 4, Experiment 2, Table 4):
    the 6144 x 16384 measurement matrix of a 128x128 frame assembled dense and
    applied with matrix-vector products, in FP64 (the paper's precision) and in
    FP32, against the matrix-free A and A^T on the same geometry."""
    from paper_2404_10928_gb300 import phantoms as ph
    from paper_2404_10928_gb300.api import Plan
    prob = ph.dense_paper_size()
    plan = Plan.from_problem(prob)
    rows, cols = prob.n_sensors * prob.n_samples, prob.n_pixels
    out = {"workload": "128x128 at 0.1 mm, 48-sensor ring R=10 mm, 128 samples at 10 MHz: "
                       "M = 6144 x 16384 (the matrix size of the paper's Table 4)",
           "paper_k40c_fp64_s": {"Mx": 7.8, "MTr": 6.4,
                                 "note": "Table 4 as printed (Tesla K40c, FP64, MATLAB/mex)"}}
    g = torch.Generator(device="cuda").manual_seed(0)
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        m = torch.empty((rows, cols), dtype=dt, device="cuda")
        plan.dense_assemble(dt, out=m)
        t_asm = _events_time(torch, lambda: plan.dense_assemble(dt, out=m), 3)
        v = torch.rand(cols, dtype=dt, device="cuda", generator=g)
        w = torch.rand(rows, dtype=dt, device="cuda", generator=g)
        yo = torch.empty(rows, dtype=dt, device="cuda")
        xo = torch.empty(cols, dtype=dt, device="cuda")
        plan.dense_matvec(m, v, out=yo)
        plan.dense_matvec(m, w, transpose=True, out=xo)
        t_mv = _events_time(torch, lambda: plan.dense_matvec(m, v, out=yo), reps)
        t_mtv = _events_time(torch, lambda: plan.dense_matvec(m, w, transpose=True, out=xo),
                             reps)
        nbytes = rows * cols * m.element_size()
        out[name] = {"assemble_ms": t_asm * 1e3, "Mx_ms": t_mv * 1e3, "MTr_ms": t_mtv * 1e3,
                     "Mx_gbs": nbytes / t_mv / 1e9, "MTr_gbs": nbytes / t_mtv / 1e9,
                     "Mx_frac_hbm": nbytes / t_mv / 1e9 / hbm_gbs,
                     "MTr_frac_hbm": nbytes / t_mtv / 1e9 / hbm_gbs,
                     "Mx_tflops": 2 * rows * cols / t_mv / 1e12}
        del m
        torch.cuda.empty_cache()
    x = torch.rand(cols, device="cuda", generator=g)
    r = torch.rand(rows, device="cuda", generator=g)
    p = torch.empty(rows, device="cuda")
    z = torch.empty(cols, device="cuda")
    plan.forward(x, out=p)
    plan.adjoint(r, out=z)
    out["matrix_free_fp32"] = {"A_ms": _events_time(torch, lambda: plan.forward(x, out=p), reps) * 1e3,
                               "AT_ms": _events_time(torch, lambda: plan.adjoint(r, out=z), reps) * 1e3}
    out["hbm_peak_gbs"] = hbm_gbs
    out["timing"] = f"median of {reps}, CUDA events; M is larger than L2, so every product streams it from HBM"
    plan.close()
    return out


def bench_freq(torch, peak_tflops: float, reps: int = 5) -> dict:
    """The frequency-domain model of Eq. 7 on the 256^2 ring geometry at 256
    frequencies (78 kHz steps up to 20 MHz): forward and adjoint rates in
    pixel-sensor-frequency terms.  Each term costs one complex multiply (the
    phase recurrence) and one complex-by-real accumulate: 10 flop."""
    from paper_2404_10928_gb300 import phantoms as ph
    from paper_2404_10928_gb300.api import Plan
    prob = ph.ring_vessels()
    q, f0, df = 256, 78125.0, 78125.0
    plan = Plan.from_problem(prob)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(prob.n_pixels, device="cuda", generator=g)
    p = torch.empty((prob.n_sensors, q), dtype=torch.complex64, device="cuda")
    z = torch.empty(prob.n_pixels, device="cuda")
    plan.freq_forward(x, q, f0, df, out=p)
    plan.freq_adjoint(p, q, f0, df, out=z)
    t_f = _events_time(torch, lambda: plan.freq_forward(x, q, f0, df, out=p), reps)
    t_a = _events_time(torch, lambda: plan.freq_adjoint(p, q, f0, df, out=z), reps)
    plan.close()
    terms = prob.pairs * q
    return {"workload": "256x256 at 0.1 mm, 256-sensor ring R=20 mm, 256 frequencies "
                        "78 kHz..20 MHz",
            "terms_per_application": terms,
            "forward_ms": t_f * 1e3, "adjoint_ms": t_a * 1e3,
            "forward_terms_per_s": terms / t_f, "adjoint_terms_per_s": terms / t_a,
            "forward_frac_fp32": terms * 10 / t_f / 1e12 / peak_tflops,
            "adjoint_frac_fp32": terms * 10 / t_a / 1e12 / peak_tflops,
            "timing": f"median of {reps}, CUDA events"}


def bench_volume(torch, tuner, peak_tflops: float, reps: int = 3) -> dict:
    """3D workload: 128^3 voxels at 0.2 mm, 32x32 planar array (0.8 mm pitch,
    5 mm from the volume), 1024 samples; A and A^T rates, a 30-iteration CGLS
    and the speed-of-sound derivative."""
    from paper_2404_10928_gb300 import phantoms as ph
    from paper_2404_10928_gb300.api import Plan
    prob = ph.planar_vessel_tree()
    t = tuner.best(prob)
    plan = Plan.from_problem(prob, **tuner.plan_options(t))
    x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
    y = plan.forward(x_true)
    # operator timings on a dense image (an all-zero tile skips its work, so the
    # sparse phantom itself would flatter the forward gather)
    x = torch.rand(prob.n_pixels, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    p = torch.empty_like(y)
    g = torch.empty_like(x)
    out = torch.zeros_like(x)
    plan.adjoint(y, out=g)
    plan.reconstruct(y, "cgls", 30, out=out)
    t_f = _events_time(torch, lambda: plan.forward(x, out=p), reps)
    t_a = _events_time(torch, lambda: plan.adjoint(y, out=g), reps)

    def cgls():
        out.zero_()
        plan.reconstruct(y, "cgls", 30, out=out)

    t_c = _events_time(torch, cgls, reps)
    t_d = _events_time(torch, lambda: plan.dc(x, y), reps)
    plan.close()
    # the same 30 CGLS iterations with the sensors split into two shards of 512
    # (pa_shard_cgls_*, host-driven, the two sums formed by the library's
    # accumulate mode): the cost of the split's extra launches on one GPU
    from paper_2404_10928_gb300 import shard
    ranges = shard.sensor_ranges(prob.n_sensors, 2)
    shards = shard.shard_plans(prob, ranges, **tuner.plan_options(t))
    yr = y.reshape(prob.n_sensors, -1)
    ys = [yr[b:e].contiguous() for b, e in ranges]
    shard.sharded_cgls(shards, ys, 30)
    t_s = _events_time(torch, lambda: shard.sharded_cgls(shards, ys, 30), reps)
    for sp in shards:
        sp.close()
    pairs = prob.pairs
    return {"workload": "3D 128^3 at 0.2 mm, 32x32 planar array 0.8 mm pitch 5 mm from the "
                        "volume, 1024 samples, vessel tree",
            "pairs_per_application": pairs,
            "autotuned": tuner.plan_options(t),
            "forward_ms": t_f * 1e3, "adjoint_ms": t_a * 1e3,
            "forward_pairs_per_s": pairs / t_f, "adjoint_pairs_per_s": pairs / t_a,
            "adjoint_frac_fp32": pairs * FLOPS_PER_PAIR / t_a / 1e12 / peak_tflops,
            "forward_frac_fp32": pairs * FLOPS_PER_PAIR / t_f / 1e12 / peak_tflops,
            "adjoint_frac_sfu": pairs * MUFU_PER_PAIR / t_a / 1e12
                                / (peak_tflops / (2 * 128) * SFU_PER_SM_CLK),
            "forward_frac_sfu": pairs * MUFU_PER_PAIR / t_f / 1e12
                                / (peak_tflops / (2 * 128) * SFU_PER_SM_CLK),
            "cgls30_ms": t_c * 1e3, "cgls30_frames_per_s": 1.0 / t_c, "dc_ms": t_d * 1e3,
            "cgls30_two_sensor_shards_ms": t_s * 1e3,
            "timing": f"median of {reps}, CUDA events (inputs far larger than L2)"}


def run_gpu(args):
    import torch

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2404_10928_gb300 import build, phantoms as ph
    build.build()
    from paper_2404_10928_gb300.api import Plan

    prob = ph.ring_vessels(seed=1002)
    # each rank reconstructs its own frame (same geometry, its own noise draw)
    noise = frame_noise(prob.noise_unit.shape, rank)
    from paper_2404_10928_gb300.autotune import Autotuner
    tuner = Autotuner()  # cache: PA_TUNE_CACHE, else ~/.cache/pa_gb300/autotune.json
    tuned = tuner.best(prob)
    plan = Plan.from_problem(prob, **tuner.plan_options(tuned))
    x_true = torch.tensor(prob.x_true, dtype=torch.float32, device=dev)
    clean = plan.forward(x_true).cpu().numpy().astype(np.float64)
    y_host = ph.add_noise(clean, noise, prob.noise_level).astype(np.float32)
    y = torch.tensor(y_host, device=dev)
    x = torch.zeros(prob.n_pixels, dtype=torch.float32, device=dev)
    flush = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_sum = torch.zeros((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def evict_l2():
        # reading a buffer twice the size of L2 leaves only its (clean) lines
        # there: the next step finds none of its data cached and has no dirty
        # lines to write back
        torch.sum(flush, dim=0, out=flush_sum)

    def step():
        x.zero_()
        plan.reconstruct(y, "cgls", N_ITER, out=x)

    for i in range(max(args.warmup, 0)):
        step()
    step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            evict_l2()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(dist, dev, sum(step_ms))
    apps = cgls_applications(N_ITER)
    pairs_rank = prob.pairs * apps * args.steps
    value = whole_job_rate(pairs_rank, world, total_ms * 1e-3)

    # end to end through the host-buffer entry point (pinned buffers, copies inside)
    y_pin = torch.empty(y_host.shape, dtype=torch.float32).pin_memory()
    y_pin.copy_(torch.from_numpy(y_host))
    x_pin = torch.zeros(prob.n_pixels, dtype=torch.float32).pin_memory()
    y_np, x_np = y_pin.numpy(), x_pin.numpy()
    for _ in range(2):
        x_np[:] = 0
        plan.reconstruct_host(y_np, "cgls", N_ITER, x_out=x_np)
    torch.cuda.synchronize()
    e2e_t = 0.0
    for _ in range(args.steps):
        x_np[:] = 0
        evict_l2()  # the same L2 state as the device-timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.reconstruct_host(y_np, "cgls", N_ITER, x_out=x_np)  # waits for the result
        e2e_t += time.perf_counter() - t0
    e2e_t = max_over_ranks(dist, dev, e2e_t)
    e2e_value = whole_job_rate(pairs_rank, world, e2e_t)

    # the gathers' own device time: back-to-back launches in the CGLS form, one
    # pair of events around each run (no event between launches)
    x_dense = torch.rand(prob.n_pixels, device=dev,
                         generator=torch.Generator(device=dev).manual_seed(0))
    gt = plan.time_gathers(x_dense, y, reps=100)
    fwd_ms, adj_ms = gt["fwd_ms"], gt["adj_ms"]

    extra = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extra["bp_vs_ir"] = bench_bp_vs_ir(torch, plan, prob, y, x, total_ms / args.steps)
        extra["batched"] = bench_batched(torch, tuner)
        extra["differentiable"] = bench_differentiable(torch)
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        sm_max = json.load(open(pk)).get("sm_max_mhz", 2070.0) if os.path.exists(pk) else 2070.0
        peak = (torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * sm_max
                * 1e6 / 1e12)
        extra["volume3d"] = bench_volume(torch, tuner, peak)
        hbm = json.load(open(pk)).get("hbm_gbs", 6800.0) if os.path.exists(pk) else 6800.0
        extra["dense_paper_size"] = bench_dense(torch, hbm)
        extra["frequency_domain"] = bench_freq(torch, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs, n_it = oracle_sample(prob, y_host.astype(np.float64))
        cpu = {"value": rate, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", cores())),
               "kind": "oracle",
               "sample": f"FP64 oracle CGLS, {n_it} iterations ({cgls_applications(n_it)} operator "
                         f"applications) of the same frame, {secs:.1f} s"}
        if not args.no_extras:
            cpu["detail"] = oracle_detail(prob, y_host.astype(np.float64))
            cpu["detail"]["ring256_cgls_all_cores_vs_1core"] = (
                rate / cpu["detail"]["ring256_cgls_1core"]["pairs_per_s"])

    if rank == 0:
        import json as _json
        peaks = {}
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pk):
            peaks = _json.load(open(pk))
        props = torch.cuda.get_device_properties(dev)
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        peak_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
        flops = prob.pairs * FLOPS_PER_PAIR
        fwd_tf = flops / (fwd_ms * 1e-3) / 1e12
        adj_tf = flops / (adj_ms * 1e-3) / 1e12
        dom_is_adj = adj_ms >= fwd_ms
        achieved = adj_tf if dom_is_adj else fwd_tf
        kname = "k_adjoint<2>" if dom_is_adj else "k_fwd_tile<2>+k_fwd_combine"
        peak_src = (f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x "
                    f"{sm_max:.0f} MHz (MEASURED_PEAKS.json has no FP32 figure)")
        sfu_peak = props.multi_processor_count * SFU_PER_SM_CLK * sm_max * 1e6  # results/s

        def ceilings(kernel, ms):
            """The gather's pairs/s against the issue ceiling (4 warp instructions =
            128 thread instructions per SM per clock) and the shared-memory one
            (one wavefront per SM per clock), with its profiled per-pair counts."""
            pp = read_per_pair(kernel)
            if pp is None:
                return None
            ipp, wpp = pp
            got = prob.pairs / (ms * 1e-3) / (props.multi_processor_count * sm_max * 1e6)
            return {"pairs_per_sm_clock": got,
                    "issue": {"instr_per_pair": ipp, "ceiling": 128.0 / ipp,
                              "frac": got * ipp / 128.0},
                    "shared": {"wavefronts_per_pair": wpp, "ceiling": 1.0 / wpp,
                               "frac": got * wpp},
                    "source": "profiles/ncu_per_pair.txt (ncu counters of the CGLS form)"}

        def sfu(ms):  # the SFU (XU pipe) roofline of a gather: two MUFU results per pair
            got = prob.pairs * MUFU_PER_PAIR / (ms * 1e-3)
            return {"achieved": got, "peak": sfu_peak, "unit": "MUFU results/s",
                    "frac": got / sfu_peak, "ops_per_pair": MUFU_PER_PAIR,
                    "peak_source": f"derived: {props.multi_processor_count} SMs x "
                                   f"{SFU_PER_SM_CLK} MUFU results x {sm_max:.0f} MHz"}
        clk = clocks.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_rank_per_step": 1,
                       "l2": "evicted before every timed step (a 256 MiB read), value and e2e alike",
                       "pairs_per_application": prob.pairs,
                       "applications_per_step": apps, "parallelism": f"frame-parallel x{world}"},
            "frames_per_s": world * args.steps / (total_ms * 1e-3),
            "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved,
                         "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": read_traffic(kname), "peak_source": peak_src,
                         "flops_per_launch": flops, "sfu": sfu(adj_ms if dom_is_adj else fwd_ms),
                         "ceilings": ceilings(kname, adj_ms if dom_is_adj else fwd_ms)},
            "roofline_adjoint": {"bound": "alu", "kernel": "k_adjoint<2>", "achieved": adj_tf,
                                 "peak": peak_tflops, "unit": "TFLOP/s",
                                 "frac": adj_tf / peak_tflops,
                                 "traffic": read_traffic("k_adjoint<2>"),
                                 "peak_source": peak_src, "flops_per_launch": flops,
                                 "sfu": sfu(adj_ms), "ceilings": ceilings("k_adjoint<2>", adj_ms)},
            "kernels": {"adjoint_ms_per_launch": adj_ms, "forward_ms_per_application": fwd_ms,
                        "adjoint_pairs_per_s": prob.pairs / (adj_ms * 1e-3),
                        "forward_pairs_per_s": prob.pairs / (fwd_ms * 1e-3),
                        "gathers_share_of_step": (adj_ms + fwd_ms) * apps / 2
                        / (total_ms / args.steps) if world == 1 else None,
                        "timed_on": "pa_plan_time_gathers: 100 back-to-back launches of each "
                                    "gather in its CGLS form (dense random image, the bench "
                                    "traces), one pair of CUDA events per run, warm L2"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(y_host.nbytes + prob.n_pixels * 4),
                    "d2h_bytes_per_step": int(prob.n_pixels * 4)},
            "autotuned": tuner.plan_options(tuned),
            "gpu_launches": cgls_launches(N_ITER) * args.steps,
            "clocks": clk,
            "wall_s_timed_region": t_wall,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_case(kind: str) -> int:
    """Small fixed workloads for ncu captures.  "2d" / "3d": one plan (the
    256x256 ring with 8 CTAs of 4 compute warps per adjoint cluster and 24
    sensors on 128 threads per forward CTA, or a 64^3 planar array with 2 CTAs
    of 8 warps and 64 sensors on 128 threads), then A on a dense random image and
    A^T on random traces, three times each.  "dense": the 6144 x 16384 matrix
    (FP64 and FP32), M x and M^T r twice each.  "freq": the frequency-domain
    model on the 256x256 ring at 256 frequencies, forward and adjoint twice
    each.  "batch": the first 16 frames of the ragged time series (FP16 y) as
    one persistent batched launch of 4 projected Landweber iterations, twice.
    "dc": on the 64^3 planar plan, the speed-of-sound derivative and the
    smoothed TV with its gradient, three times each.  "cgls": the benchmark step
    itself (256x256 ring, 50 CGLS iterations) three times.  "cgls3d": the 128^3
    planar workload's 30-iteration CGLS twice.  Prints nothing."""
    import torch

    from paper_2404_10928_gb300 import phantoms as ph
    from paper_2404_10928_gb300.api import Batch, Plan

    torch.cuda.set_device(0)
    if kind == "cgls3d":
        # the 128^3 planar workload's step: its autotuned decomposition (2-CTA
        # adjoint clusters of 8 warps, forward items of 128 sensors on 128
        # threads), y = A x_true, two 30-iteration CGLS reconstructions
        prob = ph.planar_vessel_tree()
        with Plan.from_problem(prob, adj_cluster=2, fwd_sensors_per_cta=128, fwd_threads=128,
                               adj_warps=8) as plan:
            x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
            y = plan.forward(x_true)
            x = torch.zeros(prob.n_pixels, dtype=torch.float32, device="cuda")
            for _ in range(2):
                x.zero_()
                plan.reconstruct(y, "cgls", 30, out=x)
            torch.cuda.synchronize()
            plan.sync_status()
        return 0
    if kind == "cgls":
        # the benchmark step: the 256^2 ring frame, the autotuned decomposition
        # (8-CTA adjoint clusters of 4 compute warps, 24 sensors and 128 threads
        # per forward work item), one warm-up reconstruction (graph capture) and
        # two timed-shape reconstructions of 50 CGLS iterations: 4 + 4 x 50 + 2 =
        # 206 launches each
        prob = ph.ring_vessels()
        with Plan.from_problem(prob, adj_cluster=8, fwd_sensors_per_cta=24, fwd_threads=128,
                               adj_warps=4) as plan:
            x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
            y = plan.forward(x_true)
            x = torch.zeros(prob.n_pixels, dtype=torch.float32, device="cuda")
            for _ in range(3):
                x.zero_()
                plan.reconstruct(y, "cgls", N_ITER, out=x)
            torch.cuda.synchronize()
            plan.sync_status()
        return 0
    if kind == "dc":
        prob = ph.planar_vessel_tree(n=64)
        with Plan.from_problem(prob, adj_cluster=2) as plan:
            g = torch.Generator(device="cuda").manual_seed(0)
            x = torch.rand(plan.n_pixels, device="cuda", generator=g)
            r = torch.randn(plan.n_sensors * plan.n_samples, device="cuda", generator=g)
            for _ in range(3):
                plan.dc(x, r)
                plan.tv(x, 1e-2)
            torch.cuda.synchronize()
            plan.sync_status()
        return 0
    if kind == "batch":
        plans, ys, xs, omegas = [], [], [], []
        for prob in ph.ragged_time_series()[:16]:
            plan = Plan.from_problem(prob, adj_cluster=1)
            x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
            ys.append(plan.forward(x_true).to(torch.float16))
            omegas.append(1.0 / plan.power_iteration(20))
            xs.append(torch.zeros(prob.n_pixels, dtype=torch.float32, device="cuda"))
            plans.append(plan)
        batch = Batch(plans)
        for _ in range(2):
            batch.landweber(ys, xs, omegas, 4)
        torch.cuda.synchronize()
        batch.close()
        for plan in plans:
            plan.sync_status()
            plan.close()
        return 0
    if kind == "dense":
        prob = ph.dense_paper_size()
        with Plan.from_problem(prob) as plan:
            rows, cols = prob.n_sensors * prob.n_samples, prob.n_pixels
            for dt in (torch.float64, torch.float32):
                m = plan.dense_assemble(dt)
                v = torch.rand(cols, dtype=dt, device="cuda")
                w = torch.rand(rows, dtype=dt, device="cuda")
                for _ in range(2):
                    plan.dense_matvec(m, v)
                    plan.dense_matvec(m, w, transpose=True)
                torch.cuda.synchronize()
                del m
            plan.sync_status()
        return 0
    if kind == "freq":
        prob = ph.ring_vessels()
        with Plan.from_problem(prob) as plan:
            x = torch.rand(prob.n_pixels, device="cuda")
            for _ in range(2):
                p = plan.freq_forward(x, 256, 78125.0, 78125.0)
                plan.freq_adjoint(p, 256, 78125.0, 78125.0)
            torch.cuda.synchronize()
            plan.sync_status()
        return 0
    if kind == "2d":
        prob = ph.ring_vessels()
        plan = Plan.from_problem(prob, adj_cluster=8, fwd_sensors_per_cta=24, fwd_threads=128,
                                 adj_warps=4)
    else:
        prob = ph.planar_vessel_tree(n=64)
        plan = Plan.from_problem(prob, adj_cluster=2, fwd_sensors_per_cta=64, fwd_threads=128,
                                 adj_warps=8)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(plan.n_pixels, device="cuda", generator=g)
    y = torch.randn(plan.n_sensors * plan.n_samples, device="cuda", generator=g)
    p = torch.empty_like(y)
    z = torch.empty_like(x)
    for _ in range(3):
        plan.forward(x, out=p)
        plan.adjoint(y, out=z)
    torch.cuda.synchronize()
    plan.sync_status()
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)  # ~1.2 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and differentiable workloads")
    ap.add_argument("--profile-case", choices=["2d", "3d", "dense", "freq", "batch", "dc", "cgls",
                                                "cgls3d"],
                    help="only run the small gather workload used for ncu captures")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
