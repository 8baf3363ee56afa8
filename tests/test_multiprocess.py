"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups drive the
same helpers the GPU arm uses over NCCL (max over ranks of the job's clock,
whole-job rate, per-rank frames), and the reference arm's rank behaviour."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_s = [0.25, 0.75][rank]  # rank 1 is the slow one
    job_s = bench.max_over_ranks(dist, "cpu", local_s)
    rate = bench.whole_job_rate(1000.0, world, job_s)
    noise = bench.frame_noise((4, 8), rank)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"job_s": job_s, "rate": rate, "noise": noise.tolist()}, f)


def test_two_rank_job_clock_and_rate(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # every rank sees the slowest rank's clock, and the rate counts all ranks' units
    assert res[0]["job_s"] == res[1]["job_s"] == 0.75
    assert res[0]["rate"] == res[1]["rate"] == pytest.approx(2 * 1000.0 / 0.75)
    # frames are sharded: each rank draws its own noise
    assert not np.allclose(res[0]["noise"], res[1]["noise"])


def test_single_process_helpers():
    assert bench.max_over_ranks(None, None, 1.5) == 1.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def _run_reference(rank, world, tmp_path):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", OMP_NUM_THREADS=str(min(8, os.cpu_count() or 1)))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", str(world), "--steps", "1", "--warmup", "0"],
                          capture_output=True, text=True, env=env, cwd=tmp_path, timeout=600)


def test_reference_arm_runs_on_rank0_only(tmp_path):
    # under torchrun with N > 1 the reference arm runs on rank 0 alone; the other
    # ranks exit 0 without work and print nothing
    other = _run_reference(1, 2, tmp_path)
    assert other.returncode == 0 and other.stdout.strip() == ""
    first = _run_reference(0, 2, tmp_path)
    assert first.returncode == 0, first.stderr[-2000:]
    lines = [l for l in first.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


# ----------------------------------------------------------------------------
# Sensor sharding of one large frame, checked with the oracle on two gloo ranks:
# each rank owns half of the sensors, applies A to its own rows (no exchange)
# and A^T to its own traces; the partial images are all-reduced, and so is the
# one scalar ||A p||^2 that CGLS needs per iteration (||A^T r||^2 follows from
# the reduced image on every rank).  The sharded recursion must reproduce the
# unsharded oracle CGLS: the partition changes only the order of sums.
# ----------------------------------------------------------------------------
def _sharded_problem():
    from paper_2404_10928_gb300 import phantoms as ph
    return ph.custom(2, (24, 20), (1e-4, 1e-4), ph.ring_sensors(14, 3e-3), 200, seed=91)


def _sharded_rank(rank, world, port, out_dir, n_iter):
    import torch
    import torch.distributed as dist
    from oracle import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = _sharded_problem()
    full = orc.Geometry.of(prob)
    y_full = orc.forward(full, prob.x_true)
    mine = np.array_split(np.arange(prob.n_sensors), world)[rank]
    geo = orc.Geometry(prob.dim, prob.shape, prob.spacing, prob.origin, prob.sensors[mine],
                       prob.c, prob.fs, prob.n_samples, prob.t0, prob.amp_scale)
    y = y_full[mine]

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        dist.all_reduce(t)
        return t.numpy()

    x = np.zeros(prob.n_pixels)
    r = y - orc.forward(geo, x)
    s = allreduce(orc.adjoint(geo, r))           # the image all-reduce after A^T
    p = s.copy()
    gamma = float(np.sum(s * s))
    deltas = []
    for _ in range(n_iter):
        q = orc.forward(geo, p)                   # own rows, no exchange
        delta = float(allreduce(np.array([np.sum(q * q)]))[0])  # the scalar all-reduce
        deltas.append(delta)
        alpha = gamma / delta
        x = x + alpha * p
        r = r - alpha * q
        s = allreduce(orc.adjoint(geo, r))
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    dist.barrier()
    dist.destroy_process_group()
    np.savez(os.path.join(out_dir, f"shard{rank}.npz"), x=x, deltas=np.array(deltas))


def test_sensor_sharded_cgls_matches_unsharded_oracle(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as orc
    world, n_iter = 2, 6
    mp.spawn(_sharded_rank, args=(world, _free_port(), str(tmp_path), n_iter), nprocs=world,
             join=True)
    prob = _sharded_problem()
    geo = orc.Geometry.of(prob)
    y = orc.forward(geo, prob.x_true)
    ref = []
    orc.cgls(geo, y, n_iter, nonneg=False, iterates=ref)
    res = [np.load(tmp_path / f"shard{r}.npz") for r in range(world)]
    # every rank holds the same image, equal to the unsharded CGLS iterate
    assert np.array_equal(res[0]["x"], res[1]["x"])
    err = np.linalg.norm(res[0]["x"] - ref[-1]) / np.linalg.norm(ref[-1])
    assert err <= 1e-10, err
    # and ||A p||^2 summed over the two shards is the full operator's (first
    # iteration: p = A^T y)
    q = orc.forward(geo, orc.adjoint(geo, y))
    assert abs(res[0]["deltas"][0] - np.sum(q * q)) <= 1e-12 * np.sum(q * q)
