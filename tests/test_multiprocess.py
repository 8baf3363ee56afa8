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
