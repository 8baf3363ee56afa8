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
    # the committed ncu summaries the benchmark line reads
    for k in ("k_adjoint<2>", "k_fwd_tile<2>+k_fwd_combine"):
        assert bench.read_traffic(k) > 0
        ipp, wpp = bench.read_per_pair(k)
        assert 9 <= ipp <= 64 and 0 < wpp < 1
    assert bench.read_per_pair("no-such-kernel") is None


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
# Sensor sharding of one large frame: the product's driver
# (paper_2404_10928_gb300.shard.sharded_cgls) on two gloo ranks, each holding
# one or two shards, with the library's shard steps restated on the oracle's
# operators (FP64, CPU).  Each shard applies A to its own rows (no exchange) and
# A^T to its own traces; the partial images and the scalar ||A p||^2 are summed
# over the process's shards and all-reduced over the ranks.  The sharded
# recursion must reproduce the unsharded oracle CGLS: the partition changes
# only the order of sums.
# ----------------------------------------------------------------------------
def _sharded_problem():
    from paper_2404_10928_gb300 import phantoms as ph
    return ph.custom(2, (24, 20), (1e-4, 1e-4), ph.ring_sensors(14, 3e-3), 200, seed=91)


class _OracleShard:
    """The four pa_shard_cgls_* steps of one shard on the oracle's operators."""

    def __init__(self, geo):
        import torch
        self.geo = geo
        self.n_pixels = geo.n_pixels
        self.device = torch.device("cpu")
        self.image_dtype = torch.float64

    def _out(self, t, v, accumulate):
        a = t.numpy()
        a[...] = a + v if accumulate else v

    def shard_cgls_begin(self, n_iter, y, x, s_part, accumulate):
        from oracle import oracle as orc
        self.r = y.numpy().reshape(self.geo.n_sensors, -1) - orc.forward(self.geo, x.numpy())
        self.hist = [float(np.sum(self.r * self.r))]
        self._out(s_part, orc.adjoint(self.geo, self.r), accumulate)

    def shard_cgls_direction(self, it, s, delta_part, accumulate):
        from oracle import oracle as orc
        sv = s.numpy()
        gamma = float(np.sum(sv * sv))
        self.p = sv.copy() if it == 0 else sv + (gamma / self.gamma) * self.p
        self.gamma = gamma
        self.q = orc.forward(self.geo, self.p)
        self._out(delta_part, np.array([np.sum(self.q * self.q)]), accumulate)

    def shard_cgls_update(self, it, delta, x, s_part, accumulate):
        from oracle import oracle as orc
        alpha = self.gamma / float(delta[0])
        if x is not None:
            x.numpy()[...] += alpha * self.p
        self.r = self.r - alpha * self.q
        self.hist.append(float(np.sum(self.r * self.r)))
        self._out(s_part, orc.adjoint(self.geo, self.r), accumulate)

    def shard_cgls_finish(self, x, nonneg, hist, accumulate):
        if hist is not None:
            self._out(hist, np.array(self.hist), accumulate)
        if nonneg:
            x.numpy()[...] = np.maximum(x.numpy(), 0.0)


def _sharded_rank(rank, world, port, out_dir, n_iter, per_rank):
    import torch
    import torch.distributed as dist
    from oracle import oracle as orc
    from paper_2404_10928_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = _sharded_problem()
    y_full = orc.forward(orc.Geometry.of(prob), prob.x_true)
    ranges = shard.sensor_ranges(prob.n_sensors, world * per_rank)[rank * per_rank:
                                                                   (rank + 1) * per_rank]
    shards, ys = [], []
    for b, e in ranges:
        shards.append(_OracleShard(orc.Geometry(prob.dim, prob.shape, prob.spacing, prob.origin,
                                                prob.sensors[b:e], prob.c, prob.fs,
                                                prob.n_samples, prob.t0, prob.amp_scale)))
        ys.append(torch.from_numpy(np.ascontiguousarray(y_full[b:e])))
    x, hist = shard.sharded_cgls(shards, ys, n_iter, nonneg=False,
                                 process_group=dist.group.WORLD, history=True)
    dist.barrier()
    dist.destroy_process_group()
    np.savez(os.path.join(out_dir, f"shard{rank}.npz"), x=x.numpy(), hist=hist)


@pytest.mark.parametrize("per_rank", [1, 2])
def test_sensor_sharded_cgls_matches_unsharded_oracle(tmp_path, per_rank):
    import torch.multiprocessing as mp
    from oracle import oracle as orc
    world, n_iter = 2, 6
    mp.spawn(_sharded_rank, args=(world, _free_port(), str(tmp_path), n_iter, per_rank),
             nprocs=world, join=True)
    prob = _sharded_problem()
    geo = orc.Geometry.of(prob)
    y = orc.forward(geo, prob.x_true)
    ref = []
    x_ref, h_ref = orc.cgls(geo, y, n_iter, nonneg=False, iterates=ref)
    res = [np.load(tmp_path / f"shard{r}.npz") for r in range(world)]
    # every rank holds the same image, equal to the unsharded CGLS iterate
    assert np.array_equal(res[0]["x"], res[1]["x"])
    err = np.linalg.norm(res[0]["x"] - ref[-1]) / np.linalg.norm(ref[-1])
    assert err <= 1e-10, err
    # the residual history summed over the shards is the full problem's
    np.testing.assert_allclose(res[0]["hist"], h_ref, rtol=1e-10)
    assert np.array_equal(res[0]["hist"], res[1]["hist"])


def test_sensor_ranges():
    from paper_2404_10928_gb300 import shard
    assert shard.sensor_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert shard.sensor_ranges(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    for n, k in [(256, 2), (1024, 8), (14, 4)]:
        r = shard.sensor_ranges(n, k)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(e - b for b, e in r) - min(e - b for b, e in r) <= 1
    with pytest.raises(ValueError):
        shard.sensor_ranges(3, 4)
