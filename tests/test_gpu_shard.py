"""Sensor-sharded CGLS (pa_shard_cgls_* driven by shard.sharded_cgls) on one GPU:
shards held by one process, and a one-rank NCCL group, against the FP64 oracle's
unsharded CGLS and against the library's own unsharded CGLS."""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from helpers import RECON_TOL, f32, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10928_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def ring():
    # 72 x 60 grid (ragged against the 32 x 32 tiles), 45-sensor ring, 640 samples
    prob = ph.custom(2, (72, 60), (1e-4, 1e-4), ph.ring_sensors(45, 5e-3), 640, seed=61)
    geo = orc.Geometry.of(prob)
    y = f32(orc.forward(geo, prob.x_true))
    return prob, geo, y


def _shards(torch, prob, y, n_shards):
    from paper_2404_10928_gb300 import shard
    ranges = shard.sensor_ranges(prob.n_sensors, n_shards)
    plans = shard.shard_plans(prob, ranges)
    ys = [torch.tensor(np.ascontiguousarray(y.reshape(prob.n_sensors, -1)[b:e]),
                       dtype=torch.float32, device="cuda") for b, e in ranges]
    return plans, ys


@pytest.mark.parametrize("n_shards", [1, 2, 3])
def test_sharded_cgls_matches_oracle(torch_cuda, ring, n_shards):
    """5 CGLS iterations with the sensors split over 1, 2 or 3 shards (uneven
    sizes) against the oracle's unsharded CGLS at 1e-4, history included."""
    torch = torch_cuda
    from paper_2404_10928_gb300 import shard
    prob, geo, y = ring
    x_ref, h_ref = orc.cgls(geo, y, 5)
    plans, ys = _shards(torch, prob, y, n_shards)
    try:
        x, h = shard.sharded_cgls(plans, ys, 5, history=True)
        x = x.cpu().numpy()
    finally:
        for p in plans:
            p.close()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL, atol=RECON_TOL * h_ref[0])
    assert x.min() >= 0.0


def test_sharded_cgls_repeatable_and_ordered(torch_cuda, ring):
    """The same sharded run twice gives the same bits; calls out of order are
    rejected without touching the plan's state."""
    torch = torch_cuda
    from paper_2404_10928_gb300 import shard
    from paper_2404_10928_gb300._lib import PAError
    prob, geo, y = ring
    plans, ys = _shards(torch, prob, y, 2)
    try:
        a = shard.sharded_cgls(plans, ys, 4, nonneg=False)
        b = shard.sharded_cgls(plans, ys, 4, nonneg=False)
        assert torch.equal(a, b)
        n = prob.n_pixels
        s = torch.zeros(n, device="cuda")
        d = torch.zeros(1, dtype=torch.float64, device="cuda")
        x = torch.zeros(n, device="cuda")
        p = plans[0]
        with pytest.raises(PAError):
            p.shard_cgls_update(0, d, x, s)        # update before begin / direction
        p.shard_cgls_begin(2, ys[0], x, s)
        with pytest.raises(PAError):
            p.shard_cgls_direction(1, s, d)        # wrong iteration
        p.shard_cgls_direction(0, s, d)
        with pytest.raises(PAError):
            p.shard_cgls_direction(0, s, d)        # direction twice
        p.shard_cgls_update(0, d, x, s)
        p.shard_cgls_finish(x, True, None)
        torch.cuda.synchronize()
    finally:
        for p in plans:
            p.close()


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_sharded_cgls_over_a_one_rank_nccl_group(torch_cuda, ring):
    """The all-reduce path (NCCL, one rank holding two shards): an all-reduce
    over one rank leaves the sums alone, so the result equals the local run."""
    torch = torch_cuda
    import torch.distributed as dist
    if not dist.is_nccl_available():
        pytest.skip("NCCL not available")
    from paper_2404_10928_gb300 import shard
    prob, geo, y = ring
    plans, ys = _shards(torch, prob, y, 2)
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0,
                            world_size=1)
    try:
        x_g, h_g = shard.sharded_cgls(plans, ys, 5, process_group=dist.group.WORLD, history=True)
        x_l, h_l = shard.sharded_cgls(plans, ys, 5, history=True)
        assert torch.equal(x_g, x_l)
        np.testing.assert_array_equal(h_g, h_l)
    finally:
        dist.destroy_process_group()
        for p in plans:
            p.close()


def test_sharded_cgls_planar_128_full_size(torch_cuda):
    """The 128^3 volume with its 32 x 32 planar array split into two shards of
    512 sensors: 5 sharded CGLS iterations against the library's unsharded CGLS
    on the same input (the split changes only the order of sums), and the
    residual history against the unsharded one."""
    torch = torch_cuda
    from paper_2404_10928_gb300 import shard
    from paper_2404_10928_gb300.api import Plan
    prob = ph.planar_vessel_tree()
    x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
    with Plan.from_problem(prob) as full:
        y = full.forward(x_true)
        x_u, h_u = full.reconstruct(y, "cgls", 5, history=True)
    ranges = shard.sensor_ranges(prob.n_sensors, 2)
    plans = shard.shard_plans(prob, ranges)
    yr = y.reshape(prob.n_sensors, -1)
    try:
        x_s, h_s = shard.sharded_cgls(plans, [yr[b:e].contiguous() for b, e in ranges], 5,
                                      history=True)
    finally:
        for p in plans:
            p.close()
    err = rel_l2(x_s.cpu().numpy(), x_u.cpu().numpy())
    assert err <= RECON_TOL, err
    np.testing.assert_allclose(h_s, h_u, rtol=RECON_TOL)


def test_sharded_cgls_with_f16_traces(torch_cuda, ring):
    """Shards whose plans take FP16 measured traces (the time-series storage):
    the sharded run equals the unsharded FP16 reconstruction up to the order
    of sums, 5 iterations."""
    torch = torch_cuda
    from paper_2404_10928_gb300 import shard
    from paper_2404_10928_gb300.api import Plan
    prob, geo, y = ring
    y16 = torch.tensor(y.reshape(prob.n_sensors, -1), dtype=torch.float16, device="cuda")
    with Plan.from_problem(prob, y_dtype="f16") as full:
        x_u, h_u = full.reconstruct(y16, "cgls", 5, history=True)
    ranges = shard.sensor_ranges(prob.n_sensors, 3)
    plans = shard.shard_plans(prob, ranges, y_dtype="f16")
    try:
        x_s, h_s = shard.sharded_cgls(plans, [y16[b:e].contiguous() for b, e in ranges], 5,
                                      history=True)
    finally:
        for p in plans:
            p.close()
    assert rel_l2(x_s.cpu().numpy(), x_u.cpu().numpy()) <= 1e-5
    np.testing.assert_allclose(h_s, h_u, rtol=1e-5)
