"""Host logic of the sensor-sharded CGLS driver (shard.sharded_cgls) on CPU:
the shard steps restated on the oracle's operators, several shards in one
process (the library's accumulate mode), argument checks."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from test_multiprocess import _OracleShard


def _problem():
    return ph.custom(2, (22, 18), (1e-4, 1e-4), ph.ring_sensors(11, 3e-3), 180, seed=93)


def _shards(prob, n):
    import torch
    from paper_2404_10928_gb300 import shard
    y = orc.forward(orc.Geometry.of(prob), prob.x_true)
    out, ys = [], []
    for b, e in shard.sensor_ranges(prob.n_sensors, n):
        out.append(_OracleShard(orc.Geometry(prob.dim, prob.shape, prob.spacing, prob.origin,
                                             prob.sensors[b:e], prob.c, prob.fs, prob.n_samples,
                                             prob.t0, prob.amp_scale)))
        ys.append(torch.from_numpy(np.ascontiguousarray(y[b:e])))
    return out, ys, y


@pytest.mark.parametrize("n_shards", [1, 3, 5])
def test_local_shards_reproduce_unsharded_cgls(n_shards):
    from paper_2404_10928_gb300 import shard
    prob = _problem()
    shards, ys, y = _shards(prob, n_shards)
    x, h = shard.sharded_cgls(shards, ys, 7, nonneg=True, history=True)
    x_ref, h_ref = orc.cgls(orc.Geometry.of(prob), y, 7, nonneg=True)
    assert np.linalg.norm(x.numpy() - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    np.testing.assert_allclose(h, h_ref, rtol=1e-10)
    assert x.numpy().min() >= 0.0


def test_warm_start_and_zero_iterations():
    import torch
    from paper_2404_10928_gb300 import shard
    prob = _problem()
    shards, ys, y = _shards(prob, 2)
    x0 = np.random.default_rng(3).uniform(0.0, 0.5, prob.n_pixels)
    x, h = shard.sharded_cgls(shards, ys, 0, x0=torch.from_numpy(x0), nonneg=False,
                              history=True)
    np.testing.assert_array_equal(x.numpy(), x0)        # no iteration: x0 itself
    r = y - orc.forward(orc.Geometry.of(prob), x0)
    assert h.shape == (1,) and abs(h[0] - np.sum(r * r)) <= 1e-10 * np.sum(r * r)
    x4, _ = shard.sharded_cgls(shards, ys, 4, x0=torch.from_numpy(x0), nonneg=False,
                               history=True)
    x_ref, _ = orc.cgls(orc.Geometry.of(prob), y, 4, x0=x0, nonneg=False)
    assert np.linalg.norm(x4.numpy() - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_argument_checks():
    from paper_2404_10928_gb300 import shard
    prob = _problem()
    shards, ys, _ = _shards(prob, 2)
    with pytest.raises(ValueError):
        shard.sharded_cgls([], [], 3)
    with pytest.raises(ValueError):
        shard.sharded_cgls(shards, ys[:1], 3)
    other = _OracleShard(orc.Geometry.of(ph.custom(2, (10, 10), (1e-4, 1e-4),
                                                   ph.ring_sensors(5, 3e-3), 100, seed=1)))
    with pytest.raises(ValueError):
        shard.sharded_cgls([shards[0], other], [ys[0], ys[1]], 3)
