"""Failure paths, exercised without faulting or hanging the GPU.

* A bounded device wait that runs out: the batched launch's grid-barrier limit
  is set to zero, so a CTA that reaches a barrier before the others gives up
  at its first poll instead of waiting; the launch ends, pa_batch_landweber
  reports PA_ERR_TIMEOUT, and the next call (default limit) is exact again.
* Device allocations that fail: pa_debug_fail_allocations makes the n-th
  allocation report out-of-memory; every entry point that allocates returns
  PA_ERR_OOM, frees what it had taken, and leaves the library usable.
"""
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


def _frames():
    R = ph.ring_sensors
    return [ph.custom(2, (64, 48), (1e-4, 1e-4), R(24, 5e-3), 700, seed=71),
            ph.custom(2, (100, 90), (1e-4, 1e-4), R(40, 8e-3), 1500, seed=72),
            ph.custom(2, (37, 53), (1e-4, 1e-4), R(13, 4e-3), 301, seed=73)]


def _batch_inputs(torch, frames):
    ys, omegas = [], []
    for prob in frames:
        geo = orc.Geometry.of(prob)
        ys.append(torch.tensor(f32(orc.forward(geo, prob.x_true)), dtype=torch.float32,
                               device="cuda"))
        omegas.append(1.0 / orc.power_iteration(geo, ph.power_start(prob.n_pixels), 30))
    return ys, omegas


def test_batch_barrier_wait_limit_gives_up_and_recovers(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300 import _lib
    from paper_2404_10928_gb300.api import Batch, Plan
    frames = _frames()
    ys, omegas = _batch_inputs(torch, frames)
    plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
    try:
        zeros = lambda: [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda")
                         for p in frames]
        with Batch(plans) as batch:
            batch.set_wait_limit(0.0)
            with pytest.raises(_lib.PAError) as exc:
                batch.landweber(ys, zeros(), omegas, 4, history=True)
            assert exc.value.status == _lib.PA_ERR_TIMEOUT
            batch.set_wait_limit(2.0)
            xa = zeros()
            ha = batch.landweber(ys, xa, omegas, 4, history=True)
        with Batch(plans) as fresh:
            xb = zeros()
            hb = fresh.landweber(ys, xb, omegas, 4, history=True)
        for a, b in zip(xa, xb):
            assert torch.equal(a, b)
        assert np.array_equal(ha, hb)
        for plan in plans:
            plan.sync_status()
    finally:
        for p in plans:
            p.close()


def _free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_plan_and_workspace_allocation_failures(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300 import _lib
    from paper_2404_10928_gb300.api import Plan
    lib = _lib.load()
    prob = ph.ring_vessels()  # a 16 MB plan: a leaked table or window buffer shows
    small = _frames()[2]
    geo = orc.Geometry.of(small)
    y = f32(orc.forward(geo, small.x_true))
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    Plan.from_problem(small).close()  # module load and kernel set-up happen here
    free0 = _free_bytes(torch)
    try:
        failures = 0
        for after in range(64):
            _lib.check(lib.pa_debug_fail_allocations(after), "pa_debug_fail_allocations")
            try:
                plan = Plan.from_problem(prob)
            except _lib.PAError as e:
                assert e.status == _lib.PA_ERR_OOM, e
                failures += 1
                continue
            plan.close()
            break
        _lib.check(lib.pa_debug_fail_allocations(-1), "pa_debug_fail_allocations")
        assert failures >= 10  # each of the plan's allocations failed once
        # the reconstruction workspace: allocated on first use, partially when
        # a later allocation fails; a retry completes it
        with Plan.from_problem(small) as plan:
            for after in (0, 3):
                _lib.check(lib.pa_debug_fail_allocations(after), "pa_debug_fail_allocations")
                with pytest.raises(_lib.PAError) as exc:
                    plan.reconstruct(yd, "cgls", 3)
                assert exc.value.status == _lib.PA_ERR_OOM
            _lib.check(lib.pa_debug_fail_allocations(-1), "pa_debug_fail_allocations")
            x = plan.reconstruct(yd, "cgls", 3).cpu().numpy()
        assert rel_l2(x, orc.cgls(geo, y, 3)[0]) <= RECON_TOL
    finally:
        lib.pa_debug_fail_allocations(-1)
    assert abs(_free_bytes(torch) - free0) <= 8 << 20


def test_batch_allocation_failures(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300 import _lib
    from paper_2404_10928_gb300.api import Batch, Plan
    lib = _lib.load()
    frames = _frames()
    ys, omegas = _batch_inputs(torch, frames)
    plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
    try:
        failures = 0
        for after in range(32):
            lib.pa_debug_fail_allocations(after)
            try:
                batch = Batch(plans)
            except _lib.PAError as e:
                assert e.status == _lib.PA_ERR_OOM, e
                failures += 1
                continue
            lib.pa_debug_fail_allocations(-1)
            xs = [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda") for p in frames]
            batch.landweber(ys, xs, omegas, 2)
            batch.close()
            break
        assert failures >= 5 + len(frames)
    finally:
        lib.pa_debug_fail_allocations(-1)
        for p in plans:
            p.close()
