"""The allocation-free adjoint (pa_adjoint_static) against the plan-based
adjoint (pa_adjoint), through the C ABI.

pa_adjoint_static serves callers that may not allocate device memory while
running (a memory pool that owns the device, a host framework that forbids
foreign allocations, a fixed real-time budget): it keeps its working memory in
a statically declared device array.  This file is collected last so that a
failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_10928_gb300 import phantoms as ph

from helpers import OP_TOL, rel_l2

pytestmark = pytest.mark.gpu


def _grid(prob):
    from paper_2404_10928_gb300 import _lib
    return _lib.pa_grid(prob.dim, *prob.shape, *prob.spacing, (ctypes.c_double * 3)(*prob.origin))


def test_static_adjoint_matches_plan_adjoint_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10928_gb300 import _lib, build
    from paper_2404_10928_gb300.api import Plan
    build.build()
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream

    # two different geometries in a row: the second call must not see the
    # first call's leftovers in the shared scratch array
    cases = [ph.ring_vessels(),
             ph.custom(2, (37, 53), (1e-4, 1e-4), ph.ring_sensors(13, 4e-3), 301, seed=3,
                       t0=2 / ph.SAMPLE_RATE, amp_scale=0.5)]
    for prob in cases:
        rng = np.random.default_rng(11)
        p = torch.tensor(rng.standard_normal((prob.n_sensors, prob.n_samples)),
                         dtype=torch.float32, device="cuda")
        with Plan.from_problem(prob) as plan:
            ref = plan.adjoint(p).cpu().numpy()
        sensors = np.ascontiguousarray(prob.sensors, dtype=np.float64)
        grid = _grid(prob)
        # plan defaults, then 2-CTA clusters of 4 compute warps
        for opts in (_lib.pa_plan_opts(prob.t0, prob.amp_scale, _lib.PA_F32, 0, 0),
                     _lib.pa_plan_opts(prob.t0, prob.amp_scale, _lib.PA_F32, 2, 0, 0, 4)):
            x = torch.full((prob.n_pixels,), float("nan"), dtype=torch.float32, device="cuda")
            st = lib.pa_adjoint_static(sensors.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       prob.n_sensors, ctypes.byref(grid), prob.c, prob.fs,
                                       prob.n_samples, ctypes.byref(opts), p.data_ptr(),
                                       x.data_ptr(), stream)
            _lib.check(st, "pa_adjoint_static")
            got = x.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_l2(got, ref) <= OP_TOL, rel_l2(got, ref)


def test_static_adjoint_rejects_oversized_geometry():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10928_gb300 import _lib
    lib = _lib.load()
    prob = ph.planar_vessel_tree(n=128)  # ~75 MB of tables and traces
    sensors = np.ascontiguousarray(prob.sensors, dtype=np.float64)
    grid = _grid(prob)
    dummy = torch.zeros(1, device="cuda")
    st = lib.pa_adjoint_static(sensors.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               prob.n_sensors, ctypes.byref(grid), prob.c, prob.fs,
                               prob.n_samples, None, dummy.data_ptr(), dummy.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == _lib.PA_ERR_UNSUPPORTED
    assert b"static scratch" in lib.pa_last_error()
