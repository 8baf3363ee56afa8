"""Frequency-domain model of Eq. 7 (pa_freq_forward / pa_freq_adjoint) against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from helpers import f32, rel_l2

pytestmark = pytest.mark.gpu

# FP32 phase bound: 2 pi f_max |pixel - tile centre| / c * 2^-24 ~ 1.1e-5 rad at
# 20 MHz on 32x32 tiles of 0.1 mm; relative L2 errors sit near that bound
FREQ_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10928_gb300 import build
    build.build()
    return torch


def _plan(prob):
    from paper_2404_10928_gb300.api import Plan
    return Plan.from_problem(prob)


CASES = {
    "ragged-37x53-ring13": (ph.custom(2, (37, 53), (1e-4, 1e-4), ph.ring_sensors(13, 4e-3), 301,
                                      seed=43), 40, 0.25e6, 0.5e6),
    "ring64-disks-20MHz": (ph.custom(2, (64, 64), (1e-4, 1e-4), ph.ring_sensors(32, 6e-3), 512,
                                     seed=44), 64, 0.3125e6, 0.3125e6),
    "3d-20x17x12-planar": (ph.custom(3, (20, 17, 12), (2e-4, 2e-4, 2e-4),
                                     ph.planar_array(6, 5, 0.8e-3, 3.5e-3), 200, seed=45),
                           33, 0.5e6, 0.25e6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_freq_forward_adjoint_match_oracle(torch_cuda, name):
    torch = torch_cuda
    prob, q, f0, df = CASES[name]
    geo = orc.Geometry.of(prob)
    rng = np.random.default_rng(46)
    x = f32(prob.x_true if prob.x_true is not None else rng.uniform(0, 1, prob.n_pixels))
    pq = (rng.standard_normal((prob.n_sensors, q)) + 1j * rng.standard_normal((prob.n_sensors, q)))
    pq = pq.astype(np.complex64).astype(np.complex128)
    with _plan(prob) as plan:
        p_gpu = plan.freq_forward(torch.tensor(x, dtype=torch.float32, device="cuda"), q, f0, df)
        g_gpu = plan.freq_adjoint(torch.tensor(pq, dtype=torch.complex64, device="cuda"), q, f0, df)
        p2 = plan.freq_forward(torch.tensor(x, dtype=torch.float32, device="cuda"), q, f0, df)
        torch.cuda.synchronize()
        plan.sync_status()
        p_gpu, g_gpu, p2 = p_gpu.cpu().numpy(), g_gpu.cpu().numpy(), p2.cpu().numpy()
    assert np.array_equal(p_gpu, p2)  # bitwise reproducible
    p_ref = orc.freq_forward(geo, x, q, f0, df)
    g_ref = orc.freq_adjoint(geo, pq, q, f0, df)
    assert rel_l2(p_gpu, p_ref) <= FREQ_TOL, rel_l2(p_gpu, p_ref)
    assert rel_l2(g_gpu, g_ref) <= FREQ_TOL, rel_l2(g_gpu, g_ref)
