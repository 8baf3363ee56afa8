"""Dense-matrix mode (the paper's own method, Sec. 4 Experiment 2, Table 4)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from helpers import OP_TOL, f32, rel_l2

pytestmark = pytest.mark.gpu


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


# 9x7 pixels: 63 columns, not a multiple of the 16-byte vector width (the
# scalar path); 8x8 pixels: 64 columns (the vector path)
SMALL = {
    "9x7-ring3-k60": ph.custom(2, (9, 7), (1e-4, 1e-4), ph.ring_sensors(3, 2e-3), 60, seed=21),
    "8x8-ring4-k48-t0": ph.custom(2, (8, 8), (1e-4, 1e-4), ph.ring_sensors(4, 2e-3), 48, seed=22,
                                  t0=5 / ph.SAMPLE_RATE),
    "3d-5x4x3-planar": ph.custom(3, (5, 4, 3), (2e-4, 2e-4, 2e-4),
                                 ph.planar_array(2, 2, 0.8e-3, 2e-3), 40, seed=23),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_assembled_matrix_matches_bruteforce(torch_cuda, name):
    torch = torch_cuda
    prob = SMALL[name]
    geo = orc.Geometry.of(prob)
    ref = orc.matrix(geo)  # the hat evaluated at every sample
    with _plan(prob) as plan:
        m64 = plan.dense_assemble(torch.float64).cpu().numpy()
        m32 = plan.dense_assemble(torch.float32).cpu().numpy()
        plan.sync_status()
    assert m64.shape == ref.shape
    assert np.allclose(m64, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert np.array_equal(m32, m64.astype(np.float32))  # one rounding of the FP64 entry


@pytest.mark.parametrize("name", sorted(SMALL))
def test_matvec_pair(torch_cuda, name):
    torch = torch_cuda
    prob = SMALL[name]
    rng = np.random.default_rng(24)
    with _plan(prob) as plan:
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
            m = plan.dense_assemble(dt)
            mn = m.cpu().numpy().astype(np.float64)
            v = rng.standard_normal(prob.n_pixels)
            w = rng.standard_normal(prob.n_sensors * prob.n_samples)
            vt = torch.tensor(v, dtype=dt, device="cuda")
            wt = torch.tensor(w, dtype=dt, device="cuda")
            mv = plan.dense_matvec(m, vt).cpu().numpy()
            mtw = plan.dense_matvec(m, wt, transpose=True).cpu().numpy()
            vv = vt.cpu().numpy().astype(np.float64)
            ww = wt.cpu().numpy().astype(np.float64)
            assert rel_l2(mv, mn @ vv) <= tol
            assert rel_l2(mtw, mn.T @ ww) <= tol
            # bitwise reproducible
            assert np.array_equal(mv, plan.dense_matvec(m, vt).cpu().numpy())
            assert np.array_equal(mtw, plan.dense_matvec(m, wt, transpose=True).cpu().numpy())


def test_paper_size_against_oracle_operators(torch_cuda):
    # the 6144 x 16384 matrix of the paper's Table 4: M x = A x and M^T r = A^T r
    torch = torch_cuda
    prob = ph.dense_paper_size()
    geo = orc.Geometry.of(prob)
    rng = np.random.default_rng(25)
    x = f32(prob.x_true)
    r = f32(rng.standard_normal((prob.n_sensors, prob.n_samples)))
    p_ref, g_ref = orc.forward(geo, x), orc.adjoint(geo, r)
    with _plan(prob) as plan:
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, OP_TOL)):
            m = plan.dense_assemble(dt)
            assert m.shape == (6144, 16384)
            p = plan.dense_matvec(m, torch.tensor(x, dtype=dt, device="cuda")).cpu().numpy()
            g = plan.dense_matvec(m, torch.tensor(r.ravel(), dtype=dt, device="cuda"),
                                  transpose=True).cpu().numpy()
            del m
            torch.cuda.empty_cache()
            assert rel_l2(p, p_ref) <= tol, (dt, rel_l2(p, p_ref))
            assert rel_l2(g, g_ref) <= tol, (dt, rel_l2(g, g_ref))
        plan.sync_status()


def test_matvec_unaligned_views(torch_cuda):
    # a matrix and vector starting one element past a 16-byte boundary: M x then
    # takes scalar loads (the 16-byte path needs aligned rows and v); both
    # products still match the FP64 product of the same entries
    torch = torch_cuda
    prob = SMALL["8x8-ring4-k48-t0"]  # 64 columns: aligned rows would take 16-byte loads
    rng = np.random.default_rng(26)
    with _plan(prob) as plan:
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
            m = plan.dense_assemble(dt)
            rows, cols = m.shape
            big = torch.empty(m.numel() + 1, dtype=dt, device="cuda")
            big[1:] = m.reshape(-1)
            vbig = torch.empty(cols + 1, dtype=dt, device="cuda")
            vbig[1:] = torch.tensor(rng.standard_normal(cols), dtype=dt, device="cuda")
            m_off, v_off = big[1:], vbig[1:]
            assert m_off.data_ptr() % 16 != 0 and v_off.data_ptr() % 16 != 0
            mn = m.cpu().numpy().astype(np.float64)
            out = plan.dense_matvec(m_off, v_off).cpu().numpy()
            assert rel_l2(out, mn @ v_off.cpu().numpy().astype(np.float64)) <= tol
            w = torch.tensor(rng.standard_normal(rows), dtype=dt, device="cuda")
            out_t = plan.dense_matvec(m_off, w, transpose=True).cpu().numpy()
            assert rel_l2(out_t, mn.T @ w.cpu().numpy().astype(np.float64)) <= tol
        plan.sync_status()
