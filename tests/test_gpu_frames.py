"""Several frames on one plan (one launch per operator for all frames) against
the single-frame entry points (bitwise) and the FP64 oracle."""
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


def _dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


CASES = {
    "ragged-2d": lambda: ph.custom(2, (37, 53), (1e-4, 1e-4), ph.ring_sensors(13, 4e-3), 301, seed=3),
    "3d": lambda: ph.custom(3, (20, 17, 12), (2e-4, 2e-4, 2e-4),
                            ph.planar_array(6, 5, 0.8e-3, 3.5e-3), 200, seed=8),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_frames_match_single_frame_calls_and_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Plan
    prob = CASES[name]()
    geo = orc.Geometry.of(prob)
    F = 3
    rng = np.random.default_rng(11)
    xs = f32(rng.uniform(0.0, 1.0, (F, prob.n_pixels)))
    ps = f32(rng.standard_normal((F, prob.n_sensors, prob.n_samples)))
    with Plan.from_problem(prob) as plan:
        xf = plan.forward_frames(_dev(torch, xs)).cpu().numpy()
        gf = plan.adjoint_frames(_dev(torch, ps)).cpu().numpy()
        single_f = [plan.forward(_dev(torch, xs[f])).cpu().numpy() for f in range(F)]
        single_g = [plan.adjoint(_dev(torch, ps[f])).cpu().numpy() for f in range(F)]
        plan.sync_status()
    for f in range(F):
        assert np.array_equal(xf[f].ravel(), single_f[f].ravel())   # same kernels, same order
        assert np.array_equal(gf[f], single_g[f])
        assert rel_l2(xf[f], orc.forward(geo, xs[f])) <= OP_TOL
        assert rel_l2(gf[f], orc.adjoint(geo, ps[f])) <= OP_TOL


def test_residual_axpy_dc_tv_and_landweber_step(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Plan
    prob = CASES["ragged-2d"]()
    geo = orc.Geometry.of(prob)
    F = 3
    rng = np.random.default_rng(12)
    xs = f32(rng.uniform(0.0, 1.0, (F, prob.n_pixels)))
    ys = f32(rng.standard_normal((F, prob.n_sensors, prob.n_samples)))
    tg = f32(rng.standard_normal((F, prob.n_pixels)))
    nx, ny = prob.shape[0], prob.shape[1]
    with Plan.from_problem(prob) as plan:
        r, sq = plan.residual_frames(_dev(torch, xs), _dev(torch, ys), norms=True)
        r, sq = r.cpu().numpy(), sq.cpu().numpy()
        out = plan.adjoint_axpy_frames(_dev(torch, ys), -0.7, xin=_dev(torch, xs),
                                       tvg=_dev(torch, tg), tv_weight=0.3, nonneg=True)
        out = out.cpu().numpy()
        dc = plan.dc_frames(_dev(torch, xs), _dev(torch, ys), scale=2.0).item()
        tv, tvg = plan.tv_frames(_dev(torch, xs), 1e-3)
        tv, tvg = tv.cpu().numpy(), tvg.cpu().numpy()
        step = plan.landweber_step_frames(_dev(torch, xs), _dev(torch, ys), 3e-8, True).cpu().numpy()
    dc_ref = 0.0
    for f in range(F):
        r_ref = ys[f] - orc.forward(geo, xs[f])
        assert rel_l2(r[f], r_ref) <= OP_TOL
        assert abs(sq[f] - np.sum(r_ref ** 2)) <= 2 * OP_TOL * np.sum(r_ref ** 2)
        o_ref = np.maximum(xs[f] - 0.7 * orc.adjoint(geo, ys[f]) + 0.3 * tg[f], 0.0)
        assert rel_l2(out[f], o_ref) <= OP_TOL
        dc_ref += 2.0 * orc.dc(geo, xs[f], ys[f])
        img = xs[f].reshape(ny, nx)
        assert abs(tv[f] - orc.tv(img, 1e-3)) <= 1e-6 * orc.tv(img, 1e-3)
        assert rel_l2(tvg[f], orc.tv_grad(img, 1e-3).ravel()) <= OP_TOL
        s_ref = np.maximum(xs[f] + 3e-8 * orc.adjoint(geo, r_ref), 0.0)
        assert rel_l2(step[f], s_ref) <= OP_TOL
    flips = sum(2.0 * orc.dc_flip_bound(geo, xs[f], ys[f], 5e-5) for f in range(F))
    assert abs(dc - dc_ref) <= 1e-3 * abs(dc_ref) + flips, (dc, dc_ref, flips)


def test_frames_argument_checks(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300 import _lib
    from paper_2404_10928_gb300.api import Plan
    prob = CASES["ragged-2d"]()
    lib = _lib.load()
    with Plan.from_problem(prob) as plan:
        assert lib.pa_forward_frames(plan._h, 0, None, None, None) == _lib.PA_ERR_INVALID_ARG
        too_many = 65535 // prob.n_sensors + 1
        assert lib.pa_forward_frames(plan._h, too_many, 1, 1, None) == _lib.PA_ERR_UNSUPPORTED
        with pytest.raises(ValueError):
            plan.forward_frames(torch.zeros(prob.n_pixels + 1, device="cuda"))
