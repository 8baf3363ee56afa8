"""Batched persistent Landweber over ragged frames (one cooperative launch for all
frames and iterations) against the single-frame path and the FP64 oracle."""
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


def _ragged_frames():
    R = ph.ring_sensors
    return [
        ph.custom(2, (64, 48), (1e-4, 1e-4), R(24, 5e-3), 700, seed=61),
        ph.custom(2, (100, 90), (1e-4, 1e-4), R(40, 8e-3), 1500, seed=62),
        ph.custom(2, (37, 53), (1e-4, 1e-4), R(13, 4e-3), 301, seed=63),
        ph.custom(2, (33, 33), (1e-4, 1e-4), R(7, 3e-3), 90, seed=64),  # truncated arrivals
    ]


def test_batch_matches_single_frame_and_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Batch, Plan
    frames = _ragged_frames()
    n_iter = 20
    ys, omegas, refs = [], [], []
    for prob in frames:
        geo = orc.Geometry.of(prob)
        y16 = orc.forward(geo, prob.x_true).astype(np.float16)
        lam = orc.power_iteration(geo, ph.power_start(prob.n_pixels), 50)
        x_ref, h_ref = orc.landweber(geo, y16.astype(np.float64), n_iter, omega=1.0 / lam)
        ys.append(y16)
        omegas.append(1.0 / lam)
        refs.append((x_ref, h_ref))
    plans = [Plan.from_problem(p, y_dtype="f16", adj_cluster=1) for p in frames]
    try:
        yd = [torch.tensor(y, dtype=torch.float16, device="cuda") for y in ys]
        single = []
        for plan, y, om in zip(plans, yd, omegas):
            x, h = plan.reconstruct(y, "landweber", n_iter, omega=om, history=True)
            single.append((x.cpu().numpy(), h))
        xb = [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda") for p in frames]
        with Batch(plans) as batch:
            hist = batch.landweber(yd, xb, omegas, n_iter, history=True)
            # a replay of the captured graph gives the same bits
            xb2 = [torch.zeros_like(x) for x in xb]
            batch.landweber(yd, xb2, omegas, n_iter)
            torch.cuda.synchronize()
        for f, prob in enumerate(frames):
            got = xb[f].cpu().numpy()
            assert np.array_equal(got, single[f][0]), f
            assert np.array_equal(got, xb2[f].cpu().numpy()), f
            np.testing.assert_allclose(hist[f], single[f][1], rtol=1e-12)
            assert rel_l2(got, refs[f][0]) <= RECON_TOL, (f, rel_l2(got, refs[f][0]))
            np.testing.assert_allclose(hist[f], refs[f][1], rtol=RECON_TOL)
    finally:
        for p in plans:
            p.close()


def test_batch_time_series_sample(torch_cuda):
    """Four frames of the 64-frame ragged time series (grids up to 512^2, up to
    512 sensors and 4096 samples, FP16 traces): batched == single-frame, bitwise."""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Batch, Plan
    frames = ph.ragged_time_series(n_frames=4)
    plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
    try:
        ys, xs_single, xs_batch, omegas = [], [], [], []
        for plan, prob in zip(plans, frames):
            x_true = torch.tensor(prob.x_true, dtype=torch.float32, device="cuda")
            ys.append(plan.forward(x_true).to(torch.float16))
            omegas.append(1.0 / plan.power_iteration(20))
            xs_single.append(plan.reconstruct(ys[-1], "landweber", 3, omega=omegas[-1]))
            xs_batch.append(torch.zeros(prob.n_pixels, dtype=torch.float32, device="cuda"))
        with Batch(plans) as batch:
            batch.landweber(ys, xs_batch, omegas, 3, history=True)
        for a, b in zip(xs_single, xs_batch):
            assert torch.equal(a, b)
    finally:
        for p in plans:
            p.close()


def test_batch_cgls_matches_single_frame_and_oracle(torch_cuda):
    """Batched CGLS (one persistent launch for all frames and iterations) on
    four ragged frames: 5 iterations within RECON_TOL of the oracle and of the
    single-frame path; 20 iterations within the perturbed-oracle envelope of
    each frame (past the knee FP32-level perturbations move CGLS by >1e-3);
    the clamp, the residual history and a graph replay."""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Batch, Plan
    from helpers import CGLS_ENVELOPE_FACTOR, cgls_spread, cgls_with_iterates
    frames = _ragged_frames()
    ys = [f32(orc.forward(orc.Geometry.of(p), p.x_true)) for p in frames]
    plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
    try:
        yd = [torch.tensor(y, dtype=torch.float32, device="cuda") for y in ys]
        zeros = lambda: [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda")
                         for p in frames]
        with Batch(plans) as batch:
            x5 = zeros()
            h5 = batch.reconstruct(yd, x5, "cgls", 5, nonneg=False, history=True)
            x20 = zeros()
            h20 = batch.reconstruct(yd, x20, "cgls", 20, nonneg=False, history=True)
            x20b = zeros()
            batch.reconstruct(yd, x20b, "cgls", 20, nonneg=False)  # graph replay
            x20c = zeros()
            batch.reconstruct(yd, x20c, "cgls", 20, nonneg=True)
        for f, (prob, plan) in enumerate(zip(frames, plans)):
            geo = orc.Geometry.of(prob)
            ref, href = cgls_with_iterates(orc, geo, ys[f], 20)
            single = plan.reconstruct(yd[f], "cgls", 5, nonneg=False).cpu().numpy()
            got5 = x5[f].cpu().numpy()
            assert rel_l2(got5, ref[4]) <= RECON_TOL, (f, rel_l2(got5, ref[4]))
            assert rel_l2(got5, single) <= RECON_TOL, (f, rel_l2(got5, single))
            np.testing.assert_allclose(h5[f], href[:6], rtol=RECON_TOL, atol=RECON_TOL * href[0])
            dx, dh, _ = cgls_spread(orc, geo, ys[f], 20, ref, href)
            got20 = x20[f].cpu().numpy()
            e = rel_l2(got20, ref[19])
            assert e <= max(CGLS_ENVELOPE_FACTOR * dx[19], RECON_TOL), (f, e, dx[19])
            assert np.max(np.abs(h20[f] - href)) / href[0] <= max(CGLS_ENVELOPE_FACTOR * dh.max(),
                                                                 RECON_TOL)
            assert np.all(np.diff(h20[f]) <= 1e-7 * h20[f][0])
            assert torch.equal(x20[f], x20b[f])
            assert np.array_equal(x20c[f].cpu().numpy(), np.maximum(got20, 0.0))
    finally:
        for p in plans:
            p.close()


def test_batch_cgls_3d_and_fista_rejected(torch_cuda):
    torch = torch_cuda
    from paper_2404_10928_gb300 import _lib
    from paper_2404_10928_gb300.api import Batch, Plan
    frames = [ph.custom(3, (20, 17, 12), (2e-4, 2e-4, 2e-4), ph.planar_array(6, 5, 0.8e-3, 3.5e-3),
                        200, seed=81),
              ph.custom(3, (33, 9, 17), (1.5e-4, 2e-4, 1e-4), ph.planar_array(4, 7, 0.6e-3, -3e-3),
                        151, seed=82)]
    ys = [f32(orc.forward(orc.Geometry.of(p), p.x_true)) for p in frames]
    plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
    try:
        yd = [torch.tensor(y, dtype=torch.float32, device="cuda") for y in ys]
        xs = [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda") for p in frames]
        with Batch(plans) as batch:
            batch.reconstruct(yd, xs, "cgls", 5)
            with pytest.raises(_lib.PAError) as exc:
                batch.reconstruct(yd, xs, "fista", 5)
            assert exc.value.status == _lib.PA_ERR_UNSUPPORTED
        for f, prob in enumerate(frames):
            ref, _ = orc.cgls(orc.Geometry.of(prob), ys[f], 5)
            assert rel_l2(xs[f].cpu().numpy(), ref) <= RECON_TOL
    finally:
        for p in plans:
            p.close()


def test_batch_time_series_frames_full_size_against_oracle(torch_cuda):
    """Four frames of the 64-frame ragged time series at their full sizes (grids up
    to 512^2, up to 512 sensors and 4096 samples, FP16 traces), batched Landweber
    (the persistent launch the benchmark times) and batched CGLS, 5 iterations,
    against the FP64 oracle at the reconstruction tolerance."""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Batch, Plan
    frames = ph.ragged_time_series(n_frames=4)
    plans = [Plan.from_problem(p, adj_cluster=1) for p in frames]
    try:
        ys, omegas, geos = [], [], []
        for prob in frames:
            geo = orc.Geometry.of(prob)
            y16 = orc.forward(geo, prob.x_true).astype(np.float16)
            ys.append(y16)
            omegas.append(1.0 / orc.power_iteration(geo, ph.power_start(prob.n_pixels), 20))
            geos.append(geo)
        yd = [torch.tensor(y, dtype=torch.float16, device="cuda") for y in ys]
        xl = [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda") for p in frames]
        xc = [torch.zeros(p.n_pixels, dtype=torch.float32, device="cuda") for p in frames]
        with Batch(plans) as batch:
            batch.reconstruct(yd, xl, "landweber", 5, omegas=omegas)
            batch.reconstruct(yd, xc, "cgls", 5)
        for f, geo in enumerate(geos):
            y64 = ys[f].astype(np.float64)
            ref_l, _ = orc.landweber(geo, y64, 5, omega=omegas[f])
            ref_c, _ = orc.cgls(geo, y64, 5)
            assert rel_l2(xl[f].cpu().numpy(), ref_l) <= RECON_TOL, f
            assert rel_l2(xc[f].cpu().numpy(), ref_c) <= RECON_TOL, f
    finally:
        for p in plans:
            p.close()
