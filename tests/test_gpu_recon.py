"""GPU Landweber / CGLS / power iteration against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from helpers import (CGLS_ENSEMBLE, CGLS_ENVELOPE_FACTOR, OP_TOL, RECON_TOL, cgls_spread,
                     cgls_with_iterates, f32, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10928_gb300 import build
    build.build()
    return torch


def _plan(prob, **kw):
    from paper_2404_10928_gb300.api import Plan
    return Plan.from_problem(prob, **kw)


def _dev(torch, a, dtype=None):
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float32, device="cuda")


@pytest.fixture(scope="module")
def disks():
    prob = ph.linear_array_disks()
    geo = orc.Geometry.of(prob)
    y = f32(orc.forward(geo, prob.x_true))
    v0 = f32(ph.power_start(prob.n_pixels))
    lam = orc.power_iteration(geo, v0, 50)
    return prob, geo, y, v0, lam


def test_power_iteration(torch_cuda, disks):
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    with _plan(prob) as plan:
        lam_gpu = plan.power_iteration(50, _dev(torch, v0))
    assert abs(lam_gpu - lam) <= OP_TOL * lam, (lam_gpu, lam)


def test_landweber_given_step(torch_cuda, disks):
    """10 projected Landweber steps (the linear-array disk workload), step 1/sigma^2."""
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    x_ref, h_ref = orc.landweber(geo, y, 10, omega=1.0 / lam)
    with _plan(prob) as plan:
        x, h = plan.reconstruct(_dev(torch, y), "landweber", 10, omega=1.0 / lam, history=True)
        x = x.cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL, atol=RECON_TOL * h_ref[0])
    assert np.all(np.diff(h) <= 1e-7 * h[0])
    assert np.all(x >= 0.0)


def test_landweber_own_power_iteration(torch_cuda, disks):
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    x_ref, _ = orc.landweber(geo, y, 10, omega=1.0 / lam)
    with _plan(prob) as plan:
        x = plan.reconstruct(_dev(torch, y), "landweber", 10, omega=0.0, power_iters=50,
                             power_v0=_dev(torch, v0)).cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)


@pytest.fixture(scope="module")
def vessels():
    prob = ph.ring_vessels()
    geo = orc.Geometry.of(prob)
    clean = orc.forward(geo, prob.x_true)
    y = f32(ph.add_noise(clean, prob.noise_unit, prob.noise_level))
    return prob, geo, y


def test_cgls_ring_vessels_early(torch_cuda, vessels):
    """CGLS before the semi-convergence knee: parity with the FP64 oracle at 1e-4."""
    torch = torch_cuda
    prob, geo, y = vessels
    x_ref, h_ref = orc.cgls(geo, y, 5)
    with _plan(prob) as plan:
        x, h = plan.reconstruct(_dev(torch, y), "cgls", 5, history=True)
    assert rel_l2(x.cpu().numpy(), x_ref) <= RECON_TOL
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL)


def test_pcgls_ring_vessels_early(torch_cuda, vessels):
    """Projected CGLS (restart every 3) on the full 256^2 ring workload with 1%
    noise, 5 iterations, with the benchmark's decomposition: parity with the
    FP64 oracle at 1e-4."""
    torch = torch_cuda
    prob, geo, y = vessels
    x_ref, h_ref = orc.pcgls(geo, y, 5, restart=3)
    with _plan(prob, adj_cluster=8, fwd_sensors_per_cta=24, fwd_threads=128,
               adj_warps=4) as plan:
        x, h = plan.reconstruct(_dev(torch, y), "pcgls", 5, restart=3, history=True)
    assert rel_l2(x.cpu().numpy(), x_ref) <= RECON_TOL
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL)


def test_sharded_cgls_ring_vessels_early(torch_cuda, vessels):
    """The full 256^2 ring workload with its 256 sensors split into 4 shards
    (sensor-sharded CGLS, one process): 5 iterations against the oracle's
    unsharded CGLS at 1e-4."""
    torch = torch_cuda
    from paper_2404_10928_gb300 import shard
    prob, geo, y = vessels
    x_ref, h_ref = orc.cgls(geo, y, 5)
    ranges = shard.sensor_ranges(prob.n_sensors, 4)
    plans = shard.shard_plans(prob, ranges)
    yr = y.reshape(prob.n_sensors, -1)
    try:
        x, h = shard.sharded_cgls(plans, [_dev(torch, np.ascontiguousarray(yr[b:e]))
                                          for b, e in ranges], 5, history=True)
    finally:
        for p in plans:
            p.close()
    assert rel_l2(x.cpu().numpy(), x_ref) <= RECON_TOL
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL)


def test_cgls_ring_vessels_full(torch_cuda, vessels):
    """CGLS on the full 256^2 ring workload with 1% noise, at 10, 20 and 50
    iterations.  Past the semi-convergence knee FP32-level perturbations move
    CGLS by 1e-3 and more (tests/test_cgls_sensitivity.py), so x and the
    residual history are held to CGLS_ENVELOPE_FACTOR times the spread of the
    perturbed oracle ensemble (helpers.cgls_spread), computed here on the same
    frame."""
    torch = torch_cuda
    prob, geo, y = vessels
    ref, href = cgls_with_iterates(orc, geo, y, 50)
    dx, dh, _ = cgls_spread(orc, geo, y, 50, ref, href)
    with _plan(prob) as plan:
        yd = _dev(torch, y)
        for n in (10, 20, 50):
            x, h = plan.reconstruct(yd, "cgls", n, nonneg=False, history=True)
            x = x.cpu().numpy()
            e = rel_l2(x, ref[n - 1])
            assert e <= CGLS_ENVELOPE_FACTOR * dx[n - 1], (n, e, dx[n - 1])
            eh = np.max(np.abs(h - href[:n + 1])) / href[0]
            assert eh <= CGLS_ENVELOPE_FACTOR * dh[:n + 1].max(), (n, eh, dh[:n + 1].max())
            assert np.all(np.diff(h) <= 1e-7 * h[0])
        # the benchmark's setting: the same 50 iterations, clamped once at the end
        xc = plan.reconstruct(yd, "cgls", 50).cpu().numpy()
    assert np.array_equal(xc, np.maximum(x, 0.0).astype(np.float32))
    # same reconstruction quality against the phantom
    x_ref = np.maximum(ref[-1], 0.0)
    e_gpu, e_ref = rel_l2(xc, prob.x_true), rel_l2(x_ref, prob.x_true)
    assert abs(e_gpu - e_ref) <= 0.02 * e_ref, (e_gpu, e_ref)


def test_graph_direct_and_host_paths_agree(torch_cuda, vessels):
    """Graph replay, direct launches and the host-buffer entry point give
    bitwise identical results (fixed-order reductions, no atomics)."""
    torch = torch_cuda
    prob, geo, y = vessels
    with _plan(prob) as plan:
        yd = _dev(torch, y)
        a = plan.reconstruct(yd, "cgls", 8, use_graph=True).cpu().numpy()
        b = plan.reconstruct(yd, "cgls", 8, use_graph=True).cpu().numpy()  # replay
        c = plan.reconstruct(yd, "cgls", 8, use_graph=False).cpu().numpy()
        d = plan.reconstruct_host(np.ascontiguousarray(y, dtype=np.float32), "cgls", 8)
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)


def test_zero_iterations_and_warm_start(torch_cuda, disks):
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    rng = np.random.default_rng(3)
    x0 = f32(rng.normal(size=prob.n_pixels))
    with _plan(prob) as plan:
        xl = plan.reconstruct(_dev(torch, y), "landweber", 0, x0=_dev(torch, x0), omega=1.0 / lam)
        xc = plan.reconstruct(_dev(torch, y), "cgls", 0, x0=_dev(torch, x0))
        xw, hw = plan.reconstruct(_dev(torch, y), "cgls", 5, x0=_dev(torch, x0), nonneg=False,
                                  history=True)
    assert np.array_equal(xl.cpu().numpy(), x0.astype(np.float32))  # untouched
    assert np.array_equal(xc.cpu().numpy(), np.maximum(x0, 0).astype(np.float32))
    x_ref, h_ref = orc.cgls(geo, y, 5, x0=x0, nonneg=False)
    assert rel_l2(xw.cpu().numpy(), x_ref) <= RECON_TOL
    np.testing.assert_allclose(hw, h_ref, rtol=RECON_TOL, atol=RECON_TOL * h_ref[0])


def test_f16_measurements(torch_cuda, disks):
    """Measured traces stored as FP16 (the ragged time-series workload's format);
    both sides consume the same quantised values, arithmetic stays FP32."""
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    y16 = y.astype(np.float16)
    x_ref, _ = orc.landweber(geo, y16.astype(np.float64), 10, omega=1.0 / lam)
    with _plan(prob, y_dtype="f16") as plan:
        x = plan.reconstruct(_dev(torch, y16, torch.float16), "landweber", 10,
                             omega=1.0 / lam).cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL


def test_cgls_3d_small(torch_cuda):
    """3D planar-array vessel tree at 32^3 (the 128^3 workload's geometry, scaled):
    5 CGLS iterations at 1e-4; 30 iterations within the perturbed-oracle envelope."""
    torch = torch_cuda
    prob = ph.planar_vessel_tree(n=32)
    geo = orc.Geometry.of(prob)
    y = f32(orc.forward(geo, prob.x_true))
    ref, href = cgls_with_iterates(orc, geo, y, 30)
    dx, dh, _ = cgls_spread(orc, geo, y, 30, ref, href)
    with _plan(prob) as plan:
        g5, gh5 = plan.reconstruct(_dev(torch, y), "cgls", 5, nonneg=False, history=True)
        g30, gh30 = plan.reconstruct(_dev(torch, y), "cgls", 30, nonneg=False, history=True)
    assert rel_l2(g5.cpu().numpy(), ref[4]) <= RECON_TOL
    np.testing.assert_allclose(gh5, href[:6], rtol=RECON_TOL)
    g30 = g30.cpu().numpy()
    assert rel_l2(g30, ref[29]) <= CGLS_ENVELOPE_FACTOR * dx[29], (rel_l2(g30, ref[29]), dx[29])
    assert np.max(np.abs(gh30 - href)) / href[0] <= CGLS_ENVELOPE_FACTOR * dh.max()
    assert np.all(np.diff(gh30) <= 1e-7 * gh30[0])
    assert rel_l2(g30, prob.x_true) <= 2.0 * rel_l2(ref[29], prob.x_true)


def test_cgls_planar_128_full_size(torch_cuda):
    """The 3D workload at full size: 128^3 voxels at 0.2 mm, 32x32 planar array,
    1024 samples, 30 CGLS iterations (2.15 G pixel-sensor pairs per operator
    application).  5 iterations at 1e-4; after 30, x within the envelope of an
    oracle run whose operator outputs carry noise at the operator tolerance, and
    the objective ||r_30||^2 within CGLS_ENVELOPE_FACTOR times that run's (FP32
    CGLS on this noise-free problem converges more slowly than FP64)."""
    torch = torch_cuda
    prob = ph.planar_vessel_tree()
    geo = orc.Geometry.of(prob)
    y = f32(orc.forward(geo, prob.x_true))
    ref, href = cgls_with_iterates(orc, geo, y, 30)
    member = CGLS_ENSEMBLE[1]  # operator outputs perturbed at OP_TOL
    its, hist = cgls_with_iterates(orc, geo, y, 30, **member)
    with _plan(prob) as plan:
        yd = _dev(torch, y)
        g5 = plan.reconstruct(yd, "cgls", 5, nonneg=False).cpu().numpy()
        g30, gh30 = plan.reconstruct(yd, "cgls", 30, nonneg=False, history=True)
    g30 = g30.cpu().numpy()
    assert rel_l2(g5, ref[4]) <= RECON_TOL, rel_l2(g5, ref[4])
    spread = rel_l2(its[29], ref[29])
    assert rel_l2(g30, ref[29]) <= CGLS_ENVELOPE_FACTOR * spread, (rel_l2(g30, ref[29]), spread)
    assert gh30[-1] <= CGLS_ENVELOPE_FACTOR * max(hist[-1], href[-1]), (gh30[-1], hist[-1],
                                                                         href[-1])
    assert np.all(np.diff(gh30) <= 1e-7 * gh30[0])


@pytest.mark.parametrize("alpha_rel,beta_rel,nonneg", [(0.02, 0.0, True), (0.02, 0.05, True),
                                                       (0.01, 0.05, False)])
def test_fista_full_objective(torch_cuda, disks, alpha_rel, beta_rel, nonneg):
    """30 FISTA steps on the full objective of Eq. 8 (data, L1 and smoothed TV)."""
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    eps = 1e-2
    alpha = alpha_rel * float(np.abs(orc.adjoint(geo, y)).max())
    beta = beta_rel * lam * eps  # TV curvature 8 beta / eps: 0.4 of the data term's 2 lam
    tau = 1.0 / (2.0 * lam + 8.0 * beta / eps)
    x_ref, h_ref = orc.fista(geo, y, 30, tau, alpha, beta, eps, nonneg=nonneg)
    with _plan(prob) as plan:
        x, h = plan.reconstruct(_dev(torch, y), "fista", 30, omega=tau, nonneg=nonneg,
                                history=True, l1=alpha, tv=beta, tv_eps=eps)
        x = x.cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL, atol=RECON_TOL * h_ref[0])
    if nonneg:
        assert x.min() >= 0.0


def test_fista_default_step_from_power_iteration(torch_cuda, disks):
    # omega <= 0: tau = 1 / (2 sigma^2 + 8 beta / eps), sigma^2 from the power iteration
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    eps, beta = 1e-2, 0.05 * lam * 1e-2
    alpha = 0.02 * float(np.abs(orc.adjoint(geo, y)).max())
    tau = 1.0 / (2.0 * lam + 8.0 * beta / eps)
    x_ref, _ = orc.fista(geo, y, 20, tau, alpha, beta, eps)
    with _plan(prob) as plan:
        x = plan.reconstruct(_dev(torch, y), "fista", 20, omega=0.0, power_iters=50,
                             power_v0=_dev(torch, v0), l1=alpha, tv=beta, tv_eps=eps)
        x = x.cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)


@pytest.mark.parametrize("restart,nonneg", [(0, True), (3, True), (1, True), (0, False)])
def test_pcgls_matches_oracle(torch_cuda, disks, restart, nonneg):
    """Projected, restarted CGLS (x >= 0 every step, r recomputed from x) on the
    linear-array disk workload: 5 iterations against the oracle at 1e-4."""
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    x_ref, h_ref = orc.pcgls(geo, y, 5, restart=restart, project=nonneg)
    with _plan(prob) as plan:
        x, h = plan.reconstruct(_dev(torch, y), "pcgls", 5, nonneg=nonneg, restart=restart,
                                history=True)
        x = x.cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL, atol=RECON_TOL * h_ref[0])
    if nonneg:
        assert x.min() >= 0.0


def test_pcgls_reaches_nnls_on_a_small_system(torch_cuda):
    """With a restart every step the projected iteration converges to the
    non-negative least-squares solution (scipy's Lawson-Hanson NNLS on the
    explicit matrix), to FP32 accuracy."""
    torch = torch_cuda
    from scipy.optimize import nnls
    prob = ph.custom(2, (6, 5), (1e-4, 1e-4), ph.ring_sensors(9, 1.5e-3), 80, seed=51)
    geo = orc.Geometry.of(prob)
    m = orc.matrix(geo)
    rng = np.random.default_rng(52)
    truth = np.where(rng.uniform(size=prob.n_pixels) < 0.5, rng.uniform(0.2, 1.0, prob.n_pixels),
                     0.0)
    y = f32(m @ truth + 0.05 * rng.standard_normal(m.shape[0]))
    ref = nnls(m, y)[0]
    with _plan(prob) as plan:
        x = plan.reconstruct(_dev(torch, y), "pcgls", 3000, restart=1).cpu().numpy()
    assert np.all(x >= 0.0)
    assert rel_l2(x, ref) <= 1e-3, rel_l2(x, ref)


def test_pcgls_warm_start_is_projected_first(torch_cuda, disks):
    """A start image with negative entries is projected onto x >= 0 before the
    first residual (oracle: x = max(0, x0) first), then 4 projected steps."""
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    rng = np.random.default_rng(71)
    x0 = f32(rng.standard_normal(prob.n_pixels) * 0.05)
    x_ref, h_ref = orc.pcgls(geo, y, 4, restart=2, x0=x0)
    with _plan(prob) as plan:
        x, h = plan.reconstruct(_dev(torch, y), "pcgls", 4, x0=_dev(torch, x0), restart=2,
                                history=True)
        x = x.cpu().numpy()
    assert rel_l2(x, x_ref) <= RECON_TOL, rel_l2(x, x_ref)
    np.testing.assert_allclose(h, h_ref, rtol=RECON_TOL, atol=RECON_TOL * h_ref[0])


def test_cgls_bits_do_not_depend_on_thread_layouts(torch_cuda):
    """Threads and sensors per forward item only move pixels between threads
    and split the sensors differently: 6 CGLS iterations (the forward's
    direction prologue included) give the same bits for every forward layout.
    (The adjoint's warp count regroups the terms of its norm partials, so it is
    held fixed here.)"""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Plan
    prob = ph.custom(2, (70, 45), (1e-4, 1e-4), ph.ring_sensors(33, 5e-3), 400, seed=73)
    y = _dev(torch, f32(orc.forward(orc.Geometry.of(prob), prob.x_true)))
    outs = []
    for nt, aw, spc in ((128, 4, 0), (64, 4, 12), (256, 4, 8), (128, 4, 20)):
        with Plan.from_problem(prob, adj_cluster=2, fwd_threads=nt, adj_warps=aw,
                               fwd_sensors_per_cta=spc) as plan:
            x, h = plan.reconstruct(y, "cgls", 6, history=True)
            outs.append((x, h))
    for x, h in outs[1:]:
        assert torch.equal(x, outs[0][0])
        np.testing.assert_array_equal(h, outs[0][1])


def test_graph_cache_is_bounded(torch_cuda, disks):
    """Each distinct argument set is captured once; past 64 of them the plan
    starts its cache again and every result stays the same."""
    torch = torch_cuda
    prob, geo, y, v0, lam = disks
    yd = _dev(torch, y)
    with _plan(prob) as plan:
        ref = plan.reconstruct(yd, "cgls", 2)
        keep = []
        for i in range(70):
            x = torch.zeros(prob.n_pixels, device="cuda")
            keep.append(x)  # distinct buffers: distinct graphs
            plan.reconstruct(yd, "cgls", 2, out=x)
        torch.cuda.synchronize()
        for x in keep:
            assert torch.equal(x, ref)
