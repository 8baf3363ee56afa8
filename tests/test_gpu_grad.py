"""Differentiation on the GPU: d/dc kernel, TV kernel, autograd Functions and the
checkpointed unrolled Landweber module, against the FP64 oracle and FP64 finite
differences."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from helpers import OP_TOL, f32, operator_cases, rel_l2

pytestmark = pytest.mark.gpu

# d/dc sums terms g[k0+1] - g[k0] whose tap k0 flips where u crosses an integer:
# the hat's derivative is discontinuous there, and both one-sided values are
# correct for a pair whose FP32 arrival lies within its rounding error of the
# integer.  The comparison allows 1e-3 relative for the FP32 sums plus the
# oracle's bound on what such pairs can change (dc_flip_bound), with DC_DELTA
# well above the FP32 arrival error (< 2e-5 samples for windows of 128).
DC_TOL = 1e-3
DC_DELTA = 5e-5


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


def _dev(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def _dc_cases():
    cases = {k: v for k, v in operator_cases().items()
             if k in ("ragged-37x53-ring13-k301", "truncated-40x40-k90", "t0-amp-33x20")}
    # 3D: sensors off the voxel lattice.  On a lattice-aligned planar array many
    # arrivals fall exactly on a sample, where the hat's derivative jumps and
    # even FP64 rounding decides which side is taken.
    sens = ph.planar_array(6, 5, 0.8e-3, 3.5e-3) + np.array([1.37e-5, 2.91e-5, 1.13e-5])
    cases["3d-20x17x12-planar-offlattice"] = ph.custom(3, (20, 17, 12), (2e-4, 2e-4, 2e-4), sens,
                                                       200, seed=8)
    # the ragged 2D case has pixels whose arrival is exactly an integer (d a
    # multiple of c/fs on the sensor's axis): its flip bound is large, so the
    # same frame is also checked with the ring shifted to a position where no
    # arrival of a nonzero pixel lies within DC_DELTA of an integer
    for j in range(1, 200):
        ring = ph.ring_sensors(13, 4e-3) + j * np.array([1.37e-6, 2.91e-6])
        prob = ph.custom(2, (37, 53), (1e-4, 1e-4), ring, 301, seed=3)
        if _min_integer_gap(prob) > 2 * DC_DELTA:
            cases["ragged-37x53-ring13-offlattice"] = prob
            break
    return cases


def _min_integer_gap(prob, all_pixels=False):
    """Smallest |u - round(u)| over pairs with a nonzero pixel (or any pixel)
    (numpy, FP64)."""
    xs, ys, _ = prob.pixel_axes()
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    nz = np.ones(prob.n_pixels, bool) if all_pixels else prob.x_true.ravel() != 0
    px, py = gx.ravel()[nz], gy.ravel()[nz]
    d = np.hypot(px[None, :] - prob.sensors[:, :1], py[None, :] - prob.sensors[:, 1:])
    u = d * prob.fs / prob.c - prob.t0 * prob.fs
    return float(np.min(np.abs(u - np.rint(u))))


@pytest.mark.parametrize("name", sorted(_dc_cases()))
def test_dc_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    prob = _dc_cases()[name]
    geo = orc.Geometry.of(prob)
    rng = np.random.default_rng(5)
    x = f32(prob.x_true)
    g = f32(rng.standard_normal((prob.n_sensors, prob.n_samples)))
    with _plan(prob) as plan:
        d = plan.dc(_dev(torch, x), _dev(torch, g)).item()
    ref = orc.dc(geo, x, g)
    flips = orc.dc_flip_bound(geo, x, g, DC_DELTA)
    assert abs(d - ref) <= DC_TOL * abs(ref) + flips, (d, ref, flips)


@pytest.mark.parametrize("shape", [(256, 256), (37, 53), (1, 9)])
def test_tv_matches_oracle(torch_cuda, shape):
    torch = torch_cuda
    prob = ph.custom(2, shape, (1e-4, 1e-4), ph.ring_sensors(4, 2e-2), 64, seed=3, density=0.5)
    img = f32(np.random.default_rng(8).uniform(0, 1, prob.n_pixels) * (prob.x_true > 0))
    with _plan(prob) as plan:
        val, grad = plan.tv(_dev(torch, img), 1e-4)
        val, grad = val.item(), grad.cpu().numpy()
    img2 = img.reshape(shape[1], shape[0])
    assert abs(val - orc.tv(img2)) <= 1e-6 * orc.tv(img2)
    assert rel_l2(grad, orc.tv_grad(img2).ravel()) <= OP_TOL


@pytest.mark.parametrize("shape", [(64, 64, 64), (33, 9, 17), (1, 5, 7)])
def test_tv_3d_matches_oracle(torch_cuda, shape):
    """pa_tv on 3D grids (forward differences along x, y and z) against the
    oracle's 3D TV, pinned by finite differences and a hand-worked volume."""
    torch = torch_cuda
    prob = ph.custom(3, shape, (2e-4, 2e-4, 2e-4), ph.planar_array(2, 2, 1e-3, 2e-2), 64, seed=4,
                     density=0.5)
    img = f32(np.random.default_rng(9).uniform(0, 1, prob.n_pixels) * (prob.x_true > 0))
    with _plan(prob) as plan:
        val, grad = plan.tv(_dev(torch, img), 1e-4)
        val, grad = val.item(), grad.cpu().numpy()
    vol = img.reshape(shape[2], shape[1], shape[0])
    assert abs(val - orc.tv(vol)) <= 1e-6 * orc.tv(vol)
    assert rel_l2(grad, orc.tv_grad(vol).ravel()) <= OP_TOL


def _batch(n_frames=2):
    sensors = ph.ring_sensors(11, 4e-3)
    frames = [ph.custom(2, (29, 23), (1e-4, 1e-4), sensors, 260, seed=40 + b) for b in range(n_frames)]
    return frames


def test_autograd_loss_gradients(torch_cuda):
    """d/dx and d/dc of ||A(x;c) - p||^2 + 1e-3 TV(x) over a batch of frames."""
    torch = torch_cuda
    from paper_2404_10928_gb300.autograd import data_tv_loss
    frames = _batch()
    prob = frames[0]
    geo_true = orc.Geometry.of(prob, c=1540.0)
    geo = orc.Geometry.of(prob, c=1500.0)
    xs = np.stack([f32(f.x_true) for f in frames])
    ps = np.stack([f32(orc.forward(geo_true, f.x_true)) for f in frames])
    rng = np.random.default_rng(1)
    x0 = f32(xs + 0.05 * rng.standard_normal(xs.shape))
    with _plan(prob) as plan:
        x = _dev(torch, x0).requires_grad_(True)
        c = torch.tensor(1500.0, dtype=torch.float64, device="cuda", requires_grad=True)
        loss = data_tv_loss(plan, x, c, _dev(torch, ps), 1e-3)
        loss.backward()
        gx, gc = x.grad.cpu().numpy(), c.grad.item()
    nx, ny = prob.shape[0], prob.shape[1]
    ref_gx, ref_gc, flips = [], 0.0, 0.0
    for b in range(len(frames)):
        r = orc.forward(geo, x0[b]) - ps[b]
        ref_gx.append(2 * orc.adjoint(geo, r) + 1e-3 * orc.tv_grad(x0[b].reshape(ny, nx)).ravel())
        ref_gc += 2 * orc.dc(geo, x0[b], r)
        flips += 2 * orc.dc_flip_bound(geo, x0[b], r, DC_DELTA)
    assert rel_l2(gx, np.stack(ref_gx)) <= OP_TOL
    assert abs(gc - ref_gc) <= DC_TOL * abs(ref_gc) + flips, (gc, ref_gc, flips)


def test_autograd_dc_against_finite_differences(torch_cuda):
    """GPU d/dc against FP64 central differences of the oracle's data term, on a
    geometry where no arrival crosses a sample boundary within +-delta_c."""
    torch = torch_cuda
    from paper_2404_10928_gb300.autograd import ForwardOp
    dcs = 1e-2
    for seed in range(200):
        rng = np.random.default_rng(seed)
        th = rng.uniform(0, 2 * np.pi, 4)
        rad = rng.uniform(1.0e-3, 1.5e-3, 4)
        sensors = np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
        prob = ph.custom(2, (6, 5), (1e-4, 1e-4), sensors, 128, seed=seed, density=1.0)
        geo = orc.Geometry.of(prob)
        xs, ys, _ = prob.pixel_axes()
        gy, gx = np.meshgrid(ys, xs, indexing="ij")
        d = np.hypot(gx.ravel()[None, :] - prob.sensors[:, :1], gy.ravel()[None, :] - prob.sensors[:, 1:])
        if np.all(np.floor(d * prob.fs / (prob.c + dcs)) == np.floor(d * prob.fs / (prob.c - dcs))):
            break
    else:
        pytest.fail("no geometry without sample-boundary crossings")
    x = f32(prob.x_true)
    p = f32(np.random.default_rng(3).standard_normal((prob.n_sensors, prob.n_samples)))
    f = lambda cc: float(np.sum((orc.forward(geo, x, c=cc) - p) ** 2))
    fd = (f(prob.c + dcs) - f(prob.c - dcs)) / (2 * dcs)
    with _plan(prob) as plan:
        c = torch.tensor(prob.c, dtype=torch.float64, device="cuda", requires_grad=True)
        r = ForwardOp.apply(_dev(torch, x), c, plan) - _dev(torch, p)
        (r.double() ** 2).sum().backward()
        gc = c.grad.item()
    assert abs(gc - fd) <= DC_TOL * abs(fd), (gc, fd)


def _oracle_unrolled(geo, x0, y, omega, n, target):
    """FP64 reverse mode through n projected Landweber steps (written out with the
    oracle's operators): returns (dL/dx0, dL/dc) for L = ||x_n - target||^2."""
    xs, zs, rs = [x0], [], []
    for _ in range(n):
        r = orc.forward(geo, xs[-1]) - y
        z = xs[-1] - omega * orc.adjoint(geo, r)
        rs.append(r)
        zs.append(z)
        xs.append(np.maximum(z, 0.0))
    lam = 2 * (xs[-1] - target)
    gc = 0.0
    for k in reversed(range(n)):
        mu = lam * (zs[k] > 0)
        amu = orc.forward(geo, mu)
        gc += -omega * (orc.dc(geo, mu, rs[k]) + orc.dc(geo, xs[k], amu))
        lam = mu - omega * orc.adjoint(geo, amu)
    return lam, gc


def test_unrolled_landweber_gradients(torch_cuda):
    """3 checkpointed unrolled steps: bitwise equal with and without checkpointing,
    and equal to an FP64 reverse-mode pass built from the oracle.  The iterates
    are dense, so the ring is placed where no pixel's arrival lies within
    DC_DELTA of an integer sample (d/dc is discontinuous there)."""
    torch = torch_cuda
    from paper_2404_10928_gb300.autograd import UnrolledLandweber
    for j in range(1, 400):
        ring = ph.ring_sensors(11, 4e-3) + j * np.array([1.37e-6, 2.91e-6])
        prob = ph.custom(2, (29, 23), (1e-4, 1e-4), ring, 260, seed=40)
        if _min_integer_gap(prob, all_pixels=True) > 2 * DC_DELTA:
            break
    else:
        pytest.fail("no ring position without near-integer arrivals")
    geo = orc.Geometry.of(prob)
    y = f32(orc.forward(orc.Geometry.of(prob, c=1540.0), prob.x_true))
    lam = orc.power_iteration(geo, ph.power_start(prob.n_pixels), 50)
    omega = 1.0 / lam
    rng = np.random.default_rng(2)
    x0 = f32(0.5 + 0.1 * rng.standard_normal(prob.n_pixels))
    target = f32(prob.x_true)
    grads = []
    with _plan(prob) as plan:
        for ckpt in (True, False):
            x = _dev(torch, x0).requires_grad_(True)
            c = torch.tensor(1500.0, dtype=torch.float64, device="cuda", requires_grad=True)
            net = UnrolledLandweber(plan, 3, omega, checkpointing=ckpt)
            out = net(x, _dev(torch, y), c)
            ((out.double() - _dev(torch, target).double()) ** 2).sum().backward()
            grads.append((x.grad.cpu().numpy(), c.grad.item()))
    assert np.array_equal(grads[0][0], grads[1][0]) and grads[0][1] == grads[1][1]
    ref_gx, ref_gc = _oracle_unrolled(geo, x0, y, omega, 3, target)
    assert rel_l2(grads[0][0], ref_gx) <= 1e-4
    assert abs(grads[0][1] - ref_gc) <= DC_TOL * abs(ref_gc), (grads[0][1], ref_gc)


def test_gradients_ring128_batch8(torch_cuda):
    """The differentiation workload: batch of 8 vessel frames (256^2, 128-sensor ring,
    2048 samples), traces at c = 1540, gradients at c = 1500."""
    torch = torch_cuda
    from paper_2404_10928_gb300.autograd import data_tv_loss
    frames = ph.ring_vessels_batch()
    prob = frames[0]
    geo_true = orc.Geometry.of(prob, c=1540.0)
    geo = orc.Geometry.of(prob, c=1500.0)
    xs = np.stack([f32(f.x_true) for f in frames])
    ps = np.stack([f32(orc.forward(geo_true, f.x_true)) for f in frames])
    with _plan(prob) as plan:
        x = _dev(torch, xs).requires_grad_(True)
        c = torch.tensor(1500.0, dtype=torch.float64, device="cuda", requires_grad=True)
        data_tv_loss(plan, x, c, _dev(torch, ps), 1e-3).backward()
        gx, gc = x.grad.cpu().numpy(), c.grad.item()
    ny, nx = prob.shape[1], prob.shape[0]
    ref_gc = 0.0
    worst = 0.0
    for b in range(len(frames)):
        r = orc.forward(geo, xs[b]) - ps[b]
        ref = 2 * orc.adjoint(geo, r) + 1e-3 * orc.tv_grad(xs[b].reshape(ny, nx)).ravel()
        worst = max(worst, rel_l2(gx[b], ref))
        ref_gc += 2 * orc.dc(geo, xs[b], r)
    assert worst <= OP_TOL, worst
    assert abs(gc - ref_gc) <= DC_TOL * abs(ref_gc), (gc, ref_gc)
