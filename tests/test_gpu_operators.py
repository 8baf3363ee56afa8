"""GPU operators A and A^T against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

from helpers import OP_TOL, f32, operator_cases, rel_l2

pytestmark = pytest.mark.gpu

CASES = operator_cases()


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


def _inputs(prob, seed=0):
    rng = np.random.default_rng(seed)
    x = f32(prob.x_true if prob.x_true is not None else rng.uniform(0, 1, prob.n_pixels))
    y = f32(rng.standard_normal((prob.n_sensors, prob.n_samples)))
    return x, y


@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_adjoint_match_oracle(torch_cuda, name):
    torch = torch_cuda
    prob = CASES[name]
    geo = orc.Geometry.of(prob)
    x, y = _inputs(prob)
    with _plan(prob) as plan:
        p_gpu = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda"))
        g_gpu = plan.adjoint(torch.tensor(y, dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
        plan.sync_status()
        p_gpu, g_gpu = p_gpu.cpu().numpy(), g_gpu.cpu().numpy()
    p_ref = orc.forward(geo, x)
    g_ref = orc.adjoint(geo, y)
    assert rel_l2(p_gpu, p_ref) <= OP_TOL, rel_l2(p_gpu, p_ref)
    assert rel_l2(g_gpu, g_ref) <= OP_TOL, rel_l2(g_gpu, g_ref)


@pytest.mark.parametrize("name", ["ragged-37x53-ring13-k301", "3d-33x9x17-ragged"])
def test_adjoint_identity_and_determinism(torch_cuda, name):
    torch = torch_cuda
    prob = CASES[name]
    x, y = _inputs(prob, seed=1)
    rng = np.random.default_rng(2)
    x = f32(rng.normal(size=prob.n_pixels))  # signed image
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    with _plan(prob) as plan:
        a1, b1 = plan.forward(xt).cpu().numpy(), plan.adjoint(yt).cpu().numpy()
        a2, b2 = plan.forward(xt).cpu().numpy(), plan.adjoint(yt).cpu().numpy()
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)  # bitwise reproducible
    lhs = float(np.dot(a1.astype(np.float64).ravel(), y.ravel()))
    rhs = float(np.dot(x, b1.astype(np.float64)))
    scale = np.linalg.norm(a1) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs)


def test_linearity_and_zero(torch_cuda):
    torch = torch_cuda
    prob = CASES["ragged-37x53-ring13-k301"]
    rng = np.random.default_rng(5)
    a = torch.tensor(rng.normal(size=prob.n_pixels), dtype=torch.float32, device="cuda")
    with _plan(prob) as plan:
        z = plan.forward(torch.zeros_like(a)).cpu().numpy()
        assert np.all(z == 0.0)
        pa = plan.forward(a).cpu().numpy()
        pb = plan.forward(2.0 * a).cpu().numpy()
    assert rel_l2(pb, 2.0 * pa) <= 1e-6


@pytest.mark.parametrize("factory", ["ring_vessels", "planar_vessel_tree"])
def test_full_size_operators(torch_cuda, factory):
    """The benchmark workloads at full size (2D 256^2 x 256 sensors x 2048 samples;
    3D 128^3 x 1024 sensors x 1024 samples), with the plan defaults and with
    every work decomposition the autotuner can pick for the benchmark (adjoint
    clusters change the order of the final per-pixel sum, forward chunks the
    windows' grouping)."""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Plan
    from paper_2404_10928_gb300.autotune import candidates
    prob = getattr(ph, factory)()
    geo = orc.Geometry.of(prob)
    x, y = _inputs(prob, seed=3)
    p_ref, g_ref = orc.forward(geo, x), orc.adjoint(geo, y)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    shapes = [(0, 0, 0, 0)] + list(candidates(prob.n_sensors))
    p_first = None
    for c, spc, nt, aw in shapes:
        with Plan.from_problem(prob, adj_cluster=c, fwd_sensors_per_cta=spc,
                               fwd_threads=nt, adj_warps=aw) as plan:
            p_gpu = plan.forward(xt).cpu().numpy()
            g_gpu = plan.adjoint(yt).cpu().numpy()
            plan.sync_status()
        assert rel_l2(p_gpu, p_ref) <= OP_TOL, (c, spc, nt, aw, rel_l2(p_gpu, p_ref))
        assert rel_l2(g_gpu, g_ref) <= OP_TOL, (c, spc, nt, aw, rel_l2(g_gpu, g_ref))
        # the forward's window sums are exact integer sums: every decomposition
        # gives the same bits
        if p_first is None:
            p_first = p_gpu
        assert np.array_equal(p_gpu, p_first), (c, spc, nt)


def test_sound_speed_change(torch_cuda):
    torch = torch_cuda
    prob = CASES["ragged-37x53-ring13-k301"]
    x, y = _inputs(prob, seed=4)
    with _plan(prob) as plan:
        plan.set_sound_speed(1540.0)
        p_gpu = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel_l2(p_gpu, orc.forward(orc.Geometry.of(prob, c=1540.0), x)) <= OP_TOL


def test_bad_tensor_arguments(torch_cuda):
    torch = torch_cuda
    prob = CASES["ragged-37x53-ring13-k301"]
    with _plan(prob) as plan:
        with pytest.raises(ValueError):
            plan.forward(torch.zeros(prob.n_pixels + 1, device="cuda"))
        with pytest.raises(ValueError):
            plan.forward(torch.zeros(prob.n_pixels, device="cuda", dtype=torch.float64))


@pytest.mark.parametrize("name", ["ragged-37x53-ring13-k301", "3d-20x17x12-planar"])
def test_thread_layouts_give_the_same_bits(torch_cuda, name):
    """Threads per forward tile and compute warps per adjoint CTA only change
    which thread holds which pixels: A and A^T are bitwise the same."""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Plan
    prob = CASES[name]
    x, y = _inputs(prob, seed=12)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    outs = []
    for nt, aw in ((64, 4), (128, 8), (256, 4), (128, 4)):
        with Plan.from_problem(prob, adj_cluster=2, fwd_threads=nt, adj_warps=aw) as plan:
            assert plan.info()["fwd_threads"] == nt and plan.info()["adj_warps"] == aw
            outs.append((plan.forward(xt), plan.adjoint(yt)))
            plan.sync_status()
    for p, g in outs[1:]:
        assert torch.equal(p, outs[0][0]) and torch.equal(g, outs[0][1])


def autotune_sizes():
    from paper_2404_10928_gb300.autotune import FWD_SENSORS
    return FWD_SENSORS


def test_autotuned_plan_matches_default(torch_cuda, tmp_path):
    """The autotuner picks a valid decomposition; the tuned plan computes the same
    operators (A bitwise; A^T up to the order of the per-pixel cluster sum)."""
    torch = torch_cuda
    from paper_2404_10928_gb300.api import Plan
    from paper_2404_10928_gb300.autotune import Autotuner
    prob = CASES["ragged-37x53-ring13-k301"]
    best = Autotuner(str(tmp_path / "t.json")).best(prob)
    assert best["adj_cluster"] in (1, 2, 4, 8)
    assert best["fwd_sensors_per_cta"] in autotune_sizes()
    x, y = _inputs(prob, seed=9)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    assert best["fwd_threads"] in (64, 128, 256)
    with Plan.from_problem(prob) as a, Plan.from_problem(
            prob, **Autotuner.plan_options(best)) as b:
        assert torch.equal(a.forward(xt), b.forward(xt))
        assert rel_l2(a.adjoint(yt).cpu().numpy(), b.adjoint(yt).cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("name", ["linear64-disks", "ragged-37x53-ring13-k301", "t0-amp-33x20",
                                  "3d-20x17x12-planar"])
@pytest.mark.parametrize("filt", ["ubp", "none"])
def test_backproject_matches_oracle(torch_cuda, name, filt):
    # back-projection (Sec. 4, Experiment 1): A^T of the filtered traces
    torch = torch_cuda
    prob = CASES[name]
    geo = orc.Geometry.of(prob)
    x, y = _inputs(prob, seed=13)
    p = f32(orc.forward(geo, x))  # traces with the structure of a measurement
    with _plan(prob) as plan:
        b_gpu = plan.backproject(torch.tensor(p, dtype=torch.float32, device="cuda"), filt)
        torch.cuda.synchronize()
        plan.sync_status()
        b_gpu = b_gpu.cpu().numpy()
    b_ref = orc.backproject(geo, p, filt)
    assert rel_l2(b_gpu, b_ref) <= OP_TOL, rel_l2(b_gpu, b_ref)


def test_backproject_full_size_ring(torch_cuda):
    torch = torch_cuda
    prob = ph.ring_vessels()
    geo = orc.Geometry.of(prob)
    p = f32(orc.forward(geo, f32(prob.x_true)))
    with _plan(prob) as plan:
        b_gpu = plan.backproject(torch.tensor(p, dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
        plan.sync_status()
        b_gpu = b_gpu.cpu().numpy()
    b_ref = orc.backproject(geo, p, "ubp")
    assert rel_l2(b_gpu, b_ref) <= OP_TOL, rel_l2(b_gpu, b_ref)
