"""Pins of the FP64 oracle to facts fixed outside the oracle itself.

Each test checks the oracle against something it cannot agree with by
construction: hand-worked closed forms (``tests/golden``), partition-of-unity
sums of the hat, an independently written adjoint loop, a brute-force matrix
that evaluates the hat at every sample, library solvers (lstsq, NNLS, SVD) and
finite differences.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2404_10928_gb300 import phantoms as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _single_pixel_geo(case):
    dim = case["dim"]
    shape = (1, 1, 1)
    spacing = (1e-4, 1e-4, 1e-4)
    origin = (0.0, 0.0, 0.0)
    sensors = np.array([case["sensor"]], dtype=np.float64)
    return orc.Geometry(dim, shape, spacing, origin, sensors, case["c"], case["fs"], case["K"],
                        case["t0"], case["amp"])


def _load_cases():
    with open(os.path.join(GOLDEN, "single_pixel.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _load_cases(), ids=lambda c: c["name"])
def test_single_pixel_closed_form(case):
    geo = _single_pixel_geo(case)
    p = orc.forward(geo, np.ones(1))[0]
    expect = np.zeros(case["K"])
    for k, v in case["taps"].items():
        expect[int(k)] = v
    # FP64 rounding of d*fs/c can put u a hair below an integer: that moves
    # at most ~1e-12 of the weight to the neighbouring tap.
    np.testing.assert_allclose(p, expect, rtol=1e-10, atol=1e-9)
    # the brute-force form and the adjoint see the same two taps
    np.testing.assert_allclose(orc.forward_dense(geo, np.ones(1))[0], expect, rtol=1e-10, atol=1e-9)
    y = np.arange(case["K"], dtype=np.float64)[None, :] + 1.0
    np.testing.assert_allclose(orc.adjoint(geo, y)[0], float(expect @ y[0]), rtol=1e-12)


def _random_geo(dim, shape, n_sensors, K, seed, radius=None, spacing=1e-4, t0=0.0, amp=1.0):
    rng = np.random.default_rng(seed)
    shape3 = tuple(shape) + (1,) * (3 - len(shape))
    sp = (spacing, spacing, spacing)
    origin = ph.centred_origin(shape3, sp)
    ext = max(shape) * spacing
    if radius is None:
        radius = ext + 1e-3
    dirs = rng.normal(size=(n_sensors, dim))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    sensors = dirs * radius * rng.uniform(1.0, 1.5, size=(n_sensors, 1))
    return orc.Geometry(dim, shape3, sp, origin, sensors, 1500.0, 40e6, K, t0, amp)


def _distances(geo):
    """Pixel-sensor distances computed here with numpy broadcasting, [S][N]."""
    nx, ny, nz = geo.shape
    xs = geo.origin[0] + geo.spacing[0] * np.arange(nx)
    ys = geo.origin[1] + geo.spacing[1] * np.arange(ny)
    zs = geo.origin[2] + geo.spacing[2] * np.arange(nz)
    gz, gy, gx = np.meshgrid(zs, ys, xs, indexing="ij")
    pts = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)[:, :geo.dim]
    return np.linalg.norm(pts[None, :, :] - geo.sensors[:, None, :], axis=2)


@pytest.mark.parametrize("dim,shape", [(2, (7, 5)), (3, (4, 3, 5))])
def test_sum_rule_partition_of_unity(dim, shape):
    """sum_k p[s,k] = sum_i x_i / d_is when every tap lies inside [0, K)."""
    geo = _random_geo(dim, shape, 6, 4096, seed=11)
    x = np.random.default_rng(3).uniform(0, 1, geo.n_pixels)
    p = orc.forward(geo, x)
    d = _distances(geo)
    np.testing.assert_allclose(p.sum(axis=1), (x[None, :] / d).sum(axis=1), rtol=1e-12)


@pytest.mark.parametrize("dim,shape", [(2, (6, 4)), (3, (3, 4, 2))])
def test_adjoint_of_ones(dim, shape):
    """(A^T 1)_i = sum_s 1/d_is when both taps of every pair lie inside [0, K)."""
    geo = _random_geo(dim, shape, 5, 4096, seed=5)
    g = orc.adjoint(geo, np.ones((geo.n_sensors, geo.n_samples)))
    np.testing.assert_allclose(g, (1.0 / _distances(geo)).sum(axis=0), rtol=1e-12)


@pytest.mark.parametrize("dim,shape,K,t0", [(2, (4, 4), 64, 0.0), (3, (3, 3, 3), 64, 0.0),
                                            (2, (5, 3), 40, 3e-7)])
def test_bruteforce_matrix(dim, shape, K, t0):
    """A equals the explicitly assembled matrix (hat evaluated at every sample,
    no floor) and A^T equals its transpose, including truncated taps."""
    geo = _random_geo(dim, shape, 4, K, seed=21, radius=1.2e-3, t0=t0)
    M = orc.matrix(geo)
    rng = np.random.default_rng(0)
    x = rng.normal(size=geo.n_pixels)
    y = rng.normal(size=(geo.n_sensors, K))
    np.testing.assert_allclose(orc.forward(geo, x).ravel(), M @ x, rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(orc.adjoint(geo, y), M.T @ y.ravel(), rtol=1e-11, atol=1e-9)
    assert np.count_nonzero(M) > 0


@pytest.mark.parametrize("dim,shape,S,K", [(2, (33, 21), 17, 300), (3, (9, 7, 6), 11, 200),
                                           (2, (20, 20), 8, 90)])
def test_adjoint_identity(dim, shape, S, K):
    """<A x, y> = <x, A^T y> with independently written forward and adjoint loops
    (the last case truncates most arrivals)."""
    geo = _random_geo(dim, shape, S, K, seed=99)
    rng = np.random.default_rng(1)
    x = rng.normal(size=geo.n_pixels)
    y = rng.normal(size=(S, K))
    lhs = float(np.sum(orc.forward(geo, x) * y))
    rhs = float(x @ orc.adjoint(geo, y))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


def test_linearity():
    geo = _random_geo(2, (12, 9), 5, 256, seed=2)
    rng = np.random.default_rng(4)
    a, b = rng.normal(size=(2, geo.n_pixels))
    np.testing.assert_allclose(orc.forward(geo, 2.5 * a - 0.5 * b),
                               2.5 * orc.forward(geo, a) - 0.5 * orc.forward(geo, b),
                               rtol=1e-11, atol=1e-9)


def _tiny_system(seed=8):
    geo = _random_geo(2, (3, 3), 4, 64, seed=seed, radius=1.0e-3)
    M = orc.matrix(geo)
    return geo, M


def test_cgls_matches_lstsq():
    """CGLS on a tiny full-rank system reaches numpy.linalg.lstsq."""
    geo, M = _tiny_system()
    assert np.linalg.matrix_rank(M) == geo.n_pixels
    y = np.random.default_rng(6).normal(size=M.shape[0])
    x_ls = np.linalg.lstsq(M, y, rcond=None)[0]
    x, hist = orc.cgls(geo, y, n_iter=3 * geo.n_pixels, nonneg=False)
    np.testing.assert_allclose(x, x_ls, rtol=1e-8, atol=1e-10 * np.abs(x_ls).max())
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])


def test_landweber_matches_nnls():
    """Projected Landweber with omega = 1/sigma_max^2 converges to the NNLS
    solution (Lawson-Hanson, scipy.optimize.nnls) with active constraints."""
    from scipy.optimize import nnls

    geo, M = _tiny_system(seed=12)
    x_star = np.array([1.0, -0.5, 0.8, 0.3, -0.2, 1.2, 0.0, 0.5, 0.9])
    y = M @ x_star
    x_nn, _ = nnls(M, y, maxiter=10000)
    assert np.any(x_nn == 0.0)
    sig = np.linalg.svd(M, compute_uv=False)
    omega = 1.0 / sig[0] ** 2
    x, hist = orc.landweber(geo, y, n_iter=20000, omega=omega, nonneg=True)
    np.testing.assert_allclose(x, x_nn, atol=1e-8 * np.abs(x_nn).max())
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])


def test_power_iteration_matches_svd():
    geo, M = _tiny_system(seed=14)
    lam = orc.power_iteration(geo, ph.power_start(geo.n_pixels), n_iter=200)
    sig = np.linalg.svd(M, compute_uv=False)
    assert abs(lam - sig[0] ** 2) <= 1e-6 * sig[0] ** 2


def test_dc_matches_finite_differences():
    """d/dc <g, A(x;c)> against central differences, on a geometry where no
    arrival crosses a sample boundary within +-delta_c."""
    for seed in range(50):
        geo = _random_geo(2, (6, 5), 4, 128, seed=100 + seed)
        d = _distances(geo)
        c, dc_step = geo.c, 1e-2
        u_lo = d * geo.fs / (c + dc_step)
        u_hi = d * geo.fs / (c - dc_step)
        if np.all(np.floor(u_lo) == np.floor(u_hi)):
            break
    else:
        pytest.fail("no seed without sample-boundary crossings")
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, geo.n_pixels)
    g = rng.normal(size=(geo.n_sensors, geo.n_samples))
    f = lambda cc: float(np.sum(g * orc.forward(geo, x, c=cc)))
    fd = (f(c + dc_step) - f(c - dc_step)) / (2 * dc_step)
    an = orc.dc(geo, x, g)
    assert abs(an - fd) <= 1e-6 * abs(fd)


def test_dc_flip_bound_is_the_derivative_jump():
    """A pixel whose arrival sits on an integer sample m: the bound equals the
    jump between the one-sided finite-difference derivatives of <g, A(x; c)>
    in c, and vanishes once delta is below the distance to the integer."""
    fs, c0, m = 40e6, 1500.0, 57
    d = m * c0 / fs
    geo = orc.Geometry(2, (1, 1, 1), (1e-4, 1e-4, 1e-4), (0.0, 0.0, 0.0),
                       np.array([[d, 0.0]]), c0, fs, 128, 0.0, 0.7)
    rng = np.random.default_rng(11)
    x = np.array([0.8])
    g = rng.normal(size=(1, 128))
    f = lambda cc: float(np.sum(g * orc.forward(geo, x, c=cc)))
    h = 1e-3
    d_plus = (f(c0 + h) - f(c0)) / h    # u just below m: taps (m-1, m)
    d_minus = (f(c0) - f(c0 - h)) / h   # u just above m: taps (m, m+1)
    jump = abs(d_plus - d_minus)
    assert jump > 0.0
    bound = orc.dc_flip_bound(geo, x, g, 1e-6)
    assert abs(bound - jump) <= 1e-4 * jump, (bound, jump)
    # moving the sensor a quarter sample away takes the pair out of range
    geo2 = orc.Geometry(2, (1, 1, 1), (1e-4, 1e-4, 1e-4), (0.0, 0.0, 0.0),
                        np.array([[d + 0.25 * c0 / fs, 0.0]]), c0, fs, 128, 0.0, 0.7)
    assert orc.dc_flip_bound(geo2, x, g, 0.2) == 0.0
    assert orc.dc_flip_bound(geo2, x, g, 0.3) > 0.0


def test_tv_constant_and_fd():
    eps = 1e-4
    img = np.full((5, 7), 0.3)
    assert abs(orc.tv(img, eps) - img.size * eps) <= 1e-15
    assert np.all(orc.tv_grad(img, eps) == 0.0)
    rng = np.random.default_rng(9)
    img = rng.uniform(0, 1, (6, 5))
    g = orc.tv_grad(img, eps)
    h = 1e-6
    fd = np.zeros_like(img)
    for idx in np.ndindex(img.shape):
        e = np.zeros_like(img)
        e[idx] = h
        fd[idx] = (orc.tv(img + e, eps) - orc.tv(img - e, eps)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-7)


def test_tv_hand_value():
    """2x2 image [[0,1],[0,0]]: four terms worked out by hand."""
    eps = 1e-4
    img = np.array([[0.0, 1.0], [0.0, 0.0]])
    # (0,0): dx=1, dy=0; (0,1): dx=0, dy=-1; (1,0): dx=0, dy=0; (1,1): 0, 0
    expect = 2 * np.sqrt(1 + eps * eps) + 2 * eps
    assert abs(orc.tv(img, eps) - expect) <= 1e-15


def test_monotone_residual_landweber():
    prob = ph.custom(2, (16, 16), (1e-4, 1e-4), ph.ring_sensors(12, 2.5e-3), 160, seed=4)
    geo = orc.Geometry.of(prob)
    y = orc.forward(geo, prob.x_true)
    lam = orc.power_iteration(geo, ph.power_start(geo.n_pixels), 50)
    _, hist = orc.landweber(geo, y, 25, omega=1.0 / lam)
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    assert hist[-1] < 0.5 * hist[0]


def test_ubp_filter_hand_values():
    # worked by hand from b(t) = 2 p(t) - 2 t dp/dt, dp/dt = fs (p[k+1] - p[k-1]) / 2,
    # p[-1] = p[K] = 0:  p = (1, 2, 4)
    #   t0 = 0, fs = 1:   dp/dt = (1, 1.5, -1),  t = (0, 1, 2)     -> b = (2, 1, 12)
    #   t0 = 0.5, fs = 2: dp/dt = (2, 3, -2),    t = (0.5, 1, 1.5) -> b = (0, -2, 14)
    p = np.array([[1.0, 2.0, 4.0]])
    assert np.allclose(orc.ubp_filter(p, 0.0, 1.0), [[2.0, 1.0, 12.0]], rtol=0, atol=1e-14)
    assert np.allclose(orc.ubp_filter(p, 0.5, 2.0), [[0.0, -2.0, 14.0]], rtol=0, atol=1e-14)


def test_ubp_filter_quadratic_closed_form():
    # a central difference is exact on a quadratic: for p[k] = a + b k + c k^2 the
    # interior derivative is fs (b + 2 c k), so the filter is the polynomial
    # 2 (a + b k + c k^2) - 2 (t0 fs + k)(b + 2 c k) away from the two ends
    a, b, c, fs, t0, K = 0.3, -1.7, 0.05, 40e6, 2.5e-8, 64
    k = np.arange(K, dtype=np.float64)
    p = (a + b * k + c * k * k)[None, :]
    got = orc.ubp_filter(p, t0, fs)[0]
    expect = 2 * (a + b * k + c * k * k) - 2 * (t0 * fs + k) * (b + 2 * c * k)
    assert np.allclose(got[1:-1], expect[1:-1], rtol=1e-12, atol=1e-12)
    # the ends see the zero extension: dp/dt = fs p[1] / 2 and -fs p[K-2] / 2
    assert np.isclose(got[0], 2 * p[0, 0] - 2 * t0 * fs * p[0, 1] / 2, rtol=1e-12)
    assert np.isclose(got[-1], 2 * p[0, -1] + 2 * (t0 * fs + K - 1) * p[0, -2] / 2, rtol=1e-12)


def test_backproject_is_adjoint_of_filtered_traces():
    # <BP(p), x> = <F(p), A x>: the back-projection is the adjoint (an independent
    # loop, pinned above) applied to the filtered traces
    prob = ph.custom(2, (21, 17), (1e-4, 1e-4), ph.ring_sensors(7, 3e-3), 180, seed=11,
                     t0=2 / ph.SAMPLE_RATE)
    geo = orc.Geometry.of(prob)
    rng = np.random.default_rng(12)
    p = rng.standard_normal((prob.n_sensors, prob.n_samples))
    x = rng.standard_normal(prob.n_pixels)
    lhs = float(np.dot(orc.backproject(geo, p, "ubp"), x))
    rhs = float(np.sum(orc.ubp_filter(p, geo.t0, geo.fs) * orc.forward(geo, x)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    assert np.array_equal(orc.backproject(geo, p, "none"), orc.adjoint(geo, p))


def _tiny_fista_problem(seed):
    prob = ph.custom(2, (5, 4), (1e-4, 1e-4), ph.ring_sensors(6, 1.5e-3), 70, seed=seed)
    geo = orc.Geometry.of(prob)
    m = orc.matrix(geo)
    sigma2 = float(np.linalg.svd(m, compute_uv=False)[0] ** 2)
    return prob, geo, m, sigma2


def test_fista_unregularised_reaches_lstsq():
    # alpha = beta = 0, no projection: FISTA minimises ||A x - y||^2
    prob, geo, m, sigma2 = _tiny_fista_problem(31)
    rng = np.random.default_rng(32)
    y = m @ rng.uniform(0.2, 1.0, prob.n_pixels) + 0.01 * rng.standard_normal(m.shape[0])
    x, hist = orc.fista(geo, y, 4000, tau=1.0 / (2.0 * sigma2), nonneg=False)
    ref = np.linalg.lstsq(m, y, rcond=None)[0]
    assert np.allclose(x, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
    assert hist[-1] <= hist[0]


def test_fista_meets_the_optimality_conditions():
    # minimiser of ||A x - y||^2 + alpha ||x||_1 + beta TV_eps(x) over x >= 0: with
    # G the gradient of the smooth part, G_i + alpha = 0 where x_i > 0 and
    # G_i + alpha >= 0 where x_i = 0 (KKT)
    prob, geo, m, sigma2 = _tiny_fista_problem(33)
    rng = np.random.default_rng(34)
    truth = np.where(rng.uniform(size=prob.n_pixels) < 0.5, rng.uniform(0.5, 1.0, prob.n_pixels), 0.0)
    y = m @ truth + 0.02 * rng.standard_normal(m.shape[0])
    # beta such that the TV term's curvature bound 8 beta / eps is half the data
    # term's 2 sigma^2: both terms shape the minimiser
    alpha, eps = 0.05 * np.abs(m.T @ y).max(), 1e-2
    beta = 0.125 * sigma2 * eps
    tau = 1.0 / (2.0 * sigma2 + 8.0 * beta / eps)
    x, _ = orc.fista(geo, y, 20000, tau, alpha, beta, eps)
    nx, ny, _ = prob.shape
    g = -2.0 * m.T @ (y - m @ x) + beta * orc.tv_grad(x.reshape(ny, nx), eps).ravel()
    scale = alpha + np.abs(g).max()
    active = x > 1e-12 * np.abs(x).max()
    assert active.any() and (~active).any()  # both cases are exercised
    assert np.all(np.abs(g[active] + alpha) <= 1e-6 * scale)
    assert np.all(g[~active] + alpha >= -1e-6 * scale)


def test_fista_momentum_beats_plain_shrinkage():
    # the extrapolation is what makes FISTA O(1/k^2): after a few dozen steps on
    # an ill-conditioned problem its objective is below that of the same
    # proximal steps without momentum (ISTA)
    prob, geo, m, sigma2 = _tiny_fista_problem(35)
    rng = np.random.default_rng(36)
    y = m @ rng.uniform(0.0, 1.0, prob.n_pixels)
    tau, alpha = 1.0 / (2.0 * sigma2), 1e-3 * np.abs(m.T @ y).max()

    def objective(x):
        return float(np.sum((m @ x - y) ** 2) + alpha * np.abs(x).sum())

    f_star = objective(orc.fista(geo, y, 20000, tau, alpha)[0])
    x_f, _ = orc.fista(geo, y, 40, tau, alpha)
    x_i = np.zeros(prob.n_pixels)  # ISTA: the same step, no extrapolation
    for _ in range(40):
        v = x_i - tau * (-2.0 * m.T @ (y - m @ x_i))
        x_i = np.maximum(v - tau * alpha, 0.0)
    assert objective(x_f) - f_star < 0.5 * (objective(x_i) - f_star)


def test_freq_single_pixel_hand_values():
    # Eq. 7 for one pixel 3 mm from the sensor, c = 1500 m/s, amp = 1:
    #   f = 1 MHz:    f d / c = 2 cycles, exp(-i k d) = 1,  P = i c k / d = i 2 pi f / d
    #   f = 1.125 MHz: 2.25 cycles, exp(-i k d) = -i,    P = c k / d = 2 pi f / d (real)
    geo = orc.Geometry(2, (1, 1, 1), (1e-4, 1e-4, 1e-4), (0.0, 0.0, 0.0),
                       np.array([[0.0, 3e-3]]), 1500.0, 40e6, 16)
    p = orc.freq_forward(geo, np.ones(1), 2, 1.0e6, 0.125e6)[0]
    two_pi_over_d = 2 * np.pi / 3e-3
    assert abs(p[0] - 1j * two_pi_over_d * 1.0e6) <= 1e-9 * two_pi_over_d * 1e6
    assert abs(p[1] - two_pi_over_d * 1.125e6) <= 1e-9 * two_pi_over_d * 1e6


def test_freq_adjoint_identity():
    # <K x, P> = <x, K^H P> between the two independently written loops
    prob = ph.custom(2, (9, 7), (1e-4, 1e-4), ph.ring_sensors(5, 2e-3), 50, seed=41)
    geo = orc.Geometry.of(prob)
    rng = np.random.default_rng(42)
    x = rng.standard_normal(prob.n_pixels)
    q = 11
    pq = rng.standard_normal((5, q)) + 1j * rng.standard_normal((5, q))
    lhs = float(np.real(np.sum(np.conj(orc.freq_forward(geo, x, q, 0.5e6, 1.7e6)) * pq)))
    rhs = float(np.dot(x, orc.freq_adjoint(geo, pq, q, 0.5e6, 1.7e6)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("dim,d,t0", [(2, 3.0e-3, 0.0), (2, 3.0137e-3, 0.0), (2, 7.45e-3, 0.0),
                                       (3, 4.2311e-3, 0.0), (2, 3.0137e-3, 3.37 / 40e6)])
def test_freq_model_is_the_spectrum_of_the_time_derivative(dim, d, t0):
    # Eq. 7 against Eq. 6 for one pixel at distance d (amp = 1, x = 1, t0 = 0):
    # Eq. 6's impulse delta(t - d/c) / d has spectrum exp(-i k d) / d, and Eq. 7
    # is i c k = 2 pi i f times it (the spectrum of its time derivative).  The
    # discretised trace p[k] = h(u - k) / d samples a triangle of half-width
    # 1/fs, whose transform is (1/fs) sinc^2(f/fs), so by Poisson summation
    #   sum_k p[k] exp(-2 pi i f k / fs)
    #     = sum_m sinc^2(f/fs - m) exp(-2 pi i (f - m fs) d / c) / d.
    # The m = 0 term is sinc^2(f/fs) exp(-i k d) / d; the aliases m != 0 add at
    # most B(f) = sum_{m != 0} sinc^2(f/fs - m) / sinc^2(f/fs) relative to it
    # (they reach it when u is an integer, where the sum is exactly 1/d).  So
    # |P(f) - 2 pi i f DTFT(p)(f) / sinc^2(f/fs)| <= B(f) |P(f)|.  With a time
    # origin t0 the samples sit at t0 + k/fs, and the DTFT uses those times.
    c, fs, K = 1500.0, 40e6, 512
    sensor = [0.0, d] if dim == 2 else [0.0, 0.0, d]
    geo = orc.Geometry(dim, (1, 1, 1), (1e-4, 1e-4, 1e-4), (0.0, 0.0, 0.0),
                       np.array([sensor]), c, fs, K, t0=t0)
    p = orc.forward(geo, np.ones(1))[0]
    assert np.count_nonzero(p) in (1, 2) and abs(p.sum() - 1.0 / d) <= 1e-9 / d
    q, f0, df = 8, 0.125e6, 0.125e6
    P = orc.freq_forward(geo, np.ones(1), q, f0, df)[0]
    k = np.arange(K)
    m = np.concatenate([np.arange(-200000, 0), np.arange(1, 200001)])
    worst_conj = 0.0
    for n in range(q):
        f = f0 + n * df
        bound = np.sum(np.sinc(f / fs - m) ** 2) / np.sinc(f / fs) ** 2 * (1 + 1e-3) + 1e-12
        dtft = np.sum(p * np.exp(-2j * np.pi * f * (t0 + k / fs)))
        expected = 2j * np.pi * f * dtft / np.sinc(f / fs) ** 2
        assert abs(P[n] - expected) <= bound * abs(P[n]), (f, P[n], expected, bound)
        # a planted mistake, the conjugate phase exp(+i k d), must fail somewhere
        wrong = 2j * np.pi * f * np.conj(P[n] / (2j * np.pi * f))
        worst_conj = max(worst_conj, abs(wrong - expected) / abs(P[n]))
    assert worst_conj > 0.5


def test_tv_3d_constant_and_fd():
    eps = 1e-4
    img = np.full((3, 4, 5), -0.7)
    assert abs(orc.tv(img, eps) - img.size * eps) <= 1e-15
    assert np.all(orc.tv_grad(img, eps) == 0.0)
    rng = np.random.default_rng(19)
    img = rng.uniform(0, 1, (3, 4, 5))
    g = orc.tv_grad(img, eps)
    h = 1e-6
    fd = np.zeros_like(img)
    for idx in np.ndindex(img.shape):
        e = np.zeros_like(img)
        e[idx] = h
        fd[idx] = (orc.tv(img + e, eps) - orc.tv(img - e, eps)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-7)


def test_tv_3d_hand_value():
    """2x2x2 volume with one unit voxel at (0,0,0), worked by hand: that voxel
    has differences -1 along x, y and z (sqrt(3 + eps^2)); its three forward
    neighbours and the other four voxels have none (eps each).  dTV/dx at the
    unit voxel is 3/sqrt(3 + eps^2); at each of its three neighbours, which see
    it as their backward neighbour, -1/sqrt(3 + eps^2); elsewhere 0."""
    eps = 1e-3
    img = np.zeros((2, 2, 2))
    img[0, 0, 0] = 1.0
    m = np.sqrt(3.0 + eps * eps)
    assert abs(orc.tv(img, eps) - (m + 7 * eps)) <= 1e-15
    expect = np.zeros((2, 2, 2))
    expect[0, 0, 0] = 3.0 / m
    expect[0, 0, 1] = expect[0, 1, 0] = expect[1, 0, 0] = -1.0 / m
    np.testing.assert_allclose(orc.tv_grad(img, eps), expect, rtol=0, atol=1e-15)
    # a misplaced axis (a difference taken along the wrong stride) moves these
    # values: the z neighbour (1,0,0) must carry the backward term
    assert orc.tv_grad(img, eps)[1, 0, 0] < 0.0


def test_min_distance_bruteforce():
    rng = np.random.default_rng(41)
    for dim, shape in ((2, (7, 5, 1)), (3, (4, 6, 3))):
        spacing = (1.1e-4, 0.9e-4, 1.3e-4)
        origin = ph.centred_origin(shape, spacing)
        sensors = rng.uniform(-1e-3, 1e-3, (9, dim))
        geo = orc.Geometry(dim, shape, spacing, origin, sensors, 1500.0, 40e6, 64)
        axes = [origin[a] + spacing[a] * np.arange(shape[a]) for a in range(dim)]
        pts = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
        brute = np.min(np.linalg.norm(pts[:, None, :] - sensors[None, :, :], axis=-1))
        assert abs(orc.min_distance(geo) - brute) <= 1e-15


def _one_tap_geometry():
    # one unit pixel at the origin, one sensor 3 mm away: u = 80 exactly, so
    # the operator is the column with the single entry 1/d at sample 80 (the
    # first golden case, pinned above)
    return orc.Geometry(2, (1, 1, 1), (1e-4, 1e-4, 1e-4), (0.0, 0.0, 0.0),
                        np.array([[0.0, 3e-3]]), 1500.0, 4e7, 128)


def test_fista_signed_soft_threshold_hand_value():
    """Three FISTA steps on a one-pixel system, by hand.  With A = the column
    (1/d at sample 80), m = A^T A = 1/d^2 and g = A^T y = y_80/d; the step from
    z is v = z + 2 tau (g - m z) and the signed proximal step is
    x = sign(v) max(|v| - tau alpha, 0).  A negative measurement drives x below
    zero, so the threshold must move v towards zero from below (v + tau alpha):
    a threshold taken without the sign, or a projection onto x >= 0, fails."""
    geo = _one_tap_geometry()
    d = 3e-3
    y = np.zeros((1, 128))
    y[0, 80] = -0.02
    m, g = 1.0 / d**2, -0.02 / d
    tau = 0.3 / m
    alpha = 0.1 * abs(g)

    def shrink(v):
        return np.sign(v) * max(abs(v) - tau * alpha, 0.0)

    x_prev, z, t = 0.0, 0.0, 1.0
    for _ in range(3):
        x = shrink(z + 2.0 * tau * (g - m * z))
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        z = x + ((t - 1.0) / t_new) * (x - x_prev)
        x_prev, t = x, t_new
    # numbers: step 1 from z = 0 gives v = 2 tau g = 0.6 g/m, and the threshold
    # tau alpha = 0.03 |g|/m moves it towards zero: x1 = 0.57 g/m = -3.42e-5
    x1, _ = orc.fista(geo, y, 1, tau, alpha, nonneg=False)
    assert abs(x1[0] - (-3.42e-5)) <= 1e-15
    x3, _ = orc.fista(geo, y, 3, tau, alpha, nonneg=False)
    assert x3[0] < 0.0
    assert abs(x3[0] - x_prev) <= 1e-12 * abs(x_prev)
    # with the projection the same steps stop at zero
    xp, _ = orc.fista(geo, y, 3, tau, alpha, nonneg=True)
    assert xp[0] == 0.0


def test_fista_signed_meets_the_optimality_conditions():
    # minimiser of ||A x - y||^2 + alpha ||x||_1 (+ beta TV) without x >= 0:
    # with G the gradient of the smooth part, G_i + alpha sign(x_i) = 0 where
    # x_i != 0 and |G_i| <= alpha where x_i = 0 (the subgradient condition)
    prob, geo, m, sigma2 = _tiny_fista_problem(37)
    rng = np.random.default_rng(38)
    truth = np.where(rng.uniform(size=prob.n_pixels) < 0.5, rng.uniform(-1.0, 1.0, prob.n_pixels),
                     0.0)
    y = m @ truth + 0.02 * rng.standard_normal(m.shape[0])
    alpha, eps = 0.05 * np.abs(m.T @ y).max(), 1e-2
    beta = 0.125 * sigma2 * eps
    tau = 1.0 / (2.0 * sigma2 + 8.0 * beta / eps)
    x, _ = orc.fista(geo, y, 20000, tau, alpha, beta, eps, nonneg=False)
    nx, ny, _ = prob.shape
    g = -2.0 * m.T @ (y - m @ x) + beta * orc.tv_grad(x.reshape(ny, nx), eps).ravel()
    scale = alpha + np.abs(g).max()
    nz = np.abs(x) > 1e-12 * np.abs(x).max()
    assert (x[nz] < 0).any() and (x[nz] > 0).any() and (~nz).any()  # every case exercised
    assert np.all(np.abs(g[nz] + alpha * np.sign(x[nz])) <= 1e-6 * scale)
    assert np.all(np.abs(g[~nz]) <= alpha + 1e-6 * scale)


def test_fista_3d_tv_meets_the_optimality_conditions():
    # FISTA with the TV term on a 3D grid: the smooth part's gradient uses the
    # 3D TV pinned above; at the minimiser over x >= 0 the KKT conditions hold
    prob = ph.custom(3, (3, 3, 2), (1e-4, 1e-4, 1e-4), ph.planar_array(2, 2, 0.5e-3, 1.2e-3), 60,
                     seed=39)
    geo = orc.Geometry.of(prob)
    m = orc.matrix(geo)
    sigma2 = float(np.linalg.svd(m, compute_uv=False)[0] ** 2)
    y = m @ prob.x_true
    alpha, eps = 0.02 * np.abs(m.T @ y).max(), 1e-2
    beta = 0.1 * sigma2 * eps
    tau = 1.0 / (2.0 * sigma2 + 12.0 * beta / eps)  # 3D curvature bound 12 beta / eps
    x, _ = orc.fista(geo, y, 20000, tau, alpha, beta, eps)
    nx, ny, nz = prob.shape
    g = -2.0 * m.T @ (y - m @ x) + beta * orc.tv_grad(x.reshape(nz, ny, nx), eps).ravel()
    scale = alpha + np.abs(g).max()
    active = x > 1e-12 * np.abs(x).max()
    assert active.any()
    assert np.all(np.abs(g[active] + alpha) <= 1e-6 * scale)
    assert np.all(g[~active] + alpha >= -1e-6 * scale)


def test_pcgls_one_pixel_hand_values():
    """One pixel, operator = the column (1/d at sample 80): m = A^T A = 1/d^2 and
    g = A^T y.  From x = 0 the first CG step is the exact line search along
    s = g: alpha = g^2 / (m g^2) = 1/m, so x1 = max(0, g/m), the non-negative
    least-squares solution; with a negative measurement the projection stops at
    0 and the residual stays ||y||^2."""
    geo = orc.Geometry(2, (1, 1, 1), (1e-4, 1e-4, 1e-4), (0.0, 0.0, 0.0),
                       np.array([[0.0, 3e-3]]), 1500.0, 4e7, 128)
    d = 3e-3
    for y80, expect in ((0.02, 0.02 * d), (-0.02, 0.0)):
        y = np.zeros((1, 128))
        y[0, 80] = y80
        x, h = orc.pcgls(geo, y, 1)
        assert abs(x[0] - expect) <= 1e-15
        assert abs(h[0] - y80 * y80) <= 1e-18
        assert abs(h[1] - (0.0 if y80 > 0 else y80 * y80)) <= 1e-18


def test_pcgls_unprojected_is_cgls_and_projected_reaches_nnls():
    prob = ph.custom(2, (6, 5), (1e-4, 1e-4), ph.ring_sensors(9, 1.5e-3), 80, seed=51)
    geo = orc.Geometry.of(prob)
    m = orc.matrix(geo)
    rng = np.random.default_rng(52)
    truth = np.where(rng.uniform(size=prob.n_pixels) < 0.5, rng.uniform(0.2, 1.0, prob.n_pixels),
                     0.0)
    y = m @ truth + 0.05 * rng.standard_normal(m.shape[0])
    # without the projection the recursion is plain CGLS (r recomputed from x
    # instead of by the recurrence: the same iterates up to rounding)
    xu, hu = orc.pcgls(geo, y, 12, project=False)
    xc, hc = orc.cgls(geo, y, 12, nonneg=False)
    assert np.allclose(xu, xc, rtol=1e-9, atol=1e-12 * np.abs(xc).max())
    assert np.allclose(hu, hc, rtol=1e-9)
    # with the projection and a restart every step (projected steepest descent
    # with the exact line search) and every 3rd step, the iterates reach the
    # non-negative least-squares solution
    from scipy.optimize import nnls
    ref = nnls(m, y)[0]
    assert (ref == 0).any() and (ref > 0).any()  # active constraints exercised
    for restart in (1, 3):
        x, h = orc.pcgls(geo, y, 3000, restart=restart)
        assert np.all(x >= 0.0)
        assert np.allclose(x, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max()), restart
        assert h[-1] <= h[0]
