"""FP64 CPU oracle: plain, slow, obviously correct.

TEST INFRASTRUCTURE ONLY: only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library (``paper_2404_10928_gb300``) and imports nothing from it;
the two meet only in the seeded input generators (``phantoms``), which hold
none of the method's arithmetic.

What is computed, and where it comes from:

* ``forward`` / ``adjoint`` / ``forward_dense`` / ``dc``: the time-domain
  measurement matrix of Eq. 6 (Sec. 3.4) discretised with a linear-interpolation
  hat and a 1/distance weight (the spreading factor of Eq. 7); C loops in
  ``pa_oracle.c``.
* ``landweber``: projected gradient descent on the data term of Eq. 8,
  ``x <- max(0, x + omega * A^T (y - A x))``.  This is the gradient line the
  paper profiles (Table 3: ``t1 = 2*kn'*(kn*mk1r - y)``) with step omega/2,
  plus a non-negativity projection.
* ``cgls``: conjugate gradients on the normal equations of the same data term
  (Hestenes-Stiefel recursion for least squares), then a final clamp x >= 0.
* ``pcgls``: the same recursion projected onto x >= 0 after every step, with
  restarts (the non-negative data term by CG).
* ``power_iteration``: largest eigenvalue of A^T A (step size for Landweber).
* ``tv`` / ``tv_grad``: smoothed isotropic total variation (the TV term of
  Eq. 8 with Psi' = identity), 2D and 3D.
* ``min_distance``: the smallest pixel-sensor distance (the geometry check).
* ``freq_forward`` / ``freq_adjoint``: the frequency-domain measurement matrix
  of Eq. 7 applied to an image, and its adjoint (own loops).
* ``fista``: the full objective of Eq. 8 (data term, L1 and smoothed TV) by
  FISTA with a fixed step.
* ``ubp_filter`` / ``backproject``: the back-projection reconstruction timed
  against the iterative one in Sec. 4 (Experiment 1, Table 2), with the
  universal back-projection trace filter (a reading: the paper names no filter).

Where the paper is silent, each function states the reading it uses.  Parity
status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pa_oracle.c into liboracle.so with gcc (FP64, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            geo = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                   ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                   ctypes.c_double, ctypes.c_int]
            for name in ("oracle_forward", "oracle_forward_dense", "oracle_adjoint"):
                fn = getattr(lib, name)
                fn.argtypes = geo + [dp, dp]
                fn.restype = None
            lib.oracle_dc.argtypes = geo + [dp, dp, dp]
            lib.oracle_dc.restype = ctypes.c_double
            lib.oracle_dc_flip_bound.argtypes = geo + [dp, dp, ctypes.c_double]
            lib.oracle_dc_flip_bound.restype = ctypes.c_double
            fgeo = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                    ctypes.c_double, ctypes.c_double]
            for name in ("oracle_freq_forward", "oracle_freq_adjoint"):
                fn = getattr(lib, name)
                fn.argtypes = fgeo + [dp, dp]
                fn.restype = None
            lib.oracle_min_distance.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, dp, dp, dp, ctypes.c_int]
            lib.oracle_min_distance.restype = ctypes.c_double
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = None
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Number of host threads the C loops use (results do not depend on it)."""
    _load().oracle_set_threads(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Geometry:
    """The oracle's own copy of a problem's geometry (plain FP64 numbers)."""

    def __init__(self, dim, shape, spacing, origin, sensors, c, fs, n_samples, t0=0.0,
                 amp_scale=1.0):
        self.dim = int(dim)
        self.shape = tuple(int(v) for v in shape)
        self.spacing = _f64(spacing)
        self.origin = _f64(origin)
        self.sensors = _f64(sensors).reshape(-1, self.dim)
        self.c = float(c)
        self.fs = float(fs)
        self.n_samples = int(n_samples)
        self.t0 = float(t0)
        self.amp = float(amp_scale)

    @classmethod
    def of(cls, prob, c=None):
        return cls(prob.dim, prob.shape, prob.spacing, prob.origin, prob.sensors,
                   prob.c if c is None else c, prob.fs, prob.n_samples, prob.t0, prob.amp_scale)

    @property
    def n_pixels(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    @property
    def n_sensors(self):
        return self.sensors.shape[0]

    def _args(self, c=None):
        nx, ny, nz = self.shape
        return (self.dim, nx, ny, nz, _ptr(self.spacing), _ptr(self.origin), _ptr(self.sensors),
                self.n_sensors, self.c if c is None else float(c), self.fs, self.t0, self.amp,
                self.n_samples)


def forward(geo: Geometry, x, c=None) -> np.ndarray:
    """p = A x (Eq. 6 discretised), two-tap form.  Returns [S][K] float64."""
    x = _f64(x).ravel()
    assert x.size == geo.n_pixels
    p = np.empty((geo.n_sensors, geo.n_samples))
    _load().oracle_forward(*geo._args(c), _ptr(x), _ptr(p))
    return p


def forward_dense(geo: Geometry, x) -> np.ndarray:
    """p = A x evaluating the hat at every sample (no floor).  Tiny grids only."""
    x = _f64(x).ravel()
    p = np.empty((geo.n_sensors, geo.n_samples))
    _load().oracle_forward_dense(*geo._args(), _ptr(x), _ptr(p))
    return p


def adjoint(geo: Geometry, p, c=None) -> np.ndarray:
    """g = A^T p (delay-and-sum back-projection with the same hat and weight)."""
    p = _f64(p).reshape(geo.n_sensors, geo.n_samples)
    g = np.empty(geo.n_pixels)
    _load().oracle_adjoint(*geo._args(c), _ptr(p), _ptr(g))
    return g


def _freq_args(geo: Geometry, q: int, f0: float, df: float):
    nx, ny, nz = geo.shape
    return (geo.dim, nx, ny, nz, _ptr(geo.spacing), _ptr(geo.origin), _ptr(geo.sensors),
            geo.n_sensors, geo.c, geo.amp, int(q), float(f0), float(df))


def freq_forward(geo: Geometry, x, q: int, f0: float, df: float) -> np.ndarray:
    """The frequency-domain model of Eq. 7: P[m][n] = amp sum_i x_i i c k_n
    exp(-i k_n d_im) / d_im at f_n = f0 + n df (a reading: the paper gives q_n
    frequency samples without their values).  Returns complex [S][q]."""
    x = _f64(x).ravel()
    p = np.empty((geo.n_sensors, q, 2))
    _load().oracle_freq_forward(*_freq_args(geo, q, f0, df), _ptr(x), _ptr(p))
    return p[..., 0] + 1j * p[..., 1]


def freq_adjoint(geo: Geometry, p, q: int, f0: float, df: float) -> np.ndarray:
    """Adjoint of freq_forward for the real inner product Re sum conj(P) Q."""
    p = np.asarray(p, dtype=np.complex128).reshape(geo.n_sensors, q)
    pp = np.ascontiguousarray(np.stack([p.real, p.imag], axis=-1))
    g = np.empty(geo.n_pixels)
    _load().oracle_freq_adjoint(*_freq_args(geo, q, f0, df), _ptr(pp), _ptr(g))
    return g


def ubp_filter(p, t0: float, fs: float) -> np.ndarray:
    """Universal back-projection term b(t) = 2 p(t) - 2 t dp/dt (Xu and Wang,
    Phys. Rev. E 71, 016706, 2005), the filter of the paper's "filtered
    back-projection" (Sec. 4, Experiment 1; the paper does not give one), at the
    sample times t_k = t0 + k/fs, with dp/dt taken as the central difference
    fs (p[k+1] - p[k-1]) / 2 and zero traces before sample 0 and after K-1.
    p: [S][K]; returns [S][K] float64."""
    p = _f64(p)
    s, k = p.shape
    padded = np.zeros((s, k + 2))
    padded[:, 1:-1] = p
    dpdt = fs * (padded[:, 2:] - padded[:, :-2]) / 2.0
    t = t0 + np.arange(k) / fs
    return 2.0 * p - 2.0 * t[None, :] * dpdt


def backproject(geo: Geometry, p, filter: str = "ubp") -> np.ndarray:
    """Back-projection reconstruction x = A^T F(p) (the "BP" of Table 2):
    F = ubp_filter ("ubp") or the identity ("none"), then the adjoint."""
    p = _f64(p).reshape(geo.n_sensors, geo.n_samples)
    if filter == "ubp":
        p = ubp_filter(p, geo.t0, geo.fs)
    elif filter != "none":
        raise ValueError(filter)
    return adjoint(geo, p)


def dc(geo: Geometry, x, g, c=None) -> float:
    """d/dc <g, A(x; c)>: the speed-of-sound derivative of the forward model."""
    x = _f64(x).ravel()
    g = _f64(g).reshape(geo.n_sensors, geo.n_samples)
    per = np.empty(geo.n_sensors)
    return float(_load().oracle_dc(*geo._args(c), _ptr(x), _ptr(g), _ptr(per)))


def dc_flip_bound(geo: Geometry, x, g, delta: float, c=None) -> float:
    """Largest change of dc() that arrivals rounded by up to `delta` samples can
    cause: pairs within delta of an integer may take either one-sided derivative
    of the hat."""
    x = _f64(x).ravel()
    g = _f64(g).reshape(geo.n_sensors, geo.n_samples)
    return float(_load().oracle_dc_flip_bound(*geo._args(c), _ptr(x), _ptr(g), float(delta)))


def min_distance(geo: Geometry) -> float:
    """Smallest pixel-centre to sensor distance (metres), over all pairs."""
    nx, ny, nz = geo.shape
    return float(_load().oracle_min_distance(geo.dim, nx, ny, nz, _ptr(geo.spacing),
                                             _ptr(geo.origin), _ptr(geo.sensors), geo.n_sensors))


def matrix(geo: Geometry) -> np.ndarray:
    """Explicit [S*K][N] matrix assembled column by column with forward_dense."""
    n = geo.n_pixels
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(forward_dense(geo, e).ravel())
    return np.stack(cols, axis=1)


# ----------------------------------------------------------------------------
# iterations (numpy, FP64)
# ----------------------------------------------------------------------------

def landweber(geo: Geometry, y, n_iter: int, omega: float, x0=None, nonneg: bool = True):
    """Projected Landweber: x_{n+1} = max(0, x_n + omega * A^T (y - A x_n)).

    Reading: Table 3 gives only the gradient 2 K^T (K x - y); the update is a
    plain gradient step of size omega/2 followed by the projection onto x >= 0.
    Returns (x_n, history) with history[n] = ||y - A x_n||^2, n = 0..n_iter.
    """
    y = _f64(y).reshape(geo.n_sensors, geo.n_samples)
    x = np.zeros(geo.n_pixels) if x0 is None else _f64(x0).ravel().copy()
    hist = []
    for _ in range(n_iter):
        r = y - forward(geo, x)
        hist.append(float(np.sum(r * r)))
        x = x + omega * adjoint(geo, r)
        if nonneg:
            x = np.maximum(x, 0.0)
    r = y - forward(geo, x)
    hist.append(float(np.sum(r * r)))
    return x, np.array(hist)


def cgls(geo: Geometry, y, n_iter: int, x0=None, nonneg: bool = True, round_fp32: bool = False,
         round_steps_fp32: bool = False, op_noise: float = 0.0, noise_seed: int = 0,
         iterates=None):
    """CGLS (conjugate gradients on A^T A x = A^T y, Hestenes-Stiefel form).

    r = y - A x0; s = A^T r; p = s; gamma = ||s||^2; then per iteration
      q = A p; alpha = gamma / ||q||^2; x += alpha p; r -= alpha q;
      s = A^T r; gamma' = ||s||^2; beta = gamma'/gamma; p = s + beta p.
    A zero ||q||^2 or gamma stops the recursion (alpha = 0 / beta = 0).
    Reading: non-negativity is applied once after the last iteration.
    Returns (x, history) with history[n] = ||r_n||^2, n = 0..n_iter.

    Sensitivity models (all off by default; the recursion itself is unchanged):
    ``round_fp32`` rounds every vector the recursion stores (x, r, s, p and the
    operator outputs) to FP32, the storage any FP32 implementation uses, with
    everything else exact; ``round_steps_fp32`` rounds the step lengths alpha
    and beta to FP32; ``op_noise`` > 0 adds to every operator output
    i.i.d. Gaussian noise of rms ``op_noise`` times the output's rms (seeded by
    ``noise_seed``), a model of rounding inside the operators; ``iterates``, a
    list, receives a copy of x after every iteration (before the clamp).
    """
    y = _f64(y).reshape(geo.n_sensors, geo.n_samples)
    rng = np.random.default_rng(noise_seed)

    def keep(v):
        return v.astype(np.float32).astype(np.float64) if round_fp32 else v

    def noisy(v):
        if op_noise > 0.0:
            v = v + op_noise * np.sqrt(np.mean(v * v)) * rng.standard_normal(v.shape)
        return keep(v)

    x = keep(np.zeros(geo.n_pixels) if x0 is None else _f64(x0).ravel().copy())
    r = keep(y - noisy(forward(geo, x)))
    s = noisy(adjoint(geo, r))
    p = s.copy()
    gamma = float(np.sum(s * s))
    hist = [float(np.sum(r * r))]
    for _ in range(n_iter):
        q = noisy(forward(geo, p))
        delta = float(np.sum(q * q))
        alpha = gamma / delta if delta > 0.0 else 0.0
        if round_steps_fp32:
            alpha = float(np.float32(alpha))
        x = keep(x + alpha * p)
        r = keep(r - alpha * q)
        hist.append(float(np.sum(r * r)))
        s = noisy(adjoint(geo, r))
        gamma_new = float(np.sum(s * s))
        beta = gamma_new / gamma if gamma > 0.0 else 0.0
        if round_steps_fp32:
            beta = float(np.float32(beta))
        gamma = gamma_new
        p = keep(s + beta * p)
        if iterates is not None:
            iterates.append(x.copy())
    if nonneg:
        x = np.maximum(x, 0.0)
    return x, np.array(hist)


def pcgls(geo: Geometry, y, n_iter: int, restart: int = 0, x0=None, project: bool = True):
    """Projected, restarted CGLS for min ||A x - y||^2 over x >= 0 (the CGLS
    recursion of ``cgls`` with the iterate projected onto x >= 0 after every
    step; reading: the paper's Eq. 8 with non-negativity and no L1/TV terms).

    The projection breaks the residual recurrence, so r is recomputed from x:
      x = max(0, x0); r = y - A x; s = A^T r; p = s; gamma = ||s||^2; then
      q = A p; alpha = gamma / ||q||^2; x = max(0, x + alpha p); r = y - A x;
      s = A^T r; gamma' = ||s||^2; p = s every ``restart``-th iteration
      (restart >= 1; 0: never), else p = s + (gamma'/gamma) p.
    ``project`` False keeps every step unconstrained (then the iterates are those
    of plain CGLS).  Returns (x, history) with history[n] = ||r_n||^2."""
    y = _f64(y).reshape(geo.n_sensors, geo.n_samples)
    x = np.zeros(geo.n_pixels) if x0 is None else _f64(x0).ravel().copy()
    if project:
        x = np.maximum(x, 0.0)
    r = y - forward(geo, x)
    s = adjoint(geo, r)
    p = s.copy()
    gamma = float(np.sum(s * s))
    hist = [float(np.sum(r * r))]
    for k in range(n_iter):
        q = forward(geo, p)
        delta = float(np.sum(q * q))
        alpha = gamma / delta if delta > 0.0 else 0.0
        x = x + alpha * p
        if project:
            x = np.maximum(x, 0.0)
        r = y - forward(geo, x)
        hist.append(float(np.sum(r * r)))
        s = adjoint(geo, r)
        gamma_new = float(np.sum(s * s))
        if restart > 0 and (k + 1) % restart == 0:
            p = s.copy()
        else:
            p = s + (gamma_new / gamma if gamma > 0.0 else 0.0) * p
        gamma = gamma_new
    return x, np.array(hist)


def fista(geo: Geometry, y, n_iter: int, tau: float, alpha: float = 0.0, beta: float = 0.0,
          eps: float = 1e-4, x0=None, nonneg: bool = True):
    """The full objective of Eq. 8 with Phi = A and Psi' = I,
        F(x) = ||A x - y||^2 + alpha ||x||_1 + beta TV_eps(x),
    by FISTA (Beck and Teboulle, SIAM J. Imaging Sci. 2, 183, 2009) with a fixed
    step tau: x_k = prox(z_k - tau grad f(z_k)) for the smooth part f (data term
    and TV_eps), prox the soft threshold of tau alpha |.| (with nonneg: max(0,
    v - tau alpha)), t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 and
    z_{k+1} = x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1}).  TV is taken on the
    image's own grid (2D or 3D).
    Returns (x, history) with history = ||y - A z_k||^2 for k < n_iter and
    ||y - A x_n||^2 last."""
    y = _f64(y).reshape(geo.n_sensors, geo.n_samples)
    n = geo.n_pixels
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    z = x.copy()
    t = 1.0
    hist = []
    nx, ny, nz = geo.shape
    for _ in range(n_iter):
        r = y - forward(geo, z)
        hist.append(float(np.sum(r * r)))
        grad = -2.0 * adjoint(geo, r)
        if beta != 0.0:
            img = z.reshape(ny, nx) if nz == 1 else z.reshape(nz, ny, nx)
            grad = grad + beta * tv_grad(img, eps).ravel()
        v = z - tau * grad
        if nonneg:
            x_new = np.maximum(v - tau * alpha, 0.0)
        else:
            x_new = np.sign(v) * np.maximum(np.abs(v) - tau * alpha, 0.0)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        z = x_new + ((t - 1.0) / t_new) * (x_new - x)
        x, t = x_new, t_new
    r = y - forward(geo, x)
    hist.append(float(np.sum(r * r)))
    return x, np.array(hist)


def power_iteration(geo: Geometry, v0, n_iter: int = 50) -> float:
    """sigma_max(A)^2 by power iteration on A^T A from the given start vector.

    v <- A^T A v / ||A^T A v||; the estimate is ||A^T A v|| at the last step
    with v of unit norm.
    """
    v = _f64(v0).ravel()
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(n_iter):
        w = adjoint(geo, forward(geo, v))
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


# ----------------------------------------------------------------------------
# smoothed total variation (2D and 3D), the TV term of Eq. 8 with Psi' = I
# ----------------------------------------------------------------------------

def _forward_differences(x):
    """Forward difference of x along every axis, zero past the last index
    (Neumann).  x: [ny][nx] or [nz][ny][nx]; returns one array per axis."""
    diffs = []
    for axis in range(x.ndim):
        d = np.zeros_like(x)
        lead = [slice(None)] * x.ndim
        lag = [slice(None)] * x.ndim
        lead[axis] = slice(1, None)
        lag[axis] = slice(None, -1)
        d[tuple(lag)] = x[tuple(lead)] - x[tuple(lag)]
        diffs.append(d)
    return diffs


def tv(img, eps: float = 1e-4) -> float:
    """sum over pixels of sqrt(sum_a (x[i + e_a] - x[i])^2 + eps^2): forward
    differences along each axis a, zero difference past the last index
    (Neumann).  img: [ny][nx] (2D) or [nz][ny][nx] (3D)."""
    x = _f64(img)
    m2 = np.full_like(x, eps * eps)
    for d in _forward_differences(x):
        m2 += d * d
    return float(np.sum(np.sqrt(m2)))


def tv_grad(img, eps: float = 1e-4) -> np.ndarray:
    """Analytic gradient of ``tv``: with a_a = (difference along a) / m at each
    pixel, dTV/dx_i = -sum_a a_a(i) + sum_a a_a(i - e_a)."""
    x = _f64(img)
    diffs = _forward_differences(x)
    m = np.full_like(x, eps * eps)
    for d in diffs:
        m += d * d
    m = np.sqrt(m)
    g = np.zeros_like(x)
    for axis, d in enumerate(diffs):
        a = d / m
        g -= a
        dst = [slice(None)] * x.ndim
        src = [slice(None)] * x.ndim
        dst[axis] = slice(1, None)
        src[axis] = slice(None, -1)
        g[tuple(dst)] += a[tuple(src)]
    return g
