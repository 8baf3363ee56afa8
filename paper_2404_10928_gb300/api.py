"""Python face of the library: a ``Plan`` around the C ABI of ``include/pa.h``.

Device memory and streams come from PyTorch; every step of the computation
runs in the library's own CUDA kernels.  Methods check tensor shapes, dtypes
and devices, then pass raw pointers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (PA_BP_NONE, PA_BP_UBP, PA_CGLS, PA_F16, PA_F32, PA_F64, PA_FISTA,
                   PA_LANDWEBER, PA_PCGLS, check)

METHODS = {"landweber": PA_LANDWEBER, "cgls": PA_CGLS, "fista": PA_FISTA, "pcgls": PA_PCGLS}
BP_FILTERS = {"none": PA_BP_NONE, "ubp": PA_BP_UBP}
_DENSE_DTYPES = {torch.float64: PA_F64, torch.float32: PA_F32}


def _stream_handle(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Plan:
    """One imaging geometry on one GPU (see ``pa_plan_create``)."""

    def __init__(self, sensors, shape, spacing, origin, c: float, fs: float, n_samples: int,
                 t0: float = 0.0, amp_scale: float = 1.0, y_dtype: str = "f32",
                 dim: Optional[int] = None, device=None, adj_cluster: int = 0,
                 fwd_sensors_per_cta: int = 0, fwd_threads: int = 0, adj_warps: int = 0):
        self._lib = _lib.load()
        sensors = np.ascontiguousarray(sensors, dtype=np.float64)
        dim = int(dim if dim is not None else sensors.shape[1])
        shape = tuple(int(v) for v in shape) + (1,) * (3 - len(shape))
        spacing = tuple(float(v) for v in spacing) + (float(spacing[-1]),) * (3 - len(spacing))
        origin = tuple(float(v) for v in origin) + (0.0,) * (3 - len(origin))
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.dim, self.shape, self.spacing, self.origin = dim, shape, spacing, origin
        self.n_sensors = int(sensors.shape[0])
        self.n_samples = int(n_samples)
        self.n_pixels = shape[0] * shape[1] * shape[2]
        self.c, self.fs, self.t0, self.amp_scale = float(c), float(fs), float(t0), float(amp_scale)
        self.y_dtype = y_dtype
        self._sensors = sensors  # keep alive for the call
        grid = _lib.pa_grid(dim, shape[0], shape[1], shape[2], spacing[0], spacing[1], spacing[2],
                            (ctypes.c_double * 3)(*origin))
        opts = _lib.pa_plan_opts(self.t0, self.amp_scale, PA_F16 if y_dtype == "f16" else PA_F32,
                                 int(adj_cluster), int(fwd_sensors_per_cta), int(fwd_threads),
                                 int(adj_warps))
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self._lib.pa_plan_create(ctypes.byref(handle),
                                          sensors.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          self.n_sensors, ctypes.byref(grid), self.c, self.fs,
                                          self.n_samples, ctypes.byref(opts))
        check(st, "pa_plan_create")
        self._h = handle

    @classmethod
    def from_problem(cls, prob, c: Optional[float] = None, y_dtype: Optional[str] = None, **kw):
        return cls(prob.sensors, prob.shape, prob.spacing, prob.origin,
                   prob.c if c is None else c, prob.fs, prob.n_samples, t0=prob.t0,
                   amp_scale=prob.amp_scale,
                   y_dtype=y_dtype or prob.extra.get("y_dtype", "f32"), dim=prob.dim, **kw)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pa_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- helpers ----------------------------------------------------------
    def _check_tensor(self, t: torch.Tensor, numel: int, name: str, dtype=torch.float32):
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{name} must be contiguous with {numel} elements")

    def info(self) -> dict:
        inf = _lib.pa_plan_info()
        check(self._lib.pa_plan_query(self._h, ctypes.byref(inf)), "pa_plan_query")
        return {"n_pixels": inf.n_pixels, "n_sensors": inf.n_sensors, "n_samples": inf.n_samples,
                "pairs": inf.pairs, "tile": tuple(inf.tile), "window": inf.window,
                "cluster": inf.cluster, "fwd_sensors": inf.fwd_sensors,
                "fwd_threads": inf.fwd_threads, "adj_warps": inf.adj_warps,
                "device_bytes": inf.device_bytes}

    def set_sound_speed(self, c: float):
        check(self._lib.pa_plan_set_sound_speed(self._h, float(c)), "pa_plan_set_sound_speed")
        self.c = float(c)

    def sync_status(self):
        check(self._lib.pa_plan_sync_status(self._h), "pa_plan_sync_status")

    # -- operators --------------------------------------------------------
    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """p = A x: [N] image -> [S][K] traces."""
        self._check_tensor(x, self.n_pixels, "x")
        if out is None:
            out = torch.empty((self.n_sensors, self.n_samples), device=self.device,
                              dtype=torch.float32)
        self._check_tensor(out, self.n_sensors * self.n_samples, "out")
        check(self._lib.pa_forward(self._h, x.data_ptr(), out.data_ptr(),
                                   _stream_handle(self.device)), "pa_forward")
        return out

    def adjoint(self, p: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """x = A^T p: [S][K] traces -> [N] image."""
        self._check_tensor(p, self.n_sensors * self.n_samples, "p")
        if out is None:
            out = torch.empty(self.n_pixels, device=self.device, dtype=torch.float32)
        self._check_tensor(out, self.n_pixels, "out")
        check(self._lib.pa_adjoint(self._h, p.data_ptr(), out.data_ptr(),
                                   _stream_handle(self.device)), "pa_adjoint")
        return out

    def backproject(self, p: torch.Tensor, filter: str = "ubp",
                    out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """x = A^T F(p): back-projection of [S][K] traces, F = "ubp" (universal
        back-projection term 2p - 2t dp/dt) or "none" (see ``pa_backproject``)."""
        self._check_tensor(p, self.n_sensors * self.n_samples, "p")
        if filter not in BP_FILTERS:
            raise ValueError(f"filter must be one of {sorted(BP_FILTERS)}")
        if out is None:
            out = torch.empty(self.n_pixels, device=self.device, dtype=torch.float32)
        self._check_tensor(out, self.n_pixels, "out")
        check(self._lib.pa_backproject(self._h, p.data_ptr(), BP_FILTERS[filter], out.data_ptr(),
                                       _stream_handle(self.device)), "pa_backproject")
        return out

    # -- frequency-domain model (Eq. 7; see pa_freq_forward / pa_freq_adjoint) --
    def freq_forward(self, x: torch.Tensor, n_freq: int, f0: float, df: float,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """P = K x: [N] image -> [S][n_freq] complex64 spectra at f0 + n df."""
        self._check_tensor(x, self.n_pixels, "x")
        if out is None:
            out = torch.empty((self.n_sensors, n_freq), dtype=torch.complex64, device=self.device)
        if out.dtype != torch.complex64 or not out.is_contiguous() or \
                out.numel() != self.n_sensors * n_freq or out.device != self.device:
            raise ValueError("out must be a contiguous complex64 [S][n_freq] tensor on the device")
        check(self._lib.pa_freq_forward(self._h, int(n_freq), float(f0), float(df), x.data_ptr(),
                                        out.data_ptr(), _stream_handle(self.device)),
              "pa_freq_forward")
        return out

    def freq_adjoint(self, p: torch.Tensor, n_freq: int, f0: float, df: float,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """x = K^H p (real part): [S][n_freq] complex64 -> [N] image."""
        if p.dtype != torch.complex64 or not p.is_contiguous() or \
                p.numel() != self.n_sensors * n_freq or p.device != self.device:
            raise ValueError("p must be a contiguous complex64 [S][n_freq] tensor on the device")
        if out is None:
            out = torch.empty(self.n_pixels, dtype=torch.float32, device=self.device)
        self._check_tensor(out, self.n_pixels, "out")
        check(self._lib.pa_freq_adjoint(self._h, int(n_freq), float(f0), float(df), p.data_ptr(),
                                        out.data_ptr(), _stream_handle(self.device)),
              "pa_freq_adjoint")
        return out

    # -- dense-matrix mode (see pa_dense_assemble / pa_dense_matvec) ---------
    def dense_assemble(self, dtype: torch.dtype = torch.float64,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The matrix of A, [S*K][N] row-major, in float64 or float32."""
        code = _DENSE_DTYPES.get(dtype)
        if code is None:
            raise ValueError("dtype must be torch.float64 or torch.float32")
        rows, cols = self.n_sensors * self.n_samples, self.n_pixels
        if out is None:
            out = torch.empty((rows, cols), dtype=dtype, device=self.device)
        self._check_tensor(out, rows * cols, "out", dtype)
        check(self._lib.pa_dense_assemble(self._h, code, out.data_ptr(),
                                          _stream_handle(self.device)), "pa_dense_assemble")
        return out

    def dense_matvec(self, m: torch.Tensor, v: torch.Tensor, transpose: bool = False,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """M v ([N] -> [S*K]) or M^T v ([S*K] -> [N]) for an assembled matrix."""
        code = _DENSE_DTYPES.get(m.dtype)
        if code is None:
            raise ValueError("m must be float64 or float32")
        rows, cols = self.n_sensors * self.n_samples, self.n_pixels
        self._check_tensor(m, rows * cols, "m", m.dtype)
        n_in, n_out = (rows, cols) if transpose else (cols, rows)
        self._check_tensor(v, n_in, "v", m.dtype)
        if out is None:
            out = torch.empty(n_out, dtype=m.dtype, device=self.device)
        self._check_tensor(out, n_out, "out", m.dtype)
        check(self._lib.pa_dense_matvec(self._h, code, m.data_ptr(), int(bool(transpose)),
                                        v.data_ptr(), out.data_ptr(), _stream_handle(self.device)),
              "pa_dense_matvec")
        return out

    def dc(self, x: torch.Tensor, g: torch.Tensor, out: Optional[torch.Tensor] = None):
        """d/dc <g, A(x; c)> as a float64 scalar tensor on the device."""
        self._check_tensor(x, self.n_pixels, "x")
        self._check_tensor(g, self.n_sensors * self.n_samples, "g")
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        check(self._lib.pa_dc(self._h, x.data_ptr(), g.data_ptr(), out.data_ptr(),
                              _stream_handle(self.device)), "pa_dc")
        return out

    def tv(self, x: torch.Tensor, eps: float = 1e-4, grad: Optional[torch.Tensor] = None):
        """Smoothed TV of x and its gradient: (float64 scalar tensor, [N] float32)."""
        self._check_tensor(x, self.n_pixels, "x")
        if grad is None:
            grad = torch.empty(self.n_pixels, dtype=torch.float32, device=self.device)
        self._check_tensor(grad, self.n_pixels, "grad")
        val = torch.empty((), dtype=torch.float64, device=self.device)
        check(self._lib.pa_tv(self._h, x.data_ptr(), float(eps), val.data_ptr(), grad.data_ptr(),
                              _stream_handle(self.device)), "pa_tv")
        return val, grad

    # -- several frames on this geometry (one launch per operator) ----------
    def _frames_img(self, t: torch.Tensor, name: str) -> int:
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float32:
            raise ValueError(f"{name} must be a float32 tensor on {self.device}")
        if not t.is_contiguous() or t.numel() % self.n_pixels or t.numel() == 0:
            raise ValueError(f"{name} must be contiguous with a multiple of {self.n_pixels} elements")
        return t.numel() // self.n_pixels

    def _frames_trace(self, t: torch.Tensor, n: int, name: str, dtype=torch.float32):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise ValueError(f"{name} must be a {dtype} tensor on {self.device}")
        if not t.is_contiguous() or t.numel() != n * self.n_sensors * self.n_samples:
            raise ValueError(f"{name} must be contiguous with {n} x {self.n_sensors} x "
                             f"{self.n_samples} elements")

    def _ydtype(self):
        return torch.float16 if self.y_dtype == "f16" else torch.float32

    def forward_frames(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """p[f] = A x[f] for x of shape [F, N]; returns [F, S, K]."""
        n = self._frames_img(x, "x")
        if out is None:
            out = torch.empty((n, self.n_sensors, self.n_samples), device=self.device)
        self._frames_trace(out, n, "out")
        check(self._lib.pa_forward_frames(self._h, n, x.data_ptr(), out.data_ptr(),
                                          _stream_handle(self.device)), "pa_forward_frames")
        return out

    def adjoint_frames(self, p: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """x[f] = A^T p[f] for p of shape [F, S, K]; returns [F, N]."""
        n = p.numel() // max(self.n_sensors * self.n_samples, 1)
        self._frames_trace(p, n, "p")
        if out is None:
            out = torch.empty((n, self.n_pixels), device=self.device)
        self._frames_img(out, "out")
        check(self._lib.pa_adjoint_frames(self._h, n, p.data_ptr(), out.data_ptr(),
                                          _stream_handle(self.device)), "pa_adjoint_frames")
        return out

    def residual_frames(self, x: torch.Tensor, y: torch.Tensor, r: Optional[torch.Tensor] = None,
                        norms: bool = False):
        """r[f] = y[f] - A x[f] (and the float64 norms ||r[f]||^2 when asked)."""
        n = self._frames_img(x, "x")
        self._frames_trace(y, n, "y", self._ydtype())
        if r is None:
            r = torch.empty((n, self.n_sensors, self.n_samples), device=self.device)
        self._frames_trace(r, n, "r")
        sq = torch.empty(n, dtype=torch.float64, device=self.device) if norms else None
        check(self._lib.pa_residual_frames(self._h, n, x.data_ptr(), y.data_ptr(), r.data_ptr(),
                                           sq.data_ptr() if norms else None,
                                           _stream_handle(self.device)), "pa_residual_frames")
        return (r, sq) if norms else r

    def adjoint_axpy_frames(self, p: torch.Tensor, coef: float, xin: Optional[torch.Tensor] = None,
                            tvg: Optional[torch.Tensor] = None, tv_weight: float = 0.0,
                            nonneg: bool = False, out: Optional[torch.Tensor] = None):
        """out[f] = [max(0,)](xin[f] + coef A^T p[f] + tv_weight tvg[f])."""
        n = p.numel() // max(self.n_sensors * self.n_samples, 1)
        self._frames_trace(p, n, "p")
        for t, name in ((xin, "xin"), (tvg, "tvg")):
            if t is not None and self._frames_img(t, name) != n:
                raise ValueError(f"{name} must hold {n} frames")
        if out is None:
            out = torch.empty((n, self.n_pixels), device=self.device)
        self._frames_img(out, "out")
        check(self._lib.pa_adjoint_axpy_frames(
            self._h, n, p.data_ptr(), xin.data_ptr() if xin is not None else None, float(coef),
            tvg.data_ptr() if tvg is not None else None, float(tv_weight), int(bool(nonneg)),
            out.data_ptr(), _stream_handle(self.device)), "pa_adjoint_axpy_frames")
        return out

    def dc_frames(self, x: torch.Tensor, g: torch.Tensor, scale: float = 1.0,
                  out: Optional[torch.Tensor] = None, accumulate: bool = False):
        """scale * sum_f d/dc <g[f], A(x[f]; c)> as a float64 scalar tensor."""
        n = self._frames_img(x, "x")
        self._frames_trace(g, n, "g")
        if out is None:
            out = torch.zeros((), dtype=torch.float64, device=self.device)
        check(self._lib.pa_dc_frames(self._h, n, x.data_ptr(), g.data_ptr(), float(scale),
                                     int(bool(accumulate)), out.data_ptr(),
                                     _stream_handle(self.device)), "pa_dc_frames")
        return out

    def tv_frames(self, x: torch.Tensor, eps: float = 1e-4, grad: Optional[torch.Tensor] = None):
        """Per-frame smoothed TV (float64 [F]) and gradients ([F, N])."""
        n = self._frames_img(x, "x")
        if grad is None:
            grad = torch.empty((n, self.n_pixels), device=self.device)
        self._frames_img(grad, "grad")
        val = torch.empty(n, dtype=torch.float64, device=self.device)
        check(self._lib.pa_tv_frames(self._h, n, x.data_ptr(), float(eps), val.data_ptr(),
                                     grad.data_ptr(), _stream_handle(self.device)), "pa_tv_frames")
        return val, grad

    def landweber_step_frames(self, x: torch.Tensor, y: torch.Tensor, omega: float,
                              nonneg: bool = True, out: Optional[torch.Tensor] = None):
        """x_out[f] = [max(0,)](x[f] + omega A^T (y[f] - A x[f]))."""
        n = self._frames_img(x, "x")
        self._frames_trace(y, n, "y", self._ydtype())
        if out is None:
            out = torch.empty((n, self.n_pixels), device=self.device)
        self._frames_img(out, "out")
        check(self._lib.pa_landweber_step_frames(self._h, n, x.data_ptr(), y.data_ptr(),
                                                 float(omega), int(bool(nonneg)), out.data_ptr(),
                                                 _stream_handle(self.device)),
              "pa_landweber_step_frames")
        return out

    def landweber_step_vjp_frames(self, x, y, x_out, g_out, omega: float, nonneg: bool = True,
                                  need_y: bool = False, need_c: bool = False):
        """(gx, gy or None, gc or None) of one Landweber step for the gradient g_out."""
        n = self._frames_img(x, "x")
        self._frames_trace(y, n, "y", self._ydtype())
        for t, name in ((x_out, "x_out"), (g_out, "g_out")):
            if self._frames_img(t, name) != n:
                raise ValueError(f"{name} must hold {n} frames")
        gx = torch.empty((n, self.n_pixels), device=self.device)
        gy = torch.empty((n, self.n_sensors, self.n_samples), device=self.device) if need_y else None
        gc = torch.zeros((), dtype=torch.float64, device=self.device) if need_c else None
        check(self._lib.pa_landweber_step_vjp_frames(
            self._h, n, x.data_ptr(), y.data_ptr(), x_out.data_ptr(), g_out.data_ptr(),
            float(omega), int(bool(nonneg)), gx.data_ptr(),
            gy.data_ptr() if gy is not None else None, gc.data_ptr() if gc is not None else None,
            _stream_handle(self.device)), "pa_landweber_step_vjp_frames")
        return gx, gy, gc

    def data_tv_loss_frames(self, x: torch.Tensor, y: torch.Tensor, tv_weight: float,
                            eps: float = 1e-4):
        """(loss float64 scalar, residuals [F, S, K], TV gradients [F, N] or None)."""
        n = self._frames_img(x, "x")
        self._frames_trace(y, n, "y", self._ydtype())
        loss = torch.empty((), dtype=torch.float64, device=self.device)
        r = torch.empty((n, self.n_sensors, self.n_samples), device=self.device)
        tg = torch.empty((n, self.n_pixels), device=self.device) if tv_weight != 0.0 else None
        check(self._lib.pa_data_tv_loss_frames(
            self._h, n, x.data_ptr(), y.data_ptr(), float(tv_weight), float(eps), loss.data_ptr(),
            r.data_ptr(), tg.data_ptr() if tg is not None else None, _stream_handle(self.device)),
            "pa_data_tv_loss_frames")
        return loss, r, tg

    def data_tv_loss_vjp_frames(self, x, r, tvgrad, tv_weight: float, g_loss: float,
                                need_x: bool = True, need_c: bool = False):
        """(gx or None, gc or None) of the data + TV loss times g_loss."""
        n = self._frames_img(x, "x")
        self._frames_trace(r, n, "r")
        gx = torch.empty((n, self.n_pixels), device=self.device) if need_x else None
        gc = torch.zeros((), dtype=torch.float64, device=self.device) if need_c else None
        check(self._lib.pa_data_tv_loss_vjp_frames(
            self._h, n, x.data_ptr(), r.data_ptr(),
            tvgrad.data_ptr() if tvgrad is not None else None, float(tv_weight), float(g_loss),
            gx.data_ptr() if gx is not None else None, gc.data_ptr() if gc is not None else None,
            _stream_handle(self.device)), "pa_data_tv_loss_vjp_frames")
        return gx, gc

    def power_iteration(self, n_iter: int = 50, v0: Optional[torch.Tensor] = None) -> float:
        if v0 is not None:
            self._check_tensor(v0, self.n_pixels, "v0")
        out = ctypes.c_double()
        check(self._lib.pa_power_iteration(self._h, int(n_iter),
                                           v0.data_ptr() if v0 is not None else None,
                                           ctypes.byref(out), _stream_handle(self.device)),
              "pa_power_iteration")
        return out.value

    def _opts(self, omega, nonneg, power_iters, power_v0, hist, use_graph, kernel_timing,
              l1=0.0, tv=0.0, tv_eps=1e-4, restart=0):
        o = _lib.pa_recon_opts()
        self._lib.pa_recon_opts_default(ctypes.byref(o))
        o.restart = int(restart)
        o.l1_weight = float(l1)
        o.tv_weight = float(tv)
        o.tv_eps = float(tv_eps)
        o.omega = float(omega)
        o.nonneg = int(bool(nonneg))
        o.power_iters = int(power_iters)
        o.power_v0_dev = power_v0.data_ptr() if power_v0 is not None else None
        o.residual_history_host = (hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                   if hist is not None else None)
        o.use_graph = int(bool(use_graph))
        o.kernel_timing = int(bool(kernel_timing))
        return o

    def reconstruct(self, y: torch.Tensor, method: str = "cgls", n_iter: int = 50,
                    x0: Optional[torch.Tensor] = None, omega: float = 0.0, nonneg: bool = True,
                    power_iters: int = 50, power_v0: Optional[torch.Tensor] = None,
                    history: bool = False, use_graph: bool = True, kernel_timing: bool = False,
                    out: Optional[torch.Tensor] = None, l1: float = 0.0, tv: float = 0.0,
                    tv_eps: float = 1e-4, restart: int = 0):
        """Minimise ||A x - y||^2 (Landweber with projection, CGLS + final clamp, or
        "pcgls": CGLS projected onto x >= 0 every step, restarted every ``restart``
        iterations), or with method "fista" ||A x - y||^2 + l1 ||x||_1 + tv TV_eps(x)
        (Eq. 8).

        Returns x (and the residual history ||y - A x_n||^2, n = 0..n_iter, when
        ``history`` is set).  ``out`` (if given) is used in place: its contents
        are the start image unless ``x0`` is given."""
        ydt = torch.float16 if self.y_dtype == "f16" else torch.float32
        self._check_tensor(y, self.n_sensors * self.n_samples, "y", ydt)
        if out is None:
            out = (x0.clone() if x0 is not None else
                   torch.zeros(self.n_pixels, device=self.device, dtype=torch.float32))
        elif x0 is not None:
            out.copy_(x0)
        self._check_tensor(out, self.n_pixels, "x")
        if power_v0 is not None:
            self._check_tensor(power_v0, self.n_pixels, "power_v0")
        hist = np.zeros(n_iter + 1) if history else None
        o = self._opts(omega, nonneg, power_iters, power_v0, hist, use_graph, kernel_timing,
                       l1, tv, tv_eps, restart)
        check(self._lib.pa_reconstruct(self._h, METHODS[method], int(n_iter), y.data_ptr(),
                                       out.data_ptr(), ctypes.byref(o),
                                       _stream_handle(self.device)), "pa_reconstruct")
        return (out, hist) if history else out

    def reconstruct_host(self, y: np.ndarray, method: str = "cgls", n_iter: int = 50,
                         x0: Optional[np.ndarray] = None, omega: float = 0.0, nonneg: bool = True,
                         power_iters: int = 50, use_graph: bool = True,
                         x_out: Optional[np.ndarray] = None) -> np.ndarray:
        """Same as ``reconstruct`` with host (numpy, ideally pinned) buffers."""
        ydt = np.float16 if self.y_dtype == "f16" else np.float32
        if y.dtype != ydt or not y.flags.c_contiguous or y.size != self.n_sensors * self.n_samples:
            raise ValueError(f"y must be a contiguous {ydt} array of {self.n_sensors}x{self.n_samples}")
        if x_out is None:
            x_out = (np.array(x0, dtype=np.float32) if x0 is not None
                     else np.zeros(self.n_pixels, dtype=np.float32))
        if x_out.dtype != np.float32 or not x_out.flags.c_contiguous or x_out.size != self.n_pixels:
            raise ValueError("x_out must be a contiguous float32 array of n_pixels")
        o = self._opts(omega, nonneg, power_iters, None, None, use_graph, False)
        check(self._lib.pa_reconstruct_host(self._h, METHODS[method], int(n_iter), y.ctypes.data,
                                            x_out.ctypes.data, ctypes.byref(o),
                                            _stream_handle(self.device)), "pa_reconstruct_host")
        return x_out

    def time_gathers(self, x: torch.Tensor, p: torch.Tensor, reps: int = 20) -> dict:
        """Average device time (ms) of one application of A and of one A^T
        gather launch, each timed over `reps` back-to-back launches."""
        self._check_tensor(x, self.n_pixels, "x")
        self._check_tensor(p, self.n_sensors * self.n_samples, "p")
        fm, am = ctypes.c_double(), ctypes.c_double()
        check(self._lib.pa_plan_time_gathers(self._h, int(reps), x.data_ptr(), p.data_ptr(),
                                             ctypes.byref(fm), ctypes.byref(am),
                                             _stream_handle(self.device)), "pa_plan_time_gathers")
        return {"fwd_ms": fm.value, "adj_ms": am.value, "reps": int(reps)}

    # -- sensor-sharded CGLS (pa_shard_cgls_*; the driver is shard.sharded_cgls) --
    def shard_cgls_begin(self, n_iter: int, y: torch.Tensor, x: torch.Tensor,
                         s_part: torch.Tensor, accumulate: bool = False) -> None:
        ydt = torch.float16 if self.y_dtype == "f16" else torch.float32
        self._check_tensor(y, self.n_sensors * self.n_samples, "y", ydt)
        self._check_tensor(x, self.n_pixels, "x")
        self._check_tensor(s_part, self.n_pixels, "s_part")
        check(self._lib.pa_shard_cgls_begin(self._h, int(n_iter), y.data_ptr(), x.data_ptr(),
                                            s_part.data_ptr(), int(bool(accumulate)),
                                            _stream_handle(self.device)), "pa_shard_cgls_begin")

    def shard_cgls_direction(self, it: int, s: torch.Tensor, delta_part: torch.Tensor,
                             accumulate: bool = False) -> None:
        self._check_tensor(s, self.n_pixels, "s")
        self._check_tensor(delta_part, 1, "delta_part", torch.float64)
        check(self._lib.pa_shard_cgls_direction(self._h, int(it), s.data_ptr(),
                                                delta_part.data_ptr(), int(bool(accumulate)),
                                                _stream_handle(self.device)),
              "pa_shard_cgls_direction")

    def shard_cgls_update(self, it: int, delta: torch.Tensor, x: Optional[torch.Tensor],
                          s_part: torch.Tensor, accumulate: bool = False) -> None:
        self._check_tensor(delta, 1, "delta", torch.float64)
        if x is not None:
            self._check_tensor(x, self.n_pixels, "x")
        self._check_tensor(s_part, self.n_pixels, "s_part")
        check(self._lib.pa_shard_cgls_update(self._h, int(it), delta.data_ptr(),
                                             x.data_ptr() if x is not None else None,
                                             s_part.data_ptr(), int(bool(accumulate)),
                                             _stream_handle(self.device)), "pa_shard_cgls_update")

    def shard_cgls_finish(self, x: Optional[torch.Tensor], nonneg: bool,
                          hist: Optional[torch.Tensor], accumulate: bool = False) -> None:
        if x is not None:
            self._check_tensor(x, self.n_pixels, "x")
        if hist is not None and (hist.device != self.device or hist.dtype != torch.float64
                                 or not hist.is_contiguous()):
            raise ValueError(f"hist must be a contiguous float64 tensor on {self.device}")
        check(self._lib.pa_shard_cgls_finish(self._h, x.data_ptr() if x is not None else None,
                                             int(bool(nonneg)),
                                             hist.data_ptr() if hist is not None else None,
                                             int(bool(accumulate)), _stream_handle(self.device)),
              "pa_shard_cgls_finish")

    def kernel_times(self) -> dict:
        fm, am = ctypes.c_double(), ctypes.c_double()
        fn, an = ctypes.c_int(), ctypes.c_int()
        check(self._lib.pa_plan_kernel_times(self._h, ctypes.byref(fm), ctypes.byref(fn),
                                             ctypes.byref(am), ctypes.byref(an)),
              "pa_plan_kernel_times")
        return {"fwd_ms": fm.value, "n_fwd": fn.value, "adj_ms": am.value, "n_adj": an.value}


class Batch:
    """Several plans (frames of uneven size) reconstructed together by one
    persistent launch per call (see ``pa_batch_landweber``)."""

    def __init__(self, plans):
        self._lib = _lib.load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        check(self._lib.pa_batch_create(ctypes.byref(h), arr, len(self.plans)), "pa_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_wait_limit(self, seconds: float):
        """Limit of each grid-barrier wait of the persistent launch (seconds)."""
        check(self._lib.pa_batch_set_wait_limit(self._h, float(seconds)), "pa_batch_set_wait_limit")

    def reconstruct(self, ys, xs, method: str = "cgls", n_iter: int = 50, omegas=None,
                    nonneg: bool = True, history: bool = False):
        """Run n_iter iterations of `method` ("landweber" or "cgls") on every frame
        in one persistent launch (xs: start images, receive the results)."""
        n = len(self.plans)
        if not (len(ys) == len(xs) == n) or (omegas is not None and len(omegas) != n):
            raise ValueError("need one y and x (and omega) per frame")
        for p, y, x in zip(self.plans, ys, xs):
            ydt = torch.float16 if p.y_dtype == "f16" else torch.float32
            p._check_tensor(y, p.n_sensors * p.n_samples, "y", ydt)
            p._check_tensor(x, p.n_pixels, "x")
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        om = (ctypes.c_double * n)(*[float(o) for o in omegas]) if omegas is not None else None
        hist = np.zeros((n, n_iter + 1)) if history else None
        hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history else None
        check(self._lib.pa_batch_reconstruct(self._h, METHODS[method], int(n_iter), yp, xp, om,
                                             int(bool(nonneg)), hp,
                                             _stream_handle(self.plans[0].device)),
              "pa_batch_reconstruct")
        return hist

    def landweber(self, ys, xs, omegas, n_iter: int, nonneg: bool = True, history: bool = False):
        """Run n_iter projected Landweber steps on every frame in place (xs are the
        start images and receive the results)."""
        n = len(self.plans)
        if not (len(ys) == len(xs) == len(omegas) == n):
            raise ValueError("need one y, x and omega per frame")
        for p, y, x in zip(self.plans, ys, xs):
            ydt = torch.float16 if p.y_dtype == "f16" else torch.float32
            p._check_tensor(y, p.n_sensors * p.n_samples, "y", ydt)
            p._check_tensor(x, p.n_pixels, "x")
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        om = (ctypes.c_double * n)(*[float(o) for o in omegas])
        hist = np.zeros((n, n_iter + 1)) if history else None
        hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history else None
        check(self._lib.pa_batch_landweber(self._h, int(n_iter), yp, xp, om, int(bool(nonneg)), hp,
                                           _stream_handle(self.plans[0].device)),
              "pa_batch_landweber")
        return hist
