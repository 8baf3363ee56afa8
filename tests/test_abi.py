"""The C-ABI library builds, loads and exports every entry point of
``include/pa.h``; structure layouts agree with the binding; host-side argument
validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2404_10928_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pa.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared_functions() == sorted(_lib.SIGNATURES)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(pa_\w+)", out))
    assert set(_declared_functions()) <= exported


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "pa.h"
int main(void) {
  printf("pa_grid %zu %zu %zu\n", sizeof(pa_grid), offsetof(pa_grid, dx), offsetof(pa_grid, origin));
  printf("pa_plan_opts %zu %zu %zu %zu %zu\n", sizeof(pa_plan_opts), offsetof(pa_plan_opts, y_dtype),
         offsetof(pa_plan_opts, fwd_sensors_per_cta), offsetof(pa_plan_opts, fwd_threads),
         offsetof(pa_plan_opts, adj_warps));
  printf("pa_recon_opts %zu %zu %zu %zu %zu %zu\n", sizeof(pa_recon_opts), offsetof(pa_recon_opts, power_v0_dev),
         offsetof(pa_recon_opts, residual_history_host), offsetof(pa_recon_opts, kernel_timing),
         offsetof(pa_recon_opts, tv_eps), offsetof(pa_recon_opts, restart));
  printf("pa_plan_info %zu %zu %zu %zu %zu\n", sizeof(pa_plan_info), offsetof(pa_plan_info, tile),
         offsetof(pa_plan_info, device_bytes), offsetof(pa_plan_info, fwd_threads),
         offsetof(pa_plan_info, adj_warps));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    rows = {l.split()[0]: [int(v) for v in l.split()[1:]]
            for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                    check=True).stdout.splitlines()}
    S = _lib
    assert rows["pa_grid"] == [ctypes.sizeof(S.pa_grid), S.pa_grid.dx.offset, S.pa_grid.origin.offset]
    assert rows["pa_plan_opts"] == [ctypes.sizeof(S.pa_plan_opts), S.pa_plan_opts.y_dtype.offset,
                                    S.pa_plan_opts.fwd_sensors_per_cta.offset,
                                    S.pa_plan_opts.fwd_threads.offset,
                                    S.pa_plan_opts.adj_warps.offset]
    assert rows["pa_recon_opts"] == [ctypes.sizeof(S.pa_recon_opts), S.pa_recon_opts.power_v0_dev.offset,
                                     S.pa_recon_opts.residual_history_host.offset,
                                     S.pa_recon_opts.kernel_timing.offset,
                                     S.pa_recon_opts.tv_eps.offset, S.pa_recon_opts.restart.offset]
    assert rows["pa_plan_info"] == [ctypes.sizeof(S.pa_plan_info), S.pa_plan_info.tile.offset,
                                    S.pa_plan_info.device_bytes.offset,
                                    S.pa_plan_info.fwd_threads.offset,
                                    S.pa_plan_info.adj_warps.offset]


def _create(lib, sensors, grid, c=1500.0, fs=40e6, K=64, opts=None):
    h = ctypes.c_void_p()
    s = np.ascontiguousarray(sensors, dtype=np.float64)
    st = lib.pa_plan_create(ctypes.byref(h), s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            s.shape[0], ctypes.byref(grid) if grid is not None else None, c, fs, K,
                            ctypes.byref(opts) if opts is not None else None)
    return st, h


def _grid(dim=2, n=(8, 8, 1), h=1e-4):
    return _lib.pa_grid(dim, n[0], n[1], n[2], h, h, h, (ctypes.c_double * 3)(-3.5e-4, -3.5e-4, 0.0))


def test_argument_validation_without_gpu(lib):
    far = np.array([[0.0, 5e-3], [5e-3, 0.0]])
    assert _create(lib, far, None)[0] == _lib.PA_ERR_INVALID_ARG
    assert _create(lib, far, _grid(dim=4))[0] == _lib.PA_ERR_INVALID_ARG
    assert _create(lib, far, _grid(n=(8, 8, 2)))[0] == _lib.PA_ERR_INVALID_ARG  # 2D needs nz == 1
    assert _create(lib, far, _grid(n=(0, 8, 1)))[0] == _lib.PA_ERR_INVALID_ARG
    assert _create(lib, far, _grid(), c=0.0)[0] == _lib.PA_ERR_INVALID_ARG
    assert _create(lib, far, _grid(), fs=float("nan"))[0] == _lib.PA_ERR_INVALID_ARG
    assert _create(lib, far, _grid(), K=1)[0] == _lib.PA_ERR_INVALID_ARG
    assert _create(lib, far, _grid(h=-1e-4))[0] == _lib.PA_ERR_GEOMETRY
    assert _create(lib, np.array([[0.0, np.inf]]), _grid())[0] == _lib.PA_ERR_GEOMETRY
    # a sensor 0.2 pixel from a pixel centre is rejected (reading: d >= half a pixel)
    near = np.array([[0.5e-4 + 0.2e-4, 0.5e-4]])
    assert _create(lib, near, _grid())[0] == _lib.PA_ERR_GEOMETRY
    assert b"half the pixel" in lib.pa_last_error()
    bad_opts = _lib.pa_plan_opts(0.0, 1.0, 7, 0, 0)
    assert _create(lib, far, _grid(), opts=bad_opts)[0] == _lib.PA_ERR_INVALID_ARG
    # adjoint clusters of 1, 2, 4 or 8 CTAs only; 1..256 sensors per forward work
    # item; 64, 128 or 256 threads per forward work item; 4 or 8 adjoint warps
    for cluster, spc, nt, aw in ((3, 0, 0, 0), (9, 0, 0, 0), (-1, 0, 0, 0), (0, 257, 0, 0),
                                 (0, -2, 0, 0), (0, 0, 96, 0), (0, 0, 512, 0), (0, 0, -1, 0),
                                 (0, 0, 32, 0), (0, 0, 0, 2), (0, 0, 0, 16), (0, 0, 0, -4)):
        opts = _lib.pa_plan_opts(0.0, 1.0, _lib.PA_F32, cluster, spc, nt, aw)
        assert _create(lib, far, _grid(), opts=opts)[0] == _lib.PA_ERR_INVALID_ARG
        assert b"adj_cluster" in lib.pa_last_error()
    # the dense, frequency-domain and back-projection entry points reject NULL plans
    assert lib.pa_dense_assemble(None, _lib.PA_F64, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_dense_matvec(None, _lib.PA_F32, None, 0, None, None, None) == \
        _lib.PA_ERR_INVALID_ARG
    assert lib.pa_freq_forward(None, 16, 1e5, 1e5, None, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_freq_adjoint(None, 16, 1e5, 1e5, None, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_backproject(None, None, _lib.PA_BP_UBP, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_plan_destroy(None) == _lib.PA_OK
    assert lib.pa_forward(None, None, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_adjoint(None, None, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_reconstruct(None, 0, 1, None, None, None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_batch_set_wait_limit(None, 1.0) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_debug_fail_allocations(-2) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_debug_fail_allocations(-1) == _lib.PA_OK
    assert lib.pa_status_string(_lib.PA_ERR_TIMEOUT) == b"device wait timed out"
    assert lib.pa_version() == 1


def test_recon_opts_default(lib):
    o = _lib.pa_recon_opts()
    lib.pa_recon_opts_default(ctypes.byref(o))
    assert (o.omega, o.nonneg, o.power_iters, o.use_graph, o.kernel_timing) == (0.0, 1, 50, 1, 0)
    assert not o.power_v0_dev and not o.residual_history_host
