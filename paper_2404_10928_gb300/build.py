"""Builds the sm_103a shared library ``libpa.so`` in-tree with nvcc.

Usage: ``python -m paper_2404_10928_gb300.build`` (or ``build()`` from Python).
Each translation unit compiles in parallel; the objects go to ``_build/`` next
to this file and the library to ``libpa.so`` beside it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpa.so")
BUILD_DIR = os.path.join(HERE, "_build")
# the checked build (-DPA_CHECKED): index checks in the gathers and the combine
# that latch PA_ERR_DEVICE_CHECK instead of touching memory out of range
OUT_CHECKED = os.path.join(HERE, "libpa_checked.so")
BUILD_DIR_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["pa_plan.cu", "pa_ops.cu", "pa_recon.cu", "pa_static.cu", "pa_batch.cu", "pa_dense.cu",
           "pa_freq.cu", "pa_frames.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpa.so")


def cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _stale(extra_flags, out=OUT) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "pa.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps) or bool(extra_flags)


def build(force: bool = False, extra_flags=(), verbose: bool = False,
          checked: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link libpa.so (with checked=True
    the index-checked libpa_checked.so).  Returns the library's path."""
    out, build_dir = (OUT_CHECKED, BUILD_DIR_CHECKED) if checked else (OUT, BUILD_DIR)
    if not force and not _stale(extra_flags, out):
        return out
    nvcc = nvcc_path()
    os.makedirs(build_dir, exist_ok=True)
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]
    if checked:
        common.append("-DPA_CHECKED")
    common += list(extra_flags)
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    libdir = cuda_lib_dir(nvcc)
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", f"-rpath,{libdir}"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
