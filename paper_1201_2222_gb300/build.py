"""Build the CUDA library ``librtsc.so`` (and a bounds-checked ``librtsc_debug.so``).

nvcc for sm_103a only; the translation units compile in parallel and are linked
into one shared library in the package directory (git-ignored).  The CUDA
runtime is linked statically so the library does not depend on which
``libcudart`` the host process has loaded.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["rt_api.cu", "rt_kernels.cu", "rt_quad.cu", "rt_server.cu", "rt_gs.cu", "rt_probe.cu"]
HEADERS = ["rt_common.cuh", "rt_kernels.h", "rt_device.cuh", "rt_lockstep.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def lib_path(debug: bool = False) -> str:
    return os.path.join(HERE, "librtsc_debug.so" if debug else "librtsc.so")


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "rt_sc.h"))
    return files


def up_to_date(debug: bool = False) -> bool:
    out = lib_path(debug)
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(debug: bool = False, force: bool = False, verbose: bool = False) -> str:
    out = lib_path(debug)
    if not force and up_to_date(debug):
        return out
    nvcc = _nvcc()
    bdir = os.path.join(HERE, "_build", "debug" if debug else "release")
    os.makedirs(bdir, exist_ok=True)
    # -ftz=true: float32 subnormals flush to zero, so the sweep's fast exp and
    # reciprocal are single special-function instructions (FP64 is unaffected)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                     "-I", CSRC]
    if debug:
        common.append("-DRT_DEBUG_BOUNDS")
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + log.decode(errors="replace"))
        if verbose and log:
            sys.stdout.write(log.decode(errors="replace"))
    tmp = out + f".tmp{os.getpid()}"
    link = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(link, capture_output=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode() + r.stderr.decode())
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    dbg = "--debug" in sys.argv
    print(build(debug=dbg, force="--force" in sys.argv, verbose=True))
