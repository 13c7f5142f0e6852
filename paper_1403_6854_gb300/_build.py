"""Build the CUDA scan library in-tree (nvcc, sm_103a only, no torch extension)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libselscan_gb300.so")
SOURCES = ["api.cu", "kernels.cu", "batch.cu", "noalloc.cu", "sweep.cu", "normalize.cu", "tped.cpp"]
# the integer-pipe peak measurement, a library of its own (include/selscan_peak.h)
PEAK_SOURCES = ["intpeak.cu"]
PEAK_LIB = os.path.join(PKG, "libselscan_peak.so")
HEADERS = ["walk.cuh", "internal.h", "device_common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags(ptxas_verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "-I", os.path.join(ROOT, "include")]
    # extra nvcc flags for a debugging build (e.g. -DSELSCAN_SWEEP_CHECKS=1)
    f += [x for x in os.environ.get("SELSCAN_NVCC_FLAGS", "").split() if x]
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib, sources, headers) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in sources + HEADERS] + headers
    return any(os.path.getmtime(d) > t for d in deps)


def _build_lib(lib, sources, headers, force, ptxas_verbose, quiet):
    if not force and not _stale(lib, sources, headers):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for s in sources:
        obj = os.path.join(BUILD, os.path.splitext(s)[0] + ".o")
        objs.append(obj)
        cmd = [NVCC, "-c", os.path.join(CSRC, s), "-o", obj] + _flags(ptxas_verbose)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((cmd, text))
        elif text and (ptxas_verbose or not quiet):
            sys.stderr.write(text)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + f".tmp{os.getpid()}"
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    cmd = [NVCC, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared",
                                                         "-Xlinker", "-rpath," + cuda_lib]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True) -> str:
    """Compile every translation unit in parallel and link libselscan_gb300.so
    (the scan library) and libselscan_peak.so (the integer-peak measurement)."""
    _build_lib(PEAK_LIB, PEAK_SOURCES, [os.path.join(ROOT, "include", "selscan_peak.h")], force,
               ptxas_verbose, quiet)
    return _build_lib(LIB, SOURCES, [os.path.join(ROOT, "include", "selscan.h")], force,
                      ptxas_verbose, quiet)


if __name__ == "__main__":
    build(force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv, quiet=False)
    print(LIB)
