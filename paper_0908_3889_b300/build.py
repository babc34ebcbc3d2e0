"""Build the CUDA library ``libpn_b300.so`` in-tree for sm_103a (B300) with nvcc, and beside it its
debug build ``libpn_b300_debug.so`` (``-DPN_DEBUG``: device bounds checks reported as PN_E_CHECK)."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpn_b300.so")
DEBUG_LIB = os.path.join(HERE, "libpn_b300_debug.so")
PEAK_LIB = os.path.join(HERE, "libpn_peak.so")
PEAK_SRC = os.path.join(HERE, "csrc", "peak_probe.cu")
SOURCES = [os.path.join(HERE, "csrc", "pn_kernels.cu"), os.path.join(HERE, "csrc", "pn_capi.cu"),
           os.path.join(HERE, "csrc", "pn_noalloc.cu"), os.path.join(HERE, "csrc", "pn_analysis.cu"),
           os.path.join(HERE, "csrc", "pn_adjoint.cu")]
# the integrator's own headers (the peak probe is built separately)
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def _deps():
    return SOURCES + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(HERE, "csrc", "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(lib: str, deps) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def _nvcc(out: str, sources, verbose: bool, extra=()) -> subprocess.Popen:
    """Start one nvcc compile into out (written under a temporary name until it succeeds)."""
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-o", out + ".tmp", *sources]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    return subprocess.Popen(cmd)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the integrator, its debug build and the peak probe bench.py uses, each if missing or stale
    (the compiles run side by side); returns the release library's path."""
    jobs = []
    if force or _stale(LIB, _deps()):
        jobs.append((LIB, _nvcc(LIB, SOURCES, verbose)))
    if force or _stale(DEBUG_LIB, _deps()):
        jobs.append((DEBUG_LIB, _nvcc(DEBUG_LIB, SOURCES, verbose, ["-DPN_DEBUG"])))
    if force or _stale(PEAK_LIB, [PEAK_SRC]):
        jobs.append((PEAK_LIB, _nvcc(PEAK_LIB, [PEAK_SRC], verbose)))
    failed = [out for out, p in jobs if p.wait() != 0]
    if failed:
        for out, _ in jobs:  # no partial output is left beside the sources
            if os.path.exists(out + ".tmp"):
                os.remove(out + ".tmp")
        raise RuntimeError("nvcc failed for " + ", ".join(os.path.basename(f) for f in failed))
    for out, _ in jobs:
        os.replace(out + ".tmp", out)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
