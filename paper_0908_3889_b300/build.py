"""Build the CUDA library ``libpn_b300.so`` in-tree for sm_103a (B300) with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpn_b300.so")
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


def _nvcc(out: str, sources, verbose: bool) -> None:
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-o", out + ".tmp", *sources]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the integrator (and the peak probe bench.py uses) if missing or stale; returns the library path."""
    if force or _stale(LIB, _deps()):
        _nvcc(LIB, SOURCES, verbose)
    if force or _stale(PEAK_LIB, [PEAK_SRC]):
        _nvcc(PEAK_LIB, [PEAK_SRC], verbose)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
