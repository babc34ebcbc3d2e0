"""CPU FP64 oracle for batched post-Newtonian inspirals (arXiv:0908.3889).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference arm may import this package.  It is
independent of the CUDA library: it shares no source, header, table or
constant with ``paper_0908_3889_b300`` and does not import it.

The arithmetic lives in ``pn_oracle.cpp`` (plain C++17, FP64, compiled with
``-ffp-contract=off``); this module builds it with g++ and wraps its
``extern "C"`` functions with ctypes.  See the header of ``pn_oracle.cpp`` for
what each function computes, the paper passages it follows, the readings taken
where the paper is silent, and which functions are pinned by which tests.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pn_oracle.cpp")
_LIB = os.path.join(_HERE, "libpn_oracle.so")
ABI_VERSION = 3

# PN term bits (same meaning as the oracle's T_* enum).
T_1PN, T_SO, T_TAIL, T_2PN, T_SS, T_25PN, T_3PN, T_35PN, T_PREC = (1 << i for i in range(9))
T_ALL = 0x1FF
NEWTONIAN = T_PREC  # leading-order chirp, precession on
ST_OK, ST_MAX_STEPS, ST_H_UNDERFLOW, ST_NONFINITE, ST_BAD_INPUT, ST_LAND_MAXIT = range(6)


def _compile(src: str, out: str) -> None:
    cmd = ["g++", "-std=c++17", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-Wall", "-o", out + ".tmp", src]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    """Compile pn_oracle.cpp into libpn_oracle.so (portable -O3, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def build_variant(src_text: str, directory: str, name: str) -> str:
    """Compile a modified copy of the oracle's source (a planted mistake, for checking that the pins catch
    it) into directory/name.so with the oracle's own flags; returns the library path."""
    src = os.path.join(directory, name + ".cpp")
    with open(src, "w") as fh:
        fh.write(src_text)
    out = os.path.join(directory, name + ".so")
    _compile(src, out)
    return out


@contextlib.contextmanager
def variant(path: str):
    """Route every wrapper in this module through another build of the oracle while the block runs."""
    global _lib
    saved = lib()
    _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


class Params(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double), ("safety", C.c_double),
                ("fac_min", C.c_double), ("fac_max", C.c_double), ("h_min", C.c_double),
                ("land_tol", C.c_double), ("max_steps", C.c_int64), ("land_max_iter", C.c_int32),
                ("stop_mode", C.c_int32), ("term_mask", C.c_uint32), ("theta_mode", C.c_int32),
                ("fixed_step", C.c_int32), ("pad_", C.c_int32)]


def params(**kw) -> Params:
    """Defaults: tolerance 5e-7 and h0 = 10 (Sec. II); the rest are our readings."""
    d = dict(rtol=5e-7, atol=5e-7, h0=10.0, safety=0.9, fac_min=0.2, fac_max=10.0, h_min=1e-10,
             land_tol=1e-7, max_steps=1_000_000, land_max_iter=8, stop_mode=0, term_mask=T_ALL,
             theta_mode=0, fixed_step=0, pad_=0)
    d.update(kw)
    return Params(**d)


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)


class _BatchIn(C.Structure):
    _fields_ = [(n, _DP) for n in ("m1", "m2", "chi1", "chi2", "s1x", "s1y", "s1z", "s2x", "s2y", "s2z",
                                   "lx", "ly", "lz", "omega0", "omega_f")]


class _BatchOut(C.Structure):
    _fields_ = ([(n, _DP) for n in ("S1x", "S1y", "S1z", "S2x", "S2y", "S2z", "Lx", "Ly", "Lz", "omega", "t")]
                + [(n, _IP) for n in ("n_acc", "n_rej", "n_land", "status")]
                + [(n, _DP) for n in ("dot_s1s2", "dot_ls1", "dot_ls2")])


class _Dist(C.Structure):
    _fields_ = [("q_mode", C.c_int32), ("chi_mode", C.c_int32), ("q_lo", C.c_double), ("q_hi", C.c_double),
                ("chi_lo", C.c_double), ("chi_hi", C.c_double), ("omega0_lo", C.c_double),
                ("omega0_hi", C.c_double), ("omega_f", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(L):
    """Declare the argument and result types of the oracle's extern "C" functions on a loaded library."""
    L.oracle_abi_version.restype = C.c_int
    assert L.oracle_abi_version() == ABI_VERSION
    L.oracle_tableau.argtypes = [_DP, _DP, _DP, _DP]
    L.oracle_rhs.argtypes = [C.POINTER(Params), C.c_double, C.c_double, _DP, _DP]
    L.oracle_dp5_attempt.argtypes = [C.POINTER(Params), C.c_double, C.c_double, _DP, C.c_double, _DP]
    L.oracle_dp5_attempt.restype = C.c_double
    L.oracle_integrate_batch.argtypes = [C.c_int64, C.POINTER(_BatchIn), C.POINTER(Params),
                                         C.POINTER(_BatchOut), C.c_int]
    L.oracle_integrate_batch.restype = C.c_int
    L.oracle_trace.argtypes = [C.POINTER(_BatchIn), C.c_int64, C.POINTER(Params), _DP, C.c_int64, _DP,
                               C.c_int64]
    L.oracle_trace.restype = C.c_int64
    L.oracle_replay.argtypes = [C.POINTER(_BatchIn), C.c_int64, C.POINTER(Params), _DP, C.c_int64, _DP, _DP]
    L.oracle_replay.restype = C.c_int
    L.oracle_grad.argtypes = [C.POINTER(_BatchIn), C.c_int64, C.POINTER(Params), _DP, _DP]
    L.oracle_grad.restype = C.c_int64
    L.oracle_count_ops.argtypes = [C.POINTER(Params), C.c_double, C.c_double, _DP,
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.oracle_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
    L.oracle_splitmix64_next.restype = C.c_uint64
    L.oracle_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.oracle_uniform.restype = C.c_double
    L.oracle_sample.argtypes = [C.c_uint64, C.POINTER(_Dist), C.c_int64] + [_DP] * 15
    L.oracle_sample_at.argtypes = [C.c_uint64, C.POINTER(_Dist), C.POINTER(C.c_int64), C.c_int64] + [_DP] * 15
    return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


INPUT_KEYS = ("m1", "m2", "chi1", "chi2", "s1hat", "s2hat", "lhat", "omega0", "omega_f")
OUTPUT_KEYS = ("S1", "S2", "Lhat", "omega", "t", "n_acc", "n_rej", "n_land", "status",
               "dot_s1s2", "dot_ls1", "dot_ls2")


def _as_batch_in(inp: dict):
    """inp: dict of numpy arrays; scalars (n,), vectors (3, n) component-major."""
    keep = {}
    n = int(np.asarray(inp["m1"]).shape[0])

    def arr(x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        keep[id(a)] = a
        return a

    v = {k: arr(inp[k]) for k in INPUT_KEYS}
    for k in ("s1hat", "s2hat", "lhat"):
        assert v[k].shape == (3, n), (k, v[k].shape)
    b = _BatchIn(m1=_dp(v["m1"]), m2=_dp(v["m2"]), chi1=_dp(v["chi1"]), chi2=_dp(v["chi2"]),
                 s1x=_dp(v["s1hat"][0]), s1y=_dp(v["s1hat"][1]), s1z=_dp(v["s1hat"][2]),
                 s2x=_dp(v["s2hat"][0]), s2y=_dp(v["s2hat"][1]), s2z=_dp(v["s2hat"][2]),
                 lx=_dp(v["lhat"][0]), ly=_dp(v["lhat"][1]), lz=_dp(v["lhat"][2]),
                 omega0=_dp(v["omega0"]), omega_f=_dp(v["omega_f"]))
    return b, n, (v, keep)


def integrate(inp: dict, prm: Params | None = None, threads: int = 0) -> dict:
    """Integrate every binary of ``inp``; returns numpy outputs (vectors (3, n))."""
    prm = prm or params()
    b, n, hold = _as_batch_in(inp)
    out = {"S1": np.empty((3, n)), "S2": np.empty((3, n)), "Lhat": np.empty((3, n)),
           "omega": np.empty(n), "t": np.empty(n), "dot_s1s2": np.empty(n), "dot_ls1": np.empty(n),
           "dot_ls2": np.empty(n)}
    for k in ("n_acc", "n_rej", "n_land", "status"):
        out[k] = np.empty(n, dtype=np.int32)
    ip = lambda a: a.ctypes.data_as(_IP)
    bo = _BatchOut(S1x=_dp(out["S1"][0]), S1y=_dp(out["S1"][1]), S1z=_dp(out["S1"][2]),
                   S2x=_dp(out["S2"][0]), S2y=_dp(out["S2"][1]), S2z=_dp(out["S2"][2]),
                   Lx=_dp(out["Lhat"][0]), Ly=_dp(out["Lhat"][1]), Lz=_dp(out["Lhat"][2]),
                   omega=_dp(out["omega"]), t=_dp(out["t"]), n_acc=ip(out["n_acc"]), n_rej=ip(out["n_rej"]),
                   n_land=ip(out["n_land"]), status=ip(out["status"]), dot_s1s2=_dp(out["dot_s1s2"]),
                   dot_ls1=_dp(out["dot_ls1"]), dot_ls2=_dp(out["dot_ls2"]))
    used = lib().oracle_integrate_batch(n, C.byref(b), C.byref(prm), C.byref(bo), int(threads))
    out["threads_used"] = used
    del hold
    return out


def rhs(y, m1: float, m2: float, prm: Params | None = None) -> np.ndarray:
    prm = prm or params()
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.empty(10)
    lib().oracle_rhs(C.byref(prm), m1, m2, _dp(y), _dp(f))
    return f


def dp5_attempt(y, h: float, m1: float, m2: float, prm: Params | None = None):
    prm = prm or params()
    y = np.ascontiguousarray(y, dtype=np.float64)
    y5 = np.empty(10)
    err = lib().oracle_dp5_attempt(C.byref(prm), m1, m2, _dp(y), h, _dp(y5))
    return y5, err


def tableau():
    c, a, b, bh = np.empty(7), np.empty(42), np.empty(7), np.empty(7)
    lib().oracle_tableau(_dp(c), _dp(a), _dp(b), _dp(bh))
    return c, a.reshape(7, 6), b, bh


def trace(inp: dict, i: int, prm: Params | None = None, cap: int = 200000):
    """Accepted trajectory of binary i: rows (t, y[10]) and the accepted step sizes."""
    prm = prm or params()
    b, n, hold = _as_batch_in(inp)
    rows = np.empty((cap, 11))
    hs = np.empty(cap)
    nr = lib().oracle_trace(C.byref(b), i, C.byref(prm), _dp(rows), cap, _dp(hs), cap)
    del hold
    nr = min(nr, cap)
    return rows[:nr].copy(), hs[: nr - 1].copy()


def replay(inp: dict, i: int, hs: np.ndarray, prm: Params | None = None):
    prm = prm or params()
    b, n, hold = _as_batch_in(inp)
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    y = np.empty(10)
    t = C.c_double()
    rc = lib().oracle_replay(C.byref(b), i, C.byref(prm), _dp(hs), len(hs), _dp(y), C.byref(t))
    del hold
    if rc != 0:
        raise RuntimeError("replay failed")
    return y, t.value


GRAD_OUTPUTS = ("dot_s1s2", "dot_ls1", "dot_ls2", "Lx", "Ly", "Lz", "S1x", "S1y", "S1z", "S2x", "S2y", "S2z", "t")
GRAD_PARAMS = ("s1x", "s1y", "s1z", "s2x", "s2y", "s2z", "q")


def grad(inp: dict, i: int, prm: Params | None = None):
    """Forward-mode Jacobian (13 outputs x 7 parameters) of binary i; see GRAD_OUTPUTS/GRAD_PARAMS."""
    prm = prm or params()
    b, n, hold = _as_batch_in(inp)
    out = np.empty(13)
    jac = np.empty(13 * 7)
    nacc = lib().oracle_grad(C.byref(b), i, C.byref(prm), _dp(out), _dp(jac))
    del hold
    if nacc < 0:
        raise RuntimeError("gradient unavailable (binary did not land cleanly)")
    return out, jac.reshape(13, 7), int(nacc)


def count_ops(y, m1: float, m2: float, prm: Params | None = None):
    """(rhs_counts, step_counts), each (add, mul, div, sqrt, cbrt, log, pow)."""
    prm = prm or params()
    y = np.ascontiguousarray(y, dtype=np.float64)
    r = (C.c_int64 * 7)()
    s = (C.c_int64 * 7)()
    lib().oracle_count_ops(C.byref(prm), m1, m2, _dp(y), r, s)
    return tuple(r), tuple(s)


def splitmix64(seed: int, count: int) -> list[int]:
    st = C.c_uint64(seed)
    return [int(lib().oracle_splitmix64_next(C.byref(st))) for _ in range(count)]


def uniform(seed: int, i: int, j: int) -> float:
    return lib().oracle_uniform(seed, i, j)


@dataclass
class Dist:
    q_mode: int = 0
    chi_mode: int = 0
    q_lo: float = 1.0
    q_hi: float = 1.0
    chi_lo: float = 1.0
    chi_hi: float = 1.0
    omega0_lo: float = 0.01
    omega0_hi: float = 0.01
    omega_f: float = 0.05


def sample(seed: int, dist: Dist, n: int, idx=None) -> dict:
    """The paper's initial-data draw (Sec. V) from counter-based SplitMix64 uniforms: binaries 0..n-1,
    or the binaries with the given indices (each depends only on the seed and its own index)."""
    d = _Dist(**dist.__dict__)
    if idx is not None:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        n = idx.shape[0]
    a = {k: np.empty(n) for k in ("m1", "m2", "chi1", "chi2", "omega0", "omega_f")}
    for k in ("s1hat", "s2hat", "lhat"):
        a[k] = np.empty((3, n))
    ip = idx.ctypes.data_as(C.POINTER(C.c_int64)) if idx is not None else None
    lib().oracle_sample_at(seed, C.byref(d), ip, n, _dp(a["m1"]), _dp(a["m2"]), _dp(a["chi1"]), _dp(a["chi2"]),
                           _dp(a["s1hat"][0]), _dp(a["s1hat"][1]), _dp(a["s1hat"][2]),
                           _dp(a["s2hat"][0]), _dp(a["s2hat"][1]), _dp(a["s2hat"][2]),
                           _dp(a["lhat"][0]), _dp(a["lhat"][1]), _dp(a["lhat"][2]),
                           _dp(a["omega0"]), _dp(a["omega_f"]))
    return a
