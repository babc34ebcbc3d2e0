"""Python binding of the C ABI (include/pn_batch.h): same names, torch tensors for memory and streams.

Every function here only marshals arguments; all of the integration, the
set-up included (masses from mass ratios: pn_batch_masses), runs in the CUDA
library.  Ensembles are dicts of float64 tensors on one CUDA device:

  inputs   m1, m2, chi1, chi2, omega0, omega_f: shape (n,)
           s1hat, s2hat, lhat: shape (3, n), component-major (structure of arrays)
  outputs  S1, S2, Lhat: (3, n); omega, t, dot_s1s2, dot_ls1, dot_ls2: (n,) float64;
           n_acc, n_rej, n_land, status: (n,) int32
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N

INPUT_KEYS = ("m1", "m2", "chi1", "chi2", "s1hat", "s2hat", "lhat", "omega0", "omega_f")
VEC_INPUTS = ("s1hat", "s2hat", "lhat")
OUTPUT_KEYS = ("S1", "S2", "Lhat", "omega", "t", "n_acc", "n_rej", "n_land", "status",
               "dot_s1s2", "dot_ls1", "dot_ls2")
_ERR = {N.PN_E_ARG: "PN_E_ARG", N.PN_E_CUDA: "PN_E_CUDA", N.PN_E_NOMEM: "PN_E_NOMEM",
        N.PN_E_UNIMPLEMENTED: "PN_E_UNIMPLEMENTED"}


class PNError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR.get(code, code)}: {msg}")
        self.code = code


def _lib():
    return N.load()


def _check(rc: int, handle) -> None:
    if rc != N.PN_OK:
        raise PNError(rc, (_lib().pn_last_error(handle) or b"").decode())


def params(**kw) -> N.pn_params:
    """pn_params with the library defaults, fields overridden by keyword."""
    p = N.pn_params()
    _lib().pn_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _dptr(t: torch.Tensor):
    return C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double))


def _iptr(t: torch.Tensor):
    return C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_int32))


def _check_tensor(t: torch.Tensor, n: int, dtype, name: str, rows: int | None = None, device=None):
    """Arrays may be longer than n (the C ABI reads elements 0..n-1); rows of a vector must be contiguous."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    ok_shape = (t.dim() == 1 and rows is None) or (rows is not None and t.dim() == 2 and t.shape[0] == rows)
    if not ok_shape or t.shape[-1] < n:
        want = f"({n},)" if rows is None else f"({rows}, >= {n})"
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {want}")
    if t.stride(-1) != 1:
        raise ValueError(f"{name} must be contiguous along the binary index")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")


def inputs_struct(inp: dict, n: int | None = None) -> N.pn_inputs:
    n = int(inp["m1"].shape[0]) if n is None else n
    dev = inp["m1"].device
    for k in INPUT_KEYS:
        _check_tensor(inp[k], n, torch.float64, k, 3 if k in VEC_INPUTS else None, dev)
    s = N.pn_inputs()
    for k in ("m1", "m2", "chi1", "chi2", "omega0", "omega_f"):
        setattr(s, k, _dptr(inp[k]))
    for k, pre in (("s1hat", "s1"), ("s2hat", "s2"), ("lhat", "l")):
        for c, ax in enumerate("xyz"):
            setattr(s, pre + ax, _dptr(inp[k][c]))
    return s


def outputs_struct(out: dict, n: int | None = None) -> N.pn_outputs:
    n = int(out["omega"].shape[0]) if n is None else n
    dev = out["omega"].device
    s = N.pn_outputs()
    for k, pre in (("S1", "S1"), ("S2", "S2"), ("Lhat", "L")):
        _check_tensor(out[k], n, torch.float64, k, 3, dev)
        for c, ax in enumerate("xyz"):
            setattr(s, pre + ax, _dptr(out[k][c]))
    for k in ("omega", "t", "dot_s1s2", "dot_ls1", "dot_ls2"):
        _check_tensor(out[k], n, torch.float64, k, None, dev)
        setattr(s, k, _dptr(out[k]))
    for k in ("n_acc", "n_rej", "n_land", "status"):
        _check_tensor(out[k], n, torch.int32, k, None, dev)
        setattr(s, k, _iptr(out[k]))
    return s


def alloc_inputs(n: int, device="cuda", pin_memory: bool = False) -> dict:
    """One (15, n) float64 block with per-field views."""
    kw = dict(dtype=torch.float64, device=device)
    blk = torch.empty((15, n), **kw) if not pin_memory else torch.empty((15, n), dtype=torch.float64, pin_memory=True)
    d = {"m1": blk[0], "m2": blk[1], "chi1": blk[2], "chi2": blk[3], "s1hat": blk[4:7], "s2hat": blk[7:10],
         "lhat": blk[10:13], "omega0": blk[13], "omega_f": blk[14]}
    d["_block"] = blk
    return d


def alloc_outputs(n: int, device="cuda", pin_memory: bool = False) -> dict:
    """One (14, n) float64 block and one (4, n) int32 block with per-field views."""
    if pin_memory:
        fb = torch.empty((14, n), dtype=torch.float64, pin_memory=True)
        ib = torch.empty((4, n), dtype=torch.int32, pin_memory=True)
    else:
        fb = torch.empty((14, n), dtype=torch.float64, device=device)
        ib = torch.empty((4, n), dtype=torch.int32, device=device)
    return {"S1": fb[0:3], "S2": fb[3:6], "Lhat": fb[6:9], "omega": fb[9], "t": fb[10], "dot_s1s2": fb[11],
            "dot_ls1": fb[12], "dot_ls2": fb[13], "n_acc": ib[0], "n_rej": ib[1], "n_land": ib[2], "status": ib[3],
            "_block": fb, "_iblock": ib}


def to_device(ens: dict, device="cuda", pin_memory: bool = False) -> dict:
    """Copy a NumPy ensemble (workloads layout) into a fresh input block."""
    n = int(np.asarray(ens["m1"]).shape[0])
    d = alloc_inputs(n, device, pin_memory)
    for k in INPUT_KEYS:
        d[k].copy_(torch.from_numpy(np.ascontiguousarray(ens[k], dtype=np.float64)))
    return d


def segment(tensors: dict, lo: int, hi: int) -> dict:
    """Views of binaries lo .. hi - 1 of an input or output dict (pointers offset by lo, no copy), for
    calling any entry point on one ensemble of a concatenated batch."""
    return {k: v[..., lo:hi] for k, v in tensors.items() if not k.startswith("_")}


def to_numpy(out: dict) -> dict:
    return {k: out[k].cpu().numpy() for k in OUTPUT_KEYS if k in out}


# ---------------------------------------------------------------------------
# The C ABI, function by function.
# ---------------------------------------------------------------------------
def pn_abi_version() -> int:
    return _lib().pn_abi_version()


def pn_batch_init(n_max: int, prm: N.pn_params | None = None, stream=None) -> C.c_void_p:
    prm = prm or params()
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    h = C.c_void_p()
    _check(_lib().pn_batch_init(C.byref(h), int(n_max), C.byref(prm), C.c_void_p(sp)), None)
    return h


def pn_batch_set_params(h, prm: N.pn_params) -> None:
    _check(_lib().pn_batch_set_params(h, C.byref(prm)), h)


def pn_batch_sample(h, seed: int, dist: N.pn_dist, n: int, inputs: dict) -> None:
    _check(_lib().pn_batch_sample(h, C.c_uint64(seed), C.byref(dist), int(n), C.byref(inputs_struct(inputs, n))), h)


def pn_batch_integrate(h, n: int, inputs: dict, outputs: dict) -> None:
    _check(_lib().pn_batch_integrate(h, int(n), C.byref(inputs_struct(inputs, n)),
                                     C.byref(outputs_struct(outputs, n))), h)


def pn_batch_integrate_budget(h, n: int, inputs: dict, outputs: dict, budget: int) -> None:
    _check(_lib().pn_batch_integrate_budget(h, int(n), C.byref(inputs_struct(inputs, n)),
                                            C.byref(outputs_struct(outputs, n)), int(budget)), h)


def pn_batch_resume(h, n: int, inputs: dict, outputs: dict, budget: int = 0) -> None:
    _check(_lib().pn_batch_resume(h, int(n), C.byref(inputs_struct(inputs, n)), C.byref(outputs_struct(outputs, n)),
                                  int(budget)), h)


def _host_inputs_struct(inp: dict, n: int) -> N.pn_inputs:
    for k in INPUT_KEYS:
        _check_tensor(inp[k], n, torch.float64, k, 3 if k in VEC_INPUTS else None, torch.device("cpu"))
    return inputs_struct(inp, n)


def pn_batch_integrate_host(h, n: int, host_inputs: dict, host_outputs: dict) -> None:
    """Host (CPU, ideally pinned) tensors in and out; copies happen inside the call, which synchronises."""
    _check(_lib().pn_batch_integrate_host(h, int(n), C.byref(_host_inputs_struct(host_inputs, n)),
                                          C.byref(outputs_struct(host_outputs, n))), h)


def pn_batch_integrate_host_async(h, n: int, host_inputs: dict, host_outputs: dict) -> None:
    """Enqueue a host-buffer integration and return; consecutive calls overlap their copies with the
    neighbouring integrations.  The host tensors must stay untouched until pn_batch_host_wait."""
    _check(_lib().pn_batch_integrate_host_async(h, int(n), C.byref(_host_inputs_struct(host_inputs, n)),
                                                C.byref(outputs_struct(host_outputs, n))), h)


def pn_batch_timing(h) -> tuple:
    """(ms of the last integration call, ms of its integration kernel alone), CUDA events; waits for it."""
    mc, mk = C.c_double(), C.c_double()
    _check(_lib().pn_batch_timing(h, C.byref(mc), C.byref(mk)), h)
    return mc.value, mk.value


def pn_batch_host_wait(h) -> None:
    """Wait for every pn_batch_integrate_host_async call on the batch to have copied its outputs back."""
    _check(_lib().pn_batch_host_wait(h), h)


def pn_batch_autotune(h, n: int, inputs: dict, scratch: dict) -> dict:
    r = N.pn_tune_result()
    _check(_lib().pn_batch_autotune(h, int(n), C.byref(inputs_struct(inputs, n)),
                                    C.byref(outputs_struct(scratch, n)), C.byref(r)), h)
    return {f: getattr(r, f) for f, _ in N.pn_tune_result._fields_}


def pn_batch_adjoint(h, n: int, inputs: dict, cotangents: dict, grads: dict, outputs: dict | None = None) -> None:
    cs = N.pn_cotangents()
    dev = inputs["m1"].device
    for f in N.COT_FIELDS:
        t = cotangents.get(f)
        if t is not None:
            _check_tensor(t, n, torch.float64, f, None, dev)
            setattr(cs, f, _dptr(t))
    gs = N.pn_grads()
    for f in N.GRAD_FIELDS:
        _check_tensor(grads[f], n, torch.float64, f, None, dev)
        setattr(gs, f, _dptr(grads[f]))
    for f in N.GRAD_TAN_FIELDS + N.GRAD_ANGLE_FIELDS:  # optional
        if grads.get(f) is not None:
            _check_tensor(grads[f], n, torch.float64, f, None, dev)
            setattr(gs, f, _dptr(grads[f]))
    os_ = C.byref(outputs_struct(outputs, n)) if outputs is not None else None
    _check(_lib().pn_batch_adjoint(h, int(n), C.byref(inputs_struct(inputs, n)), C.byref(cs), C.byref(gs), os_), h)


def pn_batch_eval_rhs(h, n: int, m1: torch.Tensor, m2: torch.Tensor, y: torch.Tensor, f: torch.Tensor) -> None:
    """f(y) of Eqs. (1)-(4) at n states in the batch's precision; y, f: (10, n) float64 CUDA tensors, contiguous."""
    for t, rows in ((m1, None), (m2, None), (y, 10), (f, 10)):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise PNError("pn_batch_eval_rhs needs contiguous float64 CUDA tensors")
        if (rows is None and t.shape != (n,)) or (rows is not None and t.shape != (rows, n)):
            raise PNError("pn_batch_eval_rhs: m1, m2 must be (n,), y and f (10, n)")
    _check(_lib().pn_batch_eval_rhs(h, int(n), _dptr(m1), _dptr(m2), _dptr(y), _dptr(f)), h)


def pn_batch_masses(h, n: int, q: torch.Tensor, m1: torch.Tensor, m2: torch.Tensor) -> None:
    """m1 = q/(1+q), m2 = 1/(1+q) on the device (the set-up's first step, M = 1)."""
    dev = q.device
    for t, name in ((q, "q"), (m1, "m1"), (m2, "m2")):
        _check_tensor(t, n, torch.float64, name, None, dev)
    _check(_lib().pn_batch_masses(h, int(n), _dptr(q), _dptr(m1), _dptr(m2)), h)


def _stats_dict(s: N.pn_stats) -> dict:
    d = {f: getattr(s, f) for f, _ in N.pn_stats._fields_}
    d["count_by_status"] = list(s.count_by_status)
    return d


def pn_batch_stats(h, n: int, inputs: dict, outputs: dict) -> dict:
    s = N.pn_stats()
    _check(_lib().pn_batch_stats(h, int(n), C.byref(inputs_struct(inputs, n)), C.byref(outputs_struct(outputs, n)),
                                 C.byref(s)), h)
    return _stats_dict(s)


def pn_batch_stats_segments(h, offsets, inputs: dict, outputs: dict) -> list:
    """Statistics of each segment [offsets[k], offsets[k + 1]) of one batch, one dict per segment."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_seg = int(off.shape[0]) - 1
    if n_seg < 0:
        raise ValueError("offsets needs at least one entry")
    n = int(off[-1])
    recs = (N.pn_stats * max(n_seg, 1))()
    _check(_lib().pn_batch_stats_segments(h, n_seg, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                          C.byref(inputs_struct(inputs, n)), C.byref(outputs_struct(outputs, n)),
                                          recs), h)
    return [_stats_dict(recs[k]) for k in range(n_seg)]


def pn_batch_histogram(h, n: int, inputs: dict, outputs: dict, quantity_x: int, nx: int, x_range=(-1.0, 1.0),
                       quantity_y: int = 0, ny: int = 1, y_range=(-1.0, 1.0)) -> np.ndarray:
    """Counts as int64: shape (nx,) for a 1-D histogram, (nx, ny) for 2-D (x = quantity_x)."""
    sp = N.pn_hist_spec(quantity_x=quantity_x, quantity_y=quantity_y, nx=nx, ny=ny, x_lo=x_range[0], x_hi=x_range[1],
                        y_lo=y_range[0], y_hi=y_range[1])
    counts = np.zeros(nx * ny, dtype=np.int64)
    _check(_lib().pn_batch_histogram(h, int(n), C.byref(inputs_struct(inputs, n)), C.byref(outputs_struct(outputs, n)),
                                     C.byref(sp), counts.ctypes.data_as(C.POINTER(C.c_int64))), h)
    return counts if ny == 1 else counts.reshape(nx, ny)


def pn_batch_kde(h, n: int, inputs: dict, outputs: dict, quantity: int, grid) -> tuple:
    """(density at grid, bandwidth h = 1.06 sigma N^-1/5)."""
    g = np.ascontiguousarray(grid, dtype=np.float64)
    dens = np.empty_like(g)
    bw = C.c_double()
    _check(_lib().pn_batch_kde(h, int(n), C.byref(inputs_struct(inputs, n)), C.byref(outputs_struct(outputs, n)),
                               int(quantity), g.ctypes.data_as(C.POINTER(C.c_double)), g.shape[0],
                               dens.ctypes.data_as(C.POINTER(C.c_double)), C.byref(bw)), h)
    return dens, bw.value


def pn_ks_uniform(counts, lo: float = -1.0, hi: float = 1.0) -> dict:
    """Kolmogorov-Smirnov test of binned counts against U[lo, hi] (host only): n, d_lo <= D <= d_hi and
    the p-values at both bounds."""
    c = np.ascontiguousarray(np.asarray(counts), dtype=np.int64)
    r = N.pn_ks_result()
    _check(_lib().pn_ks_uniform(c.ctypes.data_as(C.POINTER(C.c_int64)), int(c.shape[0]), float(lo), float(hi),
                                C.byref(r)), None)
    return {f: getattr(r, f) for f, _ in N.pn_ks_result._fields_}


def pn_integrate_noalloc(n: int, prm: N.pn_params, inputs: dict, outputs: dict, stream=None) -> None:
    """The library's no-allocation entry point (n <= 16384 binaries, persistent schedule)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(_lib().pn_integrate_noalloc(int(n), C.byref(prm), C.byref(inputs_struct(inputs, n)),
                                       C.byref(outputs_struct(outputs, n)), C.c_void_p(sp)), None)


def pn_batch_destroy(h) -> None:
    if h:
        _lib().pn_batch_destroy(h)


def pn_last_error(h=None) -> str:
    return (_lib().pn_last_error(h) or b"").decode()


# ---------------------------------------------------------------------------
# Conveniences.
# ---------------------------------------------------------------------------
@dataclass
class Batch:
    """Owns one pn_batch handle (use as a context manager)."""
    n_max: int
    prm: N.pn_params | None = None
    stream: object = None

    def __post_init__(self):
        self.handle = pn_batch_init(self.n_max, self.prm, self.stream)

    def close(self):
        if getattr(self, "handle", None):
            pn_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, prm: N.pn_params):
        pn_batch_set_params(self.handle, prm)

    def integrate(self, inputs: dict, outputs: dict | None = None, n: int | None = None) -> dict:
        n = int(inputs["m1"].shape[0]) if n is None else n
        outputs = alloc_outputs(n, inputs["m1"].device) if outputs is None else outputs
        pn_batch_integrate(self.handle, n, inputs, outputs)
        return outputs

    def eval_rhs(self, m1: torch.Tensor, m2: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
        """The right-hand side at the states y (10, n) in this batch's precision; returns f (10, n)."""
        f = torch.empty_like(y)
        pn_batch_eval_rhs(self.handle, int(y.shape[1]), m1, m2, y, f)
        return f

    def integrate_budget(self, inputs: dict, outputs: dict | None = None, budget: int = 64,
                         n: int | None = None) -> dict:
        """Start a bounded run (pn_batch_integrate_budget): at most `budget` attempts per binary."""
        n = int(inputs["m1"].shape[0]) if n is None else n
        outputs = alloc_outputs(n, inputs["m1"].device) if outputs is None else outputs
        pn_batch_integrate_budget(self.handle, n, inputs, outputs, budget)
        return outputs

    def resume(self, inputs: dict, outputs: dict, budget: int = 0, n: int | None = None) -> dict:
        """Continue the binaries left PN_ST_RUNNING (pn_batch_resume); budget 0 runs them to the end."""
        n = int(inputs["m1"].shape[0]) if n is None else n
        pn_batch_resume(self.handle, n, inputs, outputs, budget)
        return outputs

    def sample(self, seed: int, dist: N.pn_dist, n: int, inputs: dict | None = None, device="cuda") -> dict:
        inputs = alloc_inputs(n, device) if inputs is None else inputs
        pn_batch_sample(self.handle, seed, dist, n, inputs)
        return inputs

    def stats(self, inputs: dict, outputs: dict, n: int | None = None) -> dict:
        n = int(inputs["m1"].shape[0]) if n is None else n
        return pn_batch_stats(self.handle, n, inputs, outputs)

    def timing(self) -> tuple:
        return pn_batch_timing(self.handle)

    def stats_segments(self, inputs: dict, outputs: dict, offsets) -> list:
        return pn_batch_stats_segments(self.handle, offsets, inputs, outputs)

    def histogram(self, inputs: dict, outputs: dict, quantity_x: int, nx: int, **kw) -> np.ndarray:
        return pn_batch_histogram(self.handle, int(inputs["m1"].shape[0]), inputs, outputs, quantity_x, nx, **kw)

    def kde(self, inputs: dict, outputs: dict, quantity: int, grid) -> tuple:
        return pn_batch_kde(self.handle, int(inputs["m1"].shape[0]), inputs, outputs, quantity, grid)

    def autotune(self, inputs: dict, n: int | None = None) -> dict:
        n = int(inputs["m1"].shape[0]) if n is None else n
        scratch = alloc_outputs(min(n, 262144) if n else 1, inputs["m1"].device)
        # the scratch outputs only need to cover the tuning prefix
        return pn_batch_autotune(self.handle, min(n, 262144), inputs, scratch)


def dist(q=(1.0, 1.0), q_mode: int = 0, chi=(1.0, 1.0), chi_mode: int = 0, omega0=(0.01, 0.01),
         omega_f: float = 0.05) -> N.pn_dist:
    return N.pn_dist(q_mode=q_mode, chi_mode=chi_mode, q_lo=q[0], q_hi=q[1], chi_lo=chi[0], chi_hi=chi[1],
                     omega0_lo=omega0[0], omega0_hi=omega0[1], omega_f=omega_f)


def integrate(inputs: dict, **kw) -> dict:
    """Integrate a device ensemble with the given parameter overrides; returns the output dict."""
    n = int(inputs["m1"].shape[0])
    with Batch(max(n, 1), params(**kw)) as b:
        return b.integrate(inputs)


def sweep(ensembles: list, device="cuda", **kw):
    """Several NumPy ensembles (workloads layout) integrated in ONE pn_batch_integrate call, concatenated
    along the binary index, with per-ensemble statistics from one pn_batch_stats_segments reduction.
    Returns (inputs, outputs, offsets, stats): device tensors of the whole batch, the segment offsets and
    one statistics dict per ensemble."""
    sizes = [int(np.asarray(e["m1"]).shape[0]) for e in ensembles]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    cat = {k: np.concatenate([np.asarray(e[k], dtype=np.float64) for e in ensembles], axis=-1) for k in INPUT_KEYS}
    inputs = to_device(cat, device=device)
    with Batch(max(n, 1), params(**kw)) as b:
        outputs = b.integrate(inputs)
        stats = pn_batch_stats_segments(b.handle, offsets, inputs, outputs)
    return inputs, outputs, offsets, stats


class PNAdjointFn(torch.autograd.Function):
    """Final outputs as a differentiable function of the initial spin directions and the mass ratio.

    apply(s1hat (3, n), s2hat (3, n), q (n,), chi1, chi2, omega0, omega_f, lhat (3, n), prm=None)
    returns (dot_s1s2, dot_ls1, dot_ls2, Lhat (3, n), S1 (3, n), S2 (3, n), t); the library forms the
    masses m1 = q/(1+q), m2 = 1/(1+q) (M = 1, pn_batch_masses).  backward calls pn_batch_adjoint:
    reverse mode through the accepted
    Dormand-Prince steps with the step sizes held fixed and the stop at omega_f differentiated as an
    implicit function.  Needs PN_FP64 and PN_STOP_LAND.
    """

    @staticmethod
    def forward(ctx, s1hat, s2hat, q, chi1, chi2, omega0, omega_f, lhat, prm=None):
        n = int(q.shape[0])
        inp = alloc_inputs(n, q.device)
        inp["s1hat"].copy_(s1hat.detach())
        inp["s2hat"].copy_(s2hat.detach())
        for k, v in (("chi1", chi1), ("chi2", chi2), ("omega0", omega0), ("omega_f", omega_f), ("lhat", lhat)):
            inp[k].copy_(v.detach())
        b = Batch(n, prm or params())
        pn_batch_masses(b.handle, n, q.detach().contiguous(), inp["m1"], inp["m2"])
        out = b.integrate(inp)
        ctx.pn = (b, inp, n)
        return (out["dot_s1s2"].clone(), out["dot_ls1"].clone(), out["dot_ls2"].clone(), out["Lhat"].clone(),
                out["S1"].clone(), out["S2"].clone(), out["t"].clone())

    @staticmethod
    def backward(ctx, g12, gl1, gl2, gL, gS1, gS2, gt):
        b, inp, n = ctx.pn
        cot = {}
        for k, g in (("dot_s1s2", g12), ("dot_ls1", gl1), ("dot_ls2", gl2), ("t", gt)):
            if g is not None:
                cot[k] = g.contiguous()
        for name, g in (("L", gL), ("S1", gS1), ("S2", gS2)):
            if g is not None:
                g = g.contiguous()
                for c, ax in enumerate("xyz"):
                    cot[name + ax] = g[c].contiguous()
        grads = {f: torch.empty(n, dtype=torch.float64, device=inp["m1"].device) for f in N.GRAD_FIELDS}
        pn_batch_adjoint(b.handle, n, inp, cot, grads)
        b.close()
        gs1 = torch.stack([grads["s1x"], grads["s1y"], grads["s1z"]])
        gs2 = torch.stack([grads["s2x"], grads["s2y"], grads["s2z"]])
        return gs1, gs2, grads["q"], None, None, None, None, None, None


def adjoint(inputs: dict, cotangents: dict, n: int | None = None, tangent: bool = False, angles: bool = False,
            **kw) -> dict:
    """Gradients of sum_i cotangents_i . outputs_i w.r.t. s1x..s2z and q (pn_batch_adjoint); with
    tangent=True also the spin gradients projected onto the sphere's tangent plane (s1x_tan ...), with
    angles=True the derivatives w.r.t. the polar and azimuthal angles of each initial spin direction
    (s1_dtheta, s1_dphi, s2_dtheta, s2_dphi)."""
    n = int(inputs["m1"].shape[0]) if n is None else n
    fields = N.GRAD_FIELDS + (N.GRAD_TAN_FIELDS if tangent else ()) + (N.GRAD_ANGLE_FIELDS if angles else ())
    grads = {f: torch.empty(n, dtype=torch.float64, device=inputs["m1"].device) for f in fields}
    with Batch(max(n, 1), params(**kw)) as b:
        pn_batch_adjoint(b.handle, n, inputs, cotangents, grads)
        torch.cuda.synchronize()
    return grads
