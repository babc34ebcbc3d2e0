"""The debug build (libpn_b300_debug.so: device bounds checks in place of a memory checker) on a B300.

Its self-test must see the deliberate check failure come back and be cleared; on ordinary work, in
every precision and schedule and through every entry point that launches kernels, no check may
fail, and every output must be the release build's, bit for bit (the checks only guard accesses, so
the debug build runs the same arithmetic). The debug build runs in a child process
(PN_B300_DEBUG=1 selects it for a whole process); the release outputs come from this one.
"""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT_KEYS = ("S1", "S2", "Lhat", "omega", "t", "n_acc", "n_rej", "n_land", "status", "dot_s1s2", "dot_ls1", "dot_ls2")


def _flat(prefix: str, d: dict, res: dict) -> None:
    for k, v in d.items():
        a = v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)
        res[f"{prefix}/{k}"] = a


def run_all(pn) -> dict:
    """The same work in either build: integrations in every precision and schedule, both lane orders,
    the bounded and host-buffer paths, the right-hand side alone, the adjoint in both sweeps, the
    statistics and analysis reductions, and the no-allocation entry point."""
    import torch
    res = {}
    c1 = pn.to_device(workloads.config("C1", n=20_000))
    c2 = pn.to_device(workloads.config("C2", n=20_000))
    n = 20_000
    for prec in (0, 1, 2):
        for sched in (1, 2):
            out = pn.integrate(c1, precision=prec, schedule=sched, block=128)
            _flat(f"c1_p{prec}_s{sched}", {k: out[k] for k in OUT_KEYS}, res)
    out = pn.integrate(c2, precision=0, schedule=2, block=256)
    _flat("c2_fp64", {k: out[k] for k in OUT_KEYS}, res)
    out = pn.integrate(c2, precision=0, schedule=1, block=64, order=pn.native.PN_ORDER_INPUT)
    _flat("c2_fp64_input_order", {k: out[k] for k in OUT_KEYS}, res)

    with pn.Batch(n, pn.params(precision=2)) as b:
        out = b.integrate_budget(c1, budget=16)
        while b.stats(c1, out)["count_by_status"][pn.native.PN_ST_RUNNING]:
            b.resume(c1, out, budget=16)
        _flat("c1_ds_bounded", {k: out[k] for k in OUT_KEYS}, res)
        st = b.stats(c1, out)
        res["c1_ds_bounded/stats"] = np.array(st["count_by_status"] + [st["acc_total"], st["rej_total"]],
                                              dtype=np.float64)
        y = torch.stack([out["omega"]] + [out["S1"][j] for j in range(3)] + [out["S2"][j] for j in range(3)] +
                        [out["Lhat"][j] for j in range(3)]).contiguous()
        res["c1_ds_bounded/rhs"] = b.eval_rhs(c1["m1"], c1["m2"], y).cpu().numpy()

    hin = pn.to_device(workloads.config("C1", n=n), device="cpu", pin_memory=True)
    hout = pn.alloc_outputs(n, device="cpu", pin_memory=True)
    with pn.Batch(n, pn.params(precision=0)) as b:
        pn.pn_batch_integrate_host(b.handle, n, hin, hout)
        _flat("c1_host", {k: hout[k] for k in OUT_KEYS}, res)
        out = b.integrate(c1)
        res["c1_fp64/hist20"] = b.histogram(c1, out, pn.native.PN_Q_FINAL_S1S2, 20)
        res["c1_fp64/hist2d"] = b.histogram(c1, out, pn.native.PN_Q_INIT_S1S2, 79,
                                            quantity_y=pn.native.PN_Q_FINAL_S1S2, ny=79)
        res["c1_fp64/hist_fine"] = b.histogram(c1, out, pn.native.PN_Q_FINAL_S1S2, 1 << 16)
        dens, h = b.kde(c1, out, pn.native.PN_Q_FINAL_S1S2, np.linspace(-0.9, 0.9, 19))
        res["c1_fp64/kde"] = np.append(np.asarray(dens), h)
        seg = b.stats_segments(c1, out, [0, 5_000, 5_000, 20_000])
        res["c1_fp64/segments"] = np.array([[s["pearson_s1s2"], s["acc_total"]] for s in seg], dtype=np.float64)

    c4 = workloads.config("C4", n=2_048)
    inp4 = pn.to_device(c4)
    rng = np.random.default_rng(11)
    cot = {k: torch.from_numpy(rng.normal(size=2_048) * (1e-4 if k == "t" else 1.0)).cuda()
           for k in ("dot_s1s2", "dot_ls1", "dot_ls2", "Lx", "Ly", "Lz", "S1x", "S1y", "S1z", "S2x", "S2y", "S2z",
                     "t")}
    _flat("adj_fp64", pn.adjoint(inp4, cot, tangent=True, angles=True), res)
    _flat("adj_ds", pn.adjoint(inp4, cot, precision=2), res)

    lib = pn.native.load()
    na = 4_096
    out = pn.alloc_outputs(na)
    prm = pn.params(precision=0)
    s = torch.cuda.current_stream()
    rc = lib.pn_integrate_noalloc(na, C.byref(prm), C.byref(pn.inputs_struct(c1, na)),
                                  C.byref(pn.outputs_struct(out, na)), C.c_void_p(s.cuda_stream))
    assert rc == 0, lib.pn_last_error(None)
    torch.cuda.synchronize()
    _flat("noalloc", {k: out[k] for k in OUT_KEYS}, res)
    return res


def child_main(path: str) -> None:
    """Run in the child process, with the debug build loaded."""
    import paper_0908_3889_b300 as pn
    lib = pn.native.load()
    assert pn.native.LIB_PATH == pn.native.DEBUG_LIB_PATH
    assert lib.pn_debug_selftest() == pn.native.PN_OK, lib.pn_last_error(None)
    # a second self-test finds the flags clear again
    assert lib.pn_debug_selftest() == pn.native.PN_OK, lib.pn_last_error(None)
    np.savez(path, **run_all(pn))


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


def test_debug_build_checks_pass_and_outputs_equal_release(pn, tmp_path):
    assert pn.native.LIB_PATH == pn.native.RELEASE_LIB_PATH
    assert pn.native.load().pn_debug_selftest() == pn.native.PN_E_UNIMPLEMENTED
    path = str(tmp_path / "debug_outputs.npz")
    env = dict(os.environ, PN_B300_DEBUG="1")
    code = f"import sys; sys.path[:0] = [{HERE!r}, {ROOT!r}]; import test_gpu_debug_build as t; t.child_main({path!r})"
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    dbg = np.load(path)
    rel = run_all(pn)
    assert sorted(dbg.files) == sorted(rel)
    for k in rel:
        a, b = rel[k], dbg[k]
        assert a.shape == b.shape and a.dtype == b.dtype, k
        same = np.array_equal(a.view(np.uint8), b.view(np.uint8)) if a.dtype.kind == "f" else np.array_equal(a, b)
        assert same, k
