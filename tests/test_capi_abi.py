"""The C ABI on the host (no GPU needed): exports, struct layouts, argument checks."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pn_batch.h")


@pytest.fixture(scope="module")
def native():
    from paper_0908_3889_b300.build import build
    from paper_0908_3889_b300 import _native
    build()
    _native.load()
    return _native


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pn_\w+)\s*\(", src, flags=re.M)))


@pytest.mark.parametrize("build_kind", ["release", "debug"])
def test_every_declared_function_is_exported_and_bound(native, build_kind):
    """Both builds (the release library and its bounds-checked debug build) export the whole ABI."""
    path = native.RELEASE_LIB_PATH if build_kind == "release" else native.DEBUG_LIB_PATH
    names = declared_functions()
    assert len(names) >= 12
    lib = C.CDLL(path)
    for n in names:
        assert hasattr(lib, n), n
        assert n in native.SIGNATURES, n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pn_\w+)", out))
    assert set(names) <= exported
    assert lib.pn_abi_version() == native.ABI_VERSION


def test_struct_layouts_match_header(native, tmp_path):
    """Compile a probe against the header and compare sizes/offsets with the ctypes mirrors."""
    structs = {"pn_params": native.pn_params, "pn_inputs": native.pn_inputs, "pn_outputs": native.pn_outputs,
               "pn_dist": native.pn_dist, "pn_cotangents": native.pn_cotangents, "pn_grads": native.pn_grads,
               "pn_stats": native.pn_stats, "pn_tune_result": native.pn_tune_result,
               "pn_hist_spec": native.pn_hist_spec, "pn_ks_result": native.pn_ks_result}
    lines = ["#include <stddef.h>", f'#include "{HEADER}"', "long probe(int k) { switch (k) {"]
    k = 0
    expect = []
    for name, cls in structs.items():
        lines.append(f"case {k}: return (long)sizeof({name});")
        expect.append((k, C.sizeof(cls), name))
        k += 1
        for f, _ in cls._fields_:
            lines.append(f"case {k}: return (long)offsetof({name}, {f});")
            expect.append((k, getattr(cls, f).offset, f"{name}.{f}"))
            k += 1
    lines.append("} return -1; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    so = tmp_path / "probe.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-o", str(so), str(src)], check=True)
    lib = C.CDLL(str(so))
    lib.probe.restype = C.c_long
    for kk, val, what in expect:
        assert lib.probe(kk) == val, what


def test_defaults_follow_the_paper(native):
    lib = native.load()
    p = native.pn_params()
    lib.pn_params_default(C.byref(p))
    assert p.rtol == 5e-7 and p.atol == 5e-7 and p.h0 == 10.0  # Sec. II
    assert p.term_mask == native.PN_TERM_ALL and p.precision == native.PN_FP64 and p.stop_mode == 0
    assert p.ckpt_every == 64
    assert p.order == native.PN_ORDER_LENGTH  # lanes take the binaries sorted by predicted length


@pytest.mark.parametrize("build_kind", ["release", "debug"])
def test_argument_errors_before_any_cuda_call(native, build_kind):
    lib = native.load(native.RELEASE_LIB_PATH if build_kind == "release" else native.DEBUG_LIB_PATH)
    p = native.pn_params()
    lib.pn_params_default(C.byref(p))
    h = C.c_void_p()
    assert lib.pn_batch_init(None, 10, C.byref(p), None) == native.PN_E_ARG
    assert lib.pn_batch_init(C.byref(h), 0, C.byref(p), None) == native.PN_E_ARG
    assert b"n_max" in lib.pn_last_error(None)
    for field, bad in (("atol", 0.0), ("h0", -1.0), ("fac_min", 2.0), ("land_max_iter", 0), ("block", 48),
                       ("precision", 7), ("term_mask", 0x400), ("bpt", 3), ("order", 2), ("order", -1)):
        q = native.pn_params()
        lib.pn_params_default(C.byref(q))
        setattr(q, field, bad)
        assert lib.pn_batch_init(C.byref(h), 10, C.byref(q), None) == native.PN_E_ARG, field
        assert h.value is None
    assert lib.pn_batch_integrate(None, 1, None, None) == native.PN_E_ARG
    assert lib.pn_batch_stats(None, 1, None, None, None) == native.PN_E_ARG
    assert lib.pn_batch_integrate_host(None, 1, None, None) == native.PN_E_ARG
    assert lib.pn_batch_integrate_host_async(None, 1, None, None) == native.PN_E_ARG
    assert lib.pn_batch_host_wait(None) == native.PN_E_ARG
    assert lib.pn_batch_eval_rhs(None, 1, None, None, None, None) == native.PN_E_ARG
    assert lib.pn_batch_integrate_budget(None, 1, None, None, 1) == native.PN_E_ARG
    assert lib.pn_batch_resume(None, 1, None, None, 1) == native.PN_E_ARG
    assert lib.pn_batch_masses(None, 1, None, None, None) == native.PN_E_ARG
    assert lib.pn_batch_timing(None, None, None) == native.PN_E_ARG
    assert lib.pn_batch_stats_segments(None, 1, None, None, None, None) == native.PN_E_ARG
    lib.pn_batch_destroy(None)


def test_release_build_has_no_debug_checks(native):
    """The bounds-check self-test belongs to the debug build; the release library says so without a GPU."""
    lib = native.load(native.RELEASE_LIB_PATH)
    assert lib.pn_debug_selftest() == native.PN_E_UNIMPLEMENTED
    assert b"release build" in lib.pn_last_error(None)


def test_product_path_refuses_to_run_without_the_library(tmp_path):
    from paper_0908_3889_b300 import _native
    with pytest.raises(RuntimeError, match="not built"):
        _native.load(str(tmp_path / "missing.so"))
