"""pn_integrate_noalloc against pn_batch_integrate (needs a B300).

The no-allocation entry point is for callers that must not allocate device
memory (their host gives all of it to its own pool or budget).  It runs the
same kernels with their scratch in a fixed area inside the library, so its
results must match the ordinary entry point's; two calls in a row check that
what one call leaves in the shared area does not leak into the next.
"""
import ctypes as C

import numpy as np
import pytest

import workloads
from gpu_util import assert_fp64_parity

pytestmark = pytest.mark.gpu

LIMIT = 16384


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


def noalloc(pn, inp, n, **kw):
    import torch
    lib = pn.native.load()
    out = pn.alloc_outputs(n)
    prm = pn.params(**kw)
    rc = lib.pn_integrate_noalloc(n, C.byref(prm), C.byref(pn.inputs_struct(inp, n)),
                                  C.byref(pn.outputs_struct(out, n)), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.pn_last_error(None)
    torch.cuda.synchronize()
    return pn.to_numpy(out)


def test_two_calls_in_a_row_match_the_allocating_entry_point(pn):
    import torch
    first = workloads.config("C2", n=LIMIT, seed=501)
    second = workloads.config("C0", n=3000, seed=502)
    results = []
    for ens in (first, second):
        inp = pn.to_device(ens)
        n = ens["m1"].shape[0]
        results.append((noalloc(pn, inp, n), pn.to_numpy(pn.integrate(inp))))
        torch.cuda.synchronize()
    for got, ref in results:
        assert_fp64_parity(got, ref)


def test_mixed_precision_and_limits(pn):
    import torch
    ens = workloads.config("C1", n=2000, seed=503)
    inp = pn.to_device(ens)
    got = noalloc(pn, inp, 2000, precision=1)
    ref = pn.to_numpy(pn.integrate(inp, precision=1))
    for k in got:
        assert np.array_equal(got[k], ref[k], equal_nan=True), k
    lib = pn.native.load()
    big = pn.to_device(workloads.config("C1", n=LIMIT + 1, seed=504))
    out = pn.alloc_outputs(LIMIT + 1)
    prm = pn.params()
    rc = lib.pn_integrate_noalloc(LIMIT + 1, C.byref(prm), C.byref(pn.inputs_struct(big)), C.byref(pn.outputs_struct(out)),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == pn.native.PN_E_ARG and b"16384" in lib.pn_last_error(None)
