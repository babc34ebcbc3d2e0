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


def noalloc(pn, inp, n, stream=None, **kw):
    import torch
    lib = pn.native.load()
    out = pn.alloc_outputs(n)
    prm = pn.params(**kw)
    s = torch.cuda.current_stream() if stream is None else stream
    rc = lib.pn_integrate_noalloc(n, C.byref(prm), C.byref(pn.inputs_struct(inp, n)),
                                  C.byref(pn.outputs_struct(out, n)), C.c_void_p(s.cuda_stream))
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


def test_double_single_precision(pn):
    """The double-single form through the no-allocation entry point gives the ordinary entry point's bits."""
    ens = workloads.config("C4", n=3000, seed=505)
    inp = pn.to_device(ens)
    got = noalloc(pn, inp, 3000, precision=2)
    ref = pn.to_numpy(pn.integrate(inp, precision=2))
    for k in got:
        assert np.array_equal(got[k], ref[k], equal_nan=True), k


FIRST_CALL_ON_SIDE_STREAM = r"""
import sys
sys.path[:0] = [sys.argv[1], sys.argv[1] + "/tests"]
import numpy as np, torch
import paper_0908_3889_b300 as pn, workloads
from test_zz_no_alloc import noalloc
torch.cuda.set_device(0)
ens = workloads.config("C2", n=4000, seed=506)
inp = pn.to_device(ens)
torch.cuda.synchronize()
side = torch.cuda.Stream()
with torch.cuda.stream(side):
    got = noalloc(pn, inp, 4000, stream=side)  # the first call of this process, on a non-blocking stream
ref = pn.to_numpy(pn.integrate(inp))
for k in got:
    assert np.array_equal(got[k], ref[k], equal_nan=True), k
print("ok")
"""


def test_first_call_of_a_process_on_a_side_stream(pn):
    """A fresh process whose first no-allocation call runs on a non-blocking torch stream: the table the
    first call uploads must be in place before that stream's kernels read it."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", FIRST_CALL_ON_SIDE_STREAM, root], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
