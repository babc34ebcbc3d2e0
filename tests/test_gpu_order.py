"""The order in which lanes take the binaries (pn_params.order, PN_ORDER_LENGTH by default) changes no
output bit: each binary's arithmetic does not depend on its lane.  The outputs are pre-filled with
sentinels, so a binary that no lane took (or that two lanes wrote differently) would show."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


def run(pn, ens, **kw):
    import torch
    n = int(ens["m1"].shape[0])
    inp = pn.to_device(ens)
    out = pn.alloc_outputs(n)
    out["_block"].fill_(float("nan"))
    out["_iblock"].fill_(-7)
    with pn.Batch(n, pn.params(**kw)) as b:
        b.integrate(inp, out)
        torch.cuda.synchronize()
    return pn.to_numpy(out)


def with_bad_inputs(ens):
    e = {k: np.array(v, copy=True) for k, v in ens.items()}
    e["m1"][5] = np.nan           # invalid: taken last (key 0), written as bad input
    e["omega0"][7] = -1.0
    e["omega_f"][11] = e["omega0"][11] * 0.5
    e["chi1"][13] = 0.0           # zero spins: valid, shortest key of their kind
    e["chi2"][13] = 0.0
    return e


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_length_order_changes_no_output_bit(pn, precision):
    ens = with_bad_inputs(workloads.config("C2", n=3000))  # uneven lengths: q up to 10, omega_0 spread
    ref = run(pn, ens, precision=precision, order=pn.native.PN_ORDER_INPUT, schedule=1, block=128)
    assert np.all(ref["status"][[5, 7, 11]] == pn.native.PN_ST_BAD_INPUT)
    assert np.all(ref["status"] >= 0)
    for sched, block, bpt in ((1, 128, 1), (2, 128, 0), (1, 64, 2), (2, 256, 0)):
        g = run(pn, ens, precision=precision, order=pn.native.PN_ORDER_LENGTH, schedule=sched, block=block, bpt=bpt)
        for k in ref:
            if k.startswith("_"):
                continue
            assert np.array_equal(ref[k], g[k], equal_nan=True), (precision, sched, block, bpt, k)


@pytest.mark.parametrize("name, n", [("PAPER_PERF", 257), ("C1", 1), ("C1", 33), ("C0", 1024)])
def test_length_order_edge_sizes_and_equal_keys(pn, name, n):
    """Equal keys (the replicated inspiral), a single binary and ragged sizes."""
    ens = workloads.config(name, n=n)
    for sched in (1, 2):
        ref = run(pn, ens, order=pn.native.PN_ORDER_INPUT, schedule=sched)
        g = run(pn, ens, order=pn.native.PN_ORDER_LENGTH, schedule=sched)
        for k in ref:
            if k.startswith("_"):
                continue
            assert np.array_equal(ref[k], g[k], equal_nan=True), (name, n, sched, k)
        assert np.all(g["status"] == 0)

