"""Mixed precision (an FP32 or a double-single right-hand side; FP64 state accumulation and step
control) against the FP64 oracle (needs a B300).

FP32 rounding in the rates perturbs the embedded error estimate by ~1e-3 of
its value, so a few step sizes (and, rarely, an accept/reject decision) differ
from the FP64 run; the outputs then differ by the integration error itself,
which for small spins at tolerance 5e-7 is up to ~1e-3.  The typical binary
agrees to ~1e-7.  The FP32 form's error is stated, not held to the 1e-6 bar:
each bound below is about three times the error measured on the B300 for that
ensemble (max, 99th percentile and median of |dot - oracle| over its binaries,
largest of the three scalar products), so a regression in the FP32
right-hand side fails."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

DOT_TOL = 1e-6  # bar on the final spin scalar products in mixed precision

# FP32 form, bounds on |dot - oracle| as (max, p99, median).  Measured (max, p99, median):
#   C1 4,096 subsample  2.7e-6, 1.1e-6, 1.3e-7  (all 1,048,576 binaries: max 6.4e-6, p99 1.0e-6)
#   C0 2,000            9.4e-7, 3.8e-7, 6.0e-8
#   C4 2,000            5.4e-6, 2.7e-6, 3.2e-7
#   C2 2,000            3.6e-3, 9.0e-5, 4.3e-7  (q up to 10, spins down to 0: S2 far below the tolerance)
FP32_STATED = {"C3": (1e-5, 1.5e-6, 3e-7), "C0": (3e-6, 1.2e-6, 2e-7), "C4": (1.6e-5, 8e-6, 1e-6),
               "C2": (1.1e-2, 3e-4, 1.3e-6)}


def assert_stated(e, name):
    mx, p99, p50 = FP32_STATED[name]
    for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
        got = (float(np.max(e[k])), float(np.percentile(e[k], 99)), float(np.median(e[k])))
        assert got[0] <= mx and got[1] <= p99 and got[2] <= p50, (name, k, got)


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


def mixed_errors(g, o):
    e = {}
    e["t"] = np.abs(g["t"] / o["t"] - 1)
    for k in ("S1", "S2", "Lhat"):
        sc = np.linalg.norm(o[k], axis=0)
        e[k] = np.max(np.abs(g[k] - o[k]), axis=0) / np.where(sc > 0, sc, 1.0)
    for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
        e[k] = np.abs(g[k] - o[k])
    return e


def test_c3_mixed_full_size_subsample(pn, orc):
    """C1's 1,048,576-binary ensemble in mixed precision; a 4,096 subsample vs the FP64 oracle."""
    import torch
    ens = workloads.config("C3")
    n = ens["m1"].shape[0]
    inp = pn.to_device(ens)
    with pn.Batch(n, pn.params(precision=1)) as b:
        out = b.integrate(inp)
        torch.cuda.synchronize()
    idx = workloads.subsample(n, 4096, seed=workloads.SEED_BASE + 103)
    g = {k: v[..., idx] for k, v in pn.to_numpy(out).items()}
    o = orc.integrate(workloads.take(ens, idx))
    assert np.all(g["status"] == 0) and np.all(o["status"] == 0)
    e = mixed_errors(g, o)
    report = {k: (float(np.max(v)), float(np.median(v))) for k, v in e.items()}
    print("mixed-vs-FP64 (max, median):", report)
    assert_stated(e, "C3")
    for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
        assert np.mean(e[k] > DOT_TOL) < 0.025, (k, np.mean(e[k] > DOT_TOL))  # tail fraction (measured 1.3 %)
    assert report["t"][1] < 1e-6


@pytest.mark.parametrize("schedule", [1, 2])
def test_mixed_small_ensembles(pn, orc, schedule):
    import torch
    for name in ("C0", "C2", "C4"):
        ens = workloads.config(name, n=2000)
        o = orc.integrate(ens)
        g = pn.to_numpy(pn.integrate(pn.to_device(ens), precision=1, schedule=schedule))
        torch.cuda.synchronize()
        e = mixed_errors(g, o)
        assert np.array_equal(g["status"], o["status"])
        assert_stated(e, name)


# ---------------------------------------------------------------------------
# Double-single right-hand side (PN_MIXED_DS): rates accurate to ~1e-13, so the
# step decisions are those of the FP64 run and the 1e-6 bar on the final scalar
# products holds for every binary, not just the typical one.
# ---------------------------------------------------------------------------
def test_ds_full_size_subsample_meets_dot_bar(pn, orc):
    import torch
    from gpu_util import decided_alike
    ens = workloads.config("C3")
    n = ens["m1"].shape[0]
    inp = pn.to_device(ens)
    with pn.Batch(n, pn.params(precision=2)) as b:
        out = b.integrate(inp)
        torch.cuda.synchronize()
    idx = workloads.subsample(n, 4096, seed=workloads.SEED_BASE + 104)
    g = {k: v[..., idx] for k, v in pn.to_numpy(out).items()}
    o = orc.integrate(workloads.take(ens, idx))
    assert np.array_equal(g["status"], o["status"])
    e = mixed_errors(g, o)
    report = {k: (float(np.max(v)), float(np.median(v))) for k, v in e.items()}
    print("double-single vs FP64 (max, median):", report, "same decisions:", float(np.mean(decided_alike(g, o))))
    for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
        assert report[k][0] <= DOT_TOL, (k, report[k])
    assert np.mean(decided_alike(g, o)) >= 0.999


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_schedules_and_blocks_bit_identical(pn, precision):
    """Every launch shape gives the same bits in both mixed modes.  The double-single kernel's plain
    and persistent instantiations are compiled under different register caps (168 and 255) and its
    workspace layout depends on neither; the attempt's arithmetic must not change with them."""
    import torch
    ens = workloads.config("C2", n=3000)
    inp = pn.to_device(ens)
    ref = pn.to_numpy(pn.integrate(inp, precision=precision, schedule=1, block=128))
    for sched, block, bpt in ((2, 64, 0), (2, 256, 0), (1, 64, 1), (2, 128, 0), (1, 128, 2), (1, 256, 1)):
        g = pn.to_numpy(pn.integrate(inp, precision=precision, schedule=sched, block=block, bpt=bpt))
        torch.cuda.synchronize()
        for k in ref:
            assert np.array_equal(ref[k], g[k], equal_nan=True), (precision, sched, block, bpt, k)


@pytest.mark.parametrize("schedule", [1, 2])
def test_ds_small_ensembles(pn, orc, schedule):
    import torch
    for name in ("C0", "C2", "C4"):
        ens = workloads.config(name, n=2000)
        o = orc.integrate(ens)
        g = pn.to_numpy(pn.integrate(pn.to_device(ens), precision=2, schedule=schedule))
        torch.cuda.synchronize()
        e = mixed_errors(g, o)
        assert np.array_equal(g["status"], o["status"])
        for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
            assert np.max(e[k]) <= DOT_TOL, (name, k, np.max(e[k]))


@pytest.mark.parametrize("schedule", [1, 2])
def test_ds_small_ensembles_meet_dot_bar(pn, orc, schedule):
    """The double-single form on the other ensembles' shapes (C0 maximal spins, C2 uneven lengths
    with q up to 10 and small spins, C4 q in [1, 4]): every binary within the 1e-6 bar on the final
    scalar products, the oracle's statuses, and the oracle's step decisions for almost all."""
    import torch
    from gpu_util import decided_alike
    for name in ("C0", "C2", "C4"):
        ens = workloads.config(name, n=2000)
        o = orc.integrate(ens)
        g = pn.to_numpy(pn.integrate(pn.to_device(ens), precision=2, schedule=schedule))
        torch.cuda.synchronize()
        assert np.array_equal(g["status"], o["status"]), name
        e = mixed_errors(g, o)
        for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
            assert np.max(e[k]) <= DOT_TOL, (name, k, float(np.max(e[k])))
        assert np.mean(decided_alike(g, o)) >= 0.995, (name, float(np.mean(decided_alike(g, o))))
