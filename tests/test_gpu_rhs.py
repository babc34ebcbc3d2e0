"""The integration kernels' right-hand side of Eqs. (1)-(4), evaluated point by point through
pn_batch_eval_rhs, against the oracle's at random states (needs a B300).

Each rate vector is compared relative to its own magnitude: omega-dot, and the vectors dS1/dt,
dS2/dt, dL-hat/dt by their Euclidean norms."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

N = 4096
# FP64: the kernel and the oracle differ only in rounding order, FMA contraction and their
# logarithm / cube-root implementations (observed: median 2e-16, max 1e-14 where a cross product
# cancels).  FP32: single-precision rates (observed max 2.5e-6).  Double-single: pairs of FP32,
# ~2^-46 per operation (observed max 2.3e-13, with unnormalized products).
TOL = {0: 2e-14, 1: 1e-5, 2: 5e-13}


@pytest.fixture(scope="module")
def pn():
    import torch
    import paper_0908_3889_b300 as pn
    from paper_0908_3889_b300.build import build
    assert torch.cuda.is_available()
    build()
    return pn


@pytest.fixture(scope="module")
def case(orc):
    st = workloads.states(N, seed=workloads.SEED_BASE + 300)
    ref = np.stack([orc.rhs(st["y"][:, i], st["m1"][i], st["m2"][i]) for i in range(N)], axis=1)
    return st, ref


def device_rhs(pn, st, precision, **kw):
    import torch
    m1 = torch.from_numpy(st["m1"]).cuda()
    m2 = torch.from_numpy(st["m2"]).cuda()
    y = torch.from_numpy(np.ascontiguousarray(st["y"])).cuda()
    with pn.Batch(y.shape[1], pn.params(precision=precision, **kw)) as b:
        f = b.eval_rhs(m1, m2, y)
        torch.cuda.synchronize()
    return f.cpu().numpy()


def rel_errors(got, ref):
    """Per state: relative error of omega-dot and of each rate vector by its norm; a vector that is
    exactly zero in the reference (no precession terms) must be exactly zero on the device too."""
    out = {"omega_dot": np.abs(got[0] - ref[0]) / np.abs(ref[0])}
    for name, sl in (("S1_dot", slice(1, 4)), ("S2_dot", slice(4, 7)), ("L_dot", slice(7, 10))):
        scale = np.linalg.norm(ref[sl], axis=0)
        diff = np.linalg.norm(got[sl] - ref[sl], axis=0)
        out[name] = np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), np.where(diff == 0, 0.0, np.inf))
    return out


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_rhs_matches_oracle_pointwise(pn, case, precision):
    st, ref = case
    got = device_rhs(pn, st, precision)
    assert np.all(np.isfinite(got))
    e = rel_errors(got, ref)
    report = {k: (float(np.max(v)), float(np.median(v))) for k, v in e.items()}
    print("precision", precision, "relative error (max, median):", report)
    for k, v in e.items():
        assert np.max(v) <= TOL[precision], (k, report[k])


def test_rhs_fp64_term_mask_and_theta_mode(pn, orc):
    """The PN-term mask and the theta-hat reading reach the device right-hand side as they reach the
    oracle's: Newtonian order only, spin-orbit only, and the as-printed theta-hat eta^2 term."""
    st = workloads.states(512, seed=workloads.SEED_BASE + 301)
    for kw in ({"term_mask": 0}, {"term_mask": 2 | 256}, {"theta_mode": 1}):
        prm = orc.params(**kw)
        ref = np.stack([orc.rhs(st["y"][:, i], st["m1"][i], st["m2"][i], prm) for i in range(512)], axis=1)
        got = device_rhs(pn, st, 0, **kw)
        e = rel_errors(got, ref)
        for k, v in e.items():
            assert np.max(v) <= TOL[0], (kw, k, float(np.max(v)))


def test_rhs_fp64_wide_omega_range(pn, orc):
    """FP64 rates for M omega log-uniform in [2^-100, 2^100], far outside an inspiral: the logarithm's
    exponent term k ln 2 (k converted to a double by integer operations) for every k in [-100, 99],
    and its table reduction, against the oracle at the same tolerance as the inspiral range."""
    st = workloads.states(2048, seed=workloads.SEED_BASE + 303, omega_range=(2.0 ** -100, 2.0 ** 100))
    k = np.floor(np.log2(st["y"][0])).astype(int)
    assert k.min() <= -95 and k.max() >= 94
    ref = np.stack([orc.rhs(st["y"][:, i], st["m1"][i], st["m2"][i]) for i in range(2048)], axis=1)
    got = device_rhs(pn, st, 0)
    assert np.all(np.isfinite(got)) and np.all(np.isfinite(ref))
    e = rel_errors(got, ref)
    for name, v in e.items():
        assert np.max(v) <= TOL[0], (name, float(np.max(v)))


def test_rhs_out_of_range_omega_gives_non_finite_rates(pn):
    st = workloads.states(8, seed=workloads.SEED_BASE + 302)
    st["y"][0] = [0.0, -0.0, 1e-310, np.inf, np.nan, 1e300, 1e-40, 0.02]
    for precision in (0, 1, 2):
        got = device_rhs(pn, st, precision)
        assert not np.any(np.isfinite(got[:, :7])), precision
        assert np.all(np.isfinite(got[:, 7])), precision
