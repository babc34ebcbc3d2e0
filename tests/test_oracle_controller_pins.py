"""Pins of the oracle's embedded error norm and step-size controller.

Sec. II states only the tolerance (5e-7) and the first step (h = 10); the norm and the controller are
readings: e = h sum_j (b_j - bhat_j) k_j, err = RMS over the 10 components of e_i / (atol + rtol
max(|y_i|, |y5_i|)), accept if err <= 1, h_new = h clamp(0.9 err^(-1/5), 0.2, 10) with no growth right
after a rejection.  These tests check that the oracle computes exactly that reading, through
consequences that mathematics fixes and that do not reuse its formulas.

The test problem is the leading-order chirp of Eq. (1), w' = K w^(11/3) with K = (96/5) eta, with
precession off, so the spins and L-hat are frozen and only omega carries an error.  Its local
behaviour is known in closed form by the Butcher series of the Dormand-Prince tableau (tests/bseries.py;
the tableau itself is pinned by the order conditions in test_oracle_pins.py):

  * the embedded estimate is  e_omega = w sum_k D_k u^k,  u = h K w^(8/3),  with D_5 = -0.0900...;
  * so the RMS norm of one attempt is |e_omega| / (sqrt(10) sc), sc = atol + rtol max(w, w_exact(h));
  * if err = C h^5 and h_new = 0.9 err^(-1/5) h, the error of h_new at the same state is 0.9^5 = 0.59
    whatever C is (an exponent of -1/4 gives 0.9^4 ~ 0.66; a safety of 0.8 gives 0.33);
  * |e| grows faster than h^5 here (D_6/D_5 > 0), so after a rejection that shrinks h by
    0.9 err^(-1/5) the retried step's error falls just below 0.59: the controller would then grow h,
    and the no-growth rule is visible as h staying exactly the same.

Each check is also run on copies of the oracle with one plausible mistake planted in its source (a
2-norm instead of the RMS, a dropped h, a -1/4 exponent, safety 0.8, the scale taken from y alone, a
dropped stage, growth after a rejection, a missing clamp): every planted mistake must fail its check.
"""
from __future__ import annotations

import concurrent.futures as cf

import numpy as np
import pytest

import bseries as B
import workloads

P = 11.0 / 3.0            # w' = K w^P
M1 = M2 = 0.5
K = 96.0 / 5.0 * M1 * M2  # (96/5) eta
KMAX = 10                 # series order: truncation below 1e-6 of e for u <= 0.02
SAFETY5 = 0.9 ** 5


@pytest.fixture(scope="module")
def series(orc):
    _, a, b, bh = orc.tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a
    D = B.method_coefficients(A, b, P, KMAX) - B.method_coefficients(A, bh, P, KMAX)
    ex = B.exact_coefficients(P, KMAX)
    return D, ex


def u_of(w, h):
    return h * K * w ** (P - 1.0)


def err_series(series, w, h, atol, rtol):
    """The reading's norm of one attempt from w with step h, from the series alone."""
    D, ex = series
    u = u_of(w, h)
    e = w * B.series(D, u)
    w_exact = w * B.series(ex, u)
    return abs(e) / (np.sqrt(10.0) * (atol + rtol * max(w, w_exact)))


def chirp_params(orc, **kw):
    return orc.params(term_mask=0, max_steps=50_000, **kw)  # Newtonian chirp only, precession off


def one_binary(w0):
    return workloads.ensemble(1, 0x0C7, omega0=(w0, w0), omega_f=0.05)


# ---------------------------------------------------------------------------
# The checks (each raises AssertionError on a mismatch).
# ---------------------------------------------------------------------------
def check_tree_machinery(series):
    """The tree sums reproduce the closed-form chirp (1 - 8u/3)^(-3/8) term by term, and D_k vanishes below
    order 5 (both weight vectors satisfy the order-4 conditions)."""
    D, ex = series
    from math import factorial, prod
    taylor = [prod(1.0 + j * (P - 1.0) for j in range(k)) / factorial(k) for k in range(KMAX + 1)]
    assert [len(B.trees(k)) for k in range(1, 9)] == [1, 1, 2, 4, 9, 20, 48, 115]
    assert np.allclose(ex, taylor, rtol=1e-14, atol=0)
    assert np.all(np.abs(D[:5]) < 1e-14) and abs(D[5]) > 0.05


def check_norm(orc, series):
    """One attempt's err equals |e_omega| / (sqrt(10) sc) from the series, for the mixed, the purely
    relative and the purely absolute scale."""
    w = 0.02
    y = np.array([w, 0.10, 0.05, -0.20, 0.03, 0.10, 0.02, 0.30, 0.40, np.sqrt(0.75)])
    for atol, rtol in ((5e-7, 5e-7), (0.0, 1e-6), (1e-9, 0.0)):
        prm = chirp_params(orc, atol=atol, rtol=rtol)
        for u in (0.01, 0.015, 0.02):
            h = u / (K * w ** (P - 1.0))
            y5, err = orc.dp5_attempt(y, h, M1, M2, prm)
            assert np.array_equal(y5[1:], y[1:]), "precession off must freeze S and L"
            want = err_series(series, w, h, atol, rtol)
            assert abs(err / want - 1.0) < 2e-6, (atol, rtol, u, err, want)


def check_fixed_point(orc, series):
    """Over a long run at a tight absolute tolerance (no rejections), each accepted step's successor size
    h_{n+1} has, at the state w_n, the error 0.9^5 that an exponent of -1/5 and safety 0.9 predict."""
    atol = 1e-13
    prm = chirp_params(orc, atol=atol, rtol=0.0)
    ens = one_binary(0.01)
    rows, hs = orc.trace(ens, 0, prm)
    w = rows[:, 1]
    r = np.array([err_series(series, w[n], hs[n + 1], atol, 0.0) for n in range(len(hs) - 2)])
    ramp = np.argmax(hs[1:] / hs[:-1] < 10.0)  # the first steps grow by the clamp fac_max = 10
    steady = r[ramp + 2:]
    assert steady.size > 100
    assert abs(np.median(steady) / SAFETY5 - 1.0) < 0.005, float(np.median(steady))
    assert np.max(np.abs(steady / SAFETY5 - 1.0)) < 0.01, (float(steady.min()), float(steady.max()))
    assert orc.integrate(ens, prm)["n_rej"][0] == 0  # every step in the steady state accepted


def h_for_error(series, w, target, atol):
    """The step from w whose series norm (absolute scale atol) is target."""
    lo, hi = 1e-9, 0.2 / (K * w ** (P - 1.0))
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if err_series(series, w, mid, atol, 0.0) > target:
            hi = mid
        else:
            lo = mid
    return lo


def check_after_rejection(orc, series):
    """A first step with error 20 is rejected once and retried at 0.9 * 20^(-1/5) of itself; the retry's
    error is below 0.9^5, where the controller would grow h, and the next step keeps exactly its size."""
    atol, w0 = 1e-15, 0.01
    h0 = h_for_error(series, w0, 20.0, atol)
    prm = chirp_params(orc, atol=atol, rtol=0.0, h0=h0)
    ens = one_binary(w0)
    rows, hs = orc.trace(ens, 0, prm)
    assert orc.integrate(ens, prm)["n_rej"][0] == 1
    assert abs(hs[0] / (h0 * 0.9 * 20.0 ** -0.2) - 1.0) < 1e-5
    assert err_series(series, w0, hs[0], atol, 0.0) < 0.995 * SAFETY5
    assert hs[1] == hs[0], hs[1] / hs[0]


def check_clamps(orc, series):
    """Error 2500 on the first step: 0.9 * 2500^(-1/5) < 0.2, so the retry is exactly 0.2 h0.  Error 1e-7:
    0.9 * (1e-7)^(-1/5) > 10, so the second step is exactly 10 times the first."""
    atol, w0 = 1e-15, 0.01
    ens = one_binary(w0)
    h0 = h_for_error(series, w0, 2500.0, atol)
    prm = chirp_params(orc, atol=atol, rtol=0.0, h0=h0)
    rows, hs = orc.trace(ens, 0, prm)
    assert orc.integrate(ens, prm)["n_rej"][0] == 1 and hs[0] == h0 * 0.2, hs[0] / h0
    h0 = h_for_error(series, w0, 1e-7, atol)
    prm = chirp_params(orc, atol=atol, rtol=0.0, h0=h0)
    rows, hs = orc.trace(ens, 0, prm)
    assert hs[0] == h0 and hs[1] == hs[0] * 10.0, hs[1] / hs[0]


# ---------------------------------------------------------------------------
# The oracle as it stands passes every check.
# ---------------------------------------------------------------------------
def test_tree_machinery(series):
    check_tree_machinery(series)


def test_norm_is_the_rms_of_the_scaled_embedded_estimate(orc, series):
    check_norm(orc, series)


def test_accepted_errors_settle_at_the_fixed_point(orc, series):
    check_fixed_point(orc, series)


def test_no_growth_right_after_a_rejection(orc, series):
    check_after_rejection(orc, series)


def test_step_factor_clamps(orc, series):
    check_clamps(orc, series)


# ---------------------------------------------------------------------------
# Planted mistakes: (name, source text, replacement, occurrences, the check that must fail).
# ---------------------------------------------------------------------------
MUTANTS = [
    ("two_norm", "return sqrt_(sum / 10.0);", "return sqrt_(sum);", 1, check_norm),
    ("no_h", "    e = h * e;\n", "", 1, check_norm),
    ("scale_from_y", "T(ay > ay5 ? ay : ay5)", "T(ay)", 1, check_norm),
    ("dropped_stage", "T e = (DP_B[0] - DP_BHAT[0]) * k[0][i];", "T e = T(0.0);", 1, check_norm),
    ("exponent_quarter", "std::pow(err, -0.2)", "std::pow(err, -0.25)", 2, check_fixed_point),
    ("safety_08", "p.safety * std::pow(err, -0.2)", "0.8 * std::pow(err, -0.2)", 2, check_fixed_point),
    ("growth_after_reject", "const double fmax = last_rejected ? 1.0 : p.fac_max;",
     "const double fmax = p.fac_max;", 1, check_after_rejection),
    ("no_fac_min_on_reject", "      if (fac > 1.0) fac = 1.0;\n      if (fac < p.fac_min) fac = p.fac_min;\n",
     "      if (fac > 1.0) fac = 1.0;\n", 1, check_clamps),
    ("no_fac_max", "          if (fac > fmax) fac = fmax;\n", "", 1, check_clamps),
]


@pytest.fixture(scope="module")
def mutant_libs(orc, tmp_path_factory):
    src = orc.source()
    d = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = {}
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        for name, old, new, count, _ in MUTANTS:
            assert src.count(old) == count, (name, src.count(old))
            jobs[name] = ex.submit(orc.build_variant, src.replace(old, new), d, name)
        return {k: f.result() for k, f in jobs.items()}


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(orc, series, mutant_libs, mutant):
    name, _, _, _, check = mutant
    with orc.variant(mutant_libs[name]):
        with pytest.raises(AssertionError):
            check(orc, series)
    check(orc, series)  # and the oracle itself still passes once the variant is gone
