"""Pins of the CPU oracle to what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a textbook formula written in a different parametrisation, a property
the equations guarantee, an independent integrator, or a value the paper
prints (tests/golden/paper_values.txt).  Equation and section numbers refer to
arXiv:0908.3889.
"""
import math
import os

import mpmath
import numpy as np
import pytest
from scipy import stats

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, rest = line.split("=")
            v, tol = rest.split()
            vals[k.strip()] = (float(v), float(tol))
    return vals


def _rand_state(rng, m1, m2, omega=None):
    y = np.empty(10)
    y[0] = omega if omega is not None else rng.uniform(0.005, 0.06)
    for off, m in ((1, m1), (4, m2)):
        v = rng.normal(size=3)
        y[off:off + 3] = rng.uniform(0.1, 1.0) * m * m * v / np.linalg.norm(v)
    l = rng.normal(size=3)
    y[7:10] = l / np.linalg.norm(l)
    return y


def _one(m1, m2, chi1, chi2, s1, s2, omega0, omega_f, l=(0.0, 0.0, 1.0)):
    return {"m1": np.array([m1]), "m2": np.array([m2]), "chi1": np.array([chi1]), "chi2": np.array([chi2]),
            "s1hat": np.array(s1, float).reshape(3, 1), "s2hat": np.array(s2, float).reshape(3, 1),
            "lhat": np.array(l, float).reshape(3, 1), "omega0": np.array([omega0]),
            "omega_f": np.array([omega_f])}


# ---------------------------------------------------------------------------
# Dormand-Prince tableau: Butcher order conditions (Dormand & Prince 1980).
# ---------------------------------------------------------------------------
def test_tableau_order_conditions(orc):
    c, a76, b, bh = orc.tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a76
    # row sums give the nodes; the last row is b (first-same-as-last)
    assert np.allclose(A.sum(1), c, rtol=0, atol=1e-15)
    assert np.allclose(A[6], b, atol=0)
    Ac = A @ c
    conds = [  # (weight vector product, exact value) for every rooted tree up to order 5
        (lambda w: w.sum(), 1.0), (lambda w: w @ c, 1 / 2),
        (lambda w: w @ c**2, 1 / 3), (lambda w: w @ Ac, 1 / 6),
        (lambda w: w @ c**3, 1 / 4), (lambda w: w @ (c * Ac), 1 / 8),
        (lambda w: w @ (A @ c**2), 1 / 12), (lambda w: w @ (A @ Ac), 1 / 24),
        (lambda w: w @ c**4, 1 / 5), (lambda w: w @ (c**2 * Ac), 1 / 10),
        (lambda w: w @ (c * (A @ c**2)), 1 / 15), (lambda w: w @ (c * (A @ Ac)), 1 / 30),
        (lambda w: w @ (Ac * Ac), 1 / 20), (lambda w: w @ (A @ c**3), 1 / 20),
        (lambda w: w @ (A @ (c * Ac)), 1 / 40), (lambda w: w @ (A @ (A @ c**2)), 1 / 60),
        (lambda w: w @ (A @ (A @ Ac)), 1 / 120),
    ]
    for f, v in conds:  # b: order 5
        assert abs(f(b) - v) < 1e-14
    for f, v in conds[:8]:  # bhat: order 4
        assert abs(f(bh) - v) < 1e-14
    assert max(abs(f(bh) - v) for f, v in conds[8:]) > 1e-6  # and genuinely not order 5


def test_dp5_step_on_linear_ode_has_order_5(orc):
    """For y' = lambda y the step multiplies by the degree-5 Taylor polynomial of exp plus O(z^6)."""
    c, a76, b, _ = orc.tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a76
    for z in (0.1, 0.05, 0.025):
        # stability function R(z) = 1 + z b^T (I - zA)^{-1} 1
        R = 1 + z * b @ np.linalg.solve(np.eye(7) - z * A, np.ones(7))
        taylor = sum(z**k / math.factorial(k) for k in range(6))
        assert abs(R - taylor) < 2e-3 * z**6 + 1e-16


# ---------------------------------------------------------------------------
# Right-hand side, Eqs. (1)-(4).
# ---------------------------------------------------------------------------
def test_rhs_precession_preserves_norms_and_total_J(orc):
    """S_i . dS_i/dt = 0, L . dL/dt = 0 and, at fixed omega, |L_n| dL/dt + dS1/dt + dS2/dt = 0
    with |L_n| = eta M^{5/3} omega^{-1/3} (Eq. 3 and the |L_n| formula of Sec. II)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        m1 = rng.uniform(0.1, 0.9)
        m2 = 1 - m1
        y = _rand_state(rng, m1, m2)
        f = orc.rhs(y, m1, m2)
        S1, S2, L = y[1:4], y[4:7], y[7:10]
        dS1, dS2, dL = f[1:4], f[4:7], f[7:10]
        scale = np.linalg.norm(dS1) + np.linalg.norm(dS2)
        assert abs(S1 @ dS1) <= 1e-15 * np.linalg.norm(S1) * scale
        assert abs(S2 @ dS2) <= 1e-15 * np.linalg.norm(S2) * scale
        assert abs(L @ dL) <= 1e-14 * np.linalg.norm(dL)
        Ln = m1 * m2 * y[0] ** (-1 / 3)
        assert np.linalg.norm(Ln * dL + dS1 + dS2) <= 1e-14 * scale


def test_rhs_geodetic_precession_rate(orc):
    """With S2 = 0 and S1 perpendicular to L = z, dS1/dt = Omega_1 z x S1 with the textbook 1PN
    spin-orbit precession frequency Omega_1 = (2 + 3 m2 / (2 m1)) |L_N| / r^3, |L_N| = mu sqrt(M r),
    omega = sqrt(M / r^3) (Apostolatos et al. 1994; Kidder 1995), i.e. prograde precession."""
    for m1, omega in ((0.5, 0.01), (0.3, 0.03), (0.8, 0.05)):
        m2 = 1 - m1
        r = omega ** (-2 / 3)
        mu = m1 * m2
        Om = (2 + 1.5 * m2 / m1) * mu * math.sqrt(r) / r**3
        y = np.array([omega, m1 * m1, 0, 0, 0, 0, 0, 0, 0, 1.0])
        f = orc.rhs(y, m1, m2)
        expect = np.array([0.0, Om * m1 * m1, 0.0])  # z x x = +y
        assert np.allclose(f[1:4], expect, rtol=1e-13, atol=1e-30)
        assert np.allclose(f[4:7], 0, atol=0)


def test_rhs_leading_order_is_quadrupole_chirp(orc):
    """With only the Newtonian term, domega/dt = (96/5) eta M^{5/3} omega^{11/3} (Peters & Mathews)."""
    prm = orc.params(term_mask=orc.NEWTONIAN)
    for m1, omega in ((0.5, 0.02), (0.1, 0.005)):
        m2 = 1 - m1
        y = np.array([omega, 0.1, 0, 0.1, 0, -0.1, 0.05, 0, 0, 1.0])
        f = orc.rhs(y, m1, m2, prm)
        assert f[0] == pytest.approx(96 / 5 * m1 * m2 * omega ** (11 / 3), rel=1e-14)


def _taylor_t4_rhs(omega, eta, so=0.0, ss=0.0):
    """domega/dt from the literature's x-form dx/dt = (64/5) eta x^5 F(x), x = (M omega)^{2/3},
    non-spinning TaylorT4 coefficients through 3.5PN (Blanchet, Living Rev. Rel.), where the 3PN
    eta coefficient is -56198689/217728 + 451 pi^2 / 48.  so/ss add aligned-spin 1.5PN/2PN terms."""
    mp = mpmath
    x = mp.mpf(omega) ** (mp.mpf(2) / 3)
    pi = mp.pi
    g = mp.euler
    F = (1 - (mp.mpf(743) / 336 + mp.mpf(11) / 4 * eta) * x + (4 * pi - so) * x**1.5
         + (mp.mpf(34103) / 18144 + mp.mpf(13661) / 2016 * eta + mp.mpf(59) / 18 * eta**2 - ss) * x**2
         - (mp.mpf(4159) / 672 + mp.mpf(189) / 8 * eta) * pi * x**2.5
         + (mp.mpf(16447322263) / 139708800 - mp.mpf(1712) / 105 * g + mp.mpf(16) / 3 * pi**2
            - mp.mpf(856) / 105 * mp.log(16 * x)
            + (-mp.mpf(56198689) / 217728 + mp.mpf(451) / 48 * pi**2) * eta
            + mp.mpf(541) / 896 * eta**2 - mp.mpf(5605) / 2592 * eta**3) * x**3
         + (-mp.mpf(4415) / 4032 + mp.mpf(358675) / 6048 * eta + mp.mpf(91495) / 1512 * eta**2) * pi * x**3.5)
    dxdt = mp.mpf(64) / 5 * eta * x**5 * F
    return mp.mpf(3) / 2 * mp.sqrt(x) * dxdt


def test_rhs_matches_literature_taylor_t4_nonspinning(orc):
    """Eq. (1) with chi = 0 against the literature's form; pins the theta-hat reading."""
    mpmath.mp.dps = 30
    for m1 in (0.5, 0.25, 1 / 11):
        m2 = 1 - m1
        eta = m1 * m2
        for omega in (0.004, 0.01, 0.05, 0.1):
            y = np.array([omega, 0, 0, 0, 0, 0, 0, 0, 0, 1.0])
            f = orc.rhs(y, m1, m2)
            ref = float(_taylor_t4_rhs(omega, mpmath.mpf(eta)))
            assert f[0] == pytest.approx(ref, rel=5e-15)
            # the as-printed bracket differs by (88/3) theta eta (1 - eta) x^3 inside the braces
            f2 = orc.rhs(y, m1, m2, orc.params(theta_mode=1))
            lo = 96 / 5 * eta * omega ** (11 / 3)
            assert (f2[0] - f[0]) / lo == pytest.approx(88 / 3 * 1039 / 4620 * eta * (1 - eta) * omega**2, rel=1e-9)


def test_rhs_symmetric_under_relabelling(orc):
    """Swapping the labels 1 <-> 2 (masses and spins) swaps dS1/dt and dS2/dt; omega and L rates stay."""
    rng = np.random.default_rng(2)
    for _ in range(30):
        m1 = rng.uniform(0.1, 0.9)
        m2 = 1 - m1
        y = _rand_state(rng, m1, m2)
        ys = y.copy()
        ys[1:4], ys[4:7] = y[4:7], y[1:4]
        f = orc.rhs(y, m1, m2)
        g = orc.rhs(ys, m2, m1)
        assert g[0] == pytest.approx(f[0], rel=1e-14)
        sc = np.abs(f[1:]).max()
        assert np.allclose(g[1:4], f[4:7], atol=1e-14 * sc) and np.allclose(g[4:7], f[1:4], atol=1e-14 * sc)
        assert np.allclose(g[7:10], f[7:10], atol=1e-14 * sc)


def test_rhs_rotation_covariant(orc):
    rng = np.random.default_rng(3)
    for _ in range(30):
        m1 = rng.uniform(0.1, 0.9)
        m2 = 1 - m1
        y = _rand_state(rng, m1, m2)
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        yr = y.copy()
        for o in (1, 4, 7):
            yr[o:o + 3] = Q @ y[o:o + 3]
        f = orc.rhs(y, m1, m2)
        g = orc.rhs(yr, m1, m2)
        assert g[0] == pytest.approx(f[0], rel=1e-13)
        sc = np.abs(f[1:]).max()
        for o in (1, 4, 7):
            assert np.allclose(g[o:o + 3], Q @ f[o:o + 3], atol=1e-13 * sc)


def test_rhs_aligned_spins_are_fixed_points(orc):
    for m1 in (0.5, 0.3):
        m2 = 1 - m1
        for s1, s2 in ((1, 1), (1, -1), (-1, -1)):
            y = np.array([0.03, 0, 0, s1 * m1 * m1, 0, 0, s2 * 0.5 * m2 * m2, 0, 0, 1.0])
            f = orc.rhs(y, m1, m2)
            assert np.all(f[1:] == 0.0)


# ---------------------------------------------------------------------------
# Integration (Sec. II): closed forms, quadrature, invariants, convergence.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("q,w0,tf", [(1.0, 0.025, None), (1.0, 0.01, None), (10.0, 0.005, None)])
def test_newtonian_chirp_closed_form(orc, q, w0, tf):
    """Leading order: omega^{-8/3}(t) = omega_0^{-8/3} - (256/5) eta t at every accepted step and
    t_f = (5/256) eta^{-1} (omega_0^{-8/3} - omega_f^{-8/3})."""
    m1, m2 = q / (1 + q), 1 / (1 + q)
    eta = m1 * m2
    e = _one(m1, m2, 1.0, 1.0, (0.6, 0, 0.8), (0, -0.6, 0.8), w0, 0.05)
    prm = orc.params(term_mask=orc.NEWTONIAN, rtol=1e-13, atol=1e-13)
    rows, hs = orc.trace(e, 0, prm)
    t, w = rows[:, 0], rows[:, 1]
    lhs = w ** (-8 / 3)
    rhs = w0 ** (-8 / 3) - 256 / 5 * eta * t
    assert np.max(np.abs(lhs / rhs - 1)) < 1e-11
    tf = 5 / 256 / eta * (w0 ** (-8 / 3) - 0.05 ** (-8 / 3))
    assert rows[-1, 0] == pytest.approx(tf, rel=1e-11)
    assert rows[-1, 1] == pytest.approx(0.05, rel=1e-15)
    assert hs.sum() == pytest.approx(tf, rel=1e-12)


def _tf_quad(w0, wf, eta, so=0.0, ss=0.0):
    mpmath.mp.dps = 30
    return float(mpmath.quad(lambda w: 1 / _taylor_t4_rhs(w, mpmath.mpf(eta), so, ss), [w0, (w0 + wf) / 2, wf]))


@pytest.mark.parametrize("q,w0", [(1.0, 0.025), (3.0, 0.01), (10.0, 0.005)])
def test_full_pn_nonspinning_tf_by_quadrature(orc, q, w0):
    """chi = 0: L and S stay fixed, so t_f = int domega / (domega/dt) with the literature's series."""
    m1, m2 = q / (1 + q), 1 / (1 + q)
    e = _one(m1, m2, 0.0, 0.0, (0, 0, 1), (1, 0, 0), w0, 0.05)
    o = orc.integrate(e, orc.params(rtol=1e-13, atol=1e-13))
    assert o["status"][0] == 0
    assert o["t"][0] == pytest.approx(_tf_quad(w0, 0.05, m1 * m2), rel=1e-10)
    assert np.all(o["Lhat"][:, 0] == [0, 0, 1]) and np.all(o["S1"] == 0) and np.all(o["S2"] == 0)


@pytest.mark.parametrize("q,chi1,chi2,k1,k2", [(1.0, 1.0, 1.0, 1, 1), (2.5, 0.9, 0.4, 1, -1), (4.0, 0.3, 1.0, -1, -1)])
def test_aligned_spin_tf_by_quadrature(orc, q, chi1, chi2, k1, k2):
    """Spins (anti-)aligned with L stay fixed; t_f is then a quadrature of the scalar rate with the
    1.5PN spin-orbit term sum_i chi_i k_i (113 m_i^2 + 75 eta)/12 and the 2PN spin-spin term
    eta chi1 chi2 (247 k1 k2 - 721 k1 k2)/48, k_i = L.S_i-hat = +-1.  This exercises the oracle's
    vector path (S_i = chi_i m_i^2 S_i-hat, L.S_i / m_i^2, mass labels) against scalars."""
    m1, m2 = q / (1 + q), 1 / (1 + q)
    eta = m1 * m2
    e = _one(m1, m2, chi1, chi2, (0, 0, k1), (0, 0, k2), 0.01, 0.05)
    o = orc.integrate(e, orc.params(rtol=1e-13, atol=1e-13))
    so = (chi1 * k1 * (113 * m1 * m1 + 75 * eta) + chi2 * k2 * (113 * m2 * m2 + 75 * eta)) / 12
    ss = eta / 48 * chi1 * chi2 * (247 * k1 * k2 - 721 * k1 * k2)
    assert o["t"][0] == pytest.approx(_tf_quad(0.01, 0.05, eta, so, ss), rel=1e-10)
    assert np.allclose(o["S1"][:, 0], [0, 0, k1 * chi1 * m1 * m1], atol=1e-15)


def test_invariants_over_a_run(orc):
    e = workloads.config("C1", n=64)
    for tol, bound in ((5e-7, 1e-4), (1e-13, 2e-11)):
        o = orc.integrate(e, orc.params(rtol=tol, atol=tol))
        m1, m2 = e["m1"], e["m2"]
        n1 = np.linalg.norm(o["S1"], axis=0)
        n2 = np.linalg.norm(o["S2"], axis=0)
        nl = np.linalg.norm(o["Lhat"], axis=0)
        assert np.max(np.abs(n1 - e["chi1"] * m1 * m1) / (m1 * m1)) < bound
        assert np.max(np.abs(n2 - e["chi2"] * m2 * m2) / (m2 * m2)) < bound
        assert np.max(np.abs(nl - 1)) < bound


def test_nonspinning_L_stays_z(orc):
    e = workloads.config("C1", n=16)
    e["chi1"][:] = 0
    e["chi2"][:] = 0
    o = orc.integrate(e)
    assert np.all(o["Lhat"][2] == 1) and np.all(o["Lhat"][:2] == 0)
    assert np.all(o["S1"] == 0) and np.all(o["S2"] == 0)


def test_relabelling_symmetry_of_a_run(orc):
    e = workloads.config("C2", n=32)
    s = dict(e)
    s["m1"], s["m2"] = e["m2"], e["m1"]
    s["chi1"], s["chi2"] = e["chi2"], e["chi1"]
    s["s1hat"], s["s2hat"] = e["s2hat"], e["s1hat"]
    a = orc.integrate(e)
    b = orc.integrate(s)
    assert np.array_equal(a["n_acc"], b["n_acc"]) and np.array_equal(a["n_rej"], b["n_rej"])
    assert np.allclose(a["S1"], b["S2"], rtol=0, atol=1e-12) and np.allclose(a["S2"], b["S1"], rtol=0, atol=1e-12)
    assert np.allclose(a["t"], b["t"], rtol=1e-12)
    assert np.allclose(a["dot_s1s2"], b["dot_s1s2"], atol=1e-11)


def test_fifth_order_convergence_fixed_step(orc):
    """Fixed steps h = 80 ... 5: the error at omega_f falls as h^5 (least-squares order in [4.6, 5.8])."""
    e = workloads.config("C0", n=2)
    ref = orc.integrate(e, orc.params(rtol=1e-14, atol=1e-14))
    Hs = np.array([80.0, 40.0, 20.0, 10.0, 5.0])
    errs = []
    for H in Hs:
        o = orc.integrate(e, orc.params(fixed_step=1, h0=H))
        errs.append(max(np.abs(o["S1"] - ref["S1"]).max(), np.abs(o["Lhat"] - ref["Lhat"]).max()))
    order = np.polyfit(np.log2(Hs), np.log2(errs), 1)[0]
    assert 4.6 < order < 5.8, (order, errs)


def test_tolerance_scaling_against_tight_run(orc):
    e = workloads.config("C1", n=16)
    ref = orc.integrate(e, orc.params(rtol=1e-13, atol=1e-13))

    def err(o):
        return max(np.abs(o[k] - ref[k]).max() for k in ("S1", "S2", "Lhat"))

    e1 = err(orc.integrate(e))
    e2 = err(orc.integrate(e, orc.params(rtol=5e-9, atol=5e-9)))
    assert e1 < 1e-4
    assert e2 < e1 / 20


def test_independent_rk4_agrees(orc):
    """A fixed-step classical RK4 written here (own stepping and own landing by secant) on the
    oracle's RHS reproduces the oracle's tight-tolerance final state."""
    e = workloads.config("C0", n=1)
    m1, m2 = e["m1"][0], e["m2"][0]
    ref = orc.integrate(e, orc.params(rtol=1e-14, atol=1e-14))
    y = np.concatenate([[e["omega0"][0]], e["chi1"][0] * m1 * m1 * e["s1hat"][:, 0],
                        e["chi2"][0] * m2 * m2 * e["s2hat"][:, 0], e["lhat"][:, 0]])
    f = lambda z: orc.rhs(z, m1, m2)

    def rk4(z, h):
        k1 = f(z)
        k2 = f(z + h / 2 * k1)
        k3 = f(z + h / 2 * k2)
        k4 = f(z + h * k3)
        return z + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)

    h, t, wf = 0.25, 0.0, 0.05
    while True:
        z = rk4(y, h)
        if z[0] >= wf:
            break
        y, t = z, t + h
    a, b = 0.0, h  # secant on omega(h) - wf
    ga, gb = y[0] - wf, z[0] - wf
    for _ in range(30):
        c = b - gb * (b - a) / (gb - ga)
        zc = rk4(y, c)
        a, ga, b, gb = b, gb, c, zc[0] - wf
        if abs(gb) < 1e-17:
            break
    zc = rk4(y, b)
    assert t + b == pytest.approx(ref["t"][0], rel=1e-11)
    for k, sl in (("S1", slice(1, 4)), ("S2", slice(4, 7)), ("Lhat", slice(7, 10))):
        assert np.allclose(zc[sl], ref[k][:, 0], rtol=0, atol=2e-10)


# ---------------------------------------------------------------------------
# Statuses and inputs.
# ---------------------------------------------------------------------------
def test_bad_inputs_and_limits(orc):
    e = workloads.config("C0", n=6)
    e["chi1"][0] = 1.5           # chi outside [0, 1]
    e["omega0"][1] = 0.06        # omega_0 >= omega_f
    e["m1"][2] = np.nan          # non-finite
    e["m1"][3] = 0.7             # m1 + m2 != 1
    o = orc.integrate(e)
    assert list(o["status"][:4]) == [orc.ST_BAD_INPUT] * 4
    assert list(o["status"][4:]) == [orc.ST_OK] * 2
    o = orc.integrate(workloads.config("C0", n=2), orc.params(max_steps=3))
    assert np.all(o["status"] == orc.ST_MAX_STEPS) and np.all(o["n_acc"] + o["n_rej"] + o["n_land"] == 3)
    z = workloads.config("C0", n=2)
    z["chi1"][:] = 0.0
    o = orc.integrate(z)
    assert np.all(o["status"] == 0) and np.all(np.isnan(o["dot_s1s2"])) and np.all(np.isnan(o["dot_ls1"]))


def test_first_cross_mode_overshoots(orc):
    e = workloads.config("C0", n=8)
    a = orc.integrate(e)
    b = orc.integrate(e, orc.params(stop_mode=1))
    assert np.all(b["omega"] >= 0.05) and np.all(a["omega"] == 0.05)
    assert np.all(b["t"] >= a["t"])


# ---------------------------------------------------------------------------
# Sampler (Sec. V): SplitMix64 + Marsaglia.
# ---------------------------------------------------------------------------
def test_splitmix64_published_vectors(orc):
    assert orc.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert orc.splitmix64(1234567, 5) == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                          4593380528125082431, 16408922859458223821]


def test_uniform_keying_is_two_level_splitmix(orc):
    seed = 0x0908_3889_0001
    for i in (0, 1, 7, 123456):
        key = orc.splitmix64(seed, i + 1)[i]
        stream = orc.splitmix64(key, 6)
        for j in range(6):
            assert orc.uniform(seed, i, j) == (stream[j] >> 11) * 2.0**-53


def test_marsaglia_directions_are_isotropic(orc):
    a = orc.sample(99, orc.Dist(q_mode=2, q_lo=1.0, q_hi=10.0, chi_mode=1, chi_lo=0.0, chi_hi=1.0,
                                omega0_lo=0.005, omega0_hi=0.02), 100_000)
    for k in ("s1hat", "s2hat"):
        v = a[k]
        assert np.max(np.abs(np.linalg.norm(v, axis=0) - 1)) < 1e-15
        assert stats.kstest((v[2] + 1) / 2, "uniform").pvalue > 1e-3
        phi = (np.arctan2(v[1], v[0]) + np.pi) / (2 * np.pi)
        assert stats.kstest(phi, "uniform").pvalue > 1e-3
        assert np.all(np.abs(v.mean(1)) < 5 / math.sqrt(3 * 100_000))
    assert stats.kstest(np.log(a["m1"] / a["m2"]) / np.log(10), "uniform").pvalue > 1e-3
    assert stats.kstest(a["chi1"], "uniform").pvalue > 1e-3
    assert stats.kstest((a["omega0"] - 0.005) / 0.015, "uniform").pvalue > 1e-3
    assert np.all(np.abs(a["m1"] + a["m2"] - 1) < 3e-16)
    assert abs(np.corrcoef(a["s1hat"][2], a["s2hat"][2])[0, 1]) < 0.02


# ---------------------------------------------------------------------------
# Forward-mode gradient vs central finite differences of the replayed map.
# ---------------------------------------------------------------------------
def _outputs_of_state(y, t):
    S1, S2, L = y[1:4], y[4:7], y[7:10]
    n1, n2, nl = np.linalg.norm(S1), np.linalg.norm(S2), np.linalg.norm(L)
    return np.concatenate([[S1 @ S2 / (n1 * n2), L @ S1 / (nl * n1), L @ S2 / (nl * n2)], L, S1, S2, [t]])


def test_forward_gradient_matches_finite_differences(orc):
    e = workloads.config("C4", n=4)
    for i in range(4):
        out, jac, nacc = orc.grad(e, i)
        rows, hs = orc.trace(e, i)
        assert len(hs) == nacc
        fd = np.empty_like(jac)
        d = 1e-6
        for k in range(7):
            vals = []
            for sgn in (+1, -1):
                p = workloads.take(e, np.array([i]))
                if k < 3:
                    p["s1hat"][k, 0] += sgn * d
                elif k < 6:
                    p["s2hat"][k - 3, 0] += sgn * d
                else:
                    q = p["m1"][0] / p["m2"][0] + sgn * d
                    p["m1"][0], p["m2"][0] = q / (1 + q), 1 / (1 + q)
                y, t = orc.replay(p, 0, hs)
                vals.append(_outputs_of_state(y, t))
            fd[:, k] = (vals[0] - vals[1]) / (2 * d)
        scale = np.maximum(1.0, np.abs(jac))
        scale[12] = np.maximum(abs(out[12]), 1.0)  # t_f
        assert np.max(np.abs(fd - jac) / scale) < 2e-6, np.max(np.abs(fd - jac) / scale)


# ---------------------------------------------------------------------------
# Paper-printed statistics (Sec. V): weak but independent physics pins.
# ---------------------------------------------------------------------------
def _dots0(e):
    s1, s2, l = e["s1hat"], e["s2hat"], e["lhat"]
    return (s1 * s2).sum(0), (l * s1).sum(0), (l * s2).sum(0)


def test_paper_pearson_equal_mass_maximal_spin(orc):
    pv = _paper_values()
    e = workloads.config("SCIENCE", n=10_000)
    o = orc.integrate(e)
    assert np.all(o["status"] == 0)
    d12, dl1, dl2 = _dots0(e)
    for key, a, b in (("pearson_s1s2_eqmass_chi1", d12, o["dot_s1s2"]), ("pearson_ls1_eqmass_chi1", dl1, o["dot_ls1"]),
                      ("pearson_ls2_eqmass_chi1", dl2, o["dot_ls2"])):
        v, tol = pv[key]
        assert abs(np.corrcoef(a, b)[0, 1] - v) <= tol, (key, np.corrcoef(a, b)[0, 1])
    nb = int(pv["final_s1s2_uniform_bins"][0])
    h, _ = np.histogram(o["dot_s1s2"], bins=nb, range=(-1, 1))
    assert stats.chisquare(h).pvalue > 1e-3


def test_paper_pearson_chi_sweep_and_unequal_ring(orc):
    pv = _paper_values()
    lo = pv["pearson_s1s2_min_over_chi"][0]
    for chi in (0.2, 0.5, 0.8):
        e = workloads.ensemble(4000, 500 + int(chi * 10), chi=(chi, chi), omega0=(0.00395, 0.00395))
        o = orc.integrate(e)
        assert np.corrcoef(_dots0(e)[0], o["dot_s1s2"])[0, 1] > lo
    v, tol = pv["pearson_s1s2_m04_chi005"]
    e = workloads.ensemble(10_000, 77, q=(0.4 / 0.6, 0.4 / 0.6), chi=(0.05, 0.05), omega0=(0.00395, 0.00395))
    o = orc.integrate(e)
    assert abs(np.corrcoef(_dots0(e)[0], o["dot_s1s2"])[0, 1] - v) <= tol
