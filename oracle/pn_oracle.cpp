// pn_oracle.cpp -- CPU FP64 oracle for batched post-Newtonian (PN) inspirals.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
// CUDA path is checked against.  Only the test suite, the package's smoke()
// check and bench.py's cpu_baseline / reference arm may load it.  It shares no
// code, header, table or constant with the CUDA library, and neither side
// includes or calls the other.
//
// What it computes (arXiv:0908.3889, Herrmann et al. 2009):
//   * the PN right-hand side of Eqs. (1)-(4) (Sec. II): the orbital-frequency
//     chirp through 3.5PN (Eq. 1), spin precession dS_i/dt = Omega_i x S_i
//     (Eqs. 2 and 4) and the orbital-axis evolution (Eq. 3), with M = m1+m2 = 1,
//     eta = m1 m2 and S_i = chi_i m_i^2 S_i-hat (Sec. II);
//   * its integration in t by the Dormand-Prince method with error tolerance
//     5e-7 and first step h = 10 (Sec. II), from a circular orbit at omega_0
//     with L-hat = z-hat (Sec. V) up to omega_f;
//   * isotropic spin directions by Marsaglia's (1972) rejection method
//     (Sec. V) driven by the SplitMix64 generator (Steele, Lea & Flood 2014);
//   * a forward-mode (dual-number) gradient of the final outputs with respect
//     to the initial spin directions and the mass ratio, with the accepted
//     step sizes held fixed and the stop at omega_f treated as an implicit
//     function of the parameters.
//
// Readings where the paper is silent or garbled (each used identically by the
// CUDA path, each an input the caller can select where there is a choice):
//   * 3PN theta-hat term: the printed bracket multiplies theta-hat by eta twice;
//     the default (THETA_BCV2) multiplies it once, which reproduces the standard
//     3PN coefficient -56198689/217728 + 451 pi^2/48 exactly.  THETA_AS_PRINTED
//     keeps the printed form.
//   * log in Eq. (1) is the natural log; gamma_E = 0.5772156649015329,
//     theta-hat = 1039/4620.
//   * chi_i L-hat.S_i-hat is taken as L.S_i / m_i^2 from the current state, and
//     eta chi1 chi2 S1-hat.S2-hat as eta S1.S2/(m1^2 m2^2); L is not renormalised.
//   * t is the independent variable; "from omega_0 to omega_f" is the start and
//     stop rule.  Tolerance: atol = rtol = 5e-7 with the RMS norm over the 10
//     components, scale atol + rtol*max(|y_i|, |y_new_i|); err <= 1 accepts.
//   * Step control: h_new = h * clamp(safety * err^(-1/5), fac_min, fac_max),
//     safety 0.9, fac_min 0.2, fac_max 10, no growth right after a rejection.
//   * Stop (STOP_LAND, default): when an accepted step crosses omega_f the step
//     is retaken from its start with a Newton iteration on h whose slope is the
//     omega-rate of the last stage (FSAL), seeded by the root of the step's
//     cubic Hermite interpolant and bracketed, until |omega - omega_f| <=
//     land_tol * omega_f (1e-7); the retaken state is then moved along f by
//     dh = -(omega - omega_f)/(domega/dt), which lands omega to O(dh^2).
//     STOP_FIRST_CROSS returns the first accepted state with omega >= omega_f.
//
// Precision: FP64 throughout, compiled with -ffp-contract=off so every
// operation rounds as written; cbrt, log and pow come from the C library.
//
// Parity status per function:
//   rhs            pinned: leading-order chirp closed form, textbook geodetic
//                  precession rate, J conservation at fixed omega, S.dS = 0,
//                  1<->2 symmetry, rotation covariance, literature TaylorT4
//                  coefficients (non-spinning), paper-printed Pearson r values.
//   dp5 tableau    pinned: Butcher order conditions (orders 5 and 4).
//   integrate      pinned: Newtonian t_f closed form, quadrature of t_f for
//                  non-spinning and aligned-spin binaries, 5th-order convergence,
//                  tolerance scaling vs a tight run and an independent RK4.
//   err_norm and the step-size controller   pinned to the reading above (the
//                  paper states only the tolerance and h0; the constants are
//                  the reading's): on the leading-order chirp the norm of one
//                  attempt equals the RMS of the embedded estimate from the
//                  Butcher series of the tableau, for absolute, relative and
//                  mixed scales; accepted steps settle at the 0.9^5 error fixed
//                  point of safety 0.9 and exponent -1/5; the 0.2 / 10 clamps
//                  and the no-growth rule after a rejection act where the series
//                  says they must.  Planted mistakes in a copy of this file
//                  (2-norm, dropped h, -1/4, safety 0.8, ...) fail these pins.
//   landing        pinned: omega lands on omega_f; Newtonian t_f closed form
//                  and quadrature of t_f for non-spinning and aligned spins.
//   sample         pinned: SplitMix64 published output vectors; isotropy tests.
//   grad           pinned: central finite differences of the replayed map.

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ----------------------------------------------------------------------------
// Public structs (mirrored by ctypes in oracle.py).
// ----------------------------------------------------------------------------
struct OParams {
  double rtol, atol, h0, safety, fac_min, fac_max, h_min, land_tol;
  int64_t max_steps;      // cap on attempts (accepted + rejected + landing retakes)
  int32_t land_max_iter;  // Newton retakes allowed at the stop
  int32_t stop_mode;      // 0 = land on omega_f, 1 = first crossing
  uint32_t term_mask;     // PN terms switched on (bits below)
  int32_t theta_mode;     // 0 = BCV2 reading (theta*eta), 1 = as printed (theta*eta^2)
  int32_t fixed_step;     // 1: every attempt accepted with h = h0 (convergence tests)
  int32_t pad_;
};

enum : uint32_t {
  T_1PN = 1u << 0,    // -(743+924 eta)/336 x
  T_SO = 1u << 1,     // spin-orbit part of the 1.5PN bracket
  T_TAIL = 1u << 2,   // +4 pi x^{3/2}
  T_2PN = 1u << 3,    // non-spin 2PN
  T_SS = 1u << 4,     // spin-spin 2PN
  T_25PN = 1u << 5,
  T_3PN = 1u << 6,    // 3PN incl. log
  T_35PN = 1u << 7,
  T_PREC = 1u << 8,   // spin precession (Eqs. 2-4); off => S and L frozen
  T_ALL = 0x1ffu,
};

enum : int32_t { ST_OK = 0, ST_MAX_STEPS = 1, ST_H_UNDERFLOW = 2, ST_NONFINITE = 3,
                 ST_BAD_INPUT = 4, ST_LAND_MAXIT = 5 };

struct OBatchIn {  // structure of arrays, each of length n (vectors: 3 arrays)
  const double *m1, *m2, *chi1, *chi2;
  const double *s1x, *s1y, *s1z, *s2x, *s2y, *s2z;
  const double *lx, *ly, *lz;
  const double *omega0, *omega_f;
};
struct OBatchOut {
  double *S1x, *S1y, *S1z, *S2x, *S2y, *S2z, *Lx, *Ly, *Lz;
  double *omega, *t;
  int32_t *n_acc, *n_rej, *n_land, *status;
  double *dot_s1s2, *dot_ls1, *dot_ls2;
};

struct OBinary {
  double m1, m2, chi1, chi2, s1[3], s2[3], l0[3], omega0, omega_f;
};
struct OResult {
  double y[10];
  double t;
  int32_t n_acc, n_rej, n_land, status;
};

// ----------------------------------------------------------------------------
// Scalar types.  The RHS and the DP5 stage map are templates so the same plain
// code runs on double, on forward-mode dual numbers and on an op counter.
// ----------------------------------------------------------------------------
constexpr int ND = 8;  // dual directions: s1hat(3), s2hat(3), q, h (landing)
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0) { for (int i = 0; i < ND; i++) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < ND; i++) d[i] = 0; }
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < ND; i++) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < ND; i++) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < ND; i++) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < ND; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int i = 0; i < ND; i++) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { return a * Dual(b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a) * b; }
inline Dual operator/(const Dual& a, double b) { return a / Dual(b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual cbrt_(const Dual& a) {  // d cbrt(x) = cbrt(x) / (3x) dx
  Dual r(std::cbrt(a.v));
  for (int i = 0; i < ND; i++) r.d[i] = a.d[i] * r.v / (3.0 * a.v);
  return r;
}
inline Dual log_(const Dual& a) { Dual r(std::log(a.v)); for (int i = 0; i < ND; i++) r.d[i] = a.d[i] / a.v; return r; }
inline Dual sqrt_(const Dual& a) { Dual r(std::sqrt(a.v)); for (int i = 0; i < ND; i++) r.d[i] = a.d[i] / (2.0 * r.v); return r; }
inline double cbrt_(double a) { return std::cbrt(a); }
inline double log_(double a) { return std::log(a); }
inline double sqrt_(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }

// Operation counter: every +, -, *, / is one floating-point operation (no FMA
// contraction in this file); cbrt / log / pow / sqrt are counted apart.
struct OpCount { int64_t add, mul, div, sqrt, cbrt, log, pow; };
thread_local OpCount g_ops;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt operator+(Cnt a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, Cnt b) { return Cnt(a) + b; }
inline Cnt operator-(Cnt a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, Cnt b) { return Cnt(a) - b; }
inline Cnt operator*(Cnt a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, Cnt b) { return Cnt(a) * b; }
inline Cnt operator/(Cnt a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, Cnt b) { return Cnt(a) / b; }
inline Cnt cbrt_(Cnt a) { g_ops.cbrt++; return Cnt(std::cbrt(a.v)); }
inline Cnt log_(Cnt a) { g_ops.log++; return Cnt(std::log(a.v)); }
inline Cnt sqrt_(Cnt a) { g_ops.sqrt++; return Cnt(std::sqrt(a.v)); }
inline double val(Cnt a) { return a.v; }

// ----------------------------------------------------------------------------
// Constants of Eq. (1).
// ----------------------------------------------------------------------------
const double PI = 3.141592653589793238462643383279502884;
const double GAMMA_E = 0.5772156649015328606065120900824024310;  // Euler's constant
const double THETA_HAT = 1039.0 / 4620.0;

// Per-binary constants of Eqs. (1) and (4) with M = m1 + m2 = 1 (Sec. II):
// the masses, eta = m1 m2 / M^2, and every bracket coefficient that depends on
// the masses only.  They are computed once per binary; the RHS below then does
// only the work that depends on the state.
template <class T>
struct Coeffs {
  T m1, m2, eta;
  T inv_m1sq, inv_m2sq;  // chi_i S_i-hat = S_i / m_i^2
  T so1, so2;            // (113 m_i^2 / M^2 + 75 eta) / 12        (1.5PN spin-orbit)
  T c1, c2, c25, c3, c35;  // non-spin coefficients of x, x^2, x^{5/2}, x^3, x^{7/2}
  T ss;                  // eta / 48                                (2PN spin-spin)
  T a1, a2;              // eta (4 + 3 m2/m1), eta (4 + 3 m1/m2)    (Eq. 4)
  T inv_eta;             // 1 / (eta M^2)                           (Eq. 3)
};
template <class T>
Coeffs<T> make_coeffs(const T& m1, const T& m2, const OParams& p) {
  Coeffs<T> c;
  c.m1 = m1;
  c.m2 = m2;
  c.eta = m1 * m2;  // M = 1
  const T eta = c.eta;
  c.inv_m1sq = 1.0 / (m1 * m1);
  c.inv_m2sq = 1.0 / (m2 * m2);
  c.so1 = (113.0 * m1 * m1 + 75.0 * eta) / 12.0;
  c.so2 = (113.0 * m2 * m2 + 75.0 * eta) / 12.0;
  c.c1 = -(743.0 + 924.0 * eta) / 336.0;
  c.c2 = 34103.0 / 18144.0 + 13661.0 / 2016.0 * eta + 59.0 / 18.0 * eta * eta;
  c.c25 = -(4159.0 + 15876.0 * eta) * PI / 672.0;
  T c3 = T(16447322263.0 / 139708800.0 - 1712.0 / 105.0 * GAMMA_E + 16.0 / 3.0 * PI * PI);
  if (p.theta_mode == 0)  // theta-hat multiplies eta once (reading of the garbled bracket)
    c3 = c3 + (-273811877.0 / 1088640.0 + 451.0 / 48.0 * PI * PI - 88.0 / 3.0 * THETA_HAT) * eta;
  else                    // as printed: theta-hat eta^2
    c3 = c3 + (-273811877.0 / 1088640.0 + 451.0 / 48.0 * PI * PI - 88.0 / 3.0 * THETA_HAT * eta) * eta;
  c.c3 = c3 + 541.0 / 896.0 * eta * eta - 5605.0 / 2592.0 * eta * eta * eta;
  c.c35 = (-4415.0 / 4032.0 + 358675.0 / 6048.0 * eta + 91495.0 / 1512.0 * eta * eta) * PI;
  c.ss = eta / 48.0;
  c.a1 = eta * (4.0 + 3.0 * m2 / m1);
  c.a2 = eta * (4.0 + 3.0 * m1 / m2);
  c.inv_eta = 1.0 / eta;
  return c;
}

template <class T>
T dot3(const T* a, const T* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T>
void cross3(const T* a, const T* b, T* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Right-hand side f(y), y = (omega, S1[3], S2[3], L[3]), M = 1, x = M omega.
//   Eq. (1): domega/dt = omega^2 (96/5) eta x^{5/3} { 1 + c1 x^{2/3}
//              - (sum_i chi_i L.S_i-hat (113 m_i^2 + 75 eta)/12 - 4 pi) x
//              + (c2 - eta chi1 chi2 (247 S1-hat.S2-hat - 721 L.S1-hat L.S2-hat)/48) x^{4/3}
//              + c25 x^{5/3} + (c3 - 856/105 ln(16 x^{2/3})) x^2 + c35 x^{7/3} }
//   Eq. (4): Omega_1 = x^2/(2M) [ eta x^{-1/3} (4 + 3 m2/m1) L + (S2 - 3 (S2.L) L)/M^2 ],
//            Omega_2 by 1<->2
//   Eq. (2): dS_i/dt = Omega_i x S_i
//   Eq. (3): dL/dt = -x^{1/3}/(eta M^2) (dS1/dt + dS2/dt)
template <class T>
void rhs(const Coeffs<T>& cf, const OParams& p, const T* y, T* f) {
  const T omega = y[0];
  const T* S1 = y + 1;
  const T* S2 = y + 4;
  const T* L = y + 7;
  const uint32_t mask = p.term_mask;

  const T x = omega;
  const T x13 = cbrt_(x);
  const T x23 = x13 * x13;
  const T x43 = x * x13;
  const T x53 = x * x23;
  const T x2 = x * x;
  const T x73 = x2 * x13;

  const T LS1 = dot3(L, S1);
  const T LS2 = dot3(L, S2);
  const T chiLS1 = LS1 * cf.inv_m1sq;  // chi_1 L.S1-hat
  const T chiLS2 = LS2 * cf.inv_m2sq;  // chi_2 L.S2-hat

  T P = T(1.0);
  if (mask & T_1PN) P = P + cf.c1 * x23;
  T so = T(0.0);
  if (mask & T_SO) so = chiLS1 * cf.so1 + chiLS2 * cf.so2;
  if (mask & T_TAIL) so = so - 4.0 * PI;
  if (mask & (T_SO | T_TAIL)) P = P - so * x;
  T c2 = T(0.0);
  if (mask & T_2PN) c2 = cf.c2;
  if (mask & T_SS) {
    const T chi12 = dot3(S1, S2) * cf.inv_m1sq * cf.inv_m2sq;  // chi1 chi2 S1-hat.S2-hat
    c2 = c2 - cf.ss * (247.0 * chi12 - 721.0 * (chiLS1 * chiLS2));
  }
  if (mask & (T_2PN | T_SS)) P = P + c2 * x43;
  if (mask & T_25PN) P = P + cf.c25 * x53;
  if (mask & T_3PN) P = P + (cf.c3 - 856.0 / 105.0 * log_(16.0 * x23)) * x2;
  if (mask & T_35PN) P = P + cf.c35 * x73;

  f[0] = (96.0 / 5.0) * cf.eta * (omega * omega) * x53 * P;

  if (mask & T_PREC) {
    const T pre = 0.5 * x2;
    const T b1 = cf.a1 / x13;  // eta x^{-1/3} (4 + 3 m2/m1)
    const T b2 = cf.a2 / x13;
    T Om1[3], Om2[3];
    for (int c = 0; c < 3; c++) {
      Om1[c] = pre * (b1 * L[c] + (S2[c] - 3.0 * LS2 * L[c]));
      Om2[c] = pre * (b2 * L[c] + (S1[c] - 3.0 * LS1 * L[c]));
    }
    T dS1[3], dS2[3];
    cross3(Om1, S1, dS1);  // Eq. (2)
    cross3(Om2, S2, dS2);
    const T lfac = x13 * cf.inv_eta;
    for (int c = 0; c < 3; c++) {
      f[1 + c] = dS1[c];
      f[4 + c] = dS2[c];
      f[7 + c] = -(lfac * (dS1[c] + dS2[c]));  // Eq. (3)
    }
  } else {
    for (int c = 1; c < 10; c++) f[c] = T(0.0);
  }
}

// ----------------------------------------------------------------------------
// Dormand & Prince (1980) RK5(4)7M tableau, typed from the published table.
// ----------------------------------------------------------------------------
const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0},
};
const double DP_B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
const double DP_BHAT[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                           -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

// One DP5 attempt from y with step h.  k[0] = f(y) must be supplied (FSAL).
// Fills k[1..6] and y5 = y + h sum_j b_j k_j; k[6] = f(y5).
template <class T>
void dp5_attempt(const Coeffs<T>& ms, const OParams& p, const T* y, const T& h, T k[7][10], T* y5) {
  T ys[10];
  for (int s = 1; s < 7; s++) {
    for (int i = 0; i < 10; i++) {
      T acc = DP_A[s][0] * k[0][i];
      for (int j = 1; j < s; j++)
        if (DP_A[s][j] != 0.0) acc = acc + DP_A[s][j] * k[j][i];
      ys[i] = y[i] + h * acc;
    }
    rhs(ms, p, ys, k[s]);
  }
  for (int i = 0; i < 10; i++) y5[i] = ys[i];  // row 7 of A is b (FSAL)
}

// Error norm of Sec. II's tolerance reading: RMS over the 10 components of
// e_i / (atol + rtol * max(|y_i|, |y5_i|)) with e = h sum_j (b_j - bhat_j) k_j.
template <class T>
T err_norm(const OParams& p, const T* y, const T* y5, const T& h, T k[7][10]) {
  T sum = T(0.0);
  for (int i = 0; i < 10; i++) {
    T e = (DP_B[0] - DP_BHAT[0]) * k[0][i];
    for (int j = 1; j < 7; j++)
      if (DP_B[j] != DP_BHAT[j]) e = e + (DP_B[j] - DP_BHAT[j]) * k[j][i];
    e = h * e;
    const double ay = std::fabs(val(y[i])), ay5 = std::fabs(val(y5[i]));
    const T sc = p.atol + p.rtol * T(ay > ay5 ? ay : ay5);
    const T r = e / sc;
    sum = sum + r * r;
  }
  return sqrt_(sum / 10.0);
}

bool all_finite(const double* v, int n) {
  for (int i = 0; i < n; i++)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Initial state of Secs. II and V: omega = omega_0, S_i = chi_i m_i^2 S_i-hat,
// L-hat as given (z-hat in the paper).
template <class T>
void initial_state(const T& m1, const T& m2, double chi1, double chi2, const T* s1, const T* s2,
                   const double* l0, double omega0, T* y) {
  y[0] = T(omega0);
  for (int c = 0; c < 3; c++) {
    y[1 + c] = chi1 * (m1 * m1) * s1[c];
    y[4 + c] = chi2 * (m2 * m2) * s2[c];
    y[7 + c] = T(l0[c]);
  }
}

int32_t validate(const OBinary& b) {
  const double v[] = {b.m1, b.m2, b.chi1, b.chi2, b.s1[0], b.s1[1], b.s1[2], b.s2[0], b.s2[1],
                      b.s2[2], b.l0[0], b.l0[1], b.l0[2], b.omega0, b.omega_f};
  if (!all_finite(v, 15)) return ST_BAD_INPUT;
  if (!(b.m1 > 0.0) || !(b.m2 > 0.0) || std::fabs(b.m1 + b.m2 - 1.0) > 1e-12) return ST_BAD_INPUT;
  if (b.chi1 < 0.0 || b.chi1 > 1.0 || b.chi2 < 0.0 || b.chi2 > 1.0) return ST_BAD_INPUT;
  if (!(b.omega0 > 0.0) || !(b.omega_f > b.omega0)) return ST_BAD_INPUT;
  const double l2 = b.l0[0] * b.l0[0] + b.l0[1] * b.l0[1] + b.l0[2] * b.l0[2];
  if (std::fabs(std::sqrt(l2) - 1.0) > 1e-12) return ST_BAD_INPUT;
  return ST_OK;
}

bool params_ok(const OParams& p) {
  return p.rtol >= 0.0 && p.atol >= 0.0 && (p.rtol > 0.0 || p.atol > 0.0) && p.h0 > 0.0 &&
         p.safety > 0.0 && p.fac_min > 0.0 && p.fac_max >= 1.0 && p.fac_min <= 1.0 && p.h_min >= 0.0 &&
         p.land_tol > 0.0 && p.max_steps > 0 && p.land_max_iter >= 1;
}

// Root in (0, 1] of the cubic Hermite interpolant of omega over one step:
// p(s) = (2s^3 - 3s^2 + 1) w0 + (s^3 - 2s^2 + s) d0 + (3s^2 - 2s^3) w1 + (s^3 - s^2) d1,
// with w0, w1 the end values and d0, d1 = h * domega/dt at the ends, solved
// for p(s) = wf by three Newton steps from the linear guess.
double hermite_root(double w0, double d0, double w1, double d1, double wf) {
  double s = (wf - w0) / (w1 - w0);
  for (int it = 0; it < 3; it++) {
    const double s2 = s * s, s3 = s2 * s;
    const double ps = (2.0 * s3 - 3.0 * s2 + 1.0) * w0 + (s3 - 2.0 * s2 + s) * d0 +
                      (3.0 * s2 - 2.0 * s3) * w1 + (s3 - s2) * d1;
    const double dps = (6.0 * s2 - 6.0 * s) * w0 + (3.0 * s2 - 4.0 * s + 1.0) * d0 +
                       (6.0 * s - 6.0 * s2) * w1 + (3.0 * s2 - 2.0 * s) * d1;
    s = s - (ps - wf) / dps;
  }
  return s;
}

// Adaptive integration of one binary, one DP5 attempt per loop iteration.
// Mode STEP: ordinary steps under error control.  An accepted attempt whose
// omega reaches omega_f either ends the run (STOP_FIRST_CROSS), lands at once
// if it is already within land_tol, or switches to mode LAND, which retakes
// the step from its start (t, y) with Newton-updated sizes until omega is
// within land_tol of omega_f, then moves the state along f onto omega_f.
// A run ends with PN status codes:
//   MAX_STEPS    max_steps attempts made without finishing (the state is the
//                last committed one; if it happens during LAND, the last retake),
//   H_UNDERFLOW  a rejection pushed h below h_min,
//   NONFINITE    an attempt produced a non-finite state or error norm,
//   LAND_MAXIT   land_max_iter retakes did not reach land_tol (last retake kept).
// If hs != nullptr the accepted step sizes (the landing step last) are appended;
// if tr != nullptr the state after every accepted step is appended (t, y[10]).
OResult integrate_one(const OBinary& b, const OParams& p, std::vector<double>* hs,
                      std::vector<double>* tr) {
  OResult r;
  std::memset(&r, 0, sizeof(r));
  r.status = validate(b);
  if (r.status != ST_OK || !params_ok(p)) {
    r.status = ST_BAD_INPUT;
    for (int i = 0; i < 10; i++) r.y[i] = NAN;
    r.t = NAN;
    return r;
  }
  const Coeffs<double> ms = make_coeffs(b.m1, b.m2, p);
  double y[10];
  initial_state(b.m1, b.m2, b.chi1, b.chi2, b.s1, b.s2, b.l0, b.omega0, y);
  double t = 0.0, h = p.h0;
  double k[7][10], y5[10];
  rhs(ms, p, y, k[0]);
  bool last_rejected = false;
  bool landing = false;
  double h_lo = 0.0, h_hi = 0.0;
  int land_it = 0;
  int64_t attempts = 0;
  if (tr) { tr->push_back(t); for (int i = 0; i < 10; i++) tr->push_back(y[i]); }

  auto commit = [&](double hc) {
    t = t + hc;
    for (int i = 0; i < 10; i++) y[i] = y5[i];
    r.n_acc++;
    if (hs) hs->push_back(hc);
    if (tr) { tr->push_back(t); for (int i = 0; i < 10; i++) tr->push_back(y[i]); }
  };
  auto land = [&](double g) {  // first-order move of the retaken state onto omega_f
    const double dh = -g / k[6][0];
    for (int i = 0; i < 10; i++) y5[i] = y5[i] + dh * k[6][i];
    commit(h + dh);
  };

  for (;;) {
    dp5_attempt(ms, p, y, h, k, y5);
    attempts++;
    const double err = p.fixed_step ? 0.0 : err_norm(p, y, y5, h, k);
    if (!all_finite(y5, 10) || !std::isfinite(err)) { r.status = ST_NONFINITE; break; }

    if (landing) {
      r.n_land++;
      land_it++;
      const double g = y5[0] - b.omega_f;
      if (std::fabs(g) <= p.land_tol * b.omega_f) { land(g); r.status = ST_OK; break; }
      if (land_it >= p.land_max_iter || attempts >= p.max_steps) {
        commit(h);
        r.status = attempts >= p.max_steps ? ST_MAX_STEPS : ST_LAND_MAXIT;
        break;
      }
      if (g > 0.0) h_hi = h; else h_lo = h;
      h = h - g / k[6][0];
      if (!(h > h_lo && h < h_hi)) h = 0.5 * (h_lo + h_hi);
      continue;
    }

    if (err <= 1.0) {
      if (y5[0] >= b.omega_f) {
        const double g = y5[0] - b.omega_f;
        if (p.stop_mode == 1) { commit(h); r.status = ST_OK; break; }
        if (std::fabs(g) <= p.land_tol * b.omega_f) { land(g); r.status = ST_OK; break; }
        // Seed the retakes from the root of the step's cubic Hermite interpolant.
        landing = true;
        land_it = 0;
        h_lo = 0.0;
        h_hi = h;
        const double hn = h * hermite_root(y[0], h * k[0][0], y5[0], h * k[6][0], b.omega_f);
        h = (hn > h_lo && hn < h_hi) ? hn : 0.5 * (h_lo + h_hi);
      } else {
        commit(h);
        for (int i = 0; i < 10; i++) k[0][i] = k[6][i];  // first same as last
        if (!p.fixed_step) {
          double fac = (err == 0.0) ? p.fac_max : p.safety * std::pow(err, -0.2);
          const double fmax = last_rejected ? 1.0 : p.fac_max;
          if (fac > fmax) fac = fmax;
          if (fac < p.fac_min) fac = p.fac_min;
          h = h * fac;
        }
        last_rejected = false;
      }
    } else {
      r.n_rej++;
      double fac = p.safety * std::pow(err, -0.2);
      if (fac > 1.0) fac = 1.0;
      if (fac < p.fac_min) fac = p.fac_min;
      h = h * fac;
      last_rejected = true;
      if (h < p.h_min) { r.status = ST_H_UNDERFLOW; break; }
    }
    if (attempts >= p.max_steps) { r.status = ST_MAX_STEPS; break; }
  }
  for (int i = 0; i < 10; i++) r.y[i] = y[i];
  r.t = t;
  return r;
}

// Output dot products of Sec. V: unit-vector products of the final state.
// A zero spin gives 0/0 = NaN, as the product is undefined there.
void dots(const double* y, double* d12, double* dl1, double* dl2) {
  const double* S1 = y + 1;
  const double* S2 = y + 4;
  const double* L = y + 7;
  const double n1 = std::sqrt(dot3(S1, S1)), n2 = std::sqrt(dot3(S2, S2)), nl = std::sqrt(dot3(L, L));
  *d12 = dot3(S1, S2) / (n1 * n2);
  *dl1 = dot3(L, S1) / (nl * n1);
  *dl2 = dot3(L, S2) / (nl * n2);
}

OBinary load(const OBatchIn& in, int64_t i) {
  OBinary b;
  b.m1 = in.m1[i]; b.m2 = in.m2[i]; b.chi1 = in.chi1[i]; b.chi2 = in.chi2[i];
  b.s1[0] = in.s1x[i]; b.s1[1] = in.s1y[i]; b.s1[2] = in.s1z[i];
  b.s2[0] = in.s2x[i]; b.s2[1] = in.s2y[i]; b.s2[2] = in.s2z[i];
  b.l0[0] = in.lx[i]; b.l0[1] = in.ly[i]; b.l0[2] = in.lz[i];
  b.omega0 = in.omega0[i]; b.omega_f = in.omega_f[i];
  return b;
}

void store(const OBatchOut& out, int64_t i, const OResult& r) {
  out.S1x[i] = r.y[1]; out.S1y[i] = r.y[2]; out.S1z[i] = r.y[3];
  out.S2x[i] = r.y[4]; out.S2y[i] = r.y[5]; out.S2z[i] = r.y[6];
  out.Lx[i] = r.y[7]; out.Ly[i] = r.y[8]; out.Lz[i] = r.y[9];
  out.omega[i] = r.y[0]; out.t[i] = r.t;
  out.n_acc[i] = r.n_acc; out.n_rej[i] = r.n_rej; out.n_land[i] = r.n_land; out.status[i] = r.status;
  dots(r.y, &out.dot_s1s2[i], &out.dot_ls1[i], &out.dot_ls2[i]);
}

// ----------------------------------------------------------------------------
// Replay with fixed steps and the implicit stop (used by the gradient and by
// the finite-difference check).
// ----------------------------------------------------------------------------

// Takes the recorded accepted steps hs[0..n-2] from the initial state, then
// lands on omega_f from the last state with a Newton iteration started at
// hs[n-1] and run to roundoff.  Returns false if the replay leaves the range.
bool replay_double(const OBinary& b, const OParams& p, const double* hs, int64_t n, double* yout,
                   double* tout) {
  const Coeffs<double> ms = make_coeffs(b.m1, b.m2, p);
  double y[10], k[7][10], y5[10];
  initial_state(b.m1, b.m2, b.chi1, b.chi2, b.s1, b.s2, b.l0, b.omega0, y);
  double t = 0.0;
  rhs(ms, p, y, k[0]);
  for (int64_t s = 0; s + 1 < n; s++) {
    dp5_attempt(ms, p, y, hs[s], k, y5);
    for (int i = 0; i < 10; i++) { y[i] = y5[i]; k[0][i] = k[6][i]; }
    t = t + hs[s];
  }
  double h = hs[n - 1];
  double best_g = INFINITY, best_h = h;
  double ybest[10];
  for (int it = 0; it < 60; it++) {
    dp5_attempt(ms, p, y, h, k, y5);
    const double g = y5[0] - b.omega_f;
    if (std::fabs(g) < best_g) {
      best_g = std::fabs(g);
      best_h = h;
      for (int i = 0; i < 10; i++) ybest[i] = y5[i];
    }
    if (g == 0.0) break;
    const double hn = h - g / k[6][0];
    if (hn == h) break;
    h = hn;
  }
  if (!std::isfinite(best_g)) return false;
  for (int i = 0; i < 10; i++) yout[i] = ybest[i];
  *tout = t + best_h;
  return true;
}

}  // namespace

// ============================================================================
// extern "C" entry points (ctypes).
// ============================================================================
extern "C" {

int oracle_abi_version() { return 3; }

// Dormand-Prince tableau as used here (for the order-condition tests).
void oracle_tableau(double* c7, double* a7x6, double* b7, double* bhat7) {
  for (int i = 0; i < 7; i++) {
    c7[i] = DP_C[i];
    b7[i] = DP_B[i];
    bhat7[i] = DP_BHAT[i];
    for (int j = 0; j < 6; j++) a7x6[i * 6 + j] = DP_A[i][j];
  }
}

// f(y) for one state.
void oracle_rhs(const OParams* p, double m1, double m2, const double* y, double* f) {
  const Coeffs<double> ms = make_coeffs(m1, m2, *p);
  rhs(ms, *p, y, f);
}

// One DP5 attempt on the PN system (returns y5 and the error norm).
double oracle_dp5_attempt(const OParams* p, double m1, double m2, const double* y, double h,
                          double* y5) {
  const Coeffs<double> ms = make_coeffs(m1, m2, *p);
  double k[7][10];
  rhs(ms, *p, y, k[0]);
  dp5_attempt(ms, *p, y, h, k, y5);
  return err_norm(*p, y, y5, h, k);
}

// Integrate n binaries on nthreads host threads (0 = all hardware threads).
// Returns the number of threads used.
int oracle_integrate_batch(int64_t n, const OBatchIn* in, const OParams* p, OBatchOut* out,
                           int nthreads) {
  if (nthreads <= 0) nthreads = (int)std::thread::hardware_concurrency();
  if (nthreads < 1) nthreads = 1;
  if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= n) break;
      const OResult r = integrate_one(load(*in, i), *p, nullptr, nullptr);
      store(*out, i, r);
    }
  };
  if (nthreads == 1) {
    work();
  } else {
    std::vector<std::thread> th;
    for (int k = 0; k < nthreads; k++) th.emplace_back(work);
    for (auto& x : th) x.join();
  }
  return nthreads;
}

// Integrate one binary and return the accepted trajectory: up to cap rows of
// (t, y[10]).  Returns the number of rows (may exceed cap; extra rows dropped).
int64_t oracle_trace(const OBatchIn* in, int64_t i, const OParams* p, double* rows, int64_t cap,
                     double* hs, int64_t hcap) {
  std::vector<double> tr, hv;
  integrate_one(load(*in, i), *p, &hv, &tr);
  const int64_t nr = (int64_t)tr.size() / 11;
  for (int64_t r = 0; r < nr && r < cap; r++)
    for (int c = 0; c < 11; c++) rows[r * 11 + c] = tr[r * 11 + c];
  for (int64_t s = 0; s < (int64_t)hv.size() && s < hcap; s++) hs[s] = hv[s];
  return nr;
}

// Replay binary i of a batch with the given accepted step sizes (last entry is
// the landing step, re-solved to roundoff) and return (y[10], t).
int oracle_replay(const OBatchIn* in, int64_t i, const OParams* p, const double* hs, int64_t n,
                  double* y_out, double* t_out) {
  return replay_double(load(*in, i), *p, hs, n, y_out, t_out) ? 0 : -1;
}

// Forward-mode gradient for binary i.  The accepted step sizes of the adaptive
// run are held fixed; the last (landing) step h* is the root of
// omega5(y_{n-1}, h*; theta) = omega_f, so dh*/dtheta = -(d omega5/d theta)/(d omega5/d h).
// Directions: 0..2 = S1-hat components, 3..5 = S2-hat components, 6 = q = m1/m2
// (M = 1 and chi_i fixed, so m1 = q/(1+q), m2 = 1/(1+q)).
// jac (13 x 7, row-major) = d(out)/d(theta) for
//   out = (dot_s1s2, dot_ls1, dot_ls2, Lx, Ly, Lz, S1x, S1y, S1z, S2x, S2y, S2z, t).
// Also returns the primal out[13].  Returns n_acc or a negative status.
int64_t oracle_grad(const OBatchIn* in, int64_t i, const OParams* p, double* out13, double* jac13x7) {
  const OBinary b = load(*in, i);
  std::vector<double> hs;
  const OResult r = integrate_one(b, *p, &hs, nullptr);
  if (r.status != ST_OK || p->stop_mode != 0) return -1;
  const int64_t n = (int64_t)hs.size();

  // Dual parameters.
  Dual s1[3], s2[3];
  for (int c = 0; c < 3; c++) {
    s1[c] = Dual(b.s1[c]); s1[c].d[c] = 1.0;
    s2[c] = Dual(b.s2[c]); s2[c].d[3 + c] = 1.0;
  }
  Dual m1(b.m1), m2(b.m2);
  m1.d[6] = b.m2 * b.m2;   // dm1/dq = 1/(1+q)^2 = m2^2
  m2.d[6] = -b.m2 * b.m2;  // dm2/dq = -1/(1+q)^2
  const Coeffs<Dual> ms = make_coeffs(m1, m2, *p);

  Dual y[10], k[7][10], y5[10];
  initial_state(m1, m2, b.chi1, b.chi2, s1, s2, b.l0, b.omega0, y);
  rhs(ms, *p, y, k[0]);
  double t = 0.0;
  for (int64_t s = 0; s + 1 < n; s++) {
    dp5_attempt(ms, *p, y, Dual(hs[s]), k, y5);
    for (int c = 0; c < 10; c++) { y[c] = y5[c]; k[0][c] = k[6][c]; }
    t = t + hs[s];
  }
  // Landing step with h as direction 7.
  Dual hd(hs[n - 1]);
  hd.d[7] = 1.0;
  dp5_attempt(ms, *p, y, hd, k, y5);
  const double domega_dh = y5[0].d[7];
  double dh_dth[7];
  for (int q = 0; q < 7; q++) dh_dth[q] = -y5[0].d[q] / domega_dh;
  Dual yf[10];
  for (int c = 0; c < 10; c++) {
    yf[c] = Dual(y5[c].v);
    for (int q = 0; q < 7; q++) yf[c].d[q] = y5[c].d[q] + y5[c].d[7] * dh_dth[q];
  }
  Dual tf(t + hs[n - 1]);
  for (int q = 0; q < 7; q++) tf.d[q] = dh_dth[q];

  // Outputs.
  const Dual* S1 = yf + 1;
  const Dual* S2 = yf + 4;
  const Dual* L = yf + 7;
  const Dual n1 = sqrt_(dot3(S1, S1)), n2 = sqrt_(dot3(S2, S2)), nl = sqrt_(dot3(L, L));
  Dual o[13];
  o[0] = dot3(S1, S2) / (n1 * n2);
  o[1] = dot3(L, S1) / (nl * n1);
  o[2] = dot3(L, S2) / (nl * n2);
  for (int c = 0; c < 3; c++) { o[3 + c] = L[c]; o[6 + c] = S1[c]; o[9 + c] = S2[c]; }
  o[12] = tf;
  for (int a = 0; a < 13; a++) {
    out13[a] = o[a].v;
    for (int q = 0; q < 7; q++) jac13x7[a * 7 + q] = o[a].d[q];
  }
  return n;
}

// Floating-point operation counts of one RHS evaluation and of one DP5
// attempt's own work (stages, error norm; RHS calls excluded), at state y.
// counts7 = (add, mul, div, sqrt, cbrt, log, pow); the attempt's pow is the
// controller's err^(-1/5).
void oracle_count_ops(const OParams* p, double m1, double m2, const double* y, int64_t* rhs7,
                      int64_t* step7) {
  const Coeffs<Cnt> ms = make_coeffs(Cnt(m1), Cnt(m2), *p);
  Cnt yc[10], f[10];
  for (int i = 0; i < 10; i++) yc[i] = Cnt(y[i]);
  g_ops = OpCount{0, 0, 0, 0, 0, 0, 0};
  rhs(ms, *p, yc, f);
  const OpCount r = g_ops;
  rhs7[0] = r.add; rhs7[1] = r.mul; rhs7[2] = r.div; rhs7[3] = r.sqrt;
  rhs7[4] = r.cbrt; rhs7[5] = r.log; rhs7[6] = 0;
  Cnt k[7][10], y5[10];
  rhs(ms, *p, yc, k[0]);
  g_ops = OpCount{0, 0, 0, 0, 0, 0, 0};
  dp5_attempt(ms, *p, yc, Cnt(10.0), k, y5);
  const OpCount a = g_ops;  // includes 6 RHS calls
  g_ops = OpCount{0, 0, 0, 0, 0, 0, 0};
  (void)err_norm(*p, yc, y5, Cnt(10.0), k);
  const OpCount e = g_ops;
  step7[0] = a.add - 6 * r.add + e.add;
  step7[1] = a.mul - 6 * r.mul + e.mul + 2;  // + the controller's safety * err^-0.2 and h * fac
  step7[2] = a.div - 6 * r.div + e.div;
  step7[3] = a.sqrt - 6 * r.sqrt + e.sqrt;
  step7[4] = a.cbrt - 6 * r.cbrt;
  step7[5] = a.log - 6 * r.log;
  step7[6] = 1;
}

// ----------------------------------------------------------------------------
// Initial-data sampler (Sec. V): SplitMix64 counter-based uniforms and
// Marsaglia's rejection method for isotropic directions.
// ----------------------------------------------------------------------------
struct ODist {
  int32_t q_mode;    // 0 fixed q_lo, 1 uniform [q_lo, q_hi], 2 log-uniform [q_lo, q_hi]
  int32_t chi_mode;  // 0 fixed chi_lo, 1 uniform [chi_lo, chi_hi]
  double q_lo, q_hi, chi_lo, chi_hi;
  double omega0_lo, omega0_hi;  // uniform; equal bounds give a fixed value
  double omega_f;
};

// SplitMix64 (Steele, Lea & Flood 2014): state advances by the golden gamma,
// output is the state passed through the variant-13 finaliser.
uint64_t oracle_splitmix64_next(uint64_t* state) {
  *state += 0x9e3779b97f4a7c15ull;
  uint64_t z = *state;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Draw j of binary i: binary i owns the SplitMix64 stream seeded with the
// i-th output (i counted from 0) of the stream seeded with `seed`; draw j is
// that stream's j-th output (from 0), as a 53-bit uniform in [0, 1).
double oracle_uniform(uint64_t seed, uint64_t i, uint64_t j) {
  uint64_t s = seed + i * 0x9e3779b97f4a7c15ull;
  const uint64_t key = oracle_splitmix64_next(&s);
  uint64_t s2 = key + j * 0x9e3779b97f4a7c15ull;
  const uint64_t z = oracle_splitmix64_next(&s2);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Draw slots: 0 q, 1 chi1, 2 chi2, 3 omega0, then pairs for Marsaglia's method
// (S1-hat first, S2-hat continuing from the next unused slot; at most 64 pairs each).
// Binary idx[k] of the draw (every binary's values depend only on the seed and
// its own index) written to position k; idx == nullptr means idx[k] = k.
void oracle_sample_at(uint64_t seed, const ODist* d, const int64_t* idx, int64_t n, double* m1, double* m2,
                      double* chi1, double* chi2, double* s1x, double* s1y, double* s1z, double* s2x, double* s2y,
                      double* s2z, double* lx, double* ly, double* lz, double* omega0, double* omega_f) {
  for (int64_t i = 0; i < n; i++) {
    const uint64_t ui = (uint64_t)(idx ? idx[i] : i);
    double q;
    const double u0 = oracle_uniform(seed, ui, 0);
    if (d->q_mode == 0) q = d->q_lo;
    else if (d->q_mode == 1) q = d->q_lo + (d->q_hi - d->q_lo) * u0;
    else q = d->q_lo * std::exp(u0 * std::log(d->q_hi / d->q_lo));
    m1[i] = q / (1.0 + q);
    m2[i] = 1.0 / (1.0 + q);
    const double u1 = oracle_uniform(seed, ui, 1), u2 = oracle_uniform(seed, ui, 2);
    chi1[i] = d->chi_mode == 0 ? d->chi_lo : d->chi_lo + (d->chi_hi - d->chi_lo) * u1;
    chi2[i] = d->chi_mode == 0 ? d->chi_lo : d->chi_lo + (d->chi_hi - d->chi_lo) * u2;
    const double u3 = oracle_uniform(seed, ui, 3);
    omega0[i] = d->omega0_lo + (d->omega0_hi - d->omega0_lo) * u3;
    omega_f[i] = d->omega_f;
    uint64_t j = 4;
    double* outs[2][3] = {{s1x, s1y, s1z}, {s2x, s2y, s2z}};
    for (int b = 0; b < 2; b++) {
      double v[3] = {0.0, 0.0, 1.0};
      for (int tries = 0; tries < 64; tries++) {
        const double x1 = 2.0 * oracle_uniform(seed, ui, j) - 1.0;
        const double x2 = 2.0 * oracle_uniform(seed, ui, j + 1) - 1.0;
        j += 2;
        const double s = x1 * x1 + x2 * x2;
        if (s >= 1.0) continue;
        const double r = std::sqrt(1.0 - s);
        v[0] = 2.0 * x1 * r;
        v[1] = 2.0 * x2 * r;
        v[2] = 1.0 - 2.0 * s;
        break;
      }
      outs[b][0][i] = v[0];
      outs[b][1][i] = v[1];
      outs[b][2][i] = v[2];
    }
    lx[i] = 0.0; ly[i] = 0.0; lz[i] = 1.0;
  }
}

void oracle_sample(uint64_t seed, const ODist* d, int64_t n, double* m1, double* m2, double* chi1,
                   double* chi2, double* s1x, double* s1y, double* s1z, double* s2x, double* s2y,
                   double* s2z, double* lx, double* ly, double* lz, double* omega0, double* omega_f) {
  oracle_sample_at(seed, d, nullptr, n, m1, m2, chi1, chi2, s1x, s1y, s1z, s2x, s2y, s2z, lx, ly, lz, omega0,
                   omega_f);
}

}  // extern "C"
