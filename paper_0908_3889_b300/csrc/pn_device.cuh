// pn_device.cuh -- device arithmetic of the batched PN inspiral integrator (sm_103a).
//
// One binary per lane, its state in registers.  The method is that of
// arXiv:0908.3889 Sec. II: Eqs. (1)-(4) integrated in t with the Dormand-Prince
// 5(4) pair (Dormand & Prince 1980), error tolerance 5e-7, first step h = 10,
// from omega_0 up to omega_f.
//
// B300 shapes this file: the FP64 pipe issues ~2 lanes/clk/SM (64x below FP32),
// and the CUDA FP64 cbrt / log / pow / divide cost roughly 17 / 37 / 100 / 8
// FMA-equivalents there.  So every FP64 instruction counts.  The inverse cube
// root, reciprocals and the step control's power are computed from FP32 seeds
// plus short FP64 corrections whose truncation error is below 1e-17 relative;
// the logarithm, which enters only P's v^6 term, keeps only k ln 2 and the
// final sum in FP64 and takes the rest in double-single on the FP32 pipe
// (within ~4e-15 absolute); comparisons, absolute values and maxima of doubles use integer
// instructions on the bit patterns; and in mixed precision the FP32<->FP64
// conversions are done with integer instructions, not the FP64 pipe.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pn {

// ---------------------------------------------------------------------------
// Bit-level helpers (integer pipe).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hi32(double d) { return (uint32_t)__double2hiint(d); }
__device__ __forceinline__ uint32_t lo32(double d) { return (uint32_t)__double2loint(d); }
__device__ __forceinline__ double mk64(uint32_t hi, uint32_t lo) { return __hiloint2double((int)hi, (int)lo); }
__device__ __forceinline__ double dnan() { return __longlong_as_double(0x7ff8000000000000ll); }

// |d| (clears the sign bit).
__device__ __forceinline__ double dabs(double d) { return mk64(hi32(d) & 0x7fffffffu, lo32(d)); }

// max(|a|, |b|) by integer comparison of the magnitudes' bit patterns (which
// order like the values for non-negative doubles; NaN sorts above Inf).
__device__ __forceinline__ double max_abs(double a, double b) {
  const unsigned long long x = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
  const unsigned long long y = (unsigned long long)__double_as_longlong(b) & 0x7fffffffffffffffull;
  return __longlong_as_double((long long)(x > y ? x : y));
}

// a <= b for a, b >= 0 (not NaN), by integer comparison.
__device__ __forceinline__ bool le_pos(double a, double b) {
  return (unsigned long long)__double_as_longlong(a) <= (unsigned long long)__double_as_longlong(b);
}

// True if d is finite (exponent field not all ones).
__device__ __forceinline__ bool finite64(double d) { return (hi32(d) & 0x7ff00000u) != 0x7ff00000u; }

// Seed conversion double -> float for positive normal d in [2^-126, 2^128):
// drops the exponent bias difference and keeps the top 23 fraction bits
// (truncation).  Two integer instructions.
__device__ __forceinline__ float seed_f32(double d) {
  return __uint_as_float(__funnelshift_l(lo32(d), hi32(d), 3) - (384u << 23));
}

// Exact conversion float -> double for positive normal f.
__device__ __forceinline__ double seed_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  return mk64((b >> 3) + (896u << 20), b << 29);
}

// double -> float rounded to nearest (ties away from zero), any sign;
// |d| < 2^-126 flushes to a signed zero, overflow gives Inf, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double d) {
  const uint32_t hi = hi32(d), lo = lo32(d);
  const uint32_t ahi = hi & 0x7fffffffu;
  uint32_t b = (__funnelshift_l(lo, ahi, 3) - (384u << 23)) + ((lo >> 28) & 1u);
  if (ahi < (897u << 20)) b = 0u;
  else if (ahi >= (1151u << 20)) b = (ahi > 0x7ff00000u || (ahi == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float(b | (hi & 0x80000000u));
}

// float -> double, exact for normal floats; subnormals flush to a signed zero;
// Inf and NaN are kept.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t a = b & 0x7fffffffu;
  uint32_t hi = (a >> 3) + (896u << 20);
  uint32_t lo = a << 29;
  if (a < 0x00800000u) { hi = 0u; lo = 0u; }
  else if (a >= 0x7f800000u) { hi = (a > 0x7f800000u) ? 0x7ff80000u : 0x7ff00000u; lo = 0u; }
  return mk64(hi | (b & 0x80000000u), lo);
}

// ---------------------------------------------------------------------------
// FP64 functions from FP32 seeds (each relative error below one ulp).
// ---------------------------------------------------------------------------

// x^(-1/3), odd in x, for |x| in [2^-126, 2^128).  Seed: FP32 rcbrtf of the
// truncated |x|.  One third-order step of the binomial series
// (1 - e)^(-1/3) = 1 + e/3 + 2e^2/9 + O(e^3), e = 1 - |x| r^3.
__device__ __forceinline__ double inv_cbrt(double x) {
  const uint32_t hx = hi32(x);
  const double ax = mk64(hx & 0x7fffffffu, lo32(x));
  double r = seed_f64(rcbrtf(seed_f32(ax)));
  const double r3 = (r * r) * r;
  const double e = fma(-ax, r3, 1.0);
  r = fma(r, e * fma(e, 2.0 / 9.0, 1.0 / 3.0), r);
  return mk64(hi32(r) | (hx & 0x80000000u), lo32(r));
}

// 1/x for positive normal x: FP32 reciprocal seed, then r (1 + e + e^2),
// e = 1 - x r (the series of 1/(1 - e)).
__device__ __forceinline__ double rcp_pos(double x) {
  const double r = seed_f64(__frcp_rn(seed_f32(x)));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// 1/x for positive normal x to within 3.3e-14 relative, for the error norm:
// FP32 reciprocal seed r (|e| <= 1.8e-7), then r (1 + e), e = 1 - x r.  The
// norm only feeds the accept test and the step-size factor, where a relative
// change of 1e-13 moves the next step size by ~1e-14 of itself.
__device__ __forceinline__ double rcp_norm(double x) {
  const double r = seed_f64(__frcp_rn(seed_f32(x)));
  return fma(r, fma(-x, r, 1.0), r);
}

// s^(-1/10) for s in [2^-126, 2^128): FP32 exp2/log2 seed, then
// z (1 + e/10 + 11 e^2/200), e = 1 - s z^10 (the series of (1 - e)^(-1/10)).
__device__ __forceinline__ double pow_m_tenth(double s) {
  double z = seed_f64(exp2f(-0.1f * log2f(seed_f32(s))));
  const double z2 = z * z;
  const double z4 = z2 * z2;
  const double z10 = (z4 * z4) * z2;
  const double e = fma(-s, z10, 1.0);
  return fma(z, e * fma(e, 11.0 / 200.0, 0.1), z);
}

// ---------------------------------------------------------------------------
// Per-binary coefficients of Eqs. (1) and (4) (M = m1 + m2 = 1, eta = m1 m2).
// ---------------------------------------------------------------------------
template <class R>
struct Coef {
  R K;             // (96/5) eta                     -- Eq. (1) prefactor
  R w1, w2;        // (113 m_i^2 + 75 eta) / (12 m_i^2): 1.5PN spin-orbit weight on L.S_i
  R tail;          // 4 pi                            -- 1.5PN tail
  R ss247, ss721;  // 247 eta / (48 m1^2 m2^2), 721 eta / (48 m1^2 m2^2): 2PN spin-spin
  R c1, c2, c25, c35;  // non-spin coefficients of x^{2/3}, x^{4/3}, x^{5/3}, x^{7/3}
  R c3l;           // 3PN non-log coefficient minus (856/105) ln 16
  R clog;          // -(856/105)(2/3): coefficient of ln(M omega) in the 3PN bracket
  R a1, a2;        // eta (4 + 3 m2/m1), eta (4 + 3 m1/m2)   -- Eq. (4)
  R prec;          // 1/2 (precession on) or 0
  R nie;           // -1/eta                                  -- Eq. (3)
};

struct TermCfg {
  uint32_t mask;
  int32_t theta_mode;
};

#define PN_PI 3.141592653589793
#define PN_EULER_GAMMA 0.5772156649015329

// Coefficients from the masses, in FP64 (once per binary).
__device__ __forceinline__ Coef<double> make_coef(double m1, double m2, TermCfg tc) {
  Coef<double> c;
  const double eta = m1 * m2;
  const double e2 = eta * eta;
  const double im1 = 1.0 / (m1 * m1), im2 = 1.0 / (m2 * m2);
  const uint32_t mk = tc.mask;
  c.K = (96.0 / 5.0) * eta;
  c.w1 = (mk & 2u) ? (113.0 * (m1 * m1) + 75.0 * eta) / 12.0 * im1 : 0.0;
  c.w2 = (mk & 2u) ? (113.0 * (m2 * m2) + 75.0 * eta) / 12.0 * im2 : 0.0;
  c.tail = (mk & 4u) ? 4.0 * PN_PI : 0.0;
  const double ss = (mk & 16u) ? eta / 48.0 * im1 * im2 : 0.0;
  c.ss247 = 247.0 * ss;
  c.ss721 = 721.0 * ss;
  c.c1 = (mk & 1u) ? -(743.0 + 924.0 * eta) / 336.0 : 0.0;
  c.c2 = (mk & 8u) ? 34103.0 / 18144.0 + 13661.0 / 2016.0 * eta + 59.0 / 18.0 * e2 : 0.0;
  c.c25 = (mk & 32u) ? -(4159.0 + 15876.0 * eta) * PN_PI / 672.0 : 0.0;
  // 3PN: theta-hat = 1039/4620 multiplies eta once (default) or eta^2 (as printed).
  const double theta = 1039.0 / 4620.0;
  const double th_eta = (tc.theta_mode == 0) ? theta : theta * eta;
  const double c3 = 16447322263.0 / 139708800.0 - 1712.0 / 105.0 * PN_EULER_GAMMA + 16.0 / 3.0 * PN_PI * PN_PI +
                    (-273811877.0 / 1088640.0 + 451.0 / 48.0 * PN_PI * PN_PI - 88.0 / 3.0 * th_eta) * eta +
                    541.0 / 896.0 * e2 - 5605.0 / 2592.0 * e2 * eta;
  c.c3l = (mk & 64u) ? c3 - 856.0 / 105.0 * (4.0 * 0.6931471805599453) : 0.0;
  c.clog = (mk & 64u) ? -1712.0 / 315.0 : 0.0;
  c.c35 = (mk & 128u) ? (-4415.0 / 4032.0 + 358675.0 / 6048.0 * eta + 91495.0 / 1512.0 * e2) * PN_PI : 0.0;
  c.a1 = eta * (4.0 + 3.0 * m2 / m1);
  c.a2 = eta * (4.0 + 3.0 * m1 / m2);
  c.prec = (mk & 256u) ? 0.5 : 0.0;
  c.nie = -1.0 / eta;
  return c;
}

// The coefficients of P multiplied by the prefactor K = (96/5) eta, once per
// binary: P_K = K + v^2 (K c1 - K so v + ...), so the right-hand side skips one
// FP64 multiplication (rhs64).  K itself stays as P_K's constant term.
__device__ __forceinline__ Coef<double> fold_K(const Coef<double>& c) {
  Coef<double> f = c;
  f.w1 = c.K * c.w1;
  f.w2 = c.K * c.w2;
  f.tail = c.K * c.tail;
  f.ss247 = c.K * c.ss247;
  f.ss721 = c.K * c.ss721;
  f.c1 = c.K * c.c1;
  f.c2 = c.K * c.c2;
  f.c25 = c.K * c.c25;
  f.c35 = c.K * c.c35;
  f.c3l = c.K * c.c3l;
  f.clog = c.K * c.clog;
  return f;
}

// prec * x for prec in {0, 1/2} (the precession switch of make_coef) and x = w^2,
// with no FP64 instruction.  Where rhs64's r = w^{-1/3} is a number, x lies in
// [2^-252, 2^256): normal, so halving is the exponent minus one, exact.  Outside
// that range every rate that takes this factor is NaN through r, whatever it is.
__device__ __forceinline__ double half_or_zero(double prec, double x) {
  return (hi32(prec) & 0x7fffffffu) == 0u ? 0.0 : mk64(hi32(x) - (1u << 20), lo32(x));
}

// The FP32 coefficients, rounded with the same integer conversion the kernels use.
__device__ __forceinline__ Coef<float> to_f32(const Coef<double>& c) {
  Coef<float> f;
  const double* s = &c.K;
  float* d = &f.K;
#pragma unroll
  for (int k = 0; k < 16; k++) d[k] = f64_to_f32(s[k]);
  return f;
}

__device__ __forceinline__ double log_w(double x, const float* __restrict__ tabf);

// ---------------------------------------------------------------------------
// Right-hand side f(y), y = (omega, S1, S2, L), M = 1, x = omega, v = x^{1/3}.
//   Eq. (1): domega/dt = (96/5) eta omega^2 v^5 P, P = 1 + c1 v^2 - SO v^3
//            + (c2 - SS) v^4 + c25 v^5 + (c3 - 856/105 ln(16 v^2)) v^6 + c35 v^7,
//            SO = sum_i chi_i L.S_i-hat (113 m_i^2 + 75 eta)/12 - 4 pi,
//            SS = eta chi1 chi2 (247 S1-hat.S2-hat - 721 L.S1-hat L.S2-hat)/48,
//            with chi_i S_i-hat = S_i / m_i^2.
//   Eq. (4): Omega_1 = (x^2/2) [eta v^{-1} (4 + 3 m2/m1) L + S2 - 3 (S2.L) L], 1<->2.
//   Eq. (2): dS_i/dt = Omega_i x S_i.   Eq. (3): dL/dt = -(v/eta)(dS1/dt + dS2/dt).
// With a_i = eta (4 + 3 m_j/m_i) and q_i = a_i/v - 3 L.S_j (j the other body):
//   Omega_i = (x^2/2) U_i,  U_i = q_i L + S_j,  dS_i/dt = (x^2/2) (U_i x S_i).
// ---------------------------------------------------------------------------
// c holds the coefficients of P with the prefactor K folded in (fold_K), so that
// omega-dot = omega^2 v^5 P_K with P_K = K P.
//
// keep(k, x) receives the intermediate values the adjoint's reverse sweep
// needs (indices below), in the order they are formed; the integration kernels
// pass NoKeep, which compiles to nothing.
enum KeepIdx {
  KP_R, KP_V, KP_V2, KP_LW, KP_LS1, KP_LS2, KP_S12, KP_P6, KP_P5, KP_P4, KP_P3, KP_P2, KP_P, KP_W2, KP_Q,
  KP_Q1, KP_Q2, KP_U1, KP_U2 = KP_U1 + 3, KP_PRE = KP_U2 + 3, KP_X1, KP_X2 = KP_X1 + 3, KP_LF = KP_X2 + 3,
  KP_F, KP_COUNT = KP_F + 10  // KP_F..: the rates f themselves
};
struct NoKeep {
  __device__ __forceinline__ void operator()(int, double) const {}
};
template <class Keep = NoKeep>
__device__ __forceinline__ void rhs64(const Coef<double>& c,
                                      const float* __restrict__ tabf, const double* y, double* f,
                                      Keep keep = Keep()) {
  const double w = y[0];
  const double S1x = y[1], S1y = y[2], S1z = y[3];
  const double S2x = y[4], S2y = y[5], S2z = y[6];
  const double Lx = y[7], Ly = y[8], Lz = y[9];

  // r = w^{-1/3}, v = w^{1/3}; |w| outside [2^-126, 2^128) (incl. 0, Inf, NaN) gives NaN.
  double r = inv_cbrt(w);
  if ((hi32(w) & 0x7fffffffu) - (897u << 20) >= ((1151u - 897u) << 20)) r = dnan();
  const double v = w * (r * r);
  const double v2 = v * v;
  const double lw = log_w(w, tabf);

  const double LS1 = fma(Lz, S1z, fma(Ly, S1y, Lx * S1x));
  const double LS2 = fma(Lz, S2z, fma(Ly, S2y, Lx * S2x));
  const double S12 = fma(S1z, S2z, fma(S1y, S2y, S1x * S2x));

  const double so = fma(c.w1, LS1, fma(c.w2, LS2, -c.tail));
  const double c2p = fma(c.ss721, LS1 * LS2, fma(-c.ss247, S12, c.c2));
  const double c3p = fma(c.clog, lw, c.c3l);
  const double P6 = fma(v, c.c35, c3p);
  const double P5 = fma(v, P6, c.c25);
  const double P4 = fma(v, P5, c2p);
  const double P3 = fma(v, P4, -so);
  const double P2 = fma(v, P3, c.c1);
  const double w2 = w * w;
  const double P = fma(v2, P2, c.K);
  const double Q = (w2 * w) * v2;
  f[0] = Q * P;

  // Eq. (4) as Omega_i = pre U_i with U_1 = q1 L + S2, q1 = a1/v - 3 L.S2 (1 <-> 2),
  // and dS_i/dt = pre (U_i x S_i): 29 FP64 operations for both spins.
  const double q1 = fma(c.a1, r, -3.0 * LS2);
  const double q2 = fma(c.a2, r, -3.0 * LS1);
  const double U1x = fma(q1, Lx, S2x), U1y = fma(q1, Ly, S2y), U1z = fma(q1, Lz, S2z);
  const double U2x = fma(q2, Lx, S1x), U2y = fma(q2, Ly, S1y), U2z = fma(q2, Lz, S1z);
  const double pre = half_or_zero(c.prec, w2);
  const double X1x = fma(U1y, S1z, -U1z * S1y), X1y = fma(U1z, S1x, -U1x * S1z), X1z = fma(U1x, S1y, -U1y * S1x);
  const double X2x = fma(U2y, S2z, -U2z * S2y), X2y = fma(U2z, S2x, -U2x * S2z), X2z = fma(U2x, S2y, -U2y * S2x);
  const double d1x = pre * X1x, d1y = pre * X1y, d1z = pre * X1z;
  const double d2x = pre * X2x, d2y = pre * X2y, d2z = pre * X2z;
  f[1] = d1x; f[2] = d1y; f[3] = d1z;
  f[4] = d2x; f[5] = d2y; f[6] = d2z;
  const double lf = v * c.nie;
  f[7] = lf * (d1x + d2x);
  f[8] = lf * (d1y + d2y);
  f[9] = lf * (d1z + d2z);

  keep(KP_R, r); keep(KP_V, v); keep(KP_V2, v2); keep(KP_LW, lw);
  keep(KP_LS1, LS1); keep(KP_LS2, LS2); keep(KP_S12, S12);
  keep(KP_P6, P6); keep(KP_P5, P5); keep(KP_P4, P4); keep(KP_P3, P3); keep(KP_P2, P2); keep(KP_P, P);
  keep(KP_W2, w2); keep(KP_Q, Q); keep(KP_Q1, q1); keep(KP_Q2, q2);
  keep(KP_U1, U1x); keep(KP_U1 + 1, U1y); keep(KP_U1 + 2, U1z);
  keep(KP_U2, U2x); keep(KP_U2 + 1, U2y); keep(KP_U2 + 2, U2z);
  keep(KP_PRE, pre);
  keep(KP_X1, X1x); keep(KP_X1 + 1, X1y); keep(KP_X1 + 2, X1z);
  keep(KP_X2, X2x); keep(KP_X2 + 1, X2y); keep(KP_X2 + 2, X2z);
  keep(KP_LF, lf);
#pragma unroll
  for (int k = 0; k < 10; k++) keep(KP_F + k, f[k]);
}

// x^(-1/3) to ~5e-7 relative from the special function unit's approximate
// base-2 logarithm and exponential (two instructions), odd in x.
__device__ __forceinline__ float rcbrt_sfu(float x) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(fabsf(x)));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-0.333333343f * l));
  return copysignf(r, x);
}
// x^(-1/3) in FP32 to about an ulp: the SFU seed and one Newton step r (1 + (1 - x r^3)/3).
__device__ __forceinline__ float rcbrt_f32(float x) {
  const float r0 = rcbrt_sfu(x);
  return __fmaf_rn(r0, (1.0f / 3.0f) * __fmaf_rn(-x, (r0 * r0) * r0, 1.0f), r0);
}

// The same right-hand side in FP32 (mixed precision).  r = w^(-1/3) is the
// special-function seed refined by one Newton step (about an FP32 ulp), and
// ln w the fast approximate logarithm: ln w enters only P's v^6 term, through
// the coefficient 1712/315, so an absolute error of a few 1e-7 in it moves P by
// under 1e-8 of itself, below the FP32 rounding of the rates.  (Both replace
// the library rcbrtf and logf: 119 -> 127 M inspirals/s with the approximate
// division of the error norm below; the FP32 form's error against FP64 keeps
// its statistics.)
__device__ __forceinline__ void rhs32(const Coef<float>& c, const float* y, float* f) {
  const float w = y[0];
  const float S1x = y[1], S1y = y[2], S1z = y[3];
  const float S2x = y[4], S2y = y[5], S2z = y[6];
  const float Lx = y[7], Ly = y[8], Lz = y[9];
  const float r = rcbrt_f32(w);
  const float v = w * (r * r);
  const float v2 = v * v;
  const float lw = __logf(fabsf(w));
  const float LS1 = fmaf(Lz, S1z, fmaf(Ly, S1y, Lx * S1x));
  const float LS2 = fmaf(Lz, S2z, fmaf(Ly, S2y, Lx * S2x));
  const float S12 = fmaf(S1z, S2z, fmaf(S1y, S2y, S1x * S2x));
  const float so = fmaf(c.w1, LS1, fmaf(c.w2, LS2, -c.tail));
  const float c2p = fmaf(c.ss721, LS1 * LS2, fmaf(-c.ss247, S12, c.c2));
  const float c3p = fmaf(c.clog, lw, c.c3l);
  float P = fmaf(v, c.c35, c3p);
  P = fmaf(v, P, c.c25);
  P = fmaf(v, P, c2p);
  P = fmaf(v, P, -so);
  P = fmaf(v, P, c.c1);
  P = fmaf(v2, P, 1.0f);
  const float w2 = w * w;
  f[0] = (((w2 * w) * v2) * c.K) * P;
  // Eq. (4) as in rhs64: dS_i/dt = pre (U_i x S_i), U_1 = q1 L + S2, q1 = a1/v - 3 L.S2.
  const float q1 = fmaf(c.a1, r, -3.0f * LS2);
  const float q2 = fmaf(c.a2, r, -3.0f * LS1);
  const float U1x = fmaf(q1, Lx, S2x), U1y = fmaf(q1, Ly, S2y), U1z = fmaf(q1, Lz, S2z);
  const float U2x = fmaf(q2, Lx, S1x), U2y = fmaf(q2, Ly, S1y), U2z = fmaf(q2, Lz, S1z);
  const float pre = c.prec * w2;
  const float d1x = pre * fmaf(U1y, S1z, -U1z * S1y), d1y = pre * fmaf(U1z, S1x, -U1x * S1z),
              d1z = pre * fmaf(U1x, S1y, -U1y * S1x);
  const float d2x = pre * fmaf(U2y, S2z, -U2z * S2y), d2y = pre * fmaf(U2z, S2x, -U2x * S2z),
              d2z = pre * fmaf(U2x, S2y, -U2y * S2x);
  f[1] = d1x; f[2] = d1y; f[3] = d1z;
  f[4] = d2x; f[5] = d2y; f[6] = d2z;
  const float lf = v * c.nie;
  f[7] = lf * (d1x + d2x);
  f[8] = lf * (d1y + d2y);
  f[9] = lf * (d1z + d2z);
}

// ---------------------------------------------------------------------------
// Double-single ("pair of FP32") arithmetic for the PN_MIXED_DS right-hand
// side: a value is hi + lo with |lo| <= ulp(hi)/2, about 48 significand bits.
// Error-free transformations: Knuth's two-sum and Dekker's fast two-sum for
// addition, the FMA-based exact product for multiplication; the
// double-single add and multiply follow the usual pair-arithmetic recipes
// (Dekker 1971; Bailey's DSFUN).  Every operation is an explicitly rounded
// FP32 instruction (no reassociation or contraction) on the FP32 pipe, which
// on B300 has 64x the FP64 pipe's throughput.
// ---------------------------------------------------------------------------
struct ds {
  float hi, lo;
};

__device__ __forceinline__ ds ds_of(float h) { return ds{h, 0.0f}; }
// s + e = a + b exactly, given |a| >= |b| or a == 0.
__device__ __forceinline__ ds fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ds{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// s + e = a + b exactly.
__device__ __forceinline__ ds two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return ds{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
// p + e = a * b exactly.
__device__ __forceinline__ ds two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ds{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ds ds_add(ds a, ds b) {
  const ds s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ds ds_neg(ds a) { return ds{-a.hi, -a.lo}; }
__device__ __forceinline__ ds ds_sub(ds a, ds b) { return ds_add(a, ds_neg(b)); }
__device__ __forceinline__ ds ds_mul(ds a, ds b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ds ds_mul_f(ds a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}
// a b + c: the product's exact leading part p = a.hi b.hi joins c through
// two-sum, and its rounding and cross terms go straight into the low part
// (no separate normalisation of the product).
__device__ __forceinline__ ds ds_fma(ds a, ds b, ds c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const ds s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
// a0 b0 + a1 b1 + a2 b2 in the same way: leading products summed by two-sum,
// every rounding error and cross term collected in one FP32 correction.
__device__ __forceinline__ ds ds_dot3(ds a0, ds b0, ds a1, ds b1, ds a2, ds b2) {
  const float p0 = __fmul_rn(a0.hi, b0.hi), p1 = __fmul_rn(a1.hi, b1.hi), p2 = __fmul_rn(a2.hi, b2.hi);
  float e = __fmaf_rn(a0.hi, b0.hi, -p0);
  e = __fmaf_rn(a0.hi, b0.lo, e);
  e = __fmaf_rn(a0.lo, b0.hi, e);
  e = __fadd_rn(e, __fmaf_rn(a1.hi, b1.hi, -p1));
  e = __fmaf_rn(a1.hi, b1.lo, e);
  e = __fmaf_rn(a1.lo, b1.hi, e);
  e = __fadd_rn(e, __fmaf_rn(a2.hi, b2.hi, -p2));
  e = __fmaf_rn(a2.hi, b2.lo, e);
  e = __fmaf_rn(a2.lo, b2.hi, e);
  const ds s = two_sum(p0, p1);
  const ds t = two_sum(s.hi, p2);
  return fast_two_sum(t.hi, __fadd_rn(e, __fadd_rn(s.lo, t.lo)));
}
// a b - c d (one component of a cross product).
__device__ __forceinline__ ds ds_diff_prod(ds a, ds b, ds c, ds d) {
  const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float f = __fmaf_rn(c.hi, d.hi, -q);
  f = __fmaf_rn(c.hi, d.lo, f);
  f = __fmaf_rn(c.lo, d.hi, f);
  const ds s = two_sum(p, -q);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(e, f)));
}
// Exact scaling by a power of two given as a float.
__device__ __forceinline__ ds ds_scale(ds a, float p2) { return ds{a.hi * p2, a.lo * p2}; }

// Lazy forms of the products: the same arithmetic as ds_mul / ds_mul_f without
// the final renormalization of the result (fast_two_sum), so lo may reach a few
// ulp of hi instead of half an ulp.  The pair still carries the product to
// ~2^-46 and every later operation takes both parts; a product cannot cancel, so
// lo stays within a few ulp of hi.  Three dependent FP32 operations per product
// leave the critical path of the double-single right-hand side.  The sum-type
// operations (ds_add, ds_fma, ds_dot3, ds_diff_prod) keep their
// renormalization: after a cancellation an unnormalized result would carry a
// low part as large as its high part into the next product, which drops lo*lo
// (lazy sums were measured to raise the right-hand side's error ~6x, and lazy
// plain additions to change step decisions).
__device__ __forceinline__ ds ds_mul_l(ds a, ds b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ds{p, e};
}
__device__ __forceinline__ ds ds_mul_f_l(ds a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return ds{p, e};
}

// double -> double-single: hi is d rounded to FP32 (f64_to_f32); the residual
// d - hi is the low 29 significand bits of d (minus 2^29 when hi was rounded
// up), an integer R with |R| <= 2^28, so lo = R * 2^(E - 1075) rounded to FP32.
// Integer and FP32 instructions only.  For |d| outside [2^-74, 2^180) lo is 0.
__device__ __forceinline__ ds split64(double d) {
  const float hi = f64_to_f32(d);
  const uint32_t lw = lo32(d), hw = hi32(d);
  const uint32_t E = (hw >> 20) & 0x7ffu;
  const int32_t R = ((int32_t)(lw << 3)) >> 3;
  float lo = __fmul_rn(__int2float_rn(R), __uint_as_float((E - 948u) << 23));
  lo = __uint_as_float(__float_as_uint(lo) ^ (hw & 0x80000000u));
  if (E - 949u > 253u) lo = 0.0f;
  return ds{hi, lo};
}

// double-single -> double (exact sum of the two parts).
__device__ __forceinline__ double ds_to_f64(ds a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }

// An int k, |k| < 2^31, as a double, exactly, by integer operations (no FP64
// instruction): the leading bit of |k| becomes the implicit one.
__device__ __forceinline__ double i32_to_f64(int k) {
  if (k == 0) return 0.0;
  const uint32_t a = (k < 0) ? (uint32_t)(-k) : (uint32_t)k;
  const int e = 31 - __clz(a);  // a in [2^e, 2^(e+1))
  const uint32_t n = a << (31 - e);  // leading bit at bit 31
  return mk64(((uint32_t)(1023 + e) << 20) | ((n >> 11) & 0x000fffffu) | ((uint32_t)k & 0x80000000u), n << 21);
}

// ln|x| for the FP64 right-hand side, for |x| in the normal double range, by
// Tang's table-driven reduction (P. T. P. Tang, ACM TOMS 16, 1990): |x| = 2^k m
// with m in [1, 2), F = 1 + (2j+1)/256 where j is the top 7 bits of m's
// fraction, so f = m - F is exact and |f| <= 2^-8; then
// ln|x| = k ln2 + (ln F + ln(1 + u)), u = f/F.  Only k ln2 and the final sum
// are FP64 (one FMA with the double nearest ln 2, and the conversion of the
// bracket to a double: two FP64 instructions; an all-FP64 evaluation with the
// series to u^6 takes thirteen).  The bracket is formed in double-single on
// the FP32 pipe: f from the significand bits by integer operations (exact),
// u, u^2/2 and u^3/3 as pairs, u^4 (-1/4 + u/5 - u^2/6) in FP32 (below 1.1e-10,
// so its rounding is under 1e-16 of it), truncation u^7/7 < 2.4e-18, and
// ln F_j as a pair.  The bracket (|.| < 0.7) is then within ~3e-15 absolute,
// and ln|x| within ~4e-15 absolute for x in [0.003, 0.2].  The right-hand side
// takes the logarithm only in the v^6 term of P, with the coefficient 1712/315,
// so this moves P by under 1e-16 of itself for v < 0.6.
// tabf[4j..4j+3] = 1/F_j (hi, lo), ln F_j (hi, lo) (computed on the host in
// extended precision).
__device__ __forceinline__ double log_w(double x, const float* __restrict__ tabf) {
  const uint32_t hx = hi32(x) & 0x7fffffffu;
  const int k = (int)(hx >> 20) - 1023;
  const uint32_t j = (hx >> 13) & 127u;
  // f = m - F_j in units of 2^-52: m's 52 fraction bits minus F_j's, |D| <= 2^44,
  // split into a high part of 24 bits and a low part of 21 bits (both exact floats).
  const int64_t D = (int64_t)((((uint64_t)(hx & 0x000fffffu)) << 32) | lo32(x)) - ((int64_t)(2u * j + 1u) << 44);
  const float fh = __fmul_rn(__int2float_rn((int)(D >> 21)), 4.656612873077393e-10f);  // 2^-31
  const float fl = __fmul_rn(__int2float_rn((int)(D & 0x1fffff)), 2.220446049250313e-16f);  // 2^-52
  const ds u = ds_mul(two_sum(fh, fl), ds{tabf[4 * j], tabf[4 * j + 1]});
  const ds u2 = ds_mul(u, u);
  const ds t3 = ds_mul(ds_mul(u2, u), ds{(float)(1.0 / 3.0), (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0))});
  const float uh = u.hi;
  float q = __fmaf_rn(uh, -1.0f / 6.0f, 0.2f);
  q = __fmaf_rn(q, uh, -0.25f);
  const float t4 = __fmul_rn(__fmul_rn(u2.hi, u2.hi), q);
  const ds rem = ds_add(u, ds_add(ds_scale(u2, -0.5f), ds_add(t3, ds_of(t4))));
  const ds br = ds_add(ds{tabf[4 * j + 2], tabf[4 * j + 3]}, rem);
  return fma(i32_to_f64(k), 0.6931471805599453, ds_to_f64(br));
}

// x^(-1/3) in double-single: FP32 seed r0 = rcbrtf(hi), then
// r0 (1 + e/3 + 2e^2/9) with e = 1 - x r0^3 formed in double-single.
__device__ __forceinline__ ds ds_inv_cbrt(ds x) {
  const float r0 = rcbrtf(x.hi);
  const ds r3 = ds_mul_f_l(two_prod(r0, r0), r0);
  const ds e = ds_sub(ds_of(1.0f), ds_mul_l(x, r3));
  const float t = __fmul_rn(e.hi, __fmaf_rn(e.hi, 2.0f / 9.0f, 1.0f / 3.0f));
  return two_sum(r0, __fmul_rn(r0, t));
}

// ln(2) = PN_LN2F_1 + PN_LN2F_2 + PN_LN2F_3 (16, 24, 24 significant bits), so
// k * PN_LN2F_1 is exact in FP32 for |k| < 256.
#define PN_LN2F_1 0.693145751953125f
#define PN_LN2F_2 1.428606765330187e-06f
#define PN_LN2F_3 5.497923148104107e-14f

// ln|x| in double-single by Tang's table method on the FP32 high part:
// |x| = 2^k m, F = 1 + (2j+1)/256 with j the top 7 fraction bits of m,
// u = (m - F + lo/2^k) / F (|u| < 2^-8), ln(1 + u) = u - u^2/2 (double-single)
// + u^3 (1/3 - u/4 + u^2/5 - u^3/6) (FP32), and ln|x| = k ln2 + ln F + ln(1 + u).
// tabf[4j..4j+3] = 1/F_j (hi, lo), ln F_j (hi, lo).  |x| must be a normal FP32 value.
__device__ __forceinline__ ds ds_log(ds x, const float* __restrict__ tabf) {
  const bool neg = x.hi < 0.0f;
  const float h = neg ? -x.hi : x.hi, l = neg ? -x.lo : x.lo;
  const uint32_t hb = __float_as_uint(h);
  const int k = (int)(hb >> 23) - 127;
  const uint32_t j = (hb >> 16) & 127u;
  const float m = __uint_as_float((hb & 0x007fffffu) | 0x3f800000u);
  const float F = __uint_as_float(0x3f800000u | ((2u * j + 1u) << 15));
  const float l_scaled = __fmul_rn(l, __uint_as_float((uint32_t)(127 - k) << 23));
  const ds f = two_sum(__fsub_rn(m, F), l_scaled);
  const ds u = ds_mul_l(f, ds{tabf[4 * j], tabf[4 * j + 1]});
  const ds u2h = ds_scale(ds_mul_l(u, u), -0.5f);
  const float uh = u.hi;
  float q = __fmaf_rn(uh, -1.0f / 6.0f, 0.2f);
  q = __fmaf_rn(q, uh, -0.25f);
  q = __fmaf_rn(q, uh, 1.0f / 3.0f);
  const float tail = __fmul_rn(__fmul_rn(__fmul_rn(uh, uh), uh), q);
  const ds ln1pu = ds_add(ds_add(u, u2h), ds_of(tail));
  const float kf = (float)k;
  ds kl = ds_add(ds_of(__fmul_rn(kf, PN_LN2F_1)), two_prod(kf, PN_LN2F_2));
  kl = ds_add(kl, ds_of(__fmul_rn(kf, PN_LN2F_3)));
  return ds_add(ds_add(kl, ds{tabf[4 * j + 2], tabf[4 * j + 3]}), ln1pu);
}

// The right-hand side of Eqs. (1)-(4) in double-single arithmetic, the same
// formulation as rhs64, with the lazy products (ds_mul_l).  |omega| outside
// the FP32 normal range gives NaN.
__device__ __forceinline__ void rhs_ds(const Coef<ds>& c, const float* __restrict__ tabf, const ds* y, ds* f) {
  const ds w = y[0];
  const ds S1x = y[1], S1y = y[2], S1z = y[3];
  const ds S2x = y[4], S2y = y[5], S2z = y[6];
  const ds Lx = y[7], Ly = y[8], Lz = y[9];
  ds r = ds_inv_cbrt(w);
  if ((__float_as_uint(w.hi) & 0x7fffffffu) - 0x00800000u >= 0x7f000000u) r = ds{__int_as_float(0x7fc00000), 0.0f};
  const ds v = ds_mul_l(w, ds_mul_l(r, r));
  const ds v2 = ds_mul_l(v, v);
  const ds lw = ds_log(w, tabf);
  const ds LS1 = ds_dot3(Lx, S1x, Ly, S1y, Lz, S1z);
  const ds LS2 = ds_dot3(Lx, S2x, Ly, S2y, Lz, S2z);
  const ds S12 = ds_dot3(S1x, S2x, S1y, S2y, S1z, S2z);
  const ds so = ds_fma(c.w1, LS1, ds_fma(c.w2, LS2, ds_neg(c.tail)));
  const ds c2p = ds_fma(c.ss721, ds_mul_l(LS1, LS2), ds_fma(ds_neg(c.ss247), S12, c.c2));
  const ds c3p = ds_fma(c.clog, lw, c.c3l);
  ds P = ds_fma(v, c.c35, c3p);
  P = ds_fma(v, P, c.c25);
  P = ds_fma(v, P, c2p);
  P = ds_fma(v, P, ds_neg(so));
  P = ds_fma(v, P, c.c1);
  P = ds_fma(v2, P, ds_of(1.0f));
  const ds w2 = ds_mul_l(w, w);
  f[0] = ds_mul_l(ds_mul_l(ds_mul_l(ds_mul_l(w2, w), v2), c.K), P);
  // Eq. (4) as in rhs64: dS_i/dt = pre (U_i x S_i), U_1 = q1 L + S2, q1 = a1/v - 3 L.S2.
  const ds q1 = ds_fma(c.a1, r, ds_mul_f_l(LS2, -3.0f));
  const ds q2 = ds_fma(c.a2, r, ds_mul_f_l(LS1, -3.0f));
  const ds U1x = ds_fma(q1, Lx, S2x), U1y = ds_fma(q1, Ly, S2y), U1z = ds_fma(q1, Lz, S2z);
  const ds U2x = ds_fma(q2, Lx, S1x), U2y = ds_fma(q2, Ly, S1y), U2z = ds_fma(q2, Lz, S1z);
  const ds pre = ds_mul_l(c.prec, w2);
  const ds d1x = ds_mul_l(pre, ds_diff_prod(U1y, S1z, U1z, S1y));
  const ds d1y = ds_mul_l(pre, ds_diff_prod(U1z, S1x, U1x, S1z));
  const ds d1z = ds_mul_l(pre, ds_diff_prod(U1x, S1y, U1y, S1x));
  const ds d2x = ds_mul_l(pre, ds_diff_prod(U2y, S2z, U2z, S2y));
  const ds d2y = ds_mul_l(pre, ds_diff_prod(U2z, S2x, U2x, S2z));
  const ds d2z = ds_mul_l(pre, ds_diff_prod(U2x, S2y, U2y, S2x));
  f[1] = d1x; f[2] = d1y; f[3] = d1z;
  f[4] = d2x; f[5] = d2y; f[6] = d2z;
  const ds lf = ds_mul_l(v, c.nie);
  f[7] = ds_mul_l(lf, ds_add(d1x, d2x));
  f[8] = ds_mul_l(lf, ds_add(d1y, d2y));
  f[9] = ds_mul_l(lf, ds_add(d1z, d2z));
}

__device__ __forceinline__ Coef<ds> to_ds(const Coef<double>& c) {
  Coef<ds> r;
  const double* s = &c.K;
  ds* d = &r.K;
#pragma unroll
  for (int k = 0; k < 16; k++) d[k] = split64(s[k]);
  return r;
}

// Coefficients in the precisions the kernels use, and the two logarithm tables.
struct Coefs {
  Coef<double> c64;
  Coef<float> c32;
  Coef<ds> cds;
};
struct Tabs {
  const float* f;  // 512 floats: 1/F_j, ln F_j as FP32 pairs (ds_log, log_w)
};

// ---------------------------------------------------------------------------
// Dormand & Prince (1980) RK5(4)7M coefficients (published table).
// ---------------------------------------------------------------------------
#define DP_A21 (1.0 / 5.0)
#define DP_A31 (3.0 / 40.0)
#define DP_A32 (9.0 / 40.0)
#define DP_A41 (44.0 / 45.0)
#define DP_A42 (-56.0 / 15.0)
#define DP_A43 (32.0 / 9.0)
#define DP_A51 (19372.0 / 6561.0)
#define DP_A52 (-25360.0 / 2187.0)
#define DP_A53 (64448.0 / 6561.0)
#define DP_A54 (-212.0 / 729.0)
#define DP_A61 (9017.0 / 3168.0)
#define DP_A62 (-355.0 / 33.0)
#define DP_A63 (46732.0 / 5247.0)
#define DP_A64 (49.0 / 176.0)
#define DP_A65 (-5103.0 / 18656.0)
#define DP_B1 (35.0 / 384.0)
#define DP_B3 (500.0 / 1113.0)
#define DP_B4 (125.0 / 192.0)
#define DP_B5 (-2187.0 / 6784.0)
#define DP_B6 (11.0 / 84.0)
// b - bhat (5th minus embedded 4th order weights), exact rationals
#define DP_E1 (71.0 / 57600.0)
#define DP_E3 (-71.0 / 16695.0)
#define DP_E4 (71.0 / 1920.0)
#define DP_E5 (-17253.0 / 339200.0)
#define DP_E6 (22.0 / 525.0)
#define DP_E7 (-1.0 / 40.0)

// Step-control and stop parameters as the kernels use them.
struct Ctl {
  double rtol, atol, h0, safety, fac_min, fac_max, h_min, land_tol;
  double s_lo;  // (safety/fac_max)^10: at or below it the growth factor is fac_max
  double s_hi;  // (safety/fac_min)^10: at or above it the factor is fac_min
  int32_t max_steps, land_max_iter, stop_mode, fixed_step;
  TermCfg terms;
  int32_t pad_;
};

// k = f(y) in the kernel's precision: PREC 0 FP64; 1 FP32 (state rounded to
// FP32 on the way in, rates widened on the way out); 2 double-single (state
// split into FP32 pairs, rates summed back to FP64).
template <int PREC>
__device__ __forceinline__ void eval_rhs(const Coefs& cf, const Tabs& tb, const double* y, double* k) {
  if constexpr (PREC == 0) {
    rhs64(cf.c64, tb.f, y, k);
  } else if constexpr (PREC == 1) {
    float yf[10], kf[10];
#pragma unroll
    for (int i = 0; i < 10; i++) yf[i] = f64_to_f32(y[i]);
    rhs32(cf.c32, yf, kf);
#pragma unroll
    for (int i = 0; i < 10; i++) k[i] = f32_to_f64(kf[i]);
  } else {
    ds yd[10], kd[10];
#pragma unroll
    for (int i = 0; i < 10; i++) yd[i] = split64(y[i]);
    rhs_ds(cf.cds, tb.f, yd, kd);
#pragma unroll
    for (int i = 0; i < 10; i++) k[i] = ds_to_f64(kd[i]);
  }
}

// The per-thread shared-memory workspaces of the attempts below are laid out in
// per-warp tiles: slot k of lane l of warp w at tile_w[k * 32 + l], tile_w the
// warp's slots x 32 elements.  A warp's access to one slot is 32 consecutive
// elements (conflict-free), and the lane stride is the constant 32 whatever the
// block size (any multiple of 32), so slot addresses are constant offsets from
// the lane's own base (a block-size stride cost address arithmetic per access:
// the double-single kernel ran 12 % faster persistent, 1 % plain, without it).
template <class T, int SLOTS>
__device__ __forceinline__ T* warp_tile_base(void* smem) {
  return reinterpret_cast<T*>(smem) + (size_t)(threadIdx.x >> 5) * (SLOTS * 32) + (threadIdx.x & 31u);
}

// One Dormand-Prince attempt of size h from y in FP64, with k1 = f(y) given.
// Writes y5 (the 5th-order solution), k7 = f(y5) and returns the mean of the
// squared scaled error components, s = err^2 (err = RMS norm).  The rates
// k2..k6 sit in a per-thread shared-memory workspace (per-warp tiles: rate j,
// component c in slot (j - 2) * 10 + c) and the six stages run as one loop, so
// one copy of the right-hand side serves them all; each stage's sum keeps
// exactly its own terms.
constexpr int kF64WorkBytes = 5 * 10 * 8;  // per thread
struct F64Work {
  double* base;  // warp_tile_base<double, 50>
  __device__ __forceinline__ double get(int j, int c) const { return base[((j - 2) * 10 + c) * 32]; }
  __device__ __forceinline__ void put(int j, int c, double v) const { base[((j - 2) * 10 + c) * 32] = v; }
};

__device__ __forceinline__ double dp5_attempt_ws(const Coefs& cf, const Tabs& tb, const Ctl& ctl, const double* y,
                                                 const double* k1, double h, double* y5, double* k7,
                                                 const F64Work& w) {
  double ys[10], kn[10];
#pragma unroll 1
  for (int r = 0; r < 6; r++) {
    if (r == 0) {
      const double a1 = h * DP_A21;
#pragma unroll
      for (int i = 0; i < 10; i++) ys[i] = fma(a1, k1[i], y[i]);
    } else if (r == 1) {
      const double a1 = h * DP_A31, a2 = h * DP_A32;
#pragma unroll
      for (int i = 0; i < 10; i++) ys[i] = fma(a2, w.get(2, i), fma(a1, k1[i], y[i]));
    } else if (r == 2) {
      const double a1 = h * DP_A41, a2 = h * DP_A42, a3 = h * DP_A43;
#pragma unroll
      for (int i = 0; i < 10; i++) ys[i] = fma(a3, w.get(3, i), fma(a2, w.get(2, i), fma(a1, k1[i], y[i])));
    } else if (r == 3) {
      const double a1 = h * DP_A51, a2 = h * DP_A52, a3 = h * DP_A53, a4 = h * DP_A54;
#pragma unroll
      for (int i = 0; i < 10; i++)
        ys[i] = fma(a4, w.get(4, i), fma(a3, w.get(3, i), fma(a2, w.get(2, i), fma(a1, k1[i], y[i]))));
    } else if (r == 4) {
      const double a1 = h * DP_A61, a2 = h * DP_A62, a3 = h * DP_A63, a4 = h * DP_A64, a5 = h * DP_A65;
#pragma unroll
      for (int i = 0; i < 10; i++)
        ys[i] = fma(a5, w.get(5, i), fma(a4, w.get(4, i), fma(a3, w.get(3, i), fma(a2, w.get(2, i),
                fma(a1, k1[i], y[i])))));
    } else {
      const double b1 = h * DP_B1, b3 = h * DP_B3, b4 = h * DP_B4, b5 = h * DP_B5, b6 = h * DP_B6;
#pragma unroll
      for (int i = 0; i < 10; i++) {
        y5[i] = fma(b6, w.get(6, i), fma(b5, w.get(5, i), fma(b4, w.get(4, i), fma(b3, w.get(3, i),
                fma(b1, k1[i], y[i])))));
        ys[i] = y5[i];
      }
    }
    rhs64(cf.c64, tb.f, ys, kn);  // k_{r+2}; for r = 5, k7 = f(y5)
    if (r < 5) {
#pragma unroll
      for (int i = 0; i < 10; i++) w.put(r + 2, i, kn[i]);
    }
  }
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < 10; i++) {
    k7[i] = kn[i];
    const double e = fma(DP_E7, k7[i], fma(DP_E6, w.get(6, i), fma(DP_E5, w.get(5, i), fma(DP_E4, w.get(4, i),
                     fma(DP_E3, w.get(3, i), DP_E1 * k1[i])))));
    const double sc = fma(ctl.rtol, max_abs(y[i], y5[i]), ctl.atol);
    const double q = e * rcp_norm(sc);
    sum = fma(q, q, sum);
  }
  return sum * ((h * h) * 0.1);
}

// ---------------------------------------------------------------------------
// Packed pairs of FP32 values (the f32x2 instructions of sm_100 and later): two
// independent FP32 values in one 64-bit register, one instruction for both.
// Each half of a packed instruction rounds exactly as the scalar instruction
// does (round to nearest even, subnormals kept), so packed pair arithmetic
// gives the same bits as two scalar evaluations in the same order.  On B300 a
// packed instruction takes one issue slot and the FMA pipe for two cycles, at
// the scalar latency: packing two independent chains halves their issue slots
// and doubles the independent work a rolled loop body carries, without
// growing the code (the double-single attempt is bound by dependency latency
// and instruction-cache size, not by the FMA pipe).
// ---------------------------------------------------------------------------
typedef unsigned long long f2;  // .x in bits 0..31, .y in bits 32..63

__device__ __forceinline__ f2 f2_of(float x, float y) {
  f2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(x), "f"(y));
  return d;
}
__device__ __forceinline__ f2 f2_dup(float x) { return f2_of(x, x); }
__device__ __forceinline__ float f2_x(f2 a) { return __uint_as_float((uint32_t)a); }
__device__ __forceinline__ float f2_y(f2 a) { return __uint_as_float((uint32_t)(a >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// -a in both halves (sign bits flipped: exact, like the scalar negation).
__device__ __forceinline__ f2 neg2(f2 a) { return a ^ 0x8000000080000000ull; }

// Two double-single values, halves .x and .y: hi = (x.hi, y.hi), lo = (x.lo, y.lo).
struct ds2 {
  f2 hi, lo;
};
__device__ __forceinline__ ds2 ds2_of(ds x, ds y) { return ds2{f2_of(x.hi, y.hi), f2_of(x.lo, y.lo)}; }
__device__ __forceinline__ ds ds2_x(ds2 a) { return ds{f2_x(a.hi), f2_x(a.lo)}; }
__device__ __forceinline__ ds ds2_y(ds2 a) { return ds{f2_y(a.hi), f2_y(a.lo)}; }

// The pair versions of two_sum, fast_two_sum and the double-single operations
// above, operation for operation.
__device__ __forceinline__ ds2 two_sum2(f2 a, f2 b) {
  const f2 s = add2(a, b);
  const f2 v = sub2(s, a);
  return ds2{s, add2(sub2(a, sub2(s, v)), sub2(b, v))};
}
__device__ __forceinline__ ds2 fast_two_sum2(f2 a, f2 b) {
  const f2 s = add2(a, b);
  return ds2{s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ ds2 ds2_add(ds2 a, ds2 b) {
  const ds2 s = two_sum2(a.hi, b.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(a.lo, b.lo)));
}
__device__ __forceinline__ ds2 ds2_mul(ds2 a, ds2 b) {
  const f2 p = mul2(a.hi, b.hi);
  f2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  return fast_two_sum2(p, e);
}

// The mixed-precision attempt (FP32 right-hand side).  The stage inputs
// Y_2..Y_6 only feed the FP32 right-hand side, which rounds them to FP32 on
// entry, so they are formed in FP32 from the FP32-rounded state.  The rates are
// FP32 values, so the sums over them that need more than FP32 -- the increment
// sum_j b_j k_j of the new state and the embedded error estimate, which cancels
// to ~tol of its terms -- are compensated double-single sums on the FP32 pipe
// (~2^-48 relative).  The state accumulation y5 = y + h (increment) is one FP64
// FMA per component; the error norm is taken in FP32 from the estimate's
// leading float (the FP32 rates already perturb it by ~1e-3 of itself); the
// accept test and the step-size update are FP64.  Conversions between the two
// formats are integer operations.  The
// six stages run as one loop so that the right-hand side is emitted once
// (seven inlined copies overflow the instruction cache); the rates k1..k6 sit
// in a per-thread shared-memory workspace so no register queue has to be
// shifted between stages.  The workspace holds packed pairs of components
// (2p, 2p + 1), and every sum over the components runs on the pairs with the
// packed FP32 instructions (the same bits as the scalar sums, half the issue
// slots): slot j, pair p in workspace slot j * 5 + p as 8 bytes (per-warp tiles).
// Slots 0..5 hold k1..k6; slot 1 takes k7 once k2 is spent (its weights in b and
// in b - bhat are 0); slots 6 and 7 the increment of y5 (hi, lo), then slot 6
// the error scale.
constexpr int kF32WorkBytes = 8 * 10 * 4;  // per thread
struct F32Work {
  f2* base;  // warp_tile_base<f2, 40>
  __device__ __forceinline__ f2 get2(int j, int p) const { return base[(j * 5 + p) * 32]; }
  __device__ __forceinline__ void put2(int j, int p, f2 v) const { base[(j * 5 + p) * 32] = v; }
};
// Rows of the stage tableau in FP32: coefficients of k1..k_{r+1} for stage r + 2.
__constant__ float c_dp_a_f[5][5] = {
    {(float)DP_A21, 0, 0, 0, 0},
    {(float)DP_A31, (float)DP_A32, 0, 0, 0},
    {(float)DP_A41, (float)DP_A42, (float)DP_A43, 0, 0},
    {(float)DP_A51, (float)DP_A52, (float)DP_A53, (float)DP_A54, 0},
    {(float)DP_A61, (float)DP_A62, (float)DP_A63, (float)DP_A64, (float)DP_A65},
};

// ---------------------------------------------------------------------------
// The double-single attempt.  Its stage inputs feed the double-single
// right-hand side and so need ~48-bit accuracy: they are formed on the FP32
// pipe by compensated sums (Dot2 of Ogita, Rump & Oishi 2005) of double-single
// rates, not by FP64 sums.  The state accumulation y5 = y + h sum_j b_j k_j, the
// error norm and the step control stay FP64.  The rates and stage vectors live
// in a per-thread shared-memory workspace so that the loops over the ten
// components can stay rolled: with them unrolled (or with the vectors in
// registers) the stage loop no longer fits the instruction cache.
// ---------------------------------------------------------------------------
struct dsc {  // a double-single constant: hi the nearest float, lo the nearest float to the rest
  float hi, lo;
};
#define PN_DSC(x) {(float)(x), (float)((x) - (double)(float)(x))}
// Row r: coefficients of k1..k_{r+1} for stage r + 2; row 5 is b (first same as last).
__constant__ dsc c_dp_a_ds[6][6] = {
    {PN_DSC(DP_A21), {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {PN_DSC(DP_A31), PN_DSC(DP_A32), {0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {PN_DSC(DP_A41), PN_DSC(DP_A42), PN_DSC(DP_A43), {0, 0}, {0, 0}, {0, 0}},
    {PN_DSC(DP_A51), PN_DSC(DP_A52), PN_DSC(DP_A53), PN_DSC(DP_A54), {0, 0}, {0, 0}},
    {PN_DSC(DP_A61), PN_DSC(DP_A62), PN_DSC(DP_A63), PN_DSC(DP_A64), PN_DSC(DP_A65), {0, 0}},
    {PN_DSC(DP_B1), {0, 0}, PN_DSC(DP_B3), PN_DSC(DP_B4), PN_DSC(DP_B5), PN_DSC(DP_B6)},
};
// b - bhat for k1, k3, k4, k5, k6, k7 (the k2 weight is 0).
__constant__ dsc c_dp_e_ds[6] = {PN_DSC(DP_E1), PN_DSC(DP_E3), PN_DSC(DP_E4),
                                 PN_DSC(DP_E5), PN_DSC(DP_E6), PN_DSC(DP_E7)};
#undef PN_DSC

// Compensated sum of products c_j x_j: s collects the rounded leading products
// exactly through two_sum, e the rounding errors of those sums, the products'
// own errors and the cross terms c.hi x.lo + c.lo x.hi.  dot_val(s, e) carries
// ~2^-48 relative error unless the sum cancels.
struct dacc {
  float s, e;
};
__device__ __forceinline__ dacc dot_first(dsc c, ds x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, e);
  e = __fmaf_rn(c.lo, x.hi, e);
  return dacc{p, e};
}
__device__ __forceinline__ dacc dot_add(dacc a, dsc c, ds x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, e);
  e = __fmaf_rn(c.lo, x.hi, e);
  const ds t = two_sum(a.s, p);
  return dacc{t.hi, __fadd_rn(a.e, __fadd_rn(t.lo, e))};
}
__device__ __forceinline__ ds dot_val(dacc a) { return two_sum(a.s, a.e); }

// The same for FP32 values x (exact floats: no low part).
__device__ __forceinline__ dacc dot_first_f(dsc c, float x) {
  const float p = __fmul_rn(c.hi, x);
  return dacc{p, __fmaf_rn(c.lo, x, __fmaf_rn(c.hi, x, -p))};
}
__device__ __forceinline__ dacc dot_add_f(dacc a, dsc c, float x) {
  const float p = __fmul_rn(c.hi, x);
  const float e = __fmaf_rn(c.lo, x, __fmaf_rn(c.hi, x, -p));
  const ds t = two_sum(a.s, p);
  return dacc{t.hi, __fadd_rn(a.e, __fadd_rn(t.lo, e))};
}

// Compensated sums of products c_j x_j (dot_first / dot_add / dot_val) for a
// pair of components with the same coefficients.
struct dacc2 {
  f2 s, e;
};
__device__ __forceinline__ dacc2 dot_first2(dsc c, ds2 x) {
  const f2 ch = f2_dup(c.hi), cl = f2_dup(c.lo);
  const f2 p = mul2(ch, x.hi);
  f2 e = fma2(ch, x.hi, neg2(p));
  e = fma2(ch, x.lo, e);
  e = fma2(cl, x.hi, e);
  return dacc2{p, e};
}
__device__ __forceinline__ dacc2 dot_add2(dacc2 a, dsc c, ds2 x) {
  const f2 ch = f2_dup(c.hi), cl = f2_dup(c.lo);
  const f2 p = mul2(ch, x.hi);
  f2 e = fma2(ch, x.hi, neg2(p));
  e = fma2(ch, x.lo, e);
  e = fma2(cl, x.hi, e);
  const ds2 t = two_sum2(a.s, p);
  return dacc2{t.hi, add2(a.e, add2(t.lo, e))};
}
__device__ __forceinline__ ds2 dot_val2(dacc2 a) { return two_sum2(a.s, a.e); }
// The sum unnormalized, for the product by h that follows in the double-single
// attempt: there h times the sum is added to y (or is the error estimate), so
// only its absolute error matters, and the lo*lo term the lazy product drops is
// ~2^-24 |lo| of a sum that is itself small beside y.
__device__ __forceinline__ ds2 dot_val2_l(dacc2 a) { return ds2{a.s, a.e}; }

// dot_first_f / dot_add_f for a pair of components with the same coefficients.
__device__ __forceinline__ dacc2 dot_first_f2(dsc c, f2 x) {
  const f2 ch = f2_dup(c.hi), cl = f2_dup(c.lo);
  const f2 p = mul2(ch, x);
  return dacc2{p, fma2(cl, x, fma2(ch, x, neg2(p)))};
}
__device__ __forceinline__ dacc2 dot_add_f2(dacc2 a, dsc c, f2 x) {
  const f2 ch = f2_dup(c.hi), cl = f2_dup(c.lo);
  const f2 p = mul2(ch, x);
  const f2 e = fma2(cl, x, fma2(ch, x, neg2(p)));
  const ds2 t = two_sum2(a.s, p);
  return dacc2{t.hi, add2(a.e, add2(t.lo, e))};
}

// The FP32-RHS attempt (declared with its workspace above).
__device__ __forceinline__ double dp5_attempt_f32(const Coef<float>& c, const Ctl& ctl, const double* y,
                                                  const double* k1, double h, double* y5, double* k7,
                                                  const F32Work& w) {
  f2 yf[5];
  float ys[10], kn[10];
  const float hf = f64_to_f32(h);
  const f2 hf2 = f2_dup(hf);
#pragma unroll
  for (int p = 0; p < 5; p++) {
    yf[p] = f2_of(f64_to_f32(y[2 * p]), f64_to_f32(y[2 * p + 1]));
    w.put2(0, p, f2_of(f64_to_f32(k1[2 * p]), f64_to_f32(k1[2 * p + 1])));  // k1 is an FP32 rate widened: exact
  }
#pragma unroll 1
  for (int r = 0; r < 6; r++) {
    if (r < 5) {
      const f2 a0 = f2_dup(hf * c_dp_a_f[r][0]), a1 = f2_dup(hf * c_dp_a_f[r][1]), a2 = f2_dup(hf * c_dp_a_f[r][2]),
               a3 = f2_dup(hf * c_dp_a_f[r][3]), a4 = f2_dup(hf * c_dp_a_f[r][4]);
#pragma unroll
      for (int p = 0; p < 5; p++) {
        f2 acc = fma2(a0, w.get2(0, p), yf[p]);
        if (r >= 1) acc = fma2(a1, w.get2(1, p), acc);
        if (r >= 2) acc = fma2(a2, w.get2(2, p), acc);
        if (r >= 3) acc = fma2(a3, w.get2(3, p), acc);
        if (r >= 4) acc = fma2(a4, w.get2(4, p), acc);
        ys[2 * p] = f2_x(acc);
        ys[2 * p + 1] = f2_y(acc);
      }
    } else {  // the 5th-order solution y5 = y + h inc, inc = sum_j b_j k_j compensated, then one FP64 FMA
#pragma unroll 1
      for (int p = 0; p < 5; p++) {  // rolled: the compensated sums would not fit the instruction cache x5
        dacc2 acc = dot_first_f2(c_dp_a_ds[5][0], w.get2(0, p));
        acc = dot_add_f2(acc, c_dp_a_ds[5][2], w.get2(2, p));
        acc = dot_add_f2(acc, c_dp_a_ds[5][3], w.get2(3, p));
        acc = dot_add_f2(acc, c_dp_a_ds[5][4], w.get2(4, p));
        acc = dot_add_f2(acc, c_dp_a_ds[5][5], w.get2(5, p));
        const ds2 inc = dot_val2(acc);
        w.put2(6, p, inc.hi);
        w.put2(7, p, inc.lo);
      }
#pragma unroll
      for (int p = 0; p < 5; p++) {
        // The FP32 right-hand side's input at y5 directly in FP32 (within an FP32 ulp of
        // y5 rounded), so the FP64 accumulation below is off the path to k7.
        const f2 ih = w.get2(6, p), il = w.get2(7, p);
        const f2 yy = fma2(hf2, ih, yf[p]);
        ys[2 * p] = f2_x(yy);
        ys[2 * p + 1] = f2_y(yy);
        y5[2 * p] = fma(h, f32_to_f64(f2_x(ih)) + f32_to_f64(f2_x(il)), y[2 * p]);
        y5[2 * p + 1] = fma(h, f32_to_f64(f2_y(ih)) + f32_to_f64(f2_y(il)), y[2 * p + 1]);
      }
    }
    rhs32(c, ys, kn);  // k_{r+2}; for r = 5, k7 = f(y5)
    if (r < 5) {
#pragma unroll
      for (int p = 0; p < 5; p++) w.put2(r + 1, p, f2_of(kn[2 * p], kn[2 * p + 1]));
    }
  }
  // Error estimate sum_j (b_j - bhat_j) k_j compensated (it cancels to ~tol of its terms), its
  // scaled RMS norm in FP32 from the estimate's leading float, with approximate divisions (the
  // FP32 rates already move the estimate by ~1e-3 of itself); h enters once, in FP64.
  const float rtf = f64_to_f32(ctl.rtol), atf = f64_to_f32(ctl.atol);
#pragma unroll
  for (int p = 0; p < 5; p++) {
    k7[2 * p] = f32_to_f64(kn[2 * p]);
    k7[2 * p + 1] = f32_to_f64(kn[2 * p + 1]);
    w.put2(1, p, f2_of(kn[2 * p], kn[2 * p + 1]));
    w.put2(6, p, f2_of(__fmaf_rn(rtf, fmaxf(fabsf(f2_x(yf[p])), fabsf(ys[2 * p])), atf),
                       __fmaf_rn(rtf, fmaxf(fabsf(f2_y(yf[p])), fabsf(ys[2 * p + 1])), atf)));
  }
  float sf = 0.0f;
#pragma unroll 1
  for (int p = 0; p < 5; p++) {
    dacc2 acc = dot_first_f2(c_dp_e_ds[0], w.get2(0, p));
    acc = dot_add_f2(acc, c_dp_e_ds[1], w.get2(2, p));
    acc = dot_add_f2(acc, c_dp_e_ds[2], w.get2(3, p));
    acc = dot_add_f2(acc, c_dp_e_ds[3], w.get2(4, p));
    acc = dot_add_f2(acc, c_dp_e_ds[4], w.get2(5, p));
    acc = dot_add_f2(acc, c_dp_e_ds[5], w.get2(1, p));
    const f2 e = add2(acc.s, acc.e);
    const f2 sc = w.get2(6, p);
    const float q0 = __fdividef(f2_x(e), f2_x(sc)), q1 = __fdividef(f2_y(e), f2_y(sc));
    sf = __fmaf_rn(q0, q0, sf);
    sf = __fmaf_rn(q1, q1, sf);
  }
  return f32_to_f64(sf) * ((h * h) * 0.1);
}


// Lazy forms (see ds_mul_l) for the double-single attempt's stage and error sums.
__device__ __forceinline__ ds2 ds2_mul_l(ds2 a, ds2 b) {
  const f2 p = mul2(a.hi, b.hi);
  f2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  return ds2{p, e};
}

// Per-thread workspace of dp5_attempt_ds in shared memory: vector v of ten
// double-single components as five packed pairs of components (2p, 2p + 1),
// pair p in workspace slot v * 5 + p as 16 bytes (hi_2p, hi_2p+1, lo_2p,
// lo_2p+1), in per-warp tiles so that a warp's accesses are 32 consecutive
// 16-byte words.  Vectors 0..5 hold the rates k1..k6 and 6
// the state split into pairs (then the increment of y5).  Stage s's input is
// formed in the vector its rate k_{s+1} will take (no sum of that stage reads
// it); the last stage's input, then k7, then the error estimate take vector 1,
// k2's, whose weight in b and in b - bhat is 0.  Seven vectors rather than
// eight let three 128-thread blocks share an SM's shared memory.
constexpr int kDsVectors = 7;
constexpr int kDsWorkBytes = kDsVectors * 10 * 8;  // per thread
struct DsWork {
  ulonglong2* base;  // warp_tile_base<ulonglong2, kDsVectors * 5>
  __device__ __forceinline__ ds2 get2(int v, int p) const {
    const ulonglong2 x = base[(v * 5 + p) * 32];
    return ds2{x.x, x.y};
  }
  __device__ __forceinline__ void put2(int v, int p, ds2 a) const { base[(v * 5 + p) * 32] = make_ulonglong2(a.hi, a.lo); }
  __device__ __forceinline__ void put_vec(int v, const ds* a) const {
#pragma unroll
    for (int p = 0; p < 5; p++) put2(v, p, ds2_of(a[2 * p], a[2 * p + 1]));
  }
  __device__ __forceinline__ void get_vec(int v, ds* a) const {
#pragma unroll
    for (int p = 0; p < 5; p++) {
      const ds2 x = get2(v, p);
      a[2 * p] = ds2_x(x);
      a[2 * p + 1] = ds2_y(x);
    }
  }
};

__device__ __forceinline__ double dp5_attempt_ds(const Coefs& cf, const Tabs& tb, const Ctl& ctl, const double* y,
                                                 const double* k1, double h, double* y5, double* k7,
                                                 const DsWork& w) {
  const ds hd = split64(h);
  const ds2 hd2 = ds2{f2_dup(hd.hi), f2_dup(hd.lo)};
#pragma unroll
  for (int p = 0; p < 5; p++) {
    w.put2(6, p, ds2_of(split64(y[2 * p]), split64(y[2 * p + 1])));
    w.put2(0, p, ds2_of(split64(k1[2 * p]), split64(k1[2 * p + 1])));
  }
  ds kn[10];
#pragma unroll 1
  for (int r = 0; r < 6; r++) {
    const dsc a0 = c_dp_a_ds[r][0], a1 = c_dp_a_ds[r][1], a2 = c_dp_a_ds[r][2], a3 = c_dp_a_ds[r][3],
              a4 = c_dp_a_ds[r][4], a5 = c_dp_a_ds[r][5];
#pragma unroll 1
    for (int p = 0; p < 5; p++) {
      dacc2 acc = dot_first2(a0, w.get2(0, p));
      if (r >= 1 && r < 5) acc = dot_add2(acc, a1, w.get2(1, p));  // b2 = 0
      if (r >= 2) acc = dot_add2(acc, a2, w.get2(2, p));
      if (r >= 3) acc = dot_add2(acc, a3, w.get2(3, p));
      if (r >= 4) acc = dot_add2(acc, a4, w.get2(4, p));
      if (r >= 5) acc = dot_add2(acc, a5, w.get2(5, p));
      const ds2 inc = ds2_mul_l(hd2, dot_val2_l(acc));  // h sum_j a_sj k_j
      w.put2(r < 5 ? r + 1 : 1, p, ds2_add(w.get2(6, p), inc));
      if (r == 5) w.put2(6, p, inc);
    }
    const int vs = r < 5 ? r + 1 : 1;  // the stage input, then its rate
    ds yin[10];
    w.get_vec(vs, yin);
    rhs_ds(cf.cds, tb.f, yin, kn);  // k_{r+2}; for r = 5, k7 at the double-single y5
    w.put_vec(vs, kn);
  }
#pragma unroll 1
  for (int p = 0; p < 5; p++) {  // embedded error estimate h sum_j (b_j - bhat_j) k_j
    dacc2 acc = dot_first2(c_dp_e_ds[0], w.get2(0, p));
    acc = dot_add2(acc, c_dp_e_ds[1], w.get2(2, p));
    acc = dot_add2(acc, c_dp_e_ds[2], w.get2(3, p));
    acc = dot_add2(acc, c_dp_e_ds[3], w.get2(4, p));
    acc = dot_add2(acc, c_dp_e_ds[4], w.get2(5, p));
    acc = dot_add2(acc, c_dp_e_ds[5], w.get2(1, p));
    w.put2(1, p, ds2_mul_l(hd2, dot_val2_l(acc)));
  }
  double sum = 0.0;
#pragma unroll
  for (int p = 0; p < 5; p++) {
    const ds2 inc = w.get2(6, p), err = w.get2(1, p);
#pragma unroll
    for (int h2 = 0; h2 < 2; h2++) {
      const int c = 2 * p + h2;
      const ds i1 = h2 ? ds2_y(inc) : ds2_x(inc);
      y5[c] = y[c] + (f32_to_f64(i1.hi) + f32_to_f64(i1.lo));
      k7[c] = ds_to_f64(kn[c]);
      const double e = ds_to_f64(h2 ? ds2_y(err) : ds2_x(err));
      const double sc = fma(ctl.rtol, max_abs(y[c], y5[c]), ctl.atol);
      const double q = e * rcp_norm(sc);
      sum = fma(q, q, sum);
    }
  }
  return sum * 0.1;
}

// Growth factor of the step control: clamp(safety * s^(-1/10), fac_min, fmax)
// with s = err^2, i.e. safety * err^(-1/5).
__device__ __forceinline__ double step_factor(const Ctl& ctl, double s, double fmax) {
  double fac;
  if (le_pos(s, ctl.s_lo)) fac = ctl.fac_max;
  else if (le_pos(ctl.s_hi, s)) fac = ctl.fac_min;
  else fac = ctl.safety * pow_m_tenth(s);
  if (!le_pos(fac, fmax)) fac = fmax;
  if (le_pos(fac, ctl.fac_min)) fac = ctl.fac_min;
  return fac;
}

// a / b in double-single: quotient of the leading parts, then one correction
// from the double-single remainder a - q b (b.hi a normal FP32 value).
__device__ __forceinline__ ds ds_div(ds a, ds b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ds r = ds_sub(a, ds_mul_f(b, q1));
  return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// The first retake of a step that crossed omega_f: h times the root in (0, 1]
// of the step's cubic Hermite interpolant of omega (end values w0, w1, end
// slopes dw0, dw1), by three Newton steps from the linear guess.  The
// interpolant in power form is p(s) - wf = a0 + s (a1 + s (a2 + s a3)) with
// d_i = h dw_i, a2 = 3 (w1 - w0) - 2 d0 - d1, a3 = d0 + d1 - 2 (w1 - w0).  This
// runs once per binary in a branch that usually holds one lane of the warp,
// where FP64 instructions would cost the whole warp the FP64 pipe's time, so it
// is evaluated in double-single on the FP32 pipe from the two FP64 differences
// w1 - w0 and w0 - wf: within ~1e-13 of the FP64 evaluation, a seed for the
// landing iteration, which then converges to its own tolerance.  A
// non-positive denominator gives a value the caller's bracket check rejects.
__device__ __forceinline__ double hermite_step_ds(double h, double w0, double dw0, double w1, double dw1,
                                                  double wf) {
  const ds hd = split64(h);
  const ds dw = split64(w1 - w0), a0 = split64(w0 - wf);
  const ds d0 = ds_mul(hd, split64(dw0)), d1 = ds_mul(hd, split64(dw1));
  const ds a2 = ds_sub(ds_mul_f(dw, 3.0f), ds_add(ds_scale(d0, 2.0f), d1));
  const ds a3 = ds_add(ds_scale(dw, -2.0f), ds_add(d0, d1));
  const ds b1 = ds_scale(a2, 2.0f), b2 = ds_mul_f(a3, 3.0f);
  ds s = ds_div(ds_neg(a0), dw);
#pragma unroll 1
  for (int it = 0; it < 3; it++) {
    const ds p = ds_fma(ds_fma(ds_fma(a3, s, a2), s, d0), s, a0);
    const ds dp = ds_fma(ds_fma(b2, s, b1), s, d0);
    s = ds_sub(s, ds_div(p, dp));
  }
  return ds_to_f64(ds_mul(hd, s));
}

}  // namespace pn
