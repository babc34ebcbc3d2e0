// pn_adjoint.cu -- reverse mode (discrete adjoint) of the integration (FP64,
// or double-single for pn_batch_adjoint with PN_MIXED_DS).
//
// Gradients of the loss sum_i gbar_i . out_i (final dot products, S1, S2,
// L-hat, t of each binary) with respect to the initial spin directions and the
// mass ratio q, through the accepted Dormand-Prince steps of the forward run
// (Sec. II) with their step sizes held fixed.  The stop at omega_f is
// differentiated as an implicit function: the landing step size h* is the root
// of omega5(y_{N-1}, h*) = omega_f, so with mu = ybar_f . d y5/dh + tbar and
// nu = d omega5/dh the cotangent passed back through the landing step is
// ybar_f - (mu/nu) e_omega (two reverse sweeps of that step).
//
// The forward pass (k_integrate with recording, in the sweep's precision, the
// lanes taking the binaries in the batch's order) keeps the accepted step sizes
// and the state every `every` accepted steps.  The reverse sweep takes one
// such segment at a time: it recomputes the segment's steps from its
// checkpoint with the forward kernel's stage arithmetic, keeping each step's
// six stage states, then walks the steps backwards.
//
// Work layout on the GPU:
//  - The FP64 pipe spends the same cycles on a warp instruction whatever its
//    active mask, and a binary's work is set by its accepted-step count N.  So
//    the binaries are first ordered by N (counting sort, longest first), and
//    each warp claims 32 consecutive entries of that order: its lanes walk the
//    same segments and steps in lock-step, and the longest binaries start first.
//  - The stage states go to a lane-private segment buffer (lane-contiguous so
//    the warp's accesses coalesce), in the FP64 sweep with the right-hand
//    side's intermediates at each of them.  The reverse step then runs no
//    forward stage: each stage costs the reverse half of one rhs64_vjp, which
//    hands back the kept stage rate for the step-size cotangent as well.

#include "pn_device.cuh"
#include "pn_adjoint.h"
#include "pn_debug.h"

namespace pn {
namespace {

// ---------------------------------------------------------------------------
// Reverse mode (adjoint) of the FP64 right-hand side.
// The segment recompute evaluates rhs64 at every stage state and keeps its
// intermediate values (rhs64's keep sink, KeepIdx order) beside the state, so
// the reverse sweep of one stage runs only the reverse half: rhs64_vjp returns
//   yb = (df/dy)^T fb   and adds (df/dc)^T fb to cb,
// each line undoing one line of rhs64 in reverse order, and also returns the
// kept rate f = f(y) (the stage rate the step-size cotangent needs).  c and cb
// are in rhs64's folded form (fold_K: the eleven coefficients of P times K);
// unfold_cotangents maps cb to the coefficients of make_coef at the end.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cross_vjp(const double* a, const double* b, const double* cb_, double* ab, double* bb) {
  // c = a x b:  ab += b x cb,  bb += cb x a
  ab[0] += b[1] * cb_[2] - b[2] * cb_[1];
  ab[1] += b[2] * cb_[0] - b[0] * cb_[2];
  ab[2] += b[0] * cb_[1] - b[1] * cb_[0];
  bb[0] += cb_[1] * a[2] - cb_[2] * a[1];
  bb[1] += cb_[2] * a[0] - cb_[0] * a[2];
  bb[2] += cb_[0] * a[1] - cb_[1] * a[0];
}

static_assert(kF64StageWords == 10 + KP_COUNT, "an FP64 stage block is the state and rhs64's kept values");

// Per-thread workspace of the double-single sweep in shared memory, in per-warp
// tiles (constant lane stride 32): the six stage rates of a step's recompute,
// then the six rate cotangents of its reverse step ([6][5] double-single
// component pairs, 480 bytes).  Indexed by the stage at run time, they would
// otherwise live in local memory, which the sweep's spills already crowd: the
// C4 double-single call ran 11.8 -> 10.1 ms with them here.  (The FP64 sweep,
// bound by its FP64 pipe, keeps its [6][10] arrays local: in shared memory it
// measured 25.0 against 24.7 ms.)
constexpr int kAdjWorkBytes = 480;

struct RateWorkDs {
  ulonglong2* b;  // warp_tile_base<ulonglong2, 30>
  __device__ __forceinline__ ds2 get(int j, int p) const {
    const ulonglong2 x = b[(j * 5 + p) * 32];
    return ds2{x.x, x.y};
  }
  __device__ __forceinline__ void put(int j, int p, ds2 v) const { b[(j * 5 + p) * 32] = make_ulonglong2(v.hi, v.lo); }
};

// Stores rhs64's intermediates to kp[k * ss] (the lane's segment buffer).
struct SegKeep {
  double* kp;
  size_t ss;
  __device__ __forceinline__ void operator()(int k, double x) const { kp[(size_t)k * ss] = x; }
};

__device__ __noinline__ void rhs64_vjp(const Coef<double>& c, const double* kp, size_t ss, const double* y,
                                       const double* fb, double* yb, Coef<double>& cb, double* f) {
  // ---- the kept forward values ----
  const double w = y[0];
  const double S1[3] = {y[1], y[2], y[3]}, S2[3] = {y[4], y[5], y[6]}, L[3] = {y[7], y[8], y[9]};
  const double r = kp[KP_R * ss], v = kp[KP_V * ss], v2 = kp[KP_V2 * ss], lw = kp[KP_LW * ss];
  const double LS1 = kp[KP_LS1 * ss], LS2 = kp[KP_LS2 * ss], S12 = kp[KP_S12 * ss];
  const double P6 = kp[KP_P6 * ss], P5 = kp[KP_P5 * ss], P4 = kp[KP_P4 * ss], P3 = kp[KP_P3 * ss];
  const double P2 = kp[KP_P2 * ss], P = kp[KP_P * ss], w2 = kp[KP_W2 * ss], Q = kp[KP_Q * ss];
  const double q1 = kp[KP_Q1 * ss], q2 = kp[KP_Q2 * ss], pre = kp[KP_PRE * ss], lf = kp[KP_LF * ss];
  double U1[3], U2[3], X1[3], X2[3], d1[3], d2[3];
  for (int k = 0; k < 3; k++) {
    U1[k] = kp[(KP_U1 + k) * ss];
    U2[k] = kp[(KP_U2 + k) * ss];
    X1[k] = kp[(KP_X1 + k) * ss];
    X2[k] = kp[(KP_X2 + k) * ss];
  }
  for (int k = 0; k < 10; k++) f[k] = kp[(KP_F + k) * ss];
  for (int k = 0; k < 3; k++) {
    d1[k] = f[1 + k];
    d2[k] = f[4 + k];
  }
  // ---- reverse ----
  double S1b[3] = {0, 0, 0}, S2b[3] = {0, 0, 0}, Lb[3] = {0, 0, 0};
  double d1b[3], d2b[3], X1b[3], X2b[3], U1b[3] = {0, 0, 0}, U2b[3] = {0, 0, 0};
  double lfb = 0.0;
  for (int k = 0; k < 3; k++) lfb += fb[7 + k] * (d1[k] + d2[k]);  // f_L = lf (d1 + d2)
  for (int k = 0; k < 3; k++) {
    d1b[k] = fb[1 + k] + lf * fb[7 + k];
    d2b[k] = fb[4 + k] + lf * fb[7 + k];
  }
  double vb = lfb * c.nie;  // lf = v nie
  cb.nie += lfb * v;
  double preb = 0.0;  // d_i = pre X_i
  for (int k = 0; k < 3; k++) {
    preb += X1[k] * d1b[k] + X2[k] * d2b[k];
    X1b[k] = pre * d1b[k];
    X2b[k] = pre * d2b[k];
  }
  cross_vjp(U1, S1, X1b, U1b, S1b);  // X1 = U1 x S1
  cross_vjp(U2, S2, X2b, U2b, S2b);  // X2 = U2 x S2
  double q1b = 0.0, q2b = 0.0;       // U1 = q1 L + S2, U2 = q2 L + S1
  for (int k = 0; k < 3; k++) {
    q1b += U1b[k] * L[k];
    q2b += U2b[k] * L[k];
    Lb[k] += q1 * U1b[k] + q2 * U2b[k];
    S2b[k] += U1b[k];
    S1b[k] += U2b[k];
  }
  cb.a1 += q1b * r;  // q1 = a1 r - 3 LS2, q2 = a2 r - 3 LS1
  cb.a2 += q2b * r;
  double rb = q1b * c.a1 + q2b * c.a2;
  double LS2b = -3.0 * q1b, LS1b = -3.0 * q2b;
  double w2b = preb * c.prec;  // pre = prec w2
  cb.prec += preb * w2;
  const double f0b = fb[0];  // f0 = Q P (P carries K)
  const double Qb = f0b * P;
  const double Pb = f0b * Q;
  w2b += Qb * w * v2;  // Q = w2 w v2
  double wb = Qb * w2 * v2;
  double v2b = Qb * w2 * w;
  wb += 2.0 * w * w2b;  // w2 = w^2
  v2b += Pb * P2;       // P = v2 P2 + K
  const double P2b = Pb * v2;
  cb.K += Pb;
  vb += P2b * P3;       // P2 = v P3 + c1
  const double P3b = P2b * v;
  cb.c1 += P2b;
  vb += P3b * P4;       // P3 = v P4 - so
  const double P4b = P3b * v;
  const double sob = -P3b;
  vb += P4b * P5;       // P4 = v P5 + c2p
  const double P5b = P4b * v;
  const double c2pb = P4b;
  vb += P5b * P6;       // P5 = v P6 + c25
  const double P6b = P5b * v;
  cb.c25 += P5b;
  vb += P6b * c.c35;    // P6 = v c35 + c3p
  cb.c35 += P6b * v;
  const double c3pb = P6b;
  cb.clog += c3pb * lw;  // c3p = clog lw + c3l
  const double lwb = c3pb * c.clog;
  cb.c3l += c3pb;
  cb.ss721 += c2pb * LS1 * LS2;  // c2p = ss721 LS1 LS2 - ss247 S12 + c2
  LS1b += c2pb * c.ss721 * LS2;
  LS2b += c2pb * c.ss721 * LS1;
  cb.ss247 -= c2pb * S12;
  const double S12b = -c2pb * c.ss247;
  cb.c2 += c2pb;
  cb.w1 += sob * LS1;  // so = w1 LS1 + w2 LS2 - tail
  LS1b += sob * c.w1;
  cb.w2 += sob * LS2;
  LS2b += sob * c.w2;
  cb.tail -= sob;
  for (int k = 0; k < 3; k++) {  // LS1 = L.S1, LS2 = L.S2, S12 = S1.S2
    Lb[k] += LS1b * S1[k] + LS2b * S2[k];
    S1b[k] += LS1b * L[k] + S12b * S2[k];
    S2b[k] += LS2b * L[k] + S12b * S1[k];
  }
  const double r2 = r * r;
  const double r3 = r2 * r;  // = 1/w
  wb += lwb * r3;            // lw = ln|w|
  vb += 2.0 * v * v2b;       // v2 = v^2
  wb += vb * r2;             // v = w r^2
  rb += vb * 2.0 * w * r;
  wb += rb * (-1.0 / 3.0) * r * r3;  // r = w^(-1/3): dr/dw = -r/(3w)
  yb[0] = wb;
  for (int k = 0; k < 3; k++) {
    yb[1 + k] = S1b[k];
    yb[4 + k] = S2b[k];
    yb[7 + k] = Lb[k];
  }
}

// Cotangents of rhs64's folded coefficients (fold_K: c'_i = K c_i for the eleven
// coefficients of P) mapped, in place, to those of make_coef's c: c_i-bar =
// K c'_i-bar and K-bar += sum_i c_i c'_i-bar.
__device__ __forceinline__ void unfold_cotangents(const Coef<double>& c, Coef<double>& b) {
  double* const bf[11] = {&b.w1, &b.w2, &b.tail, &b.ss247, &b.ss721, &b.c1, &b.c2, &b.c25, &b.c35, &b.c3l, &b.clog};
  const double cv[11] = {c.w1, c.w2, c.tail, c.ss247, c.ss721, c.c1, c.c2, c.c25, c.c35, c.c3l, c.clog};
  double kb = b.K;
  for (int i = 0; i < 11; i++) {
    kb += cv[i] * *bf[i];
    *bf[i] *= c.K;
  }
  b.K = kb;
}

// Reverse mode of make_coef: (m1b, m2b) += (dc/dm)^T cb, from the closed forms
// w1 = 113/12 + (25/4) m2/m1, w2 = 113/12 + (25/4) m1/m2, ss247 = 247/(48 eta),
// ss721 = 721/(48 eta), a1 = 4 m1 m2 + 3 m2^2, a2 = 4 m1 m2 + 3 m1^2, nie = -1/eta,
// and the eta-polynomials of the non-spin coefficients (M = 1, eta = m1 m2).
__device__ __forceinline__ void coef_vjp(const Coef<double>& cb, double m1, double m2, TermCfg tc, double* m1b,
                                         double* m2b) {
  const double eta = m1 * m2;
  const uint32_t mk = tc.mask;
  double etab = cb.K * (96.0 / 5.0);
  if (mk & 2u) {
    *m1b += cb.w1 * (-6.25 * m2 / (m1 * m1)) + cb.w2 * (6.25 / m2);
    *m2b += cb.w1 * (6.25 / m1) + cb.w2 * (-6.25 * m1 / (m2 * m2));
  }
  if (mk & 16u) etab += (cb.ss247 * 247.0 + cb.ss721 * 721.0) * (-1.0 / (48.0 * eta * eta));
  if (mk & 1u) etab += cb.c1 * (-924.0 / 336.0);
  if (mk & 8u) etab += cb.c2 * (13661.0 / 2016.0 + 2.0 * 59.0 / 18.0 * eta);
  if (mk & 32u) etab += cb.c25 * (-15876.0 * PN_PI / 672.0);
  if (mk & 64u) {
    const double theta = 1039.0 / 4620.0;
    const double c31 = -273811877.0 / 1088640.0 + 451.0 / 48.0 * PN_PI * PN_PI;
    const double dth = (tc.theta_mode == 0) ? c31 - 88.0 / 3.0 * theta : c31 - 2.0 * 88.0 / 3.0 * theta * eta;
    etab += cb.c3l * (dth + 2.0 * 541.0 / 896.0 * eta - 3.0 * 5605.0 / 2592.0 * eta * eta);
  }
  if (mk & 128u) etab += cb.c35 * (358675.0 / 6048.0 + 2.0 * 91495.0 / 1512.0 * eta) * PN_PI;
  *m1b += cb.a1 * (4.0 * m2) + cb.a2 * (4.0 * m2 + 6.0 * m1);
  *m2b += cb.a1 * (4.0 * m1 + 6.0 * m2) + cb.a2 * (4.0 * m1);
  etab += cb.nie / (eta * eta);
  *m1b += etab * m2;
  *m2b += etab * m1;
}

// Full Dormand-Prince lower-triangular tableau (rows: stages 1..6, the row of
// stage 1 empty) and the 5th-order weights.
__constant__ double c_dp_A[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {DP_A21, 0, 0, 0, 0, 0},
    {DP_A31, DP_A32, 0, 0, 0, 0},
    {DP_A41, DP_A42, DP_A43, 0, 0, 0},
    {DP_A51, DP_A52, DP_A53, DP_A54, 0, 0},
    {DP_A61, DP_A62, DP_A63, DP_A64, DP_A65, 0},
};
__constant__ double c_dp_B[6] = {DP_B1, 0.0, DP_B3, DP_B4, DP_B5, DP_B6};

// One Dormand-Prince step y -> y5 with a fixed h (the map the accepted steps
// apply; same FP64 arithmetic as the forward kernel's stages, so c holds the
// coefficients with K folded in, as there).  Stage s's block of the step's
// segment words (kF64StageWords words at sp[kF64StageWords s * ss]) holds the
// stage state Y_s (words 0..9) and the intermediates of rhs64 at Y_s that the
// reverse sweep needs (words 10.., KeepIdx order), the rate f(Y_s) among them.
// With y5 == nullptr the step's result is not formed.
__device__ __forceinline__ void dp5_stages(const Coef<double>& c,
                                           const float* __restrict__ tabf, const double* y, double h, double* sp,
                                           size_t ss, double* y5) {
  double K[6][10], ys[10];
  for (int i = 0; i < 10; i++) sp[(size_t)i * ss] = y[i];
  rhs64(c, tabf, y, K[0], SegKeep{sp + (size_t)10 * ss, ss});
#pragma unroll 1
  for (int s = 1; s < 6; s++) {
    for (int i = 0; i < 10; i++) ys[i] = y[i];
    for (int j = 0; j < s; j++) {
      const double a = h * c_dp_A[s][j];
      if (a != 0.0)
        for (int i = 0; i < 10; i++) ys[i] = fma(a, K[j][i], ys[i]);
    }
    double* const blk = sp + (size_t)(kF64StageWords * s) * ss;
    for (int i = 0; i < 10; i++) blk[(size_t)i * ss] = ys[i];
    rhs64(c, tabf, ys, K[s], SegKeep{blk + (size_t)10 * ss, ss});
  }
  if (!y5) return;
  for (int i = 0; i < 10; i++) y5[i] = y[i];
  for (int j = 0; j < 6; j++) {
    const double b = h * c_dp_B[j];
    if (b != 0.0)
      for (int i = 0; i < 10; i++) y5[i] = fma(b, K[j][i], y5[i]);
  }
}

// Prefetch of one kept stage block into L2.
__device__ __forceinline__ void prefetch_block(const double* blk, size_t ss) {
#pragma unroll 1
  for (int k = 0; k < kF64StageWords; k++) asm volatile("prefetch.global.L2 [%0];" ::"l"(blk + (size_t)k * ss));
}

// Reverse mode of one step from its kept stage blocks: on entry lam is the
// cotangent of y5, on exit the cotangent of y; the (folded) coefficient
// cotangents are added to cb; returns the cotangent of h.  With
//   y5 = y + h sum_j b_j k_j,  Y_s = y + h sum_{j<s} a_sj k_j,  k_s = f(Y_s)
// and kp_j = b_j lam + sum_{s>j} a_sj Yb_s (the cotangent of k_j is h kp_j):
//   Yb_s = J(Y_s)^T (h kp_s),  yb = lam + sum_s Yb_s,  hb = sum_j k_j . kp_j.
// While stage s is reversed, the block of the stage reversed next (s - 1, or
// for s = 0 the block pf, stage 5 of the step reversed after this one, if any)
// is prefetched: the blocks come from DRAM (the whole segment was recomputed
// first), and at two warps per scheduler their latency would otherwise stall
// the FP64 pipe.  One out-of-line copy serves the landing step's two calls and
// the other steps' one (24.8 against 25.6 ms for the C4 call inlined; the
// double-single step VJP, whose sweep is bound by instruction fetch, measured
// the other way).

__device__ __noinline__ double dp5_step_vjp(const Coef<double>& c, const double* sp, size_t ss, double h,
                                            double* lam, Coef<double>& cb, const double* pf) {
  double kp[6][10], yb[10];
  for (int j = 0; j < 6; j++)
    for (int i = 0; i < 10; i++) kp[j][i] = c_dp_B[j] * lam[i];
  for (int i = 0; i < 10; i++) yb[i] = lam[i];
  double hb = 0.0;
#pragma unroll 1
  for (int s = 5; s >= 0; s--) {
    double Ys[10], fb[10], Yb[10], ks[10];
    const double* const blk = sp + (size_t)(kF64StageWords * s) * ss;
    const double* const next = s > 0 ? blk - (size_t)kF64StageWords * ss : pf;
    if (next) prefetch_block(next, ss);
    for (int i = 0; i < 10; i++) {
      Ys[i] = blk[(size_t)i * ss];
      fb[i] = h * kp[s][i];
    }
    rhs64_vjp(c, blk + (size_t)10 * ss, ss, Ys, fb, Yb, cb, ks);
    for (int i = 0; i < 10; i++) {
      hb = fma(ks[i], kp[s][i], hb);
      yb[i] += Yb[i];
    }
    for (int j = 0; j < s; j++) {
      const double a = c_dp_A[s][j];
      if (a != 0.0)
        for (int i = 0; i < 10; i++) kp[j][i] = fma(a, Yb[i], kp[j][i]);
    }
  }
  for (int i = 0; i < 10; i++) lam[i] = yb[i];
  return hb;
}

// ---------------------------------------------------------------------------
// The same reverse sweep in double-single arithmetic (pn_batch_adjoint with
// PN_MIXED_DS): the segment recompute and the vector-Jacobian products run in
// pairs of FP32 (~48-bit significands) on the FP32 pipe, each line undoing the
// matching line of the forward pass as in rhs64_vjp.  Constants that are not
// exact in FP32 enter as double-single pairs.  The recorded step sizes and
// checkpoints are the double-single forward run's (the FP64 run's steps, its
// states within ~1e-13); the states between checkpoints are recomputed with
// double-single stage sums and FP64 state accumulation.  Products are the
// lazy (unnormalized) ones of the forward kernel; sums keep their
// renormalization.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ds dfma(ds a, ds b, ds c) { return ds_fma(a, b, c); }
__device__ __forceinline__ ds dzero() { return ds{0.0f, 0.0f}; }
__device__ __forceinline__ ds dconst(dsc k) { return ds{k.hi, k.lo}; }

// Packed pair forms (f32x2) of the double-single operations, operation for
// operation as the scalar ones (the same bits): the two spins' terms of the
// VJP below -- (L.S1, L.S2), (q1, q2), (U1, U2), the cross products and their
// cotangents -- go through them, which shortens the sweep's straight-line body.
__device__ __forceinline__ ds2 ds2_mul_f(ds2 a, f2 b) {
  const f2 p = mul2(a.hi, b);
  f2 e = fma2(a.hi, b, neg2(p));
  e = fma2(a.lo, b, e);
  return fast_two_sum2(p, e);
}
__device__ __forceinline__ ds2 ds2_fma(ds2 a, ds2 b, ds2 c) {
  const f2 p = mul2(a.hi, b.hi);
  f2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  const ds2 s = two_sum2(p, c.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(e, c.lo)));
}
__device__ __forceinline__ ds2 ds2_dot3(ds2 a0, ds2 b0, ds2 a1, ds2 b1, ds2 a2, ds2 b2) {
  const f2 p0 = mul2(a0.hi, b0.hi), p1 = mul2(a1.hi, b1.hi), p2 = mul2(a2.hi, b2.hi);
  f2 e = fma2(a0.hi, b0.hi, neg2(p0));
  e = fma2(a0.hi, b0.lo, e);
  e = fma2(a0.lo, b0.hi, e);
  e = add2(e, fma2(a1.hi, b1.hi, neg2(p1)));
  e = fma2(a1.hi, b1.lo, e);
  e = fma2(a1.lo, b1.hi, e);
  e = add2(e, fma2(a2.hi, b2.hi, neg2(p2)));
  e = fma2(a2.hi, b2.lo, e);
  e = fma2(a2.lo, b2.hi, e);
  const ds2 s = two_sum2(p0, p1);
  const ds2 t = two_sum2(s.hi, p2);
  return fast_two_sum2(t.hi, add2(e, add2(s.lo, t.lo)));
}
__device__ __forceinline__ ds2 ds2_diff_prod(ds2 a, ds2 b, ds2 c, ds2 d) {
  const f2 p = mul2(a.hi, b.hi), q = mul2(c.hi, d.hi);
  f2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  f2 f = fma2(c.hi, d.hi, neg2(q));
  f = fma2(c.hi, d.lo, f);
  f = fma2(c.lo, d.hi, f);
  const ds2 s = two_sum2(p, neg2(q));
  return fast_two_sum2(s.hi, add2(s.lo, sub2(e, f)));
}
__device__ __forceinline__ ds2 ds2_swap(ds2 a) {
  return ds2{(a.hi >> 32) | (a.hi << 32), (a.lo >> 32) | (a.lo << 32)};
}
__device__ __forceinline__ ds2 ds2_dup(ds a) { return ds2{f2_dup(a.hi), f2_dup(a.lo)}; }
__device__ __forceinline__ ds2 ds2_zero() { return ds2{0ull, 0ull}; }
// c = a x b for pairs of vectors (one per spin)
__device__ __forceinline__ void cross2(const ds2* a, const ds2* b, ds2* c) {
  c[0] = ds2_diff_prod(a[1], b[2], a[2], b[1]);
  c[1] = ds2_diff_prod(a[2], b[0], a[0], b[2]);
  c[2] = ds2_diff_prod(a[0], b[1], a[1], b[0]);
}

__device__ __noinline__ void rhs_ds_vjp(const Coef<ds>& c, const float* __restrict__ tabf, const ds* y, const ds* fb,
                                        ds* yb, Coef<ds>& cb, ds* f) {
  const dsc kThird = {(float)(1.0 / 3.0), (float)(1.0 / 3.0 - (double)(float)(1.0 / 3.0))};
  // ---- forward (as rhs_ds) ----  S[k] = (S1_k, S2_k); pairs carry the two spins' terms
  const ds w = y[0];
  const ds L[3] = {y[7], y[8], y[9]};
  const ds2 S[3] = {ds2_of(y[1], y[4]), ds2_of(y[2], y[5]), ds2_of(y[3], y[6])};
  const ds2 Ld[3] = {ds2_dup(L[0]), ds2_dup(L[1]), ds2_dup(L[2])};
  ds r = ds_inv_cbrt(w);
  if ((__float_as_uint(w.hi) & 0x7fffffffu) - 0x00800000u >= 0x7f000000u) r = ds{__int_as_float(0x7fc00000), 0.0f};
  const ds r2 = ds_mul_l(r, r);
  const ds v = ds_mul_l(w, r2);
  const ds v2 = ds_mul_l(v, v);
  const ds lw = ds_log(w, tabf);
  const ds2 LS = ds2_dot3(Ld[0], S[0], Ld[1], S[1], Ld[2], S[2]);  // (L.S1, L.S2)
  const ds LS1 = ds2_x(LS), LS2 = ds2_y(LS);
  const ds S12 = ds_dot3(ds2_x(S[0]), ds2_y(S[0]), ds2_x(S[1]), ds2_y(S[1]), ds2_x(S[2]), ds2_y(S[2]));
  const ds so = dfma(c.w1, LS1, dfma(c.w2, LS2, ds_neg(c.tail)));
  const ds c2p = dfma(c.ss721, ds_mul_l(LS1, LS2), dfma(ds_neg(c.ss247), S12, c.c2));
  const ds c3p = dfma(c.clog, lw, c.c3l);
  const ds P6 = dfma(v, c.c35, c3p);
  const ds P5 = dfma(v, P6, c.c25);
  const ds P4 = dfma(v, P5, c2p);
  const ds P3 = dfma(v, P4, ds_neg(so));
  const ds P2 = dfma(v, P3, c.c1);
  const ds P = dfma(v2, P2, ds_of(1.0f));
  const ds w2 = ds_mul_l(w, w);
  const ds Q = ds_mul_l(ds_mul_l(w2, w), v2);
  // Eq. (4) as in rhs_ds: dS_i/dt = pre (U_i x S_i), U_1 = q1 L + S2, q1 = a1 r - 3 LS2 (1 <-> 2).
  const ds pre = ds_mul_l(c.prec, w2);
  const ds2 pre2 = ds2_dup(pre);
  const ds2 q = ds2_fma(ds2_of(c.a1, c.a2), ds2_dup(r), ds2_mul_f(ds2_swap(LS), f2_dup(-3.0f)));  // (q1, q2)
  const ds q1 = ds2_x(q), q2 = ds2_y(q);
  ds2 U[3], X[3], D[3];
  for (int k = 0; k < 3; k++) U[k] = ds2_fma(q, Ld[k], ds2_swap(S[k]));  // (U1_k, U2_k)
  cross2(U, S, X);                                                       // (X1, X2) = (U1 x S1, U2 x S2)
  for (int k = 0; k < 3; k++) D[k] = ds2_mul_l(pre2, X[k]);                // (d1, d2)
  const ds lf = ds_mul_l(v, c.nie);
  f[0] = ds_mul_l(ds_mul_l(Q, c.K), P);
  ds dsum[3];
  for (int k = 0; k < 3; k++) {
    f[1 + k] = ds2_x(D[k]);
    f[4 + k] = ds2_y(D[k]);
    dsum[k] = ds_add(ds2_x(D[k]), ds2_y(D[k]));
    f[7 + k] = ds_mul_l(lf, dsum[k]);
  }
  // ---- reverse ----
  ds2 Sb[3] = {ds2_zero(), ds2_zero(), ds2_zero()};  // (S1b_k, S2b_k)
  ds Lb[3] = {dzero(), dzero(), dzero()};
  ds2 Db[3], Xb[3];
  ds2 Ub[3] = {ds2_zero(), ds2_zero(), ds2_zero()};
  ds lfb = dzero();
  for (int k = 0; k < 3; k++) lfb = dfma(fb[7 + k], dsum[k], lfb);  // f_L = lf (d1 + d2)
  const ds2 lf2 = ds2_dup(lf);
  for (int k = 0; k < 3; k++) Db[k] = ds2_fma(lf2, ds2_dup(fb[7 + k]), ds2_of(fb[1 + k], fb[4 + k]));
  ds vb = ds_mul_l(lfb, c.nie);  // lf = v nie
  cb.nie = dfma(lfb, v, cb.nie);
  ds preb = dzero();  // d_i = pre X_i
  for (int k = 0; k < 3; k++) {
    preb = dfma(ds2_x(X[k]), ds2_x(Db[k]), dfma(ds2_y(X[k]), ds2_y(Db[k]), preb));
    Xb[k] = ds2_mul_l(pre2, Db[k]);
  }
  {  // X_i = U_i x S_i:  Ub_i += S_i x Xb_i,  Sb_i += Xb_i x U_i
    ds2 t[3];
    cross2(S, Xb, t);
    for (int k = 0; k < 3; k++) Ub[k] = ds2_add(Ub[k], t[k]);
    cross2(Xb, U, t);
    for (int k = 0; k < 3; k++) Sb[k] = ds2_add(Sb[k], t[k]);
  }
  const ds2 qb = ds2_dot3(Ub[0], Ld[0], Ub[1], Ld[1], Ub[2], Ld[2]);  // U1 = q1 L + S2, U2 = q2 L + S1
  const ds q1b = ds2_x(qb), q2b = ds2_y(qb);
  for (int k = 0; k < 3; k++) {
    Lb[k] = dfma(q1, ds2_x(Ub[k]), dfma(q2, ds2_y(Ub[k]), Lb[k]));
    Sb[k] = ds2_add(Sb[k], ds2_swap(Ub[k]));
  }
  cb.a1 = dfma(q1b, r, cb.a1);  // q1 = a1 r - 3 LS2, q2 = a2 r - 3 LS1
  cb.a2 = dfma(q2b, r, cb.a2);
  ds rb = dfma(q1b, c.a1, ds_mul_l(q2b, c.a2));
  ds LS2b = ds_mul_f_l(q1b, -3.0f), LS1b = ds_mul_f_l(q2b, -3.0f);
  ds w2b = ds_mul_l(preb, c.prec);  // pre = prec w2
  cb.prec = dfma(preb, w2, cb.prec);
  const ds f0b = fb[0];  // f0 = Q K P
  const ds Qb = ds_mul_l(ds_mul_l(f0b, c.K), P);
  cb.K = dfma(ds_mul_l(f0b, Q), P, cb.K);
  const ds Pb = ds_mul_l(ds_mul_l(f0b, Q), c.K);
  w2b = dfma(ds_mul_l(Qb, w), v2, w2b);  // Q = w2 w v2
  ds wb = ds_mul_l(ds_mul_l(Qb, w2), v2);
  ds v2b = ds_mul_l(ds_mul_l(Qb, w2), w);
  wb = dfma(ds_scale(w, 2.0f), w2b, wb);  // w2 = w^2
  v2b = dfma(Pb, P2, v2b);                // P = v2 P2 + 1
  const ds P2b = ds_mul_l(Pb, v2);
  vb = dfma(P2b, P3, vb);  // P2 = v P3 + c1
  const ds P3b = ds_mul_l(P2b, v);
  cb.c1 = ds_add(cb.c1, P2b);
  vb = dfma(P3b, P4, vb);  // P3 = v P4 - so
  const ds P4b = ds_mul_l(P3b, v);
  const ds sob = ds_neg(P3b);
  vb = dfma(P4b, P5, vb);  // P4 = v P5 + c2p
  const ds P5b = ds_mul_l(P4b, v);
  const ds c2pb = P4b;
  vb = dfma(P5b, P6, vb);  // P5 = v P6 + c25
  const ds P6b = ds_mul_l(P5b, v);
  cb.c25 = ds_add(cb.c25, P5b);
  vb = dfma(P6b, c.c35, vb);  // P6 = v c35 + c3p
  cb.c35 = dfma(P6b, v, cb.c35);
  const ds c3pb = P6b;
  cb.clog = dfma(c3pb, lw, cb.clog);  // c3p = clog lw + c3l
  const ds lwb = ds_mul_l(c3pb, c.clog);
  cb.c3l = ds_add(cb.c3l, c3pb);
  cb.ss721 = dfma(ds_mul_l(c2pb, LS1), LS2, cb.ss721);  // c2p = ss721 LS1 LS2 - ss247 S12 + c2
  LS1b = dfma(ds_mul_l(c2pb, c.ss721), LS2, LS1b);
  LS2b = dfma(ds_mul_l(c2pb, c.ss721), LS1, LS2b);
  cb.ss247 = ds_sub(cb.ss247, ds_mul_l(c2pb, S12));
  const ds S12b = ds_neg(ds_mul_l(c2pb, c.ss247));
  cb.c2 = ds_add(cb.c2, c2pb);
  cb.w1 = dfma(sob, LS1, cb.w1);  // so = w1 LS1 + w2 LS2 - tail
  LS1b = dfma(sob, c.w1, LS1b);
  cb.w2 = dfma(sob, LS2, cb.w2);
  LS2b = dfma(sob, c.w2, LS2b);
  cb.tail = ds_sub(cb.tail, sob);
  const ds2 LSb = ds2_of(LS1b, LS2b), S12b2 = ds2_dup(S12b);
  for (int k = 0; k < 3; k++) {  // LS1 = L.S1, LS2 = L.S2, S12 = S1.S2
    Lb[k] = dfma(LS1b, ds2_x(S[k]), dfma(LS2b, ds2_y(S[k]), Lb[k]));
    Sb[k] = ds2_fma(LSb, Ld[k], ds2_fma(S12b2, ds2_swap(S[k]), Sb[k]));
  }
  const ds r3 = ds_mul_l(r2, r);  // = 1/w
  wb = dfma(lwb, r3, wb);       // lw = ln|w|
  vb = dfma(ds_scale(v, 2.0f), v2b, vb);  // v2 = v^2
  wb = dfma(vb, r2, wb);                  // v = w r^2
  rb = dfma(ds_mul_l(vb, ds_scale(w, 2.0f)), r, rb);
  wb = ds_sub(wb, ds_mul_l(ds_mul_l(ds_mul_l(rb, dconst(kThird)), r), r3));  // dr/dw = -r/(3w)
  yb[0] = wb;
  for (int k = 0; k < 3; k++) {
    yb[1 + k] = ds2_x(Sb[k]);
    yb[4 + k] = ds2_y(Sb[k]);
    yb[7 + k] = Lb[k];
  }
}

// One recomputed step in double-single: stage states Y_0..Y_5 (pairs) to
// sp[(10 s + k) * ss], and when y5 != nullptr the step's result, accumulated in
// FP64 from the double-single increment.  The stage sums run on packed pairs of
// components (2p, 2p + 1), operation for operation as the scalar sums.
__device__ __forceinline__ void dp5_stages_ds(const Coef<ds>& c, const float* __restrict__ tabf, const double* y,
                                              double h, float2* sp, size_t ss, double* y5, RateWorkDs K) {
  ds yd[10], kn[10];
  const ds hd = split64(h);
  const ds2 hd2 = ds2_dup(hd);
  for (int i = 0; i < 10; i++) {
    yd[i] = split64(y[i]);
    sp[(size_t)i * ss] = make_float2(yd[i].hi, yd[i].lo);
  }
  rhs_ds(c, tabf, yd, kn);
  for (int p = 0; p < 5; p++) K.put(0, p, ds2_of(kn[2 * p], kn[2 * p + 1]));
#pragma unroll 1
  for (int s = 1; s < 6; s++) {
    ds ys[10];
    for (int p = 0; p < 5; p++) {
      dacc2 acc = dot_first2(c_dp_a_ds[s - 1][0], K.get(0, p));
      for (int j = 1; j < s; j++) acc = dot_add2(acc, c_dp_a_ds[s - 1][j], K.get(j, p));
      const ds2 yy = ds2_add(ds2_of(yd[2 * p], yd[2 * p + 1]), ds2_mul_l(hd2, dot_val2_l(acc)));
      ys[2 * p] = ds2_x(yy);
      ys[2 * p + 1] = ds2_y(yy);
      sp[(size_t)(10 * s + 2 * p) * ss] = make_float2(ys[2 * p].hi, ys[2 * p].lo);
      sp[(size_t)(10 * s + 2 * p + 1) * ss] = make_float2(ys[2 * p + 1].hi, ys[2 * p + 1].lo);
    }
    if (s < 5 || y5) {
      rhs_ds(c, tabf, ys, kn);
      for (int p = 0; p < 5; p++) K.put(s, p, ds2_of(kn[2 * p], kn[2 * p + 1]));
    }
  }
  if (!y5) return;
  for (int p = 0; p < 5; p++) {
    dacc2 acc = dot_first2(c_dp_a_ds[5][0], K.get(0, p));
    for (int j = 2; j < 6; j++) acc = dot_add2(acc, c_dp_a_ds[5][j], K.get(j, p));
    const ds2 inc = ds2_mul_l(hd2, dot_val2_l(acc));
    const ds i0 = ds2_x(inc), i1 = ds2_y(inc);
    y5[2 * p] = y[2 * p] + (f32_to_f64(i0.hi) + f32_to_f64(i0.lo));
    y5[2 * p + 1] = y[2 * p + 1] + (f32_to_f64(i1.hi) + f32_to_f64(i1.lo));
  }
}

// Reverse mode of one step from its stored double-single stage states (the same
// recurrences as dp5_step_vjp): lam in/out, cb accumulated, returns h's cotangent.
// The component sums run on packed pairs of components; hb keeps its scalar order.
__device__ double dp5_step_vjp_ds(const Coef<ds>& c, const float* __restrict__ tabf, const float2* sp, size_t ss,
                                  double h, ds* lam, Coef<ds>& cb, RateWorkDs kp) {
  ds2 yb[5];
  const ds hd = split64(h);
  const ds2 hd2 = ds2_dup(hd);
  for (int j = 0; j < 6; j++)
    for (int p = 0; p < 5; p++) kp.put(j, p, ds2_mul_l(ds2_dup(dconst(c_dp_a_ds[5][j])), ds2_of(lam[2 * p], lam[2 * p + 1])));
  for (int p = 0; p < 5; p++) yb[p] = ds2_of(lam[2 * p], lam[2 * p + 1]);
  ds hb = dzero();
#pragma unroll 1
  for (int s = 5; s >= 0; s--) {
    ds Ys[10], fb[10], Yb[10], ks[10];
    for (int i = 0; i < 10; i++) {
      const float2 t = sp[(size_t)(10 * s + i) * ss];
      Ys[i] = ds{t.x, t.y};
    }
    for (int p = 0; p < 5; p++) {
      const ds2 f = ds2_mul_l(hd2, kp.get(s, p));
      fb[2 * p] = ds2_x(f);
      fb[2 * p + 1] = ds2_y(f);
    }
    rhs_ds_vjp(c, tabf, Ys, fb, Yb, cb, ks);
    ds2 Yb2[5];
    for (int p = 0; p < 5; p++) {
      hb = dfma(ks[2 * p], ds2_x(kp.get(s, p)), hb);
      hb = dfma(ks[2 * p + 1], ds2_y(kp.get(s, p)), hb);
      Yb2[p] = ds2_of(Yb[2 * p], Yb[2 * p + 1]);
      yb[p] = ds2_add(yb[p], Yb2[p]);
    }
    for (int j = 0; j < s; j++) {
      const ds a = dconst(c_dp_a_ds[s - 1][j]);
      if (a.hi != 0.0f) {
        const ds2 a2 = ds2_dup(a);
        for (int p = 0; p < 5; p++) kp.put(j, p, ds2_fma(a2, Yb2[p], kp.get(j, p)));
      }
    }
  }
  for (int p = 0; p < 5; p++) {
    lam[2 * p] = ds2_x(yb[p]);
    lam[2 * p + 1] = ds2_y(yb[p]);
  }
  return ds_to_f64(hb);
}

__device__ __forceinline__ double gval(const double* p, int64_t i) { return p ? p[i] : 0.0; }

// Sort key of binary i: its accepted-step count when the sweep walks its
// record, 0 when its gradients are NaN (status not OK, or no usable record).
__device__ __forceinline__ int32_t sweep_key(const pn_outputs& o, int64_t i, int32_t cap) {
  const int32_t N = o.n_acc[i];
  return (o.status[i] == PN_ST_OK && N >= 1 && N <= cap) ? N : 0;
}

// Counting sort of the binaries by sweep_key, largest key first.
__global__ void k_order_count(const pn_outputs o, int64_t n, int32_t cap, unsigned long long* bins) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t key = sweep_key(o, i, cap);
  const unsigned peers = __match_any_sync(__activemask(), key);
  if ((int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd(&bins[key], (unsigned long long)__popc(peers));
}

__global__ void k_order_scatter(const pn_outputs o, int64_t n, int32_t cap, unsigned long long* cursor,
                                int64_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t key = sweep_key(o, i, cap);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(__activemask(), key);
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(&cursor[key], (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  const unsigned long long pos = base + __popc(peers & ((1u << lane) - 1u));
  if (PN_DCHECK(pos < (unsigned long long)n, 20)) order[pos] = i;
}

// Derivatives of a loss with gradient gv (with respect to the components of s)
// along the polar and azimuthal angles of s at fixed |s|:
//   ds/dp = (-s_y, s_x, 0),  ds/dt = (s_z s_x / rho, s_z s_y / rho, -rho) with
//   rho = sqrt(s_x^2 + s_y^2) = |s| sin t; at a pole (rho = 0) p = 0 is taken:
//   ds/dt = (s_z, 0, 0).
__device__ __forceinline__ void angle_grads(const double* gv, const double* s, double* dt, double* dp) {
  const double rho = sqrt(s[0] * s[0] + s[1] * s[1]);
  *dp = gv[1] * s[0] - gv[0] * s[1];
  if (rho > 0.0) *dt = (gv[0] * s[0] + gv[1] * s[1]) * (s[2] / rho) - gv[2] * rho;
  else *dt = gv[0] * s[2];
}

// Gradients of binary i; sp0 is the lane's segment buffer (stride ss).
template <bool DS>
__device__ void adjoint_one(const AdjArgs& a, const float* __restrict__ tabf,
                            int64_t i, double* sp0, size_t ss, void* rw) {
  const pn_outputs& o = a.k.out;
  const pn_grads& g = a.grad;
  const int32_t N = o.n_acc[i];
  if (o.status[i] != PN_ST_OK || N < 1 || N > a.cap) {
    const double nan = dnan();
    g.s1x[i] = nan; g.s1y[i] = nan; g.s1z[i] = nan; g.s2x[i] = nan; g.s2y[i] = nan; g.s2z[i] = nan; g.q[i] = nan;
    if (g.s1x_tan) {
      g.s1x_tan[i] = nan; g.s1y_tan[i] = nan; g.s1z_tan[i] = nan;
      g.s2x_tan[i] = nan; g.s2y_tan[i] = nan; g.s2z_tan[i] = nan;
    }
    if (g.s1_dtheta) { g.s1_dtheta[i] = nan; g.s1_dphi[i] = nan; g.s2_dtheta[i] = nan; g.s2_dphi[i] = nan; }
    return;
  }
  const pn_inputs& in = a.k.in;
  const double m1 = in.m1[i], m2 = in.m2[i], chi1 = in.chi1[i], chi2 = in.chi2[i];
  const Coef<double> c = make_coef(m1, m2, a.k.ctl.terms);
  const Coef<double> cf = fold_K(c);  // the forward kernel's coefficients, for a bitwise replay
  // Cotangent of the final state from the output cotangents.
  const double S1[3] = {o.S1x[i], o.S1y[i], o.S1z[i]}, S2[3] = {o.S2x[i], o.S2y[i], o.S2z[i]};
  const double L[3] = {o.Lx[i], o.Ly[i], o.Lz[i]};
  double lam[10];
  const pn_cotangents& gb = a.gbar;
  lam[0] = 0.0;
  lam[7] = gval(gb.Lx, i); lam[8] = gval(gb.Ly, i); lam[9] = gval(gb.Lz, i);
  lam[1] = gval(gb.S1x, i); lam[2] = gval(gb.S1y, i); lam[3] = gval(gb.S1z, i);
  lam[4] = gval(gb.S2x, i); lam[5] = gval(gb.S2y, i); lam[6] = gval(gb.S2z, i);
  const double n1 = sqrt(S1[0] * S1[0] + S1[1] * S1[1] + S1[2] * S1[2]);
  const double n2 = sqrt(S2[0] * S2[0] + S2[1] * S2[1] + S2[2] * S2[2]);
  const double nl = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
  const double g12 = gval(gb.dot_s1s2, i), gl1 = gval(gb.dot_ls1, i), gl2 = gval(gb.dot_ls2, i);
  if (g12 != 0.0) {  // d (a.b/(|a||b|)) / da = (b/|b| - d a/|a|) / |a|
    const double d = (S1[0] * S2[0] + S1[1] * S2[1] + S1[2] * S2[2]) / (n1 * n2);
    for (int k = 0; k < 3; k++) {
      lam[1 + k] += g12 * (S2[k] / n2 - d * S1[k] / n1) / n1;
      lam[4 + k] += g12 * (S1[k] / n1 - d * S2[k] / n2) / n2;
    }
  }
  if (gl1 != 0.0) {
    const double d = (L[0] * S1[0] + L[1] * S1[1] + L[2] * S1[2]) / (nl * n1);
    for (int k = 0; k < 3; k++) {
      lam[7 + k] += gl1 * (S1[k] / n1 - d * L[k] / nl) / nl;
      lam[1 + k] += gl1 * (L[k] / nl - d * S1[k] / n1) / n1;
    }
  }
  if (gl2 != 0.0) {
    const double d = (L[0] * S2[0] + L[1] * S2[1] + L[2] * S2[2]) / (nl * n2);
    for (int k = 0; k < 3; k++) {
      lam[7 + k] += gl2 * (S2[k] / n2 - d * L[k] / nl) / nl;
      lam[4 + k] += gl2 * (L[k] / nl - d * S2[k] / n2) / n2;
    }
  }
  const double tbar = gval(gb.t, i);
  Coef<double> cb;
  double* cbv = &cb.K;
  for (int f = 0; f < 16; f++) cbv[f] = 0.0;

  const int32_t every = a.every;
  const int32_t nseg = (N + every - 1) / every;
  const size_t step_words = (size_t)(DS ? kAdjStepWordsDS : kAdjStepWordsF64) * ss;
  if constexpr (DS) {
    const Coef<ds> cd = to_ds(c);
    Coef<ds> cbd;
    ds* cbdv = &cbd.K;
    for (int f = 0; f < 16; f++) cbdv[f] = dzero();
    ds lamd[10];
    for (int k = 0; k < 10; k++) lamd[k] = split64(lam[k]);
    float2* sf0 = reinterpret_cast<float2*>(sp0);
#pragma unroll 1
    for (int32_t seg = nseg - 1; seg >= 0; seg--) {
      const int32_t n0 = seg * every;
      const int32_t n1s = (n0 + every < N) ? n0 + every : N;
      double y[10];
      for (int k = 0; k < 10; k++) y[k] = a.ck[((size_t)seg * 10 + k) * a.stride + i];
#pragma unroll 1
      for (int32_t n = n0; n < n1s; n++) {
        double y5[10];
        const bool more = n + 1 < n1s;
        dp5_stages_ds(cd, tabf, y, a.h[(size_t)n * a.stride + i], sf0 + (size_t)(n - n0) * step_words, ss,
                      more ? y5 : nullptr, RateWorkDs{static_cast<ulonglong2*>(rw)});
        if (more)
          for (int k = 0; k < 10; k++) y[k] = y5[k];
      }
#pragma unroll 1
      for (int32_t n = n1s - 1; n >= n0; n--) {
        const float2* sp = sf0 + (size_t)(n - n0) * step_words;
        const double hn = a.h[(size_t)n * a.stride + i];
        if (n == N - 1) {  // landing step: implicit h*
          Coef<ds> cA, cB;
          ds* av = &cA.K;
          ds* bv = &cB.K;
          for (int f = 0; f < 16; f++) { av[f] = dzero(); bv[f] = dzero(); }
          ds lA[10];
          for (int k = 0; k < 10; k++) lA[k] = dzero();
          lA[0] = ds_of(1.0f);
          const double nu = dp5_step_vjp_ds(cd, tabf, sp, ss, hn, lA, cA, RateWorkDs{static_cast<ulonglong2*>(rw)});
          const double mu = dp5_step_vjp_ds(cd, tabf, sp, ss, hn, lamd, cB, RateWorkDs{static_cast<ulonglong2*>(rw)}) + tbar;
          const ds ratio = split64(mu / nu);
          for (int k = 0; k < 10; k++) lamd[k] = ds_sub(lamd[k], ds_mul(ratio, lA[k]));
          for (int f = 0; f < 16; f++) cbdv[f] = ds_add(cbdv[f], ds_sub(bv[f], ds_mul(ratio, av[f])));
        } else {
          (void)dp5_step_vjp_ds(cd, tabf, sp, ss, hn, lamd, cbd, RateWorkDs{static_cast<ulonglong2*>(rw)});
        }
      }
    }
    for (int k = 0; k < 10; k++) lam[k] = ds_to_f64(lamd[k]);
    for (int f = 0; f < 16; f++) cbv[f] = ds_to_f64(cbdv[f]);
  } else {
#pragma unroll 1
  for (int32_t seg = nseg - 1; seg >= 0; seg--) {    const int32_t n0 = seg * every;
    const int32_t n1s = (n0 + every < N) ? n0 + every : N;
    double y[10];
    for (int k = 0; k < 10; k++) y[k] = a.ck[((size_t)seg * 10 + k) * a.stride + i];
#pragma unroll 1
    for (int32_t n = n0; n < n1s; n++) {  // recompute the segment, keeping the stage states
      double y5[10];
      const bool more = n + 1 < n1s;
      dp5_stages(cf, tabf, y, a.h[(size_t)n * a.stride + i], sp0 + (size_t)(n - n0) * step_words, ss,
                 more ? y5 : nullptr);
      if (more)
        for (int k = 0; k < 10; k++) y[k] = y5[k];
    }
#pragma unroll 1
    for (int32_t n = n1s - 1; n >= n0; n--) {
      const double* sp = sp0 + (size_t)(n - n0) * step_words;
      // stage 5 of the step reversed next (in this segment), prefetched during this one
      const double* pf = n > n0 ? sp - step_words + (size_t)(5 * kF64StageWords) * ss : nullptr;
      const double hn = a.h[(size_t)n * a.stride + i];
      if (n == N - 1) {  // landing step: implicit h*
        Coef<double> cA, cB;
        double* av = &cA.K;
        double* bv = &cB.K;
        for (int f = 0; f < 16; f++) { av[f] = 0.0; bv[f] = 0.0; }
        double lA[10];
        for (int k = 0; k < 10; k++) lA[k] = 0.0;
        lA[0] = 1.0;
        const double nu = dp5_step_vjp(cf, sp, ss, hn, lA, cA, sp + (size_t)(5 * kF64StageWords) * ss);
        const double mu = dp5_step_vjp(cf, sp, ss, hn, lam, cB, pf) + tbar;
        const double ratio = mu / nu;
        for (int k = 0; k < 10; k++) lam[k] -= ratio * lA[k];
        for (int f = 0; f < 16; f++) cbv[f] += bv[f] - ratio * av[f];
      } else {
        (void)dp5_step_vjp(cf, sp, ss, hn, lam, cb, pf);
      }
    }
  }
  unfold_cotangents(c, cb);  // the FP64 sweep's cotangents are the folded coefficients'
  }
  // Initial state S_i = chi_i m_i^2 S_i-hat, and the mass ratio q = m1/m2 (M = 1).
  const double s1[3] = {in.s1x[i], in.s1y[i], in.s1z[i]}, s2[3] = {in.s2x[i], in.s2y[i], in.s2z[i]};
  const double f1 = chi1 * (m1 * m1), f2 = chi2 * (m2 * m2);
  const double gs1[3] = {f1 * lam[1], f1 * lam[2], f1 * lam[3]}, gs2[3] = {f2 * lam[4], f2 * lam[5], f2 * lam[6]};
  g.s1x[i] = gs1[0]; g.s1y[i] = gs1[1]; g.s1z[i] = gs1[2];
  g.s2x[i] = gs2[0]; g.s2y[i] = gs2[1]; g.s2z[i] = gs2[2];
  if (g.s1x_tan) {  // g - (g . s) s / |s|^2 on each sphere
    const double c1 = (gs1[0] * s1[0] + gs1[1] * s1[1] + gs1[2] * s1[2]) /
                      (s1[0] * s1[0] + s1[1] * s1[1] + s1[2] * s1[2]);
    const double c2 = (gs2[0] * s2[0] + gs2[1] * s2[1] + gs2[2] * s2[2]) /
                      (s2[0] * s2[0] + s2[1] * s2[1] + s2[2] * s2[2]);
    g.s1x_tan[i] = gs1[0] - c1 * s1[0]; g.s1y_tan[i] = gs1[1] - c1 * s1[1]; g.s1z_tan[i] = gs1[2] - c1 * s1[2];
    g.s2x_tan[i] = gs2[0] - c2 * s2[0]; g.s2y_tan[i] = gs2[1] - c2 * s2[1]; g.s2z_tan[i] = gs2[2] - c2 * s2[2];
  }
  if (g.s1_dtheta) {  // d/dt and d/dp of s = |s| (sin t cos p, sin t sin p, cos t), |s| fixed
    double dt1, dp1, dt2, dp2;
    angle_grads(gs1, s1, &dt1, &dp1);
    angle_grads(gs2, s2, &dt2, &dp2);
    g.s1_dtheta[i] = dt1; g.s1_dphi[i] = dp1; g.s2_dtheta[i] = dt2; g.s2_dphi[i] = dp2;
  }
  double m1b = 2.0 * chi1 * m1 * (lam[1] * s1[0] + lam[2] * s1[1] + lam[3] * s1[2]);
  double m2b = 2.0 * chi2 * m2 * (lam[4] * s2[0] + lam[5] * s2[1] + lam[6] * s2[2]);
  coef_vjp(cb, m1, m2, a.k.ctl.terms, &m1b, &m2b);
  g.q[i] = (m1b - m2b) * (m2 * m2);  // dm1/dq = m2^2 = -dm2/dq
}

#ifdef PN_DEBUG
// The launch's dynamic shared memory in bytes (the debug build's checks).
__device__ __forceinline__ size_t adj_dynamic_smem_bytes() {
  unsigned int b;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(b));
  return b;
}
#endif

// Persistent sweep: each warp claims 32 consecutive entries of the order.
// blockDim.x must be a multiple of 32.  DS: the double-single sweep.
template <bool DS>
__global__ void __launch_bounds__(128) k_adjoint(const AdjArgs a) {
  __shared__ float s_tabf[512];
  extern __shared__ __align__(16) ulonglong2 s_rate[];  // double-single sweep: kAdjWorkBytes per thread
  for (int q = threadIdx.x; q < 512; q += blockDim.x) s_tabf[q] = a.k.tabf[q];
  __syncthreads();
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  // Debug builds: the segment buffer has a column for every lane of the warp,
  // and the launch's dynamic shared memory every lane's rate workspace; a
  // failure returns whole warps (the loop below shuffles across the warp).
  if (!PN_DCHECK(__all_sync(0xffffffffu, slot < a.seg_stride), 22)) return;
  if (DS && !PN_DCHECK((size_t)blockDim.x * kAdjWorkBytes <= adj_dynamic_smem_bytes(), 23)) return;
  double* sp0 = a.seg + slot;
  void* const rw = DS ? static_cast<void*>(warp_tile_base<ulonglong2, kAdjWorkBytes / 16>(s_rate)) : nullptr;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.k.queue, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)a.k.n) break;
    const int64_t p = (int64_t)base + lane;
    if (p < a.k.n) {
      const int64_t i = a.order[p];
      if (PN_DCHECK(i >= 0 && i < a.k.n, 21)) adjoint_one<DS>(a, s_tabf, i, sp0, (size_t)a.seg_stride, rw);
    }
  }
}

}  // namespace

cudaError_t launch_adjoint(const AdjArgs& a, int block, int grid, cudaStream_t s) {
  if (grid <= 0 || a.k.n <= 0) return cudaSuccess;
  const int32_t nb = a.cap + 1;
  const unsigned eg = (unsigned)((a.k.n + 255) / 256);
  cudaError_t e = cudaMemsetAsync(a.bins, 0, (size_t)nb * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_order_count<<<eg, 256, 0, s>>>(a.k.out, a.k.n, a.cap, a.bins);
  e = launch_scan_above(a.bins, nb, s);
  if (e != cudaSuccess) return e;
  k_order_scatter<<<eg, 256, 0, s>>>(a.k.out, a.k.n, a.cap, a.bins, a.order);
  e = cudaMemsetAsync(a.k.queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const size_t smem = a.ds ? (size_t)kAdjWorkBytes * block : 0;
  e = cudaFuncSetAttribute(a.ds ? (const void*)k_adjoint<true> : (const void*)k_adjoint<false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (a.ds) k_adjoint<true><<<grid, block, smem, s>>>(a);
  else k_adjoint<false><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t adjoint_occupancy(bool ds, int block, int* blocks_per_sm) {
  const void* f = ds ? (const void*)k_adjoint<true> : (const void*)k_adjoint<false>;
  const size_t smem = ds ? (size_t)kAdjWorkBytes * block : 0;
  const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

#ifdef PN_DEBUG
cudaError_t debug_take_adjoint(unsigned int* site) { return debug_take_local(site); }
#else
cudaError_t debug_take_adjoint(unsigned int* site) {
  *site = 0u;
  return cudaSuccess;
}
#endif

}  // namespace pn
