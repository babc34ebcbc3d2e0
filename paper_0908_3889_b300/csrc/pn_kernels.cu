// pn_kernels.cu -- CUDA kernels of the batched PN inspiral integrator (sm_103a).
//
// k_integrate_mx / k_integrate: one binary per lane, state in registers, one Dormand-Prince
// attempt per loop iteration for every lane that holds a binary, so a warp
// stays converged on the RHS-heavy part whatever each lane's step history.
// The per-lane control is a small state machine (STEP / LAND) that takes the
// decisions of arXiv:0908.3889 Sec. II's integrator as read here: error
// control at tolerance rtol = atol = 5e-7 with first step h0 = 10, and the stop
// at omega_f by retaking the crossing step.  Two schedules share the code:
//   plain       thread g integrates binary g (grid covers n);
//   persistent  a grid sized to the resident capacity; a lane that finishes
//               claims the next binary from a device counter, with one
//               atomicAdd per warp (ballot + popc), so binaries of very
//               different lengths do not leave lanes idle.
// Inputs and outputs are structure-of-arrays: lane i touches element i of
// each array, so every load and store of a warp is one coalesced 256-byte
// transaction.  All three precisions keep their stage rates in a per-thread
// shared-memory workspace (k_integrate_mx; k_integrate is the adjoint's recording
// pass, FP64 or double-single), so their stage loops stay small: one
// right-hand-side copy.

#include <cmath>

#include "pn_debug.h"
#include "pn_internal.h"

namespace pn {

struct Lane {
  int64_t i;
  double y[10];
  double k1[10];  // f(y), carried across accepted steps (first same as last)
  double t, h, h_lo, h_hi, wf;
  int32_t n_acc, n_rej, n_land, attempts, land_it;
  int32_t stop_at;  // attempts count at which this launch's budget runs out
  bool landing, last_rej;
  Coefs cf;
};

// Shared-memory copies of the logarithm tables the kernel's precision needs.
template <int PREC>
__device__ __forceinline__ Tabs load_tabs(const float* __restrict__ g, float* s_tabf) {
  if constexpr (PREC == 0 || PREC == 2) {
    for (int q = threadIdx.x; q < 512; q += blockDim.x) s_tabf[q] = g[q];
  }
  __syncthreads();
  return Tabs{s_tabf};
}

// Final state, time, counters and status of binary i.  The scalar products are
// filled in afterwards by k_dots, a converged pass over all binaries, so the
// integration kernel spends no FP64 work on them in divergent code.
__device__ __forceinline__ void write_result(const pn_outputs& o, int64_t i, const double* y, double t, int32_t n_acc,
                                             int32_t n_rej, int32_t n_land, int32_t status) {
  o.S1x[i] = y[1]; o.S1y[i] = y[2]; o.S1z[i] = y[3];
  o.S2x[i] = y[4]; o.S2y[i] = y[5]; o.S2z[i] = y[6];
  o.Lx[i] = y[7]; o.Ly[i] = y[8]; o.Lz[i] = y[9];
  o.omega[i] = y[0];
  o.t[i] = t;
  o.n_acc[i] = n_acc; o.n_rej[i] = n_rej; o.n_land[i] = n_land; o.status[i] = status;
}

// The output epilogue, a converged pass over all binaries.  First the final move
// of a binary that landed on omega_f: the integration kernel leaves the retaken
// state y5 and t + h in the outputs and f(y5), dh = -(omega - omega_f)/(domega/dt)
// in land (fields 0..9, 10); here y += dh f(y5), t += dh, and dh is cleared (so
// a later bounded call's epilogue does not move it again).  Doing this here
// rather than in the kernel's landing branch, which usually holds one lane of
// the warp, keeps its eleven FP64 operations out of divergent code.
// Then Sec. V's scalar products of the final unit vectors, S1-hat.S2-hat,
// L-hat.S1-hat, L-hat.S2-hat (NaN for a zero spin: 0/0; NaN for BAD_INPUT binaries).
__global__ void __launch_bounds__(256) k_dots(const pn_outputs o, int64_t n, double* __restrict__ land,
                                              int64_t stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dh = land[(size_t)10 * stride + i];
  if (dh != 0.0) {
    double* const yo[10] = {o.omega, o.S1x, o.S1y, o.S1z, o.S2x, o.S2y, o.S2z, o.Lx, o.Ly, o.Lz};
#pragma unroll
    for (int c = 0; c < 10; c++) yo[c][i] = fma(dh, land[(size_t)c * stride + i], yo[c][i]);
    o.t[i] = o.t[i] + dh;
    land[(size_t)10 * stride + i] = 0.0;
  }
  const double a0 = o.S1x[i], a1 = o.S1y[i], a2 = o.S1z[i];
  const double b0 = o.S2x[i], b1 = o.S2y[i], b2 = o.S2z[i];
  const double l0 = o.Lx[i], l1 = o.Ly[i], l2 = o.Lz[i];
  const double n1 = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
  const double n2 = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
  const double nl = sqrt(l0 * l0 + l1 * l1 + l2 * l2);
  o.dot_s1s2[i] = (a0 * b0 + a1 * b1 + a2 * b2) / (n1 * n2);
  o.dot_ls1[i] = (l0 * a0 + l1 * a1 + l2 * a2) / (nl * n1);
  o.dot_ls2[i] = (l0 * b0 + l1 * b1 + l2 * b2) / (nl * n2);
}

// Per-binary set-up table (structure of arrays, `stride` doubles per field):
// fields 0..15 the coefficients, 16..25 the initial state y0, 26..35 k1 = f(y0)
// in the kernel's precision, 36 omega_f (NaN marks a binary whose BAD_INPUT
// result is already written).  k_setup fills it with one converged pass, so a
// lane that picks up a new binary in the integration kernel only loads.  The
// kLandFields fields after them hold the deferred landing moves (k_dots).
// kSetupFields (pn_internal.h) counts the fields before them.

__device__ __forceinline__ double* fld(double* ws, int64_t stride, int f) { return ws + (size_t)f * stride; }

// f(y) of Eqs. (1)-(4) at n given states, in the precision PREC, with the
// coefficients from (m1[i], m2[i]) (pn_batch_eval_rhs).
template <int PREC>
__global__ void __launch_bounds__(256) k_eval_rhs(int64_t n, const double* __restrict__ m1,
                                                  const double* __restrict__ m2, const double* __restrict__ y,
                                                  double* __restrict__ f, const float* __restrict__ tab, TermCfg tc) {
  __shared__ float s_tabf[512];
  const Tabs tb = load_tabs<PREC>(tab, s_tabf);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Coefs cf;
  cf.c64 = make_coef(m1[i], m2[i], tc);
  if constexpr (PREC == 0) cf.c64 = fold_K(cf.c64);
  if constexpr (PREC == 1) cf.c32 = to_f32(cf.c64);
  if constexpr (PREC == 2) cf.cds = to_ds(cf.c64);
  double yy[10], k[10];
#pragma unroll
  for (int c = 0; c < 10; c++) yy[c] = y[(size_t)c * n + i];
  eval_rhs<PREC>(cf, tb, yy, k);
#pragma unroll
  for (int c = 0; c < 10; c++) f[(size_t)c * n + i] = k[c];
}

template <int PREC>
__global__ void __launch_bounds__(256) k_setup(const KArgs a, double* __restrict__ ws, int64_t stride) {
  __shared__ float s_tabf[512];
  const Tabs tb = load_tabs<PREC>(a.tabf, s_tabf);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  ws[(size_t)(kSetupFields + 10) * stride + i] = 0.0;  // no deferred landing move yet
  const pn_inputs& in = a.in;
  const double m1 = in.m1[i], m2 = in.m2[i], chi1 = in.chi1[i], chi2 = in.chi2[i];
  const double s1x = in.s1x[i], s1y = in.s1y[i], s1z = in.s1z[i];
  const double s2x = in.s2x[i], s2y = in.s2y[i], s2z = in.s2z[i];
  const double lx = in.lx[i], ly = in.ly[i], lz = in.lz[i];
  const double w0 = in.omega0[i], wf = in.omega_f[i];
  // Validation of PN_ST_BAD_INPUT (same conditions as the header states).
  bool ok = finite64(m1) && finite64(m2) && finite64(chi1) && finite64(chi2) && finite64(s1x) && finite64(s1y) &&
            finite64(s1z) && finite64(s2x) && finite64(s2y) && finite64(s2z) && finite64(lx) && finite64(ly) &&
            finite64(lz) && finite64(w0) && finite64(wf);
  ok = ok && m1 > 0.0 && m2 > 0.0 && fabs(m1 + m2 - 1.0) <= 1e-12;
  ok = ok && chi1 >= 0.0 && chi1 <= 1.0 && chi2 >= 0.0 && chi2 <= 1.0;
  ok = ok && w0 > 0.0 && wf > w0;
  ok = ok && fabs(sqrt(lx * lx + ly * ly + lz * lz) - 1.0) <= 1e-12;
  if (!ok) {
    double y[10];
    for (int c = 0; c < 10; c++) y[c] = dnan();
    write_result(a.out, i, y, dnan(), 0, 0, 0, PN_ST_BAD_INPUT);
    fld(ws, stride, 36)[i] = dnan();
    return;
  }
  Coefs cf;
  cf.c64 = make_coef(m1, m2, a.ctl.terms);
  if constexpr (PREC == 0) cf.c64 = fold_K(cf.c64);  // the FP64 kernels' right-hand side takes P_K
  if constexpr (PREC == 1) cf.c32 = to_f32(cf.c64);
  if constexpr (PREC == 2) cf.cds = to_ds(cf.c64);
  const Coef<double>& c = cf.c64;
  // Initial state (Secs. II, V): omega_0, S_i = chi_i m_i^2 S_i-hat, L-hat(0).
  double y[10], k[10];
  y[0] = w0;
  y[1] = chi1 * (m1 * m1) * s1x; y[2] = chi1 * (m1 * m1) * s1y; y[3] = chi1 * (m1 * m1) * s1z;
  y[4] = chi2 * (m2 * m2) * s2x; y[5] = chi2 * (m2 * m2) * s2y; y[6] = chi2 * (m2 * m2) * s2z;
  y[7] = lx; y[8] = ly; y[9] = lz;
  eval_rhs<PREC>(cf, tb, y, k);
  const double* cv = &c.K;
#pragma unroll
  for (int f = 0; f < 16; f++) fld(ws, stride, f)[i] = cv[f];
#pragma unroll
  for (int f = 0; f < 10; f++) {
    fld(ws, stride, 16 + f)[i] = y[f];
    fld(ws, stride, 26 + f)[i] = k[f];
  }
  fld(ws, stride, 36)[i] = wf;
}

// Pick up binary i: its coefficients from the set-up table and its state either
// from the set-up table (a fresh start) or, in a resumed launch, from the saved
// state of a binary left PN_ST_RUNNING.  Returns false if there is nothing to
// do for it (invalid input already written, or not running in a resume).
template <int PREC, bool BOUNDED>
__device__ __forceinline__ bool lane_load(Lane& L, const KArgs& a, const double* __restrict__ ws, int64_t stride,
                                          int64_t i) {
  if (BOUNDED && a.resume && a.out.status[i] != PN_ST_RUNNING) return false;
  const double wf = ws[(size_t)36 * stride + i];
  if (!finite64(wf)) return false;
  L.i = i;
  double* cv = &L.cf.c64.K;
#pragma unroll
  for (int f = 0; f < 16; f++) cv[f] = ws[(size_t)f * stride + i];
  if constexpr (PREC == 1) L.cf.c32 = to_f32(L.cf.c64);
  if constexpr (PREC == 2) L.cf.cds = to_ds(L.cf.c64);
  L.wf = wf;
  if (BOUNDED && a.resume) {
    const size_t rst = (size_t)a.rs_stride;
#pragma unroll
    for (int f = 0; f < 10; f++) {
      L.y[f] = a.rs[f * rst + i];
      L.k1[f] = a.rs[(10 + f) * rst + i];
    }
    L.t = a.rs[20 * rst + i];
    L.h = a.rs[21 * rst + i];
    L.h_lo = a.rs[22 * rst + i];
    L.h_hi = a.rs[23 * rst + i];
    L.n_acc = a.ri[0 * rst + i];
    L.n_rej = a.ri[1 * rst + i];
    L.n_land = a.ri[2 * rst + i];
    L.attempts = a.ri[3 * rst + i];
    L.land_it = a.ri[4 * rst + i];
    const int32_t fl = a.ri[5 * rst + i];
    L.landing = (fl & 1) != 0;
    L.last_rej = (fl & 2) != 0;
  } else {
#pragma unroll
    for (int f = 0; f < 10; f++) {
      L.y[f] = ws[(size_t)(16 + f) * stride + i];
      L.k1[f] = ws[(size_t)(26 + f) * stride + i];
    }
    L.t = 0.0;
    L.h = a.ctl.h0;
    L.h_lo = 0.0;
    L.h_hi = 0.0;
    L.n_acc = L.n_rej = L.n_land = L.attempts = L.land_it = 0;
    L.landing = false;
    L.last_rej = false;
  }
  if constexpr (BOUNDED)
    L.stop_at = (a.budget > 0 && L.attempts <= 0x7fffffff - a.budget) ? L.attempts + a.budget : 0x7fffffff;
  return true;
}

// Keep the state of a binary whose launch budget ran out, and report it as
// running (its current state in the outputs).
__device__ __forceinline__ void lane_save(const KArgs& a, const Lane& L) {
  const size_t rst = (size_t)a.rs_stride;
  const int64_t i = L.i;
#pragma unroll
  for (int f = 0; f < 10; f++) {
    a.rs[f * rst + i] = L.y[f];
    a.rs[(10 + f) * rst + i] = L.k1[f];
  }
  a.rs[20 * rst + i] = L.t;
  a.rs[21 * rst + i] = L.h;
  a.rs[22 * rst + i] = L.h_lo;
  a.rs[23 * rst + i] = L.h_hi;
  a.ri[0 * rst + i] = L.n_acc;
  a.ri[1 * rst + i] = L.n_rej;
  a.ri[2 * rst + i] = L.n_land;
  a.ri[3 * rst + i] = L.attempts;
  a.ri[4 * rst + i] = L.land_it;
  a.ri[5 * rst + i] = (L.landing ? 1 : 0) | (L.last_rej ? 2 : 0);
  write_result(a.out, i, L.y, L.t, L.n_acc, L.n_rej, L.n_land, PN_ST_RUNNING);
}

// Recording of the accepted steps for the adjoint: h[n * stride + i] is the
// size of accepted step n (the landing step last) and ck[(c * 10 + k) * stride + i]
// component k of the state after c * every accepted steps (c = 0 is the
// initial state).  Steps beyond cap set *overflow and are not recorded.
__device__ __forceinline__ void record_commit(const RecArgs& rec, const Lane& L, double hc) {
  const int32_t n = L.n_acc - 1;  // index of the step just committed
  if (n < rec.cap) rec.h[(size_t)n * rec.stride + L.i] = hc;
  else *rec.overflow = 1;
  if (L.n_acc % rec.every == 0) {
    const int32_t c = L.n_acc / rec.every;
    if (c <= rec.cap / rec.every)
#pragma unroll
      for (int k = 0; k < 10; k++) rec.ck[((size_t)c * 10 + k) * rec.stride + L.i] = L.y[k];
  }
}

template <bool RECORD>
__device__ __forceinline__ void lane_commit(Lane& L, const double* y5, double hc, const RecArgs& rec) {
  L.t = L.t + hc;
#pragma unroll
  for (int c = 0; c < 10; c++) L.y[c] = y5[c];
  L.n_acc++;
  if constexpr (RECORD) record_commit(rec, L, hc);
}

// The landing step: commit the retake (t advances by h) and leave its final move
// dh along f(y5) to the output epilogue (k_dots); the recording pass records the
// step as h + dh.
template <bool RECORD>
__device__ __forceinline__ void lane_land(Lane& L, const double* y5, const double* k7, double dh, double* land,
                                          int64_t stride, const RecArgs& rec) {
#pragma unroll
  for (int c = 0; c < 10; c++) land[(size_t)c * stride + L.i] = k7[c];
  land[(size_t)10 * stride + L.i] = dh;
  L.t = L.t + L.h;
#pragma unroll
  for (int c = 0; c < 10; c++) L.y[c] = y5[c];
  L.n_acc++;
  if constexpr (RECORD) record_commit(rec, L, L.h + dh);
}

// Decisions after one attempt (y5, k7 = f(y5), s = err^2).  Returns true when
// the binary is finished, with its status in *status.
// lo < h < hi for a bracket with 0 <= lo < hi (integer comparison of the bit
// patterns, which order like the values there; a negative or NaN h is outside).
__device__ __forceinline__ bool in_bracket(double h, double lo, double hi) {
  const long long b = __double_as_longlong(h);
  return b > __double_as_longlong(lo) && b < __double_as_longlong(hi);
}

// Comparisons of doubles below are integer comparisons of the bit patterns (the
// operands are finite here, and the FP64 compare would take an FP64-pipe slot).
template <bool RECORD>
__device__ __forceinline__ bool lane_decide(Lane& L, const Ctl& ctl, double* y5, const double* k7, double s,
                                            int32_t* status, const RecArgs& rec, double* land, int64_t stride) {
  bool fin = ctl.fixed_step ? true : finite64(s);
#pragma unroll
  for (int c = 0; c < 10; c++) fin = fin && finite64(y5[c]);
  if (!fin) { *status = PN_ST_NONFINITE; return true; }
  const double tolw = ctl.land_tol * L.wf;
  // Growth factor for the next step, computed by every lane of the warp at once
  // (accepted: at most fac_max, or 1 right after a rejection; rejected: at most 1).
  const bool accepted = ctl.fixed_step || le_pos(s, 1.0);
  const double fac = step_factor(ctl, s, (accepted && !L.last_rej) ? ctl.fac_max : 1.0);
  const double rk7 = rcp_pos(k7[0]);  // 1 / (domega/dt) at y5

  if (L.landing) {
    L.n_land++;
    L.land_it++;
    const double g = y5[0] - L.wf;
    if (le_pos(dabs(g), tolw)) {  // converged: move onto omega_f along f (in the epilogue)
      lane_land<RECORD>(L, y5, k7, -g * rk7, land, stride, rec);
      *status = PN_ST_OK;
      return true;
    }
    if (L.land_it >= ctl.land_max_iter || L.attempts >= ctl.max_steps) {
      lane_commit<RECORD>(L, y5, L.h, rec);
      *status = (L.attempts >= ctl.max_steps) ? PN_ST_MAX_STEPS : PN_ST_LAND_MAXIT;
      return true;
    }
    if (__double_as_longlong(g) > 0) L.h_hi = L.h; else L.h_lo = L.h;
    double hn = fma(-g, rk7, L.h);
    if (!in_bracket(hn, L.h_lo, L.h_hi)) hn = 0.5 * (L.h_lo + L.h_hi);
    L.h = hn;
    return false;
  }

  if (accepted) {
    if (__double_as_longlong(y5[0]) >= __double_as_longlong(L.wf)) {
      const double g = y5[0] - L.wf;
      if (ctl.stop_mode == PN_STOP_FIRST_CROSS) {
        lane_commit<RECORD>(L, y5, L.h, rec);
        *status = PN_ST_OK;
        return true;
      }
      if (le_pos(dabs(g), tolw)) {
        lane_land<RECORD>(L, y5, k7, -g * rk7, land, stride, rec);
        *status = PN_ST_OK;
        return true;
      }
      // Retake the crossing step, seeded by the root of its Hermite cubic.
      L.landing = true;
      L.land_it = 0;
      L.h_lo = 0.0;
      L.h_hi = L.h;
      const double hn = hermite_step_ds(L.h, L.y[0], L.k1[0], y5[0], k7[0], L.wf);
      L.h = in_bracket(hn, L.h_lo, L.h_hi) ? hn : 0.5 * (L.h_lo + L.h_hi);
    } else {
      lane_commit<RECORD>(L, y5, L.h, rec);
#pragma unroll
      for (int c = 0; c < 10; c++) L.k1[c] = k7[c];
      if (!ctl.fixed_step) L.h = L.h * fac;
      L.last_rej = false;
    }
  } else {
    L.n_rej++;
    L.h = L.h * fac;
    L.last_rej = true;
    if (__double_as_longlong(L.h) < __double_as_longlong(ctl.h_min)) { *status = PN_ST_H_UNDERFLOW; return true; }
  }
  if (L.attempts >= ctl.max_steps) { *status = PN_ST_MAX_STEPS; return true; }
  return false;
}

// BOUNDED: the launch may stop binaries at a per-launch attempt budget and may
// resume saved ones (pn_batch_integrate_budget / pn_batch_resume); the default
// launches are compiled without that bookkeeping.
// Per-thread bytes of the stage workspace of the integration kernels.
template <int PREC>
__device__ __forceinline__ constexpr size_t work_bytes() {
  return PREC == 2 ? (size_t)kDsWorkBytes : (PREC == 1 ? (size_t)kF32WorkBytes : (size_t)kF64WorkBytes);
}
#ifdef PN_DEBUG
// The launch's dynamic shared memory in bytes (the debug build's checks).
__device__ __forceinline__ size_t dynamic_smem_bytes() {
  unsigned int b;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(b));
  return b;
}
#endif

template <int PREC, bool PERSIST, bool RECORD, bool BOUNDED, bool WS>
__device__ __forceinline__ void integrate_body(const KArgs& a, const double* __restrict__ ws, int64_t stride,
                                               const RecArgs& rec) {
  __shared__ float s_tabf[512];
  extern __shared__ __align__(16) float2 s_dsw[];  // per-thread stage workspace (PREC 0: kF64WorkBytes, 1: kF32WorkBytes, 2: kDsWorkBytes)
  const Tabs tb = load_tabs<PREC>(a.tabf, s_tabf);
  // Debug builds: the launch's dynamic shared memory holds every lane's stage
  // workspace (the same outcome for the whole block, after its one barrier).
  if (!PN_DCHECK((size_t)blockDim.x * work_bytes<PREC>() <= dynamic_smem_bytes(), 1)) return;

  const unsigned lane = threadIdx.x & 31u;
  Lane L;
  bool have = false, exhausted = false;
  // Plain schedule: thread g takes binaries g, g + T, ..., g + (bpt - 1) T in turn
  // (T = threads in the grid), so every round of a warp reads consecutive binaries.
  const int32_t bpt = a.bpt > 1 ? a.bpt : 1;
  int32_t taken = 0;
  for (;;) {
    const bool need = !have && !exhausted;
    int64_t idx = -1;
    if constexpr (PERSIST) {
      const unsigned m = __ballot_sync(0xffffffffu, need);
      if (m != 0u) {
        const int leader = __ffs((int)m) - 1;
        unsigned long long base = 0ull;
        if ((int)lane == leader) base = atomicAdd(a.queue, (unsigned long long)__popc((int)m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need) idx = (int64_t)(base + (unsigned long long)__popc((int)(m & ((1u << lane) - 1u))));
      }
    } else {
      if (need) {
        idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + (int64_t)taken * gridDim.x * blockDim.x;
        taken++;
      }
    }
    if (need) {
      if (idx >= 0 && idx < a.n) {
        const int64_t bi = a.order ? a.order[idx] : idx;  // the binary this lane takes
        if (PN_DCHECK(bi >= 0 && bi < a.n, 2)) have = lane_load<PREC, BOUNDED>(L, a, ws, stride, bi);
        if (RECORD && have)
#pragma unroll
          for (int c = 0; c < 10; c++) rec.ck[(size_t)c * rec.stride + bi] = L.y[c];
      }
      if ((!PERSIST && taken >= bpt) || idx >= a.n) exhausted = true;
    }
    if (__all_sync(0xffffffffu, !have && exhausted)) break;
    if (have) {
      double y5[10], k7[10];
      double s;
      if constexpr (PREC == 2)
        s = dp5_attempt_ds(L.cf, tb, a.ctl, L.y, L.k1, L.h, y5, k7,
                           DsWork{warp_tile_base<ulonglong2, kDsVectors * 5>(s_dsw)});
      else if constexpr (PREC == 1)
        s = dp5_attempt_f32(L.cf.c32, a.ctl, L.y, L.k1, L.h, y5, k7,
                            F32Work{warp_tile_base<f2, kF32WorkBytes / 8>(s_dsw)});
      else
        s = dp5_attempt_ws(L.cf, tb, a.ctl, L.y, L.k1, L.h, y5, k7,
                           F64Work{warp_tile_base<double, kF64WorkBytes / 8>(s_dsw)});
      L.attempts++;
      int32_t st;
      if (lane_decide<RECORD>(L, a.ctl, y5, k7, s, &st, rec, a.land, stride)) {
        write_result(a.out, L.i, L.y, L.t, L.n_acc, L.n_rej, L.n_land, st);
        have = false;
      } else if (BOUNDED && L.attempts >= L.stop_at) {
        lane_save(a, L);
        have = false;
      }
    }
  }
}

// The recording pass of the adjoint (persistent, RECORD): PREC 0 the FP64
// attempt, PREC 2 the double-single one, each with its rates in the dynamic
// shared-memory workspace as in k_integrate_mx<PREC>.
template <int PREC, bool PERSIST, bool RECORD = false, bool BOUNDED = false>
__global__ void __launch_bounds__(kMaxBlock) k_integrate(const KArgs a, const double* __restrict__ ws, int64_t stride,
                                                         const RecArgs rec = RecArgs{}) {
  integrate_body<PREC, PERSIST, RECORD, BOUNDED, true>(a, ws, stride, rec);
}

// The integration kernels with their rates in a per-thread shared-memory
// workspace: PREC 0 FP64, PREC 1 FP32 right-hand side, PREC 2 double-single.
// The FP32-RHS kernels and the plain-schedule double-single kernel are held to
// 168 registers, three warps per scheduler (they are latency-bound, and measured
// faster so); the FP64 kernels and the persistent double-single kernel take up to
// 255 (two warps per scheduler), which measured faster for them.
constexpr int integrate_maxnreg(int prec, bool persist) {
  return prec == 1 ? 168 : (prec == 2 && !persist ? 168 : 255);
}
template <int PREC, bool PERSIST, bool BOUNDED = false>
__global__ void __maxnreg__(integrate_maxnreg(PREC, PERSIST)) k_integrate_mx(const KArgs a,
                                                                            const double* __restrict__ ws,
                                                                            int64_t stride) {
  integrate_body<PREC, PERSIST, false, BOUNDED, PREC == 0>(a, ws, stride, RecArgs{});
}

template <int PREC, bool PERSIST>
static const void* integrate_fn() {
  return (const void*)k_integrate_mx<PREC, PERSIST>;
}

static const void* pick(int prec, bool persistent) {
  if (prec == PN_MIXED) return persistent ? integrate_fn<1, true>() : integrate_fn<1, false>();
  if (prec == PN_MIXED_DS) return persistent ? integrate_fn<2, true>() : integrate_fn<2, false>();
  return persistent ? integrate_fn<0, true>() : integrate_fn<0, false>();
}

int setup_fields() { return kTableFields; }

cudaError_t launch_eval_rhs(int prec, int64_t n, const double* m1, const double* m2, const double* y, double* f,
                            const float* tab, TermCfg tc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (n + block - 1) / block;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  if (prec == PN_MIXED) k_eval_rhs<1><<<(unsigned)grid, block, 0, s>>>(n, m1, m2, y, f, tab, tc);
  else if (prec == PN_MIXED_DS) k_eval_rhs<2><<<(unsigned)grid, block, 0, s>>>(n, m1, m2, y, f, tab, tc);
  else k_eval_rhs<0><<<(unsigned)grid, block, 0, s>>>(n, m1, m2, y, f, tab, tc);
  return cudaGetLastError();
}

cudaError_t launch_setup(int prec, const KArgs& a, double* ws, int64_t stride, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = (unsigned)((a.n + block - 1) / block);
  if (prec == PN_MIXED) k_setup<1><<<grid, block, 0, s>>>(a, ws, stride);
  else if (prec == PN_MIXED_DS) k_setup<2><<<grid, block, 0, s>>>(a, ws, stride);
  else k_setup<0><<<grid, block, 0, s>>>(a, ws, stride);
  return cudaGetLastError();
}

// The deferred-landing fields of the set-up table ws (the same allocation,
// past the set-up fields the integration kernels read).
static double* land_fields(const double* ws, int64_t stride) {
  return const_cast<double*>(ws) + (size_t)kSetupFields * (size_t)stride;
}
static KArgs with_land(const KArgs& a, const double* ws, int64_t stride) {
  KArgs b = a;
  b.land = land_fields(ws, stride);
  return b;
}

cudaError_t launch_dots(const pn_outputs& o, int64_t n, const double* ws, int64_t stride, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_dots<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(o, n, land_fields(ws, stride), stride);
  return cudaGetLastError();
}

cudaError_t launch_integrate(int prec, bool persistent, int block, int grid, const KArgs& a, const double* ws,
                             int64_t stride, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  const cudaError_t e = launch_integrate_only(prec, persistent, block, grid, a, ws, stride, s);
  if (e != cudaSuccess) return e;
  return launch_dots(a.out, a.n, ws, stride, s);
}

// Dynamic shared memory of an integration launch: the double-single workspace.
static size_t integrate_smem(int prec, int block) {
  if (prec == PN_MIXED_DS) return (size_t)kDsWorkBytes * (size_t)block;
  if (prec == PN_MIXED) return (size_t)kF32WorkBytes * (size_t)block;
  return (size_t)kF64WorkBytes * (size_t)block;
}

cudaError_t prepare_integrate_kernels() {
  const void* ds[5] = {(const void*)k_integrate_mx<2, true>, (const void*)k_integrate_mx<2, false>,
                       (const void*)k_integrate_mx<2, true, true>, (const void*)k_integrate_mx<2, false, true>,
                       (const void*)k_integrate<2, true, true>};
  const void* f32[4] = {(const void*)k_integrate_mx<1, true>, (const void*)k_integrate_mx<1, false>,
                        (const void*)k_integrate_mx<1, true, true>, (const void*)k_integrate_mx<1, false, true>};
  for (const void* f : ds) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kDsWorkBytes * kMaxBlock);
    if (e != cudaSuccess) return e;
  }
  for (const void* f : f32) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kF32WorkBytes * kMaxBlock);
    if (e != cudaSuccess) return e;
  }
  const void* f64[5] = {(const void*)k_integrate_mx<0, true>, (const void*)k_integrate_mx<0, false>,
                        (const void*)k_integrate_mx<0, true, true>, (const void*)k_integrate_mx<0, false, true>,
                        (const void*)k_integrate<0, true, true>};
  for (const void* f : f64) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kF64WorkBytes * kMaxBlock);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool BOUNDED>
static void launch_integrate_variant(int prec, bool persistent, int block, int grid, const KArgs& a,
                                     const double* ws, int64_t stride, cudaStream_t s) {
  const size_t sm = integrate_smem(prec, block);
  if (prec == PN_MIXED) {
    if (persistent) k_integrate_mx<1, true, BOUNDED><<<grid, block, sm, s>>>(a, ws, stride);
    else k_integrate_mx<1, false, BOUNDED><<<grid, block, sm, s>>>(a, ws, stride);
  } else if (prec == PN_MIXED_DS) {
    if (persistent) k_integrate_mx<2, true, BOUNDED><<<grid, block, sm, s>>>(a, ws, stride);
    else k_integrate_mx<2, false, BOUNDED><<<grid, block, sm, s>>>(a, ws, stride);
  } else {
    if (persistent) k_integrate_mx<0, true, BOUNDED><<<grid, block, sm, s>>>(a, ws, stride);
    else k_integrate_mx<0, false, BOUNDED><<<grid, block, sm, s>>>(a, ws, stride);
  }
}

cudaError_t launch_integrate_only(int prec, bool persistent, int block, int grid, const KArgs& a_in, const double* ws,
                                  int64_t stride, cudaStream_t s) {
  const KArgs a = with_land(a_in, ws, stride);
  if (a.budget > 0 || a.resume) {
    launch_integrate_variant<true>(prec, persistent, block, grid, a, ws, stride, s);
    return cudaGetLastError();
  }
  if (prec == PN_MIXED) {
    const size_t sm = integrate_smem(prec, block);
    if (persistent) k_integrate_mx<1, true><<<grid, block, sm, s>>>(a, ws, stride);
    else k_integrate_mx<1, false><<<grid, block, sm, s>>>(a, ws, stride);
  } else if (prec == PN_MIXED_DS) {
    const size_t sm = integrate_smem(prec, block);
    if (persistent) k_integrate_mx<2, true><<<grid, block, sm, s>>>(a, ws, stride);
    else k_integrate_mx<2, false><<<grid, block, sm, s>>>(a, ws, stride);
  } else {
    const size_t sm = integrate_smem(prec, block);
    if (persistent) k_integrate_mx<0, true><<<grid, block, sm, s>>>(a, ws, stride);
    else k_integrate_mx<0, false><<<grid, block, sm, s>>>(a, ws, stride);
  }
  return cudaGetLastError();
}

cudaError_t integrate_occupancy(int prec, bool persistent, int block, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pick(prec, persistent), block,
                                                       integrate_smem(prec, block));
}

cudaError_t launch_integrate_record(int prec, const KArgs& a, const double* ws, int64_t stride, const RecArgs& rec,
                                    int block, int grid, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  const KArgs al = with_land(a, ws, stride);
  if (prec == PN_MIXED_DS) k_integrate<2, true, true><<<grid, block, integrate_smem(prec, block), s>>>(al, ws, stride, rec);
  else k_integrate<0, true, true><<<grid, block, integrate_smem(PN_FP64, block), s>>>(al, ws, stride, rec);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_dots(a.out, a.n, ws, stride, s);
}

cudaError_t record_occupancy(int prec, int block, int* blocks_per_sm) {
  if (prec == PN_MIXED_DS)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)k_integrate<2, true, true>, block,
                                                         integrate_smem(prec, block));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)k_integrate<0, true, true>, block,
                                                       integrate_smem(PN_FP64, block));
}

// ---------------------------------------------------------------------------
// Initial-data sampler (Sec. V): counter-based SplitMix64 uniforms
// (Steele, Lea & Flood 2014) and Marsaglia's (1972) isotropic directions.
// Every floating-point operation is an explicitly rounded IEEE operation, so
// the draws are reproducible bit for bit on any IEEE machine (the log-uniform
// mass ratio also uses exp and log).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {  // output for state x (already advanced)
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// j-th output (from 0) of the stream whose seed is the i-th output of the
// stream seeded with `seed`, as a 53-bit uniform in [0, 1).
__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t i, uint64_t j) {
  const uint64_t gamma = 0x9e3779b97f4a7c15ull;
  const uint64_t key = splitmix64(seed + (i + 1ull) * gamma);
  const uint64_t z = splitmix64(key + (j + 1ull) * gamma);
  return __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
}

// Masses of a binary of mass ratio q = m1/m2 and total mass M = m1 + m2 = 1
// (Sec. II sets M = 1): m1 = q/(1+q), m2 = 1/(1+q), each correctly rounded
// from the rounded 1 + q.
__device__ __forceinline__ void masses_of_q(double q, double* m1, double* m2) {
  const double one_q = __dadd_rn(1.0, q);
  *m1 = __ddiv_rn(q, one_q);
  *m2 = __ddiv_rn(1.0, one_q);
}

__global__ void k_masses(int64_t n, const double* __restrict__ q, double* __restrict__ m1, double* __restrict__ m2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a, b;
  masses_of_q(q[i], &a, &b);
  m1[i] = a;
  m2[i] = b;
}

__global__ void k_sample(uint64_t seed, pn_dist d, int64_t n, pn_inputs o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t ui = (uint64_t)i;
  const double u0 = uniform53(seed, ui, 0);
  double q;
  if (d.q_mode == 0) q = d.q_lo;
  else if (d.q_mode == 1) q = __dadd_rn(d.q_lo, __dmul_rn(__dsub_rn(d.q_hi, d.q_lo), u0));
  else q = __dmul_rn(d.q_lo, exp(__dmul_rn(u0, log(__ddiv_rn(d.q_hi, d.q_lo)))));
  masses_of_q(q, &o.m1[i], &o.m2[i]);
  const double u1 = uniform53(seed, ui, 1), u2 = uniform53(seed, ui, 2);
  const double span = __dsub_rn(d.chi_hi, d.chi_lo);
  o.chi1[i] = d.chi_mode == 0 ? d.chi_lo : __dadd_rn(d.chi_lo, __dmul_rn(span, u1));
  o.chi2[i] = d.chi_mode == 0 ? d.chi_lo : __dadd_rn(d.chi_lo, __dmul_rn(span, u2));
  const double u3 = uniform53(seed, ui, 3);
  o.omega0[i] = __dadd_rn(d.omega0_lo, __dmul_rn(__dsub_rn(d.omega0_hi, d.omega0_lo), u3));
  o.omega_f[i] = d.omega_f;
  uint64_t j = 4;
  for (int b = 0; b < 2; b++) {
    double vx = 0.0, vy = 0.0, vz = 1.0;
    for (int tries = 0; tries < 64; tries++) {
      const double x1 = __dsub_rn(__dmul_rn(2.0, uniform53(seed, ui, j)), 1.0);
      const double x2 = __dsub_rn(__dmul_rn(2.0, uniform53(seed, ui, j + 1)), 1.0);
      j += 2;
      const double s = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
      if (s >= 1.0) continue;
      const double r = __dsqrt_rn(__dsub_rn(1.0, s));
      vx = __dmul_rn(__dmul_rn(2.0, x1), r);
      vy = __dmul_rn(__dmul_rn(2.0, x2), r);
      vz = __dsub_rn(1.0, __dmul_rn(2.0, s));
      break;
    }
    if (b == 0) { o.s1x[i] = vx; o.s1y[i] = vy; o.s1z[i] = vz; }
    else { o.s2x[i] = vx; o.s2y[i] = vy; o.s2z[i] = vz; }
  }
  o.lx[i] = 0.0; o.ly[i] = 0.0; o.lz[i] = 1.0;
}

cudaError_t launch_masses(int64_t n, const double* q, double* m1, double* m2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (n + block - 1) / block;
  k_masses<<<(unsigned)grid, block, 0, s>>>(n, q, m1, m2);
  return cudaGetLastError();
}

cudaError_t launch_sample(uint64_t seed, const pn_dist& d, int64_t n, const pn_inputs& in, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (n + block - 1) / block;
  k_sample<<<(unsigned)grid, block, 0, s>>>(seed, d, n, in);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batch statistics: per-status counts, step totals and extremes, and the
// Pearson moments of initial vs final scalar products (Sec. V A).
// Layout of a stat record (kStatWords doubles):
//   0..7 count per status, 8 acc sum, 9 rej sum, 10 land sum,
//   11 acc min, 12 acc max, 13 attempts min, 14 attempts max,
//   15 pearson count, then for p in 0..2: 16+5p .. 20+5p = sum x, sum y, sum xx, sum yy, sum xy,
//   31 sum final s1s2, 32 sum final s1s2^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ bool is_minmax(int w) { return w >= 11 && w <= 14; }
__device__ __forceinline__ bool is_min(int w) { return w == 11 || w == 13; }

__device__ void block_reduce_store(double (*acc)[kStatWords], double* v, double* dst) {
  // v: this thread's kStatWords values; acc: shared [32][kStatWords]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int w = 0; w < kStatWords; w++) {
    double x = is_minmax(w) ? (is_min(w) ? warp_min(v[w]) : warp_max(v[w])) : warp_sum(v[w]);
    if (lane == 0) acc[wid][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < kStatWords) {
    const int w = threadIdx.x;
    double x = acc[0][w];
    for (int k = 1; k < nw; k++) {
      const double z = acc[k][w];
      x = is_minmax(w) ? (is_min(w) ? fmin(x, z) : fmax(x, z)) : x + z;
    }
    dst[w] = x;
  }
}

__device__ __forceinline__ double unit_dot(double ax, double ay, double az, double bx, double by, double bz) {
  const double na = sqrt(ax * ax + ay * ay + az * az), nb = sqrt(bx * bx + by * by + bz * bz);
  return (ax * bx + ay * by + az * bz) / (na * nb);
}

__device__ __forceinline__ void stat_init(double* v) {
  for (int w = 0; w < kStatWords; w++) v[w] = 0.0;
  v[11] = v[13] = 1e300;
  v[12] = v[14] = -1e300;
}

// Adds binary i to the record v.
__device__ __forceinline__ void stat_add(double* v, int64_t i, const pn_inputs& in, const pn_outputs& out) {
    const int st = out.status[i];
    v[(st >= 0 && st < 8) ? st : 7] += 1.0;
    const double a = out.n_acc[i], r = out.n_rej[i], l = out.n_land[i];
    v[8] += a; v[9] += r; v[10] += l;
    v[11] = fmin(v[11], a); v[12] = fmax(v[12], a);
    v[13] = fmin(v[13], a + r + l); v[14] = fmax(v[14], a + r + l);
    if (st == PN_ST_OK) {
      const double x0 = unit_dot(in.s1x[i], in.s1y[i], in.s1z[i], in.s2x[i], in.s2y[i], in.s2z[i]);
      const double x1 = unit_dot(in.lx[i], in.ly[i], in.lz[i], in.s1x[i], in.s1y[i], in.s1z[i]);
      const double x2 = unit_dot(in.lx[i], in.ly[i], in.lz[i], in.s2x[i], in.s2y[i], in.s2z[i]);
      const double y0 = out.dot_s1s2[i], y1 = out.dot_ls1[i], y2 = out.dot_ls2[i];
      if (isfinite(x0) && isfinite(x1) && isfinite(x2) && isfinite(y0) && isfinite(y1) && isfinite(y2)) {
        const double xs[3] = {x0, x1, x2}, ys[3] = {y0, y1, y2};
        v[15] += 1.0;
        for (int p = 0; p < 3; p++) {
          v[16 + 5 * p] += xs[p];
          v[17 + 5 * p] += ys[p];
          v[18 + 5 * p] += xs[p] * xs[p];
          v[19 + 5 * p] += ys[p] * ys[p];
          v[20 + 5 * p] += xs[p] * ys[p];
        }
        v[31] += y0;
        v[32] += y0 * y0;
      }
    }
}

__global__ void __launch_bounds__(256) k_stats_part(int64_t n, pn_inputs in, pn_outputs out, double* part) {
  __shared__ double acc[32][kStatWords];
  double v[kStatWords];
  stat_init(v);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    stat_add(v, i, in, out);
  block_reduce_store(acc, v, part + (size_t)blockIdx.x * kStatWords);
}

// Segmented records: block (x, k) covers binaries [off[k], off[k + 1]) with stride
// gridDim.x * blockDim.x and writes partial record k * gridDim.x + x.
__global__ void __launch_bounds__(256) k_stats_seg_part(const int64_t* __restrict__ off, pn_inputs in,
                                                        pn_outputs out, double* part) {
  __shared__ double acc[32][kStatWords];
  double v[kStatWords];
  stat_init(v);
  const int64_t lo = off[blockIdx.y], hi = off[blockIdx.y + 1];
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x)
    stat_add(v, i, in, out);
  block_reduce_store(acc, v, part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kStatWords);
}

// Block k reduces the nparts partial records starting at part + k * nparts records into total record k.
__global__ void __launch_bounds__(256) k_stats_total(const double* part, int nparts, double* total) {
  __shared__ double acc[32][kStatWords];
  double v[kStatWords];
  part += (size_t)blockIdx.x * nparts * kStatWords;
  for (int w = 0; w < kStatWords; w++) v[w] = is_minmax(w) ? (is_min(w) ? 1e300 : -1e300) : 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x)
    for (int w = 0; w < kStatWords; w++) {
      const double z = part[(size_t)p * kStatWords + w];
      v[w] = is_minmax(w) ? (is_min(w) ? fmin(v[w], z) : fmax(v[w], z)) : v[w] + z;
    }
  block_reduce_store(acc, v, total + (size_t)blockIdx.x * kStatWords);
}

cudaError_t launch_stats(int64_t n, const pn_inputs& in, const pn_outputs& out, double* part, double* total,
                         cudaStream_t s) {
  k_stats_part<<<kStatGrid, 256, 0, s>>>(n, in, out, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_stats_total<<<1, 256, 0, s>>>(part, kStatGrid, total);
  return cudaGetLastError();
}

int stats_seg_blocks(int32_t n_seg) {
  const int b = (2 * kStatGrid + n_seg - 1) / n_seg;
  return b < 1 ? 1 : (b > 64 ? 64 : b);
}

cudaError_t launch_stats_segments(int32_t n_seg, const int64_t* off, const pn_inputs& in, const pn_outputs& out,
                                  double* part, double* total, cudaStream_t s) {
  if (n_seg <= 0) return cudaSuccess;
  const int bps = stats_seg_blocks(n_seg);
  k_stats_seg_part<<<dim3((unsigned)bps, (unsigned)n_seg), 256, 0, s>>>(off, in, out, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_stats_total<<<(unsigned)n_seg, 256, 0, s>>>(part, bps, total);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The order in which lanes take the binaries.  The lanes of a warp run in
// lock-step, so a warp lasts as long as its longest binary and its lanes take
// a step decision's branches together only while their binaries behave alike.
// Binaries sorted by a predicted length, longest first, give a warp binaries of
// similar length and similar step sequences (and the persistent queue the
// longest ones first).  The order changes no result: each binary's arithmetic
// does not depend on its lane.
// ---------------------------------------------------------------------------

// In place: bins[k] <- the number of entries with a key above k (one block of
// 1024 threads; nb bins).
__global__ void __launch_bounds__(1024) k_scan_above(unsigned long long* bins, int32_t nb) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry;
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t base = 0; base < nb; base += 1024) {
    const int32_t r = base + (int32_t)threadIdx.x;  // rank from the top key down
    const int32_t k = nb - 1 - r;
    const unsigned long long v = (r < nb) ? bins[k] : 0ull;
    unsigned long long x = v;  // inclusive scan within the warp
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, x, d);
      if ((int)lane >= d) x += t;
    }
    if (lane == 31u) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = warp_tot[lane];
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, w, d);
        if ((int)lane >= d) w += t;
      }
      warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const unsigned long long before = carry + (wid ? warp_tot[wid - 1] : 0ull) + x - v;
    if (r < nb) bins[k] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[31];
    __syncthreads();
  }
}

cudaError_t launch_scan_above(unsigned long long* bins, int32_t nb, cudaStream_t s) {
  k_scan_above<<<1, 1024, 0, s>>>(bins, nb);
  return cudaGetLastError();
}

// Predicted length of binary i: the Newtonian count
// (omega_0^(-5/3) - omega_f^(-5/3)) / eta, which grows with the number of
// orbits between the two frequencies, times 1 + 0.2 (S + S.L + |S_perp|), with
// S = |S1| + |S2| and, for the total spin S1 + S2 at the start, S.L its
// projection on L-hat and S_perp its part across L-hat: spins lengthen the run
// (along L-hat they slow the chirp) and shorten its steps (the part across
// L-hat precesses, and the error control follows it).  The weights are
// empirical (they sorted sample ensembles' attempt counts best); only the order
// depends on them.  In FP32; invalid inputs get 0 (they are taken last and
// finish at once).
__device__ __forceinline__ float len_key(const pn_inputs& in, int64_t i) {
  const float m1 = (float)in.m1[i], m2 = (float)in.m2[i];
  const float S1 = (float)in.chi1[i] * m1 * m1, S2 = (float)in.chi2[i] * m2 * m2;
  const float lx = (float)in.lx[i], ly = (float)in.ly[i], lz = (float)in.lz[i];
  const float tx = S1 * (float)in.s1x[i] + S2 * (float)in.s2x[i];
  const float ty = S1 * (float)in.s1y[i] + S2 * (float)in.s2y[i];
  const float tz = S1 * (float)in.s1z[i] + S2 * (float)in.s2z[i];
  const float tl = tx * lx + ty * ly + tz * lz;
  const float px = tx - tl * lx, py = ty - tl * ly, pz = tz - tl * lz;
  const float nN = (exp2f(-5.0f / 3.0f * log2f((float)in.omega0[i])) -
                    exp2f(-5.0f / 3.0f * log2f((float)in.omega_f[i]))) / (m1 * m2);
  const float k = nN * (1.0f + 0.2f * (S1 + S2 + tl + sqrtf(px * px + py * py + pz * pz)));
  return (k > 0.0f && k <= 3.4e38f) ? k : 0.0f;
}

// Keys, and the range of the positive ones: range[0] (set to all ones before)
// takes the smallest key's bits, range[1] (zero before) the largest's; positive
// floats order like their bit patterns.
__global__ void k_len_key(const pn_inputs in, int64_t n, float* key, unsigned int* range) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float k = len_key(in, i);
  key[i] = k;
  const unsigned act = __activemask();
  const unsigned bits = __float_as_uint(k);
  const unsigned lo = __reduce_min_sync(act, k > 0.0f ? bits : 0xffffffffu);
  const unsigned hi = __reduce_max_sync(act, bits);
  if ((int)(threadIdx.x & 31u) == __ffs(act) - 1) {
    if (lo != 0xffffffffu) atomicMin(&range[0], lo);
    atomicMax(&range[1], hi);
  }
}

__device__ __forceinline__ int32_t len_bin(float k, const unsigned int* range) {
  const float lo = __uint_as_float(range[0]), hi = __uint_as_float(range[1]);
  if (!(k > 0.0f) || !(hi > lo)) return 0;
  const int32_t b = (int32_t)((k - lo) / (hi - lo) * (float)kOrderBins);
  return b < 0 ? 0 : (b >= kOrderBins ? kOrderBins - 1 : b);
}

__global__ void k_len_count(const float* key, int64_t n, const unsigned int* range, unsigned long long* bins) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t b = len_bin(key[i], range);
  const unsigned peers = __match_any_sync(__activemask(), b);
  if ((int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd(&bins[b], (unsigned long long)__popc(peers));
}

__global__ void k_len_scatter(const float* key, int64_t n, const unsigned int* range, unsigned long long* cursor,
                              int64_t* order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t b = len_bin(key[i], range);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(__activemask(), b);
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(&cursor[b], (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  const unsigned long long pos = base + __popc(peers & ((1u << lane) - 1u));
  if (PN_DCHECK(pos < (unsigned long long)n, 3)) order[pos] = i;
}

cudaError_t launch_order(const pn_inputs& in, int64_t n, int64_t* order, float* key, unsigned long long* bins,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unsigned int* range = reinterpret_cast<unsigned int*>(bins + kOrderBins);
  cudaError_t e = cudaMemsetAsync(bins, 0, (size_t)kOrderBins * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(range, 0xff, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(range + 1, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)((n + 255) / 256);
  k_len_key<<<g, 256, 0, s>>>(in, n, key, range);
  k_len_count<<<g, 256, 0, s>>>(key, n, range, bins);
  e = launch_scan_above(bins, kOrderBins, s);
  if (e != cudaSuccess) return e;
  k_len_scatter<<<g, 256, 0, s>>>(key, n, range, bins, order);
  return cudaGetLastError();
}

void fill_log_table(float* tabf) {
  for (int j = 0; j < 128; j++) {
    const long double F = 1.0L + (long double)(2 * j + 1) / 256.0L;
    const long double inv = 1.0L / F, ln = logl(F);
    const float ih = (float)inv, lh = (float)ln;
    tabf[4 * j] = ih;
    tabf[4 * j + 1] = (float)(inv - (long double)ih);
    tabf[4 * j + 2] = lh;
    tabf[4 * j + 3] = (float)(ln - (long double)lh);
  }
}

#ifdef PN_DEBUG
// The self-test's one check fails on purpose; it guards no memory access.
__global__ void k_debug_selftest(int v) {
  if (!PN_DCHECK(v == 0, 99)) return;
}

cudaError_t debug_take_kernels(unsigned int* site) { return debug_take_local(site); }

cudaError_t launch_debug_selftest(cudaStream_t s) {
  k_debug_selftest<<<1, 32, 0, s>>>(1);
  return cudaGetLastError();
}
#else
cudaError_t debug_take_kernels(unsigned int* site) {
  *site = 0u;
  return cudaSuccess;
}

cudaError_t launch_debug_selftest(cudaStream_t) { return cudaErrorNotSupported; }
#endif

}  // namespace pn
