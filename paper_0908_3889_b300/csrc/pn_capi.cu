// pn_capi.cu -- the extern "C" boundary declared in include/pn_batch.h.
//
// Host-side runtime of the integrator: parameter validation, the library's
// small device workspace, launch-shape choice (schedule, block size) and its
// autotuner, CUDA-graph capture of the persistent launch (queue reset +
// kernel), the host-buffer entry point, and the statistics reduction.

#include <cmath>
#include <cstdio>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>
#include <string>

#include "pn_adjoint.h"
#include "pn_analysis.h"
#include "pn_debug.h"
#include "pn_internal.h"

using pn::KArgs;

struct pn_batch {
  int64_t n_max = 0;
  pn_params p{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  int device = 0;
  int num_sms = 0;
  unsigned long long* d_queue = nullptr;
  float* d_tab = nullptr;
  double* d_stat_part = nullptr;
  double* d_stat_total = nullptr;
  double* d_segstat = nullptr;  // pn_batch_stats_segments: offsets, partial and total records
  size_t segstat_cap = 0;       // bytes
  double* d_setup = nullptr;  // per-binary set-up table, setup_fields() x n_max doubles
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // integrate, autotune, adjoint
  cudaEvent_t kev[2] = {nullptr, nullptr};  // around the integration kernel alone (in the graph too)
  bool timed_integrate = false, timed_adjoint = false;
  bool kernel_timed = false;  // kev hold a kernel of the last integration call that launched one
  // graph of the last persistent launch
  cudaGraphExec_t gexec = nullptr;
  bool have_key = false;
  KArgs key_args{};
  int key_prec = -1, key_block = 0, key_grid = 0;
  // autotuned launch shape per precision
  struct Tuned {
    bool valid = false;
    int schedule = PN_SCHED_PERSISTENT, block = 128, bpt = 1;
  } tuned[3];
  // adjoint workspace: recorded steps and checkpoints, per-lane segment states
  double* d_rec_h = nullptr;
  double* d_rec_ck = nullptr;
  int32_t rec_cap = 0, rec_every = 0;
  int* d_overflow = nullptr;
  double* d_seg = nullptr;
  int64_t seg_lanes = 0;
  int32_t seg_every = 0;
  int32_t seg_words = 0;  // words per step the segment buffer was sized for (FP64 and double-single sweeps differ)
  double* d_adj_out = nullptr;   // forward outputs when the caller passes none
  unsigned long long* d_hist = nullptr;  // analysis scratch: histogram counts (hist_cap bins)
  int64_t hist_cap = 0;
  double* d_ana = nullptr;               // analysis scratch: moments, KDE grid and density
  int64_t ana_cap = 0;
  int32_t* d_adj_out_i = nullptr;
  int64_t* d_adj_order = nullptr;        // reverse sweep: binaries ordered by step count
  unsigned long long* d_adj_bins = nullptr;
  int64_t* d_order = nullptr;           // PN_ORDER_LENGTH: the lanes' order of the binaries (n_max)
  float* d_order_key = nullptr;         // its keys (n_max)
  unsigned long long* d_order_bins = nullptr;  // its counting-sort bins (+ the key range)
  int64_t adj_bins_cap = 0;
  // saved integrator states between bounded calls (pn_batch_integrate_budget / pn_batch_resume)
  double* d_rs = nullptr;
  int32_t* d_ri = nullptr;
  int32_t bounded_prec = -1;  // precision of the bounded run the saved states belong to
  // staging for pn_batch_integrate_host(_async): two sets used in turn, with a
  // copy-in and a copy-out stream, so a call's copies overlap the integration of
  // the call before or after it
  double* d_stage_d[2] = {nullptr, nullptr};
  int32_t* d_stage_i[2] = {nullptr, nullptr};
  bool stage_used[2] = {false, false};
  int stage_next = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
  std::string err;
};

static thread_local std::string g_init_err;

static int fail(pn_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  else g_init_err = msg;
  return code;
}

static int cuda_fail(pn_batch* b, cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return fail(b, PN_E_CUDA, buf);
}

// Entry points that launch device work.  A debug build (-DPN_DEBUG) compiles
// their bodies as static functions and exports a wrapper (end of this file)
// that synchronises the device and reports the debug bounds checks' flags;
// a release build exports the bodies themselves.
#ifdef PN_DEBUG
#define PN_ENTRY(name) static int name##_body
#else
#define PN_ENTRY(name) extern "C" int name
#endif

#define PN_CUDA(b, call)                               \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(b, e_, #call); \
  } while (0)

extern "C" int pn_abi_version(void) { return PN_ABI_VERSION; }

static bool params_valid(const pn_params* p, std::string* why);
static pn::Ctl make_ctl(const pn_params& p);
static bool inputs_ok(const pn_inputs* in);
static bool outputs_ok(const pn_outputs* o);

// Helpers for entry points that run without a pn_batch (pn_noalloc.cu).
namespace pn {
int set_thread_error(int code, const std::string& msg) { return fail(nullptr, code, msg); }
bool check_params(const pn_params* p, std::string* why) { return params_valid(p, why); }
bool check_io(const pn_inputs* in, const pn_outputs* out) { return inputs_ok(in) && outputs_ok(out); }
Ctl ctl_from(const pn_params& p) { return make_ctl(p); }
}  // namespace pn

extern "C" void pn_params_default(pn_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->rtol = 5e-7;
  p->atol = 5e-7;
  p->h0 = 10.0;
  p->safety = 0.9;
  p->fac_min = 0.2;
  p->fac_max = 10.0;
  p->h_min = 1e-10;
  p->land_tol = 1e-7;
  p->max_steps = 1000000;
  p->land_max_iter = 8;
  p->stop_mode = PN_STOP_LAND;
  p->term_mask = PN_TERM_ALL;
  p->theta_mode = PN_THETA_BCV2;
  p->fixed_step = 0;
  p->precision = PN_FP64;
  p->schedule = PN_SCHED_AUTO;
  p->block = 0;
  p->bpt = 0;
  p->ckpt_every = 64;
  p->order = PN_ORDER_LENGTH;
}

// Parameter domain.  Besides the integrator's own constraints, atol >= 1e-30
// and safety/fac_max >= 1e-3, safety/fac_min <= 1e3 keep the error-norm scales
// and the step-control thresholds inside the FP32 normal range that the
// kernels' FP32 seeds need.
static bool params_valid(const pn_params* p, std::string* why) {
  auto bad = [&](const char* m) { *why = m; return false; };
  if (!(p->rtol >= 0.0 && std::isfinite(p->rtol))) return bad("rtol must be finite and >= 0");
  if (!(p->atol >= 1e-30 && std::isfinite(p->atol))) return bad("atol must be finite and >= 1e-30");
  if (!(p->h0 > 0.0 && std::isfinite(p->h0))) return bad("h0 must be finite and > 0");
  if (!(p->safety > 0.0 && p->fac_min > 0.0 && p->fac_min <= 1.0 && p->fac_max >= 1.0 && std::isfinite(p->fac_max)))
    return bad("need safety > 0 and 0 < fac_min <= 1 <= fac_max");
  if (!(p->safety / p->fac_max >= 1e-3 && p->safety / p->fac_min <= 1e3))
    return bad("need safety/fac_max >= 1e-3 and safety/fac_min <= 1e3");
  if (!(p->h_min >= 0.0)) return bad("h_min must be >= 0");
  if (!(p->land_tol > 0.0 && p->land_tol < 1.0)) return bad("land_tol must be in (0, 1)");
  if (p->max_steps < 1) return bad("max_steps must be >= 1");
  if (p->land_max_iter < 1) return bad("land_max_iter must be >= 1");
  if (p->stop_mode != PN_STOP_LAND && p->stop_mode != PN_STOP_FIRST_CROSS) return bad("bad stop_mode");
  if (p->theta_mode != PN_THETA_BCV2 && p->theta_mode != PN_THETA_AS_PRINTED) return bad("bad theta_mode");
  if (p->term_mask & ~PN_TERM_ALL) return bad("unknown term_mask bits");
  if (p->fixed_step != 0 && p->fixed_step != 1) return bad("fixed_step must be 0 or 1");
  if (p->precision != PN_FP64 && p->precision != PN_MIXED && p->precision != PN_MIXED_DS) return bad("bad precision");
  if (p->schedule < PN_SCHED_AUTO || p->schedule > PN_SCHED_PERSISTENT) return bad("bad schedule");
  if (p->block != 0 && (p->block < 32 || p->block > pn::kMaxBlock || p->block % 32 != 0))
    return bad("block must be 0 or a multiple of 32 in [32, 256]");
  if (p->bpt < 0 || p->bpt > 2) return bad("bpt must be 0 (autotuned/default), 1 or 2");
  if (p->ckpt_every < 1) return bad("ckpt_every must be >= 1");
  if (p->order != PN_ORDER_INPUT && p->order != PN_ORDER_LENGTH) return bad("bad order");
  return true;
}

static pn::Ctl make_ctl(const pn_params& p) {
  pn::Ctl c;
  c.rtol = p.rtol;
  c.atol = p.atol;
  c.h0 = p.h0;
  c.safety = p.safety;
  c.fac_min = p.fac_min;
  c.fac_max = p.fac_max;
  c.h_min = p.h_min;
  c.land_tol = p.land_tol;
  c.s_lo = std::pow(p.safety / p.fac_max, 10.0);
  c.s_hi = std::pow(p.safety / p.fac_min, 10.0);
  c.max_steps = p.max_steps > 2147483647 ? 2147483647 : (int32_t)p.max_steps;
  c.land_max_iter = p.land_max_iter;
  c.stop_mode = p.stop_mode;
  c.fixed_step = p.fixed_step;
  c.terms.mask = p.term_mask;
  c.terms.theta_mode = p.theta_mode;
  c.pad_ = 0;
  return c;
}

static bool inputs_ok(const pn_inputs* in) {
  return in && in->m1 && in->m2 && in->chi1 && in->chi2 && in->s1x && in->s1y && in->s1z && in->s2x && in->s2y &&
         in->s2z && in->lx && in->ly && in->lz && in->omega0 && in->omega_f;
}
static bool outputs_ok(const pn_outputs* o) {
  return o && o->S1x && o->S1y && o->S1z && o->S2x && o->S2y && o->S2z && o->Lx && o->Ly && o->Lz && o->omega &&
         o->t && o->n_acc && o->n_rej && o->n_land && o->status && o->dot_s1s2 && o->dot_ls1 && o->dot_ls2;
}

extern "C" const char* pn_last_error(const pn_batch* b) { return b ? b->err.c_str() : g_init_err.c_str(); }

extern "C" void pn_batch_destroy(pn_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : b->kev)
    if (e) cudaEventDestroy(e);
  cudaFree(b->d_queue);
  cudaFree(b->d_tab);
  cudaFree(b->d_stat_part);
  cudaFree(b->d_stat_total);
  cudaFree(b->d_segstat);
  cudaFree(b->d_setup);
  cudaFree(b->d_rec_h);
  cudaFree(b->d_rec_ck);
  cudaFree(b->d_overflow);
  cudaFree(b->d_seg);
  cudaFree(b->d_adj_out);
  cudaFree(b->d_hist);
  cudaFree(b->d_ana);
  cudaFree(b->d_adj_out_i);
  cudaFree(b->d_adj_order);
  cudaFree(b->d_adj_bins);
  cudaFree(b->d_order);
  cudaFree(b->d_order_key);
  cudaFree(b->d_order_bins);
  if (b->s_in) cudaStreamSynchronize(b->s_in);
  if (b->s_out) cudaStreamSynchronize(b->s_out);
  for (int k = 0; k < 2; k++) {
    cudaFree(b->d_stage_d[k]);
    cudaFree(b->d_stage_i[k]);
    if (b->ev_in[k]) cudaEventDestroy(b->ev_in[k]);
    if (b->ev_comp[k]) cudaEventDestroy(b->ev_comp[k]);
    if (b->ev_out[k]) cudaEventDestroy(b->ev_out[k]);
  }
  if (b->s_in) cudaStreamDestroy(b->s_in);
  if (b->s_out) cudaStreamDestroy(b->s_out);
  cudaFree(b->d_rs);
  cudaFree(b->d_ri);
  delete b;
}

extern "C" int pn_batch_init(pn_batch** out, int64_t n_max, const pn_params* p, void* cuda_stream) {
  if (!out) return fail(nullptr, PN_E_ARG, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, PN_E_ARG, "params is NULL");
  if (n_max < 1) return fail(nullptr, PN_E_ARG, "n_max must be >= 1");
  std::string why;
  if (!params_valid(p, &why)) return fail(nullptr, PN_E_ARG, why);
  pn_batch* b = new (std::nothrow) pn_batch();
  if (!b) return fail(nullptr, PN_E_NOMEM, "host allocation failed");
  b->n_max = n_max;
  b->p = *p;
  b->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = pn::prepare_integrate_kernels();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tab, pn::kLogTabBytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_stat_part, (size_t)pn::kStatGrid * pn::kStatWords * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_stat_total, pn::kStatWords * sizeof(double));
  for (int k = 0; k < 6 && e == cudaSuccess; k++) e = cudaEventCreate(&b->ev[k]);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaEventCreate(&b->kev[k]);
  if (e == cudaSuccess) {
    float tab[pn::kLogTabBytes / sizeof(float)];
    pn::fill_log_table(tab);
    e = cudaMemcpy(b->d_tab, tab, sizeof(tab), cudaMemcpyHostToDevice);
    // The copy from pageable memory may return before its DMA lands, and the batch's stream may be a
    // non-blocking one: wait for the table before the first kernel reads it.
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    const int rc = (e == cudaErrorMemoryAllocation) ? PN_E_NOMEM : PN_E_CUDA;
    char buf[256];
    snprintf(buf, sizeof(buf), "pn_batch_init: %s", cudaGetErrorString(e));
    pn_batch_destroy(b);
    return fail(nullptr, rc, buf);
  }
  *out = b;
  return PN_OK;
}

extern "C" int pn_batch_set_params(pn_batch* b, const pn_params* p) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (!p) return fail(b, PN_E_ARG, "params is NULL");
  std::string why;
  if (!params_valid(p, &why)) return fail(b, PN_E_ARG, why);
  b->p = *p;
  return PN_OK;
}

namespace {

struct Shape {
  bool persistent;
  int block;
  int grid;
  int bpt;  // plain schedule: binaries per thread
};

Shape choose_shape(pn_batch* b, int64_t n, int prec, int sched_override = -1, int block_override = 0,
                   int bpt_override = 0) {
  const pn_params& p = b->p;
  const pn_batch::Tuned& tu = b->tuned[prec];
  int sched = sched_override >= 0 ? sched_override : p.schedule;
  if (sched == PN_SCHED_AUTO) sched = tu.valid ? tu.schedule : PN_SCHED_PERSISTENT;
  int block = block_override ? block_override : p.block;
  if (block == 0) block = tu.valid ? tu.block : 128;
  int bpt = bpt_override ? bpt_override : p.bpt;
  if (bpt == 0) bpt = tu.valid ? tu.bpt : 1;
  Shape s;
  s.persistent = (sched == PN_SCHED_PERSISTENT);
  s.block = block;
  s.bpt = s.persistent ? 1 : bpt;
  const int64_t full = (n + (int64_t)block * s.bpt - 1) / ((int64_t)block * s.bpt);
  if (s.persistent) {
    int per_sm = 0;
    if (pn::integrate_occupancy(prec, true, block, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    const int64_t cap = (int64_t)b->num_sms * per_sm;
    s.grid = (int)(full < cap ? full : cap);
  } else {
    s.grid = (int)full;
  }
  return s;
}

// The integration kernel between the batch's kernel events, then the output epilogue.
static int launch_timed_kernel(pn_batch* b, int prec, const Shape& sh, const KArgs& a, int64_t stride, cudaStream_t s) {
  b->kernel_timed = true;
  PN_CUDA(b, cudaEventRecord(b->kev[0], s));
  cudaError_t e = pn::launch_integrate_only(prec, sh.persistent, sh.block, sh.grid, a, b->d_setup, stride, s);
  if (e != cudaSuccess) return cuda_fail(b, e, "integrate kernel launch");
  PN_CUDA(b, cudaEventRecord(b->kev[1], s));
  e = pn::launch_dots(a.out, a.n, b->d_setup, stride, s);
  if (e != cudaSuccess) return cuda_fail(b, e, "output epilogue launch");
  return PN_OK;
}

// The lanes' order of the binaries (PN_ORDER_LENGTH) and its sort workspace,
// allocated on first use (n_max entries).
static int ensure_order(pn_batch* b) {
  if (b->d_order) return PN_OK;
  if (cudaMalloc(&b->d_order, (size_t)b->n_max * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&b->d_order_key, (size_t)b->n_max * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->d_order_bins, ((size_t)pn::kOrderBins + 1) * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_order);
    cudaFree(b->d_order_key);
    b->d_order = nullptr;
    b->d_order_key = nullptr;
    b->d_order_bins = nullptr;
    return fail(b, PN_E_NOMEM, "order workspace allocation failed");
  }
  return PN_OK;
}

// Launch one integration of n binaries with the given shape on b->stream.
// The persistent shape goes through a CUDA graph (queue reset + kernel),
// captured on a private stream and re-used while the arguments repeat.
// With budget > 0 or resume set (bounded calls) the launches go straight onto
// b->stream: a resumed launch runs no set-up pass, and such calls are not the
// repeated identical launches the graph is for.
int run_integrate(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out, int prec, const Shape& sh,
                  int32_t budget = 0, int32_t resume = 0) {
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.in = *in;
  a.out = *out;
  a.n = n;
  a.queue = b->d_queue;
  a.tabf = b->d_tab;
  a.ctl = make_ctl(b->p);
  a.bpt = sh.bpt;
  a.budget = budget;
  a.resume = resume;
  if (n == 0 || sh.grid == 0) return PN_OK;
  if (!b->d_setup) {
    if (resume) return fail(b, PN_E_ARG, "resume without a bounded run to continue");
    cudaError_t e = cudaMalloc(&b->d_setup, (size_t)pn::setup_fields() * (size_t)b->n_max * sizeof(double));
    if (e != cudaSuccess) {
      b->d_setup = nullptr;
      cudaGetLastError();
      return fail(b, PN_E_NOMEM, "set-up table allocation failed");
    }
  }
  const int64_t stride = b->n_max;
  const bool ordered = b->p.order == PN_ORDER_LENGTH;
  if (ordered) {
    const int rc = ensure_order(b);
    if (rc != PN_OK) return rc;
    a.order = b->d_order;
  }
  auto order_on = [&](cudaStream_t s) -> cudaError_t {
    return ordered ? pn::launch_order(a.in, n, b->d_order, b->d_order_key, b->d_order_bins, s) : cudaSuccess;
  };
  if (budget > 0 || resume) {
    if (!b->d_rs) {
      if (resume) return fail(b, PN_E_ARG, "resume without a bounded run to continue");
      if (cudaMalloc(&b->d_rs, (size_t)pn::kResumeD * (size_t)b->n_max * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&b->d_ri, (size_t)pn::kResumeI * (size_t)b->n_max * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_rs);
        b->d_rs = nullptr;
        b->d_ri = nullptr;
        return fail(b, PN_E_NOMEM, "resume state allocation failed");
      }
    }
    a.rs = b->d_rs;
    a.ri = b->d_ri;
    a.rs_stride = b->n_max;
    if (sh.persistent) PN_CUDA(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream));
    {
      cudaError_t e = order_on(b->stream);
      if (e != cudaSuccess) return cuda_fail(b, e, "order kernels launch");
    }
    if (!resume) {
      cudaError_t e = pn::launch_setup(prec, a, b->d_setup, stride, b->stream);
      if (e != cudaSuccess) return cuda_fail(b, e, "set-up kernel launch");
    }
    return launch_timed_kernel(b, prec, sh, a, stride, b->stream);
  }
  if (!sh.persistent) {
    cudaError_t e = order_on(b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "order kernels launch");
    e = pn::launch_setup(prec, a, b->d_setup, stride, b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "set-up kernel launch");
    return launch_timed_kernel(b, prec, sh, a, stride, b->stream);
  }
  const bool same = b->gexec && b->have_key && b->key_prec == prec && b->key_block == sh.block &&
                    b->key_grid == sh.grid && std::memcmp(&b->key_args, &a, sizeof(a)) == 0;
  if (!same) {
    cudaGraph_t g = nullptr;
    PN_CUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->cap_stream);
    cudaError_t e2 = order_on(b->cap_stream);
    if (e2 == cudaSuccess) e2 = pn::launch_setup(prec, a, b->d_setup, stride, b->cap_stream);
    // External event record nodes: the events are recorded (and timed) each time the graph runs.
    if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(b->kev[0], b->cap_stream, cudaEventRecordExternal);
    if (e2 == cudaSuccess) e2 = pn::launch_integrate_only(prec, true, sh.block, sh.grid, a, b->d_setup, stride, b->cap_stream);
    if (e2 == cudaSuccess) e2 = cudaEventRecordWithFlags(b->kev[1], b->cap_stream, cudaEventRecordExternal);
    if (e2 == cudaSuccess) e2 = pn::launch_dots(a.out, a.n, b->d_setup, stride, b->cap_stream);
    cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e1 != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(b, e1, "graph capture (memset)"); }
    if (e2 != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(b, e2, "graph capture (kernel)"); }
    if (e3 != cudaSuccess) return cuda_fail(b, e3, "cudaStreamEndCapture");
    bool updated = false;
    if (b->gexec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(b->gexec, g, &info) == cudaSuccess) updated = true;
      else {
        cudaGetLastError();
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
      }
    }
    if (!updated) {
      cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
      if (e != cudaSuccess) { cudaGraphDestroy(g); b->gexec = nullptr; return cuda_fail(b, e, "cudaGraphInstantiate"); }
    }
    cudaGraphDestroy(g);
    b->have_key = true;
    b->key_args = a;
    b->key_prec = prec;
    b->key_block = sh.block;
    b->key_grid = sh.grid;
  }
  PN_CUDA(b, cudaGraphLaunch(b->gexec, b->stream));
  b->kernel_timed = true;
  return PN_OK;
}

}  // namespace

PN_ENTRY(pn_batch_integrate)(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!outputs_ok(out)) return fail(b, PN_E_ARG, "NULL output pointer");
  const int prec = b->p.precision;
  const Shape sh = choose_shape(b, n, prec);
  PN_CUDA(b, cudaEventRecord(b->ev[0], b->stream));
  const int rc = run_integrate(b, n, in, out, prec, sh);
  if (rc != PN_OK) return rc;
  PN_CUDA(b, cudaEventRecord(b->ev[1], b->stream));
  b->timed_integrate = true;
  return PN_OK;
}

extern "C" int pn_batch_timing(pn_batch* b, double* ms_call, double* ms_kernel) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (!b->timed_integrate) return fail(b, PN_E_ARG, "no integration call on this batch yet");
  PN_CUDA(b, cudaEventSynchronize(b->ev[1]));
  float mc = 0.f, mk = 0.f;
  PN_CUDA(b, cudaEventElapsedTime(&mc, b->ev[0], b->ev[1]));
  if (b->kernel_timed) PN_CUDA(b, cudaEventElapsedTime(&mk, b->kev[0], b->kev[1]));
  if (ms_call) *ms_call = mc;
  if (ms_kernel) *ms_kernel = b->kernel_timed ? (double)mk : NAN;
  return PN_OK;
}

static int integrate_bounded(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out, int32_t budget,
                             int32_t resume) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!outputs_ok(out)) return fail(b, PN_E_ARG, "NULL output pointer");
  if (resume ? budget < 0 : budget < 1) return fail(b, PN_E_ARG, resume ? "budget must be >= 0" : "budget must be >= 1");
  const int prec = b->p.precision;
  // The saved states are kept in the form the run's precision carries them: a resume must use it.
  if (resume && b->bounded_prec >= 0 && b->bounded_prec != prec)
    return fail(b, PN_E_ARG, "resume: the precision differs from the bounded run's");
  const Shape sh = choose_shape(b, n, prec);
  PN_CUDA(b, cudaEventRecord(b->ev[0], b->stream));
  const int rc = run_integrate(b, n, in, out, prec, sh, budget, resume);
  if (rc != PN_OK) return rc;
  PN_CUDA(b, cudaEventRecord(b->ev[1], b->stream));
  b->timed_integrate = true;
  if (!resume) b->bounded_prec = prec;
  return PN_OK;
}

PN_ENTRY(pn_batch_integrate_budget)(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out,
                                         int32_t budget) {
  return integrate_bounded(b, n, in, out, budget, 0);
}

PN_ENTRY(pn_batch_resume)(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out, int32_t budget) {
  return integrate_bounded(b, n, in, out, budget, 1);
}

PN_ENTRY(pn_batch_integrate_host_async)(pn_batch* b, int64_t n, const pn_inputs* hin, pn_outputs* hout) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(hin)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!outputs_ok(hout)) return fail(b, PN_E_ARG, "NULL output pointer");
  if (n == 0) return PN_OK;
  const size_t N = (size_t)b->n_max;
  if (!b->s_in) {
    PN_CUDA(b, cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking));
    PN_CUDA(b, cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking));
    for (int k = 0; k < 2; k++) {
      PN_CUDA(b, cudaEventCreateWithFlags(&b->ev_in[k], cudaEventDisableTiming));
      PN_CUDA(b, cudaEventCreateWithFlags(&b->ev_comp[k], cudaEventDisableTiming));
      PN_CUDA(b, cudaEventCreateWithFlags(&b->ev_out[k], cudaEventDisableTiming));
    }
  }
  const int st = b->stage_next;
  if (!b->d_stage_d[st]) {
    cudaError_t e = cudaMalloc(&b->d_stage_d[st], 29 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_stage_i[st], 4 * N * sizeof(int32_t));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(b->d_stage_d[st]);
      b->d_stage_d[st] = nullptr;
      b->d_stage_i[st] = nullptr;
      return fail(b, PN_E_NOMEM, "staging allocation failed");
    }
  }
  double* D = b->d_stage_d[st];
  int32_t* I = b->d_stage_i[st];
  pn_inputs din;
  double** dp[15] = {&din.m1, &din.m2, &din.chi1, &din.chi2, &din.s1x, &din.s1y, &din.s1z, &din.s2x,
                     &din.s2y, &din.s2z, &din.lx, &din.ly, &din.lz, &din.omega0, &din.omega_f};
  double* const hp[15] = {hin->m1, hin->m2, hin->chi1, hin->chi2, hin->s1x, hin->s1y, hin->s1z, hin->s2x,
                          hin->s2y, hin->s2z, hin->lx, hin->ly, hin->lz, hin->omega0, hin->omega_f};
  for (int k = 0; k < 15; k++) *dp[k] = D + (size_t)k * N;
  pn_outputs dout;
  double** op[14] = {&dout.S1x, &dout.S1y, &dout.S1z, &dout.S2x, &dout.S2y, &dout.S2z, &dout.Lx,
                     &dout.Ly, &dout.Lz, &dout.omega, &dout.t, &dout.dot_s1s2, &dout.dot_ls1, &dout.dot_ls2};
  double* const ho[14] = {hout->S1x, hout->S1y, hout->S1z, hout->S2x, hout->S2y, hout->S2z, hout->Lx,
                          hout->Ly, hout->Lz, hout->omega, hout->t, hout->dot_s1s2, hout->dot_ls1, hout->dot_ls2};
  for (int k = 0; k < 14; k++) *op[k] = D + (size_t)(15 + k) * N;
  int32_t** ip[4] = {&dout.n_acc, &dout.n_rej, &dout.n_land, &dout.status};
  int32_t* const hi[4] = {hout->n_acc, hout->n_rej, hout->n_land, hout->status};
  for (int k = 0; k < 4; k++) *ip[k] = I + (size_t)k * N;
  const size_t bytes = (size_t)n * sizeof(double);
  // Inputs: after the last integration that read this staging set.
  if (b->stage_used[st]) PN_CUDA(b, cudaStreamWaitEvent(b->s_in, b->ev_comp[st], 0));
  for (int k = 0; k < 15; k++) PN_CUDA(b, cudaMemcpyAsync(*dp[k], hp[k], bytes, cudaMemcpyHostToDevice, b->s_in));
  PN_CUDA(b, cudaEventRecord(b->ev_in[st], b->s_in));
  // Integration on the batch's stream: after this call's inputs, and after the
  // output copy of the last call that used this staging set.
  PN_CUDA(b, cudaStreamWaitEvent(b->stream, b->ev_in[st], 0));
  if (b->stage_used[st]) PN_CUDA(b, cudaStreamWaitEvent(b->stream, b->ev_out[st], 0));
  const int rc = pn_batch_integrate(b, n, &din, &dout);
  if (rc != PN_OK) return rc;
  PN_CUDA(b, cudaEventRecord(b->ev_comp[st], b->stream));
  // Outputs: after the integration.
  PN_CUDA(b, cudaStreamWaitEvent(b->s_out, b->ev_comp[st], 0));
  for (int k = 0; k < 14; k++) PN_CUDA(b, cudaMemcpyAsync(ho[k], *op[k], bytes, cudaMemcpyDeviceToHost, b->s_out));
  for (int k = 0; k < 4; k++)
    PN_CUDA(b, cudaMemcpyAsync(hi[k], *ip[k], (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, b->s_out));
  PN_CUDA(b, cudaEventRecord(b->ev_out[st], b->s_out));
  b->stage_used[st] = true;
  b->stage_next = st ^ 1;
  return PN_OK;
}

PN_ENTRY(pn_batch_host_wait)(pn_batch* b) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (b->s_in) PN_CUDA(b, cudaStreamSynchronize(b->s_in));
  if (b->s_out) PN_CUDA(b, cudaStreamSynchronize(b->s_out));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  return PN_OK;
}

PN_ENTRY(pn_batch_integrate_host)(pn_batch* b, int64_t n, const pn_inputs* hin, pn_outputs* hout) {
  const int rc = pn_batch_integrate_host_async(b, n, hin, hout);
  if (rc != PN_OK) return rc;
  return pn_batch_host_wait(b);
}

PN_ENTRY(pn_batch_eval_rhs)(pn_batch* b, int64_t n, const double* m1, const double* m2, const double* y,
                                 double* f) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0) return fail(b, PN_E_ARG, "n must be >= 0");
  if (!m1 || !m2 || !y || !f) return fail(b, PN_E_ARG, "NULL pointer");
  if (n == 0) return PN_OK;
  const cudaError_t e = pn::launch_eval_rhs(b->p.precision, n, m1, m2, y, f, b->d_tab, make_ctl(b->p).terms, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "right-hand-side kernel launch");
  return PN_OK;
}

// The autotuner's process-wide cache: device and precision, tuning prefix, parameters that change
// the work, and the prefix inputs' fingerprint -> the chosen shape and its time.
namespace {
using TuneKey = std::array<uint64_t, 4>;
struct TuneEntry {
  int schedule, block, bpt;
  double best_ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune_cache;
constexpr size_t kTuneCacheMax = 1024;  // entries kept before the cache starts over

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t k = 0; k < n; k++) h = (h ^ c[k]) * 0x100000001b3ull;
  return h;
}

// FNV-1a over the parameters that change the integration's work (not the launch shape or the
// adjoint's checkpoint stride; the precision is a key field of its own).
uint64_t params_fingerprint(const pn_params& p) {
  uint64_t h = 0xcbf29ce484222325ull;
  const double d[8] = {p.rtol, p.atol, p.h0, p.safety, p.fac_min, p.fac_max, p.h_min, p.land_tol};
  h = fnv1a(h, d, sizeof(d));
  const int64_t i[7] = {p.max_steps, p.land_max_iter, p.stop_mode, (int64_t)p.term_mask, p.theta_mode,
                        p.fixed_step, p.order};
  return fnv1a(h, i, sizeof(i));
}
}  // namespace

PN_ENTRY(pn_batch_autotune)(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* scratch,
                                 pn_tune_result* res) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 1 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [1, n_max]");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!outputs_ok(scratch)) return fail(b, PN_E_ARG, "NULL output pointer");
  const int prec = b->p.precision;
  const int64_t nt = n < 262144 ? n : 262144;
  // Candidates: plain schedule x {64, 128, 256} threads x {1, 2} binaries per thread, and the
  // persistent schedule x {64, 128, 256} threads.
  struct Cand { int sched, block, bpt; };
  const Cand cands[9] = {{PN_SCHED_PLAIN, 64, 1},  {PN_SCHED_PLAIN, 128, 1}, {PN_SCHED_PLAIN, 256, 1},
                         {PN_SCHED_PLAIN, 64, 2},  {PN_SCHED_PLAIN, 128, 2}, {PN_SCHED_PLAIN, 256, 2},
                         {PN_SCHED_PERSISTENT, 64, 1}, {PN_SCHED_PERSISTENT, 128, 1},
                         {PN_SCHED_PERSISTENT, 256, 1}};
  int dev = 0;
  PN_CUDA(b, cudaGetDevice(&dev));
  unsigned long long fp = 0ull;
  unsigned long long* d_fp = reinterpret_cast<unsigned long long*>(b->d_stat_total);  // synchronous scratch
  PN_CUDA(b, cudaMemsetAsync(d_fp, 0, sizeof(fp), b->stream));
  {
    const cudaError_t e = pn::launch_input_fingerprint(*in, nt, d_fp, b->stream);
    if (e != cudaSuccess) return cuda_fail(b, e, "input fingerprint kernel launch");
  }
  PN_CUDA(b, cudaMemcpyAsync(&fp, d_fp, sizeof(fp), cudaMemcpyDeviceToHost, b->stream));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  const TuneKey key = {((uint64_t)(uint32_t)dev << 32) | (uint32_t)prec, (uint64_t)nt, params_fingerprint(b->p),
                       (uint64_t)fp};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      b->tuned[prec].valid = true;
      b->tuned[prec].schedule = it->second.schedule;
      b->tuned[prec].block = it->second.block;
      b->tuned[prec].bpt = it->second.bpt;
      if (res) {
        res->schedule = it->second.schedule;
        res->block = it->second.block;
        res->bpt = it->second.bpt;
        res->n_candidates = 0;
        res->best_ms = it->second.best_ms;
        res->n_tuned = nt;
      }
      return PN_OK;
    }
  }
  double best = 1e300;
  int bs = PN_SCHED_PERSISTENT, bb = 128, bp = 1, nc = 0;
  for (const Cand& cd : cands) {
    const Shape sh = choose_shape(b, nt, prec, cd.sched, cd.block, cd.bpt);
    int rc = run_integrate(b, nt, in, scratch, prec, sh);  // warm-up
    if (rc != PN_OK) return rc;
    float tmin = 1e30f;
    for (int rep = 0; rep < 2; rep++) {
      PN_CUDA(b, cudaEventRecord(b->ev[2], b->stream));
      rc = run_integrate(b, nt, in, scratch, prec, sh);
      if (rc != PN_OK) return rc;
      PN_CUDA(b, cudaEventRecord(b->ev[3], b->stream));
      PN_CUDA(b, cudaEventSynchronize(b->ev[3]));
      float ms = 0.f;
      PN_CUDA(b, cudaEventElapsedTime(&ms, b->ev[2], b->ev[3]));
      if (ms < tmin) tmin = ms;
    }
    nc++;
    if (tmin < best) {
      best = tmin;
      bs = cd.sched;
      bb = cd.block;
      bp = cd.bpt;
    }
  }
  b->tuned[prec].valid = true;
  b->tuned[prec].schedule = bs;
  b->tuned[prec].block = bb;
  b->tuned[prec].bpt = bp;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_cache.size() >= kTuneCacheMax) g_tune_cache.clear();
    g_tune_cache[key] = TuneEntry{bs, bb, bp, best};
  }
  if (res) {
    res->schedule = bs;
    res->block = bb;
    res->bpt = bp;
    res->n_candidates = nc;
    res->best_ms = best;
    res->n_tuned = nt;
  }
  return PN_OK;
}

PN_ENTRY(pn_batch_adjoint)(pn_batch* b, int64_t n, const pn_inputs* in, const pn_cotangents* gbar,
                                pn_grads* grad, pn_outputs* out) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!gbar) return fail(b, PN_E_ARG, "cotangents struct is NULL");
  if (!grad || !grad->s1x || !grad->s1y || !grad->s1z || !grad->s2x || !grad->s2y || !grad->s2z || !grad->q)
    return fail(b, PN_E_ARG, "NULL gradient pointer");
  {
    const double* const tp[6] = {grad->s1x_tan, grad->s1y_tan, grad->s1z_tan,
                                 grad->s2x_tan, grad->s2y_tan, grad->s2z_tan};
    int set = 0;
    for (const double* p : tp) set += (p != nullptr);
    if (set != 0 && set != 6) return fail(b, PN_E_ARG, "tangent gradient pointers must be all set or all NULL");
    const double* const ap[4] = {grad->s1_dtheta, grad->s1_dphi, grad->s2_dtheta, grad->s2_dphi};
    set = 0;
    for (const double* p : ap) set += (p != nullptr);
    if (set != 0 && set != 4) return fail(b, PN_E_ARG, "angle gradient pointers must be all set or all NULL");
  }
  if (out && !outputs_ok(out)) return fail(b, PN_E_ARG, "NULL output pointer");
  if (b->p.precision == PN_MIXED || b->p.stop_mode != PN_STOP_LAND || b->p.fixed_step)
    return fail(b, PN_E_UNIMPLEMENTED,
                "the adjoint needs precision PN_FP64 or PN_MIXED_DS, PN_STOP_LAND and adaptive steps");
  const bool ds_sweep = b->p.precision == PN_MIXED_DS;
  if (n == 0) return PN_OK;
  const size_t N = (size_t)b->n_max;
  pn_outputs o;
  if (out) {
    o = *out;
  } else {
    if (!b->d_adj_out) {
      if (cudaMalloc(&b->d_adj_out, 14 * N * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&b->d_adj_out_i, 4 * N * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_adj_out);
        b->d_adj_out = nullptr;
        b->d_adj_out_i = nullptr;
        return fail(b, PN_E_NOMEM, "adjoint output allocation failed");
      }
    }
    double* D = b->d_adj_out;
    double** op[14] = {&o.S1x, &o.S1y, &o.S1z, &o.S2x, &o.S2y, &o.S2z, &o.Lx, &o.Ly, &o.Lz, &o.omega, &o.t,
                       &o.dot_s1s2, &o.dot_ls1, &o.dot_ls2};
    for (int k = 0; k < 14; k++) *op[k] = D + (size_t)k * N;
    o.n_acc = b->d_adj_out_i;
    o.n_rej = b->d_adj_out_i + N;
    o.n_land = b->d_adj_out_i + 2 * N;
    o.status = b->d_adj_out_i + 3 * N;
  }
  if (!b->d_overflow && cudaMalloc(&b->d_overflow, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(b, PN_E_NOMEM, "adjoint flag allocation failed");
  }
  if (!b->d_setup) {
    if (cudaMalloc(&b->d_setup, (size_t)pn::setup_fields() * N * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      b->d_setup = nullptr;
      return fail(b, PN_E_NOMEM, "set-up table allocation failed");
    }
  }
  const int every = b->p.ckpt_every;
  // The recording pass runs in the sweep's precision: FP64, or double-single for the double-single sweep.
  const int fprec = ds_sweep ? PN_MIXED_DS : PN_FP64;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.in = *in;
  a.out = o;
  a.n = n;
  a.queue = b->d_queue;
  a.tabf = b->d_tab;
  a.ctl = make_ctl(b->p);
  if (b->p.order == PN_ORDER_LENGTH) {  // lanes take the binaries longest first, as in pn_batch_integrate
    const int rc = ensure_order(b);
    if (rc != PN_OK) return rc;
    a.order = b->d_order;
  }
  PN_CUDA(b, cudaEventRecord(b->ev[4], b->stream));
  if (a.order) PN_CUDA(b, pn::launch_order(a.in, n, b->d_order, b->d_order_key, b->d_order_bins, b->stream));

  // Forward pass recording the accepted steps; grow the record and rerun if a
  // binary needed more steps than it holds.
  int32_t cap = b->rec_cap > 0 ? b->rec_cap : 256;
  for (int attempt = 0; attempt < 2; attempt++) {
    if (cap % every) cap += every - cap % every;
    if (b->rec_cap != cap || b->rec_every != every || !b->d_rec_h) {
      cudaFree(b->d_rec_h);
      cudaFree(b->d_rec_ck);
      b->d_rec_h = b->d_rec_ck = nullptr;
      b->rec_cap = b->rec_every = 0;
      if (cudaMalloc(&b->d_rec_h, (size_t)cap * N * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&b->d_rec_ck, ((size_t)cap / every + 1) * 10 * N * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_rec_h);
        b->d_rec_h = nullptr;
        b->d_rec_ck = nullptr;
        return fail(b, PN_E_NOMEM, "adjoint record allocation failed");
      }
      b->rec_cap = cap;
      b->rec_every = every;
    }
    pn::RecArgs rec;
    rec.h = b->d_rec_h;
    rec.ck = b->d_rec_ck;
    rec.overflow = b->d_overflow;
    rec.stride = b->n_max;
    rec.cap = cap;
    rec.every = every;
    const int block = 128;
    int per_sm = 0;
    PN_CUDA(b, pn::record_occupancy(fprec, block, &per_sm));
    const int64_t full = (n + block - 1) / block, capg = (int64_t)b->num_sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(full < capg ? full : capg);
    PN_CUDA(b, cudaMemsetAsync(b->d_overflow, 0, sizeof(int), b->stream));
    PN_CUDA(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream));
    PN_CUDA(b, pn::launch_setup(fprec, a, b->d_setup, b->n_max, b->stream));
    PN_CUDA(b, pn::launch_integrate_record(fprec, a, b->d_setup, b->n_max, rec, block, grid, b->stream));
    int overflow = 0;
    PN_CUDA(b, cudaMemcpyAsync(&overflow, b->d_overflow, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    PN_CUDA(b, cudaStreamSynchronize(b->stream));
    if (!overflow) break;
    if (attempt == 1) return fail(b, PN_E_ARG, "adjoint: step record overflow after growing it");
    // size the record to the longest binary
    double t[pn::kStatWords];
    PN_CUDA(b, pn::launch_stats(n, *in, o, b->d_stat_part, b->d_stat_total, b->stream));
    PN_CUDA(b, cudaMemcpyAsync(t, b->d_stat_total, sizeof(t), cudaMemcpyDeviceToHost, b->stream));
    PN_CUDA(b, cudaStreamSynchronize(b->stream));
    cap = (int32_t)t[12] + 1;
  }

  // Reverse sweep, persistent: binaries ordered by step count, 32 per warp
  // claim, lane-private stage-state buffer.
  const int block = 128;
  int per_sm = 0;
  PN_CUDA(b, pn::adjoint_occupancy(ds_sweep, block, &per_sm));
  const int64_t full = (n + block - 1) / block, capg = (int64_t)b->num_sms * (per_sm > 0 ? per_sm : 1);
  const int grid = (int)(full < capg ? full : capg);
  const int64_t lanes = (int64_t)grid * block;
  const int32_t step_words = ds_sweep ? pn::kAdjStepWordsDS : pn::kAdjStepWordsF64;
  if (!b->d_seg || b->seg_lanes < lanes || b->seg_every != every || b->seg_words < step_words) {
    cudaFree(b->d_seg);
    b->d_seg = nullptr;
    b->seg_lanes = 0;
    b->seg_words = 0;
    if (cudaMalloc(&b->d_seg, (size_t)lanes * every * step_words * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      b->d_seg = nullptr;
      return fail(b, PN_E_NOMEM, "adjoint segment allocation failed");
    }
    b->seg_lanes = lanes;
    b->seg_every = every;
    b->seg_words = step_words;
  }
  if (!b->d_adj_order || b->adj_bins_cap < (int64_t)b->rec_cap + 1) {
    cudaFree(b->d_adj_order);
    cudaFree(b->d_adj_bins);
    b->d_adj_order = nullptr;
    b->d_adj_bins = nullptr;
    b->adj_bins_cap = 0;
    if (cudaMalloc(&b->d_adj_order, N * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->d_adj_bins, ((size_t)b->rec_cap + 1) * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(b->d_adj_order);
      b->d_adj_order = nullptr;
      b->d_adj_bins = nullptr;
      return fail(b, PN_E_NOMEM, "adjoint ordering allocation failed");
    }
    b->adj_bins_cap = (int64_t)b->rec_cap + 1;
  }
  pn::AdjArgs aa;
  std::memset(&aa, 0, sizeof(aa));
  aa.k = a;
  aa.h = b->d_rec_h;
  aa.ck = b->d_rec_ck;
  aa.seg = b->d_seg;
  aa.bins = b->d_adj_bins;
  aa.order = b->d_adj_order;
  aa.stride = b->n_max;
  aa.seg_stride = b->seg_lanes;
  aa.cap = b->rec_cap;
  aa.every = every;
  aa.ds = ds_sweep ? 1 : 0;
  aa.gbar = *gbar;
  aa.grad = *grad;
  PN_CUDA(b, pn::launch_adjoint(aa, block, grid, b->stream));
  PN_CUDA(b, cudaEventRecord(b->ev[5], b->stream));
  b->timed_adjoint = true;
  return PN_OK;
}

PN_ENTRY(pn_batch_sample)(pn_batch* b, uint64_t seed, const pn_dist* d, int64_t n, const pn_inputs* in) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (!d) return fail(b, PN_E_ARG, "dist is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (d->q_mode < 0 || d->q_mode > 2 || d->chi_mode < 0 || d->chi_mode > 1) return fail(b, PN_E_ARG, "bad dist mode");
  if (!(d->q_lo > 0.0 && d->q_hi >= d->q_lo && std::isfinite(d->q_hi))) return fail(b, PN_E_ARG, "need 0 < q_lo <= q_hi");
  if (!(d->chi_lo >= 0.0 && d->chi_hi >= d->chi_lo && d->chi_hi <= 1.0)) return fail(b, PN_E_ARG, "need 0 <= chi_lo <= chi_hi <= 1");
  if (!(d->omega0_lo > 0.0 && d->omega0_hi >= d->omega0_lo && d->omega_f > d->omega0_hi))
    return fail(b, PN_E_ARG, "need 0 < omega0_lo <= omega0_hi < omega_f");
  cudaError_t e = pn::launch_sample(seed, *d, n, *in, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "sample kernel launch");
  return PN_OK;
}

PN_ENTRY(pn_batch_masses)(pn_batch* b, int64_t n, const double* q, double* m1, double* m2) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (n > 0 && (!q || !m1 || !m2)) return fail(b, PN_E_ARG, "NULL q, m1 or m2");
  cudaError_t e = pn::launch_masses(n, q, m1, m2, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "masses kernel launch");
  return PN_OK;
}

static void stats_from_record(pn_batch* b, int64_t n, const double* t, pn_stats* host);

PN_ENTRY(pn_batch_stats)(pn_batch* b, int64_t n, const pn_inputs* in, const pn_outputs* out, pn_stats* host) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!outputs_ok(out)) return fail(b, PN_E_ARG, "NULL output pointer");
  if (!host) return fail(b, PN_E_ARG, "host stats is NULL");
  double t[pn::kStatWords];
  cudaError_t e = pn::launch_stats(n, *in, *out, b->d_stat_part, b->d_stat_total, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "stats kernel launch");
  PN_CUDA(b, cudaMemcpyAsync(t, b->d_stat_total, sizeof(t), cudaMemcpyDeviceToHost, b->stream));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  stats_from_record(b, n, t, host);
  return PN_OK;
}

PN_ENTRY(pn_batch_stats_segments)(pn_batch* b, int32_t n_seg, const int64_t* host_offsets, const pn_inputs* in,
                                       const pn_outputs* out, pn_stats* host) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n_seg < 0 || n_seg > pn::kMaxSegments) return fail(b, PN_E_ARG, "n_seg must be in [0, 65535]");
  if (n_seg == 0) return PN_OK;
  if (!host_offsets || !host) return fail(b, PN_E_ARG, "NULL offsets or host stats");
  if (!inputs_ok(in)) return fail(b, PN_E_ARG, "NULL input pointer");
  if (!outputs_ok(out)) return fail(b, PN_E_ARG, "NULL output pointer");
  if (host_offsets[0] < 0 || host_offsets[n_seg] > b->n_max)
    return fail(b, PN_E_ARG, "segment offsets must lie in [0, n_max]");
  for (int32_t k = 0; k < n_seg; k++)
    if (host_offsets[k + 1] < host_offsets[k]) return fail(b, PN_E_ARG, "segment offsets must not decrease");
  const int bps = pn::stats_seg_blocks(n_seg);
  const size_t off_bytes = ((size_t)(n_seg + 1) * sizeof(int64_t) + 255) / 256 * 256;
  const size_t part_doubles = (size_t)n_seg * bps * pn::kStatWords, tot_doubles = (size_t)n_seg * pn::kStatWords;
  const size_t need = off_bytes + (part_doubles + tot_doubles) * sizeof(double);
  if (b->segstat_cap < need) {
    PN_CUDA(b, cudaStreamSynchronize(b->stream));  // the old scratch may still be read by queued work
    cudaFree(b->d_segstat);
    b->d_segstat = nullptr;
    b->segstat_cap = 0;
    if (cudaMalloc(&b->d_segstat, need) != cudaSuccess) {
      cudaGetLastError();
      b->d_segstat = nullptr;
      return fail(b, PN_E_NOMEM, "segment statistics scratch allocation failed");
    }
    b->segstat_cap = need;
  }
  int64_t* d_off = reinterpret_cast<int64_t*>(b->d_segstat);
  double* d_part = reinterpret_cast<double*>(reinterpret_cast<char*>(b->d_segstat) + off_bytes);
  double* d_tot = d_part + part_doubles;
  std::vector<double> t(tot_doubles);
  PN_CUDA(b, cudaMemcpyAsync(d_off, host_offsets, (size_t)(n_seg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                             b->stream));
  cudaError_t e = pn::launch_stats_segments(n_seg, d_off, *in, *out, d_part, d_tot, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "segment stats kernel launch");
  PN_CUDA(b, cudaMemcpyAsync(t.data(), d_tot, tot_doubles * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  for (int32_t k = 0; k < n_seg; k++)
    stats_from_record(b, host_offsets[k + 1] - host_offsets[k], t.data() + (size_t)k * pn::kStatWords, &host[k]);
  return PN_OK;
}

// pn_stats of n binaries from one reduced record t (layout in pn_kernels.cu).
static void stats_from_record(pn_batch* b, int64_t n, const double* t, pn_stats* host) {
  std::memset(host, 0, sizeof(*host));
  host->n = n;
  for (int k = 0; k < 8; k++) host->count_by_status[k] = (int64_t)t[k];
  host->acc_total = (int64_t)t[8];
  host->rej_total = (int64_t)t[9];
  host->land_total = (int64_t)t[10];
  host->acc_min = n ? (int32_t)t[11] : 0;
  host->acc_max = n ? (int32_t)t[12] : 0;
  host->attempts_min = n ? (int32_t)t[13] : 0;
  host->attempts_max = n ? (int32_t)t[14] : 0;
  const double N = t[15];
  host->pearson_count = (int64_t)N;
  double* r[3] = {&host->pearson_s1s2, &host->pearson_ls1, &host->pearson_ls2};
  for (int p = 0; p < 3; p++) {
    const double sx = t[16 + 5 * p], sy = t[17 + 5 * p], sxx = t[18 + 5 * p], syy = t[19 + 5 * p],
                 sxy = t[20 + 5 * p];
    const double num = N * sxy - sx * sy;
    const double den = std::sqrt((N * sxx - sx * sx) * (N * syy - sy * sy));
    *r[p] = (N > 1 && den > 0) ? num / den : NAN;
  }
  host->mean_final_s1s2 = N > 0 ? t[31] / N : NAN;
  host->std_final_s1s2 = N > 1 ? std::sqrt((t[32] - t[31] * t[31] / N) / (N - 1)) : NAN;
  float ms = 0.f;
  host->ms_last_integrate = (b->timed_integrate && cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) ? ms : NAN;
  host->ms_last_adjoint = (b->timed_adjoint && cudaEventElapsedTime(&ms, b->ev[4], b->ev[5]) == cudaSuccess) ? ms : NAN;
  cudaGetLastError();
}

PN_ENTRY(pn_batch_histogram)(pn_batch* b, int64_t n, const pn_inputs* in, const pn_outputs* out,
                                  const pn_hist_spec* sp, int64_t* host_counts) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in) || !outputs_ok(out) || !sp || !host_counts) return fail(b, PN_E_ARG, "NULL pointer");
  const bool two = sp->ny > 1;
  if (sp->nx < 1 || sp->ny < 1 || (int64_t)sp->nx * sp->ny > pn::kMaxHistBinsGlobal)
    return fail(b, PN_E_ARG, "bad bin counts");
  if (sp->quantity_x < 0 || sp->quantity_x > 5 || (two && (sp->quantity_y < 0 || sp->quantity_y > 5)))
    return fail(b, PN_E_ARG, "bad quantity");
  if (!(sp->x_hi > sp->x_lo) || (two && !(sp->y_hi > sp->y_lo))) return fail(b, PN_E_ARG, "need lo < hi");
  const int64_t need_bins = (int64_t)sp->nx * sp->ny > pn::kMaxHistBins ? (int64_t)sp->nx * sp->ny : pn::kMaxHistBins;
  if (b->hist_cap < need_bins) {
    cudaFree(b->d_hist);
    b->d_hist = nullptr;
    b->hist_cap = 0;
    if (cudaMalloc(&b->d_hist, (size_t)need_bins * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      b->d_hist = nullptr;
      return fail(b, PN_E_NOMEM, "histogram scratch allocation failed");
    }
    b->hist_cap = need_bins;
  }
  cudaError_t e = pn::launch_histogram(*in, *out, n, *sp, b->d_hist, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "histogram kernel launch");
  const size_t nb = (size_t)sp->nx * sp->ny;
  PN_CUDA(b, cudaMemcpyAsync(host_counts, b->d_hist, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  return PN_OK;
}

PN_ENTRY(pn_batch_kde)(pn_batch* b, int64_t n, const pn_inputs* in, const pn_outputs* out, int32_t q,
                            const double* host_grid, int64_t m, double* host_density, double* host_h) {
  if (!b) return fail(nullptr, PN_E_ARG, "batch is NULL");
  if (n < 0 || n > b->n_max) return fail(b, PN_E_ARG, "n must be in [0, n_max]");
  if (!inputs_ok(in) || !outputs_ok(out) || !host_grid || !host_density) return fail(b, PN_E_ARG, "NULL pointer");
  if (q < 0 || q > 5) return fail(b, PN_E_ARG, "bad quantity");
  if (m < 1 || m > 65536) return fail(b, PN_E_ARG, "m must be in [1, 65536]");
  const int blocks = 296;
  const int64_t need = 3 * blocks + 2 * m;
  if (b->ana_cap < need) {
    cudaFree(b->d_ana);
    b->d_ana = nullptr;
    b->ana_cap = 0;
    if (cudaMalloc(&b->d_ana, (size_t)need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(b, PN_E_NOMEM, "KDE scratch allocation failed");
    }
    b->ana_cap = need;
  }
  double* part = b->d_ana;
  double* grid = b->d_ana + 3 * blocks;
  double* dens = grid + m;
  cudaError_t e = pn::launch_moments(*in, *out, n, q, part, blocks, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "moments kernel launch");
  double hp[3 * 296];
  PN_CUDA(b, cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, b->stream));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  double s = 0, s2 = 0, cnt = 0;
  for (int k = 0; k < blocks; k++) { s += hp[3 * k]; s2 += hp[3 * k + 1]; cnt += hp[3 * k + 2]; }
  if (cnt < 2) return fail(b, PN_E_ARG, "KDE needs at least two binaries with finite values");
  const double mean = s / cnt;
  const double var = (s2 - cnt * mean * mean) / (cnt - 1.0);
  const double h = 1.06 * std::sqrt(var > 0 ? var : 0.0) * std::pow(cnt, -0.2);
  if (!(h > 0)) return fail(b, PN_E_ARG, "KDE bandwidth is zero (all values equal)");
  PN_CUDA(b, cudaMemcpyAsync(grid, host_grid, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  e = pn::launch_kde(*in, *out, n, q, grid, m, h, cnt, dens, b->stream);
  if (e != cudaSuccess) return cuda_fail(b, e, "KDE kernel launch");
  PN_CUDA(b, cudaMemcpyAsync(host_density, dens, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  PN_CUDA(b, cudaStreamSynchronize(b->stream));
  if (host_h) *host_h = h;
  return PN_OK;
}

// ---------------------------------------------------------------------------
// Debug build: every entry point that launches device work waits for it, then
// reads and clears the device bounds checks' flags (pn_debug.h).  A failed
// check becomes PN_E_CHECK, with the entry point and the site in the message.
// ---------------------------------------------------------------------------
static int debug_after(pn_batch* b, int rc, const char* what) {
#ifdef PN_DEBUG
  if (rc != PN_OK) return rc;  // an argument or CUDA error stands as it is
  cudaError_t e = cudaDeviceSynchronize();
  unsigned int site[3] = {0u, 0u, 0u};
  if (e == cudaSuccess) e = pn::debug_take_kernels(&site[0]);
  if (e == cudaSuccess) e = pn::debug_take_adjoint(&site[1]);
  if (e == cudaSuccess) e = pn::debug_take_analysis(&site[2]);
  if (e != cudaSuccess) return cuda_fail(b, e, what);
  for (unsigned int v : site)
    if (v) return fail(b, PN_E_CHECK, std::string(what) + ": debug bounds check at site " + std::to_string(v) + " failed");
#else
  (void)b;
  (void)what;
#endif
  return rc;
}

extern "C" int pn_debug_selftest(void) {
#ifdef PN_DEBUG
  unsigned int site = 0u;
  cudaError_t e = pn::launch_debug_selftest(0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = pn::debug_take_kernels(&site);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pn_debug_selftest");
  if (site != 99u) return fail(nullptr, PN_E_CHECK, "pn_debug_selftest: the deliberate check failure was not reported");
  e = pn::debug_take_kernels(&site);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pn_debug_selftest");
  if (site != 0u) return fail(nullptr, PN_E_CHECK, "pn_debug_selftest: the flag was not cleared");
  return PN_OK;
#else
  (void)debug_after;
  return fail(nullptr, PN_E_UNIMPLEMENTED, "pn_debug_selftest: release build (no bounds checks)");
#endif
}

#ifdef PN_DEBUG
extern "C" int pn_batch_integrate(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out) {
  return debug_after(b, pn_batch_integrate_body(b, n, in, out), "pn_batch_integrate");
}
extern "C" int pn_batch_integrate_budget(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out,
                                         int32_t budget) {
  return debug_after(b, pn_batch_integrate_budget_body(b, n, in, out, budget), "pn_batch_integrate_budget");
}
extern "C" int pn_batch_resume(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* out, int32_t budget) {
  return debug_after(b, pn_batch_resume_body(b, n, in, out, budget), "pn_batch_resume");
}
extern "C" int pn_batch_integrate_host_async(pn_batch* b, int64_t n, const pn_inputs* hin, pn_outputs* hout) {
  return debug_after(b, pn_batch_integrate_host_async_body(b, n, hin, hout), "pn_batch_integrate_host_async");
}
extern "C" int pn_batch_host_wait(pn_batch* b) {
  return debug_after(b, pn_batch_host_wait_body(b), "pn_batch_host_wait");
}
extern "C" int pn_batch_integrate_host(pn_batch* b, int64_t n, const pn_inputs* hin, pn_outputs* hout) {
  return debug_after(b, pn_batch_integrate_host_body(b, n, hin, hout), "pn_batch_integrate_host");
}
extern "C" int pn_batch_eval_rhs(pn_batch* b, int64_t n, const double* m1, const double* m2, const double* y,
                                 double* f) {
  return debug_after(b, pn_batch_eval_rhs_body(b, n, m1, m2, y, f), "pn_batch_eval_rhs");
}
extern "C" int pn_batch_autotune(pn_batch* b, int64_t n, const pn_inputs* in, pn_outputs* scratch,
                                 pn_tune_result* res) {
  return debug_after(b, pn_batch_autotune_body(b, n, in, scratch, res), "pn_batch_autotune");
}
extern "C" int pn_batch_adjoint(pn_batch* b, int64_t n, const pn_inputs* in, const pn_cotangents* gbar,
                                pn_grads* grad, pn_outputs* out) {
  return debug_after(b, pn_batch_adjoint_body(b, n, in, gbar, grad, out), "pn_batch_adjoint");
}
extern "C" int pn_batch_sample(pn_batch* b, uint64_t seed, const pn_dist* d, int64_t n, const pn_inputs* in) {
  return debug_after(b, pn_batch_sample_body(b, seed, d, n, in), "pn_batch_sample");
}
extern "C" int pn_batch_masses(pn_batch* b, int64_t n, const double* q, double* m1, double* m2) {
  return debug_after(b, pn_batch_masses_body(b, n, q, m1, m2), "pn_batch_masses");
}
extern "C" int pn_batch_stats(pn_batch* b, int64_t n, const pn_inputs* in, const pn_outputs* out, pn_stats* host) {
  return debug_after(b, pn_batch_stats_body(b, n, in, out, host), "pn_batch_stats");
}
extern "C" int pn_batch_stats_segments(pn_batch* b, int32_t n_seg, const int64_t* host_offsets, const pn_inputs* in,
                                       const pn_outputs* out, pn_stats* host) {
  return debug_after(b, pn_batch_stats_segments_body(b, n_seg, host_offsets, in, out, host),
                     "pn_batch_stats_segments");
}
extern "C" int pn_batch_histogram(pn_batch* b, int64_t n, const pn_inputs* in, const pn_outputs* out,
                                  const pn_hist_spec* sp, int64_t* host_counts) {
  return debug_after(b, pn_batch_histogram_body(b, n, in, out, sp, host_counts), "pn_batch_histogram");
}
extern "C" int pn_batch_kde(pn_batch* b, int64_t n, const pn_inputs* in, const pn_outputs* out, int32_t q,
                            const double* host_grid, int64_t m, double* host_density, double* host_h) {
  return debug_after(b, pn_batch_kde_body(b, n, in, out, q, host_grid, m, host_density, host_h), "pn_batch_kde");
}
#endif
