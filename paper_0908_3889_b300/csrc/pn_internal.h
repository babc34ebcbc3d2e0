// pn_internal.h -- declarations shared by the integration kernels (pn_kernels.cu)
// and the C ABI layer (pn_capi.cu).  The adjoint's and the analysis kernels'
// own declarations are in pn_adjoint.h and pn_analysis.h.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "pn_batch.h"
#include "pn_device.cuh"

namespace pn {

struct KArgs {
  pn_inputs in;
  pn_outputs out;
  int64_t n;
  unsigned long long* queue;  // persistent schedule: next unclaimed binary index
  const float* tabf;          // logarithm table: 512 floats, (1/F_j, ln F_j) as FP32 pairs
  Ctl ctl;
  int32_t bpt;                // plain schedule: binaries each thread integrates in turn (0 or 1: one)
  int32_t budget;             // attempts per binary in this launch (0: no limit)
  int32_t resume;             // 1: continue the binaries whose status is PN_ST_RUNNING from the saved state
  int32_t pad_;
  double* rs;                 // saved integrator state, kResumeD doubles per binary (field-major, rs_stride)
  int32_t* ri;                // saved integrator state, kResumeI int32 per binary (field-major, rs_stride)
  int64_t rs_stride;
  double* land;               // deferred landing moves (set by the launchers: the table's last kLandFields fields)
  const int64_t* order;       // lanes take binary order[k] as their k-th (nullptr: binary k)
};

// Saved state of a binary between bounded calls: y[10], f(y)[10], t, h, h_lo,
// h_hi; n_acc, n_rej, n_land, attempts, land_it, flags (bit 0 landing, bit 1
// last attempt rejected).
constexpr int kResumeD = 24;
constexpr int kResumeI = 6;

constexpr int kMaxBlock = 256;

// Counting sort into descending key order: in place, bins[k] <- the number of
// entries with a key above k (nb bins).
cudaError_t launch_scan_above(unsigned long long* bins, int32_t nb, cudaStream_t s);

// The order in which lanes take the binaries (PN_ORDER_LENGTH): order[0..n) is
// the permutation of the binaries by their predicted length, longest first.
// Scratch: key (n floats), bins (kOrderBins + 1 words; the last holds the key
// range).
constexpr int kOrderBins = 4096;
cudaError_t launch_order(const pn_inputs& in, int64_t n, int64_t* order, float* key, unsigned long long* bins,
                         cudaStream_t s);

// Recording of accepted steps and checkpoints by the forward pass of the adjoint.
struct RecArgs {
  double* h;         // cap x stride step sizes
  double* ck;        // (cap/every + 1) x 10 x stride checkpoint states
  int* overflow;     // set to 1 if a binary needs more than cap accepted steps
  int64_t stride;    // >= n
  int32_t cap, every;
};

// The recording forward pass of the adjoint (k_integrate<prec, persistent, RECORD>),
// prec PN_FP64 or PN_MIXED_DS.
cudaError_t launch_integrate_record(int prec, const KArgs& a, const double* ws, int64_t stride, const RecArgs& rec,
                                    int block, int grid, cudaStream_t s);
cudaError_t record_occupancy(int prec, int block, int* blocks_per_sm);

// Set-up table: setup_fields() doubles per binary, field-major with the given stride (>= n): the
// kSetupFields set-up fields (16 coefficients, y0, k1 = f(y0), omega_f), then kLandFields fields for
// the final move of a binary that lands on omega_f (f(y5) and dh, written by the integration kernel,
// applied and cleared by the output epilogue).
constexpr int kSetupFields = 37;
constexpr int kLandFields = 11;
constexpr int kTableFields = kSetupFields + kLandFields;
int setup_fields();
// Validate every binary, write BAD_INPUT results, and fill the set-up table.
cudaError_t launch_setup(int prec, const KArgs& a, double* ws, int64_t stride, cudaStream_t s);
// Integration kernel launch (reads the set-up table) followed by the output
// scalar products (k_dots).  prec: PN_FP64 / PN_MIXED / PN_MIXED_DS;
// persistent: work-queue schedule.
cudaError_t launch_integrate(int prec, bool persistent, int block, int grid, const KArgs& a, const double* ws,
                             int64_t stride, cudaStream_t s);
// The output epilogue alone: deferred landing moves and the output scalar products (k_dots).
cudaError_t launch_dots(const pn_outputs& o, int64_t n, const double* ws, int64_t stride, cudaStream_t s);
// The integration kernel alone.
cudaError_t launch_integrate_only(int prec, bool persistent, int block, int grid, const KArgs& a, const double* ws,
                                  int64_t stride, cudaStream_t s);
// Allows the mixed-precision integration kernels their shared-memory workspace
// (call once per device before launching them).
cudaError_t prepare_integrate_kernels();
// Resident blocks per SM of the integration kernel at this block size.
cudaError_t integrate_occupancy(int prec, bool persistent, int block, int* blocks_per_sm);

// f(y) at n states (component-major y[c * n + i], f likewise) in precision prec.
cudaError_t launch_eval_rhs(int prec, int64_t n, const double* m1, const double* m2, const double* y, double* f,
                            const float* tab, TermCfg tc, cudaStream_t s);

cudaError_t launch_sample(uint64_t seed, const pn_dist& d, int64_t n, const pn_inputs& in, cudaStream_t s);
// m1 = q/(1+q), m2 = 1/(1+q) for n mass ratios (the sampler's own rounding).
cudaError_t launch_masses(int64_t n, const double* q, double* m1, double* m2, cudaStream_t s);

// Statistics: partial sums per block into part (grid x kStatWords doubles), then one block reduces them.
constexpr int kStatWords = 40;
constexpr int kStatGrid = 296;
cudaError_t launch_stats(int64_t n, const pn_inputs& in, const pn_outputs& out, double* part, double* total,
                         cudaStream_t s);
// The same per segment [off[k], off[k + 1]), k < n_seg (off: n_seg + 1 device int64): partial
// records into part (n_seg x stats_seg_blocks(n_seg) records), one total record per segment.
constexpr int32_t kMaxSegments = 65535;
int stats_seg_blocks(int32_t n_seg);
cudaError_t launch_stats_segments(int32_t n_seg, const int64_t* off, const pn_inputs& in, const pn_outputs& out,
                                  double* part, double* total, cudaStream_t s);

// Parameter and pointer checks shared by the C entry points (pn_capi.cu), and
// the thread-local error message that pn_last_error(NULL) returns.
int set_thread_error(int code, const std::string& msg);
bool check_params(const pn_params* p, std::string* why);
bool check_io(const pn_inputs* in, const pn_outputs* out);
Ctl ctl_from(const pn_params& p);

// Host-side logarithm table (kLogTabBytes) for log_w and ds_log: 512 floats,
// (1/F_j hi, lo, ln F_j hi, lo), F_j = 1 + (2j+1)/256.
constexpr size_t kLogTabBytes = 512 * sizeof(float);
void fill_log_table(float* tabf);

}  // namespace pn
