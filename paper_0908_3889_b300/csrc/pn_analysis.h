// pn_analysis.h -- the device statistics of Sec. V (pn_analysis.cu), as the C
// ABI layer (pn_capi.cu) drives them.
#pragma once

#include "pn_internal.h"

namespace pn {

constexpr int kMaxHistBins = 8192;             // counts in shared memory up to this many bins
constexpr int kMaxHistBinsGlobal = 1 << 22;  // counts in global memory beyond
cudaError_t launch_histogram(const pn_inputs& in, const pn_outputs& out, int64_t n, const pn_hist_spec& sp,
                             unsigned long long* counts, cudaStream_t s);
cudaError_t launch_moments(const pn_inputs& in, const pn_outputs& out, int64_t n, int q, double* part, int blocks,
                           cudaStream_t s);
// A 64-bit fingerprint of binaries 0..n-1 of the inputs (all 15 fields, bit patterns and positions),
// added into *acc (zeroed by the caller): the autotuner's workload key.  Equal inputs give equal
// fingerprints; a change to any value or to the order changes it except with probability ~2^-64.
cudaError_t launch_input_fingerprint(const pn_inputs& in, int64_t n, unsigned long long* acc, cudaStream_t s);
cudaError_t launch_kde(const pn_inputs& in, const pn_outputs& out, int64_t n, int q, const double* grid, int64_t m,
                       double h, double count, double* density, cudaStream_t s);

}  // namespace pn
