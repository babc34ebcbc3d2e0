// pn_adjoint.h -- the adjoint's reverse sweep (pn_adjoint.cu), as the C ABI
// layer (pn_capi.cu) drives it.
#pragma once

#include "pn_internal.h"

namespace pn {

// 8-byte words the reverse sweep keeps per recomputed step.  FP64 sweep: per
// stage, the stage state (10 doubles) and the right-hand side's intermediate
// values there (41: rhs64's keep indices, the rate among them).  Double-single
// sweep: the six stage states as pairs of floats.
constexpr int kF64StageWords = 51;
constexpr int kAdjStepWordsF64 = 6 * kF64StageWords;
constexpr int kAdjStepWordsDS = 60;

struct AdjArgs {
  KArgs k;           // inputs, forward outputs, n, queue, log table, controls
  const double* h;   // recorded step sizes (RecArgs layout)
  const double* ck;  // recorded checkpoints
  double* seg;       // per-lane stage blocks: every x kAdjStepWords* x seg_stride
  unsigned long long* bins;  // cap + 1 counters for the ordering by step count
  int64_t* order;    // n binary indices, longest record first
  int64_t stride, seg_stride;
  int32_t cap, every;
  int32_t ds;        // 1: the reverse sweep in double-single arithmetic
  int32_t pad_;
  pn_cotangents gbar;
  pn_grads grad;
};

// Orders the binaries by accepted-step count (bins, order), resets the queue
// and launches the reverse sweep (pn_adjoint.cu).
cudaError_t launch_adjoint(const AdjArgs& a, int block, int grid, cudaStream_t s);
cudaError_t adjoint_occupancy(bool ds, int block, int* blocks_per_sm);

}  // namespace pn
