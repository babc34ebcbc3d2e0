// pn_debug.h -- device bounds checks of the library's debug build (libpn_b300_debug.so,
// compiled with -DPN_DEBUG), which stands in for a memory checker.
//
// PN_DCHECK(cond, site) guards a device access whose index comes from data (a
// permutation entry, a scatter position, a histogram bin) or whose extent comes
// from the launch (a per-thread shared-memory workspace).  In a debug build it
// evaluates cond; when cond is false it keeps the number of the first failing
// site in its translation unit's flag and yields false, and the caller skips
// the access (no trap, no out-of-bounds access).  The C entry points of a debug
// build then synchronise the device after their work, read and clear every
// flag, and return PN_E_CHECK with the site in pn_last_error.  A release build
// compiles PN_DCHECK(cond, site) to true: cond is not evaluated and no
// instruction is added.
//
// Sites: 1-19 in pn_kernels.cu, 20-29 in pn_adjoint.cu, 30-39 in pn_analysis.cu,
// 99 the self-test's deliberate failure.
#pragma once

#include <cuda_runtime.h>

#ifdef PN_DEBUG
namespace pn {
// One flag per translation unit (internal linkage): 0, or the first failing site.
static __device__ unsigned int g_debug_site = 0u;

__device__ __forceinline__ bool debug_check(bool ok, unsigned int site) {
  if (!ok) atomicCAS(&g_debug_site, 0u, site);
  return ok;
}

// This translation unit's flag, then cleared (the caller has synchronised the device).
static inline cudaError_t debug_take_local(unsigned int* site) {
  *site = 0u;
  cudaError_t e = cudaMemcpyFromSymbol(site, g_debug_site, sizeof(unsigned int));
  if (e != cudaSuccess || *site == 0u) return e;
  const unsigned int zero = 0u;
  return cudaMemcpyToSymbol(g_debug_site, &zero, sizeof(unsigned int));
}
}  // namespace pn
#define PN_DCHECK(cond, site) (::pn::debug_check((cond), (site)))
#else
#define PN_DCHECK(cond, site) (true)
#endif

namespace pn {
// Each translation unit's first failing site since the last take (0: none), cleared.
// Release builds: 0 and cudaSuccess, with no device access.
cudaError_t debug_take_kernels(unsigned int* site);
cudaError_t debug_take_adjoint(unsigned int* site);
cudaError_t debug_take_analysis(unsigned int* site);
// Debug builds: one kernel whose single check (site 99) fails on purpose and
// guards no memory access.  Release builds: cudaErrorNotSupported.
cudaError_t launch_debug_selftest(cudaStream_t s);
}  // namespace pn
