// pn_noalloc.cu -- pn_integrate_noalloc: integration without any device allocation.
//
// Who needs this: programs that hand all device memory to their own pool or
// budget (a framework's caching allocator, a plugin host, a service that
// reserves the GPU up front) and therefore must not have a library call
// cudaMalloc behind their back.  pn_batch_init allocates its workspace; this
// entry point instead uses one fixed scratch area that lives in the library's
// own device image, so a call allocates nothing.
//
// The scratch area is the file-scope array below (about 6 MiB).  Every GPU
// that loads the library keeps it until the process exits.  It holds the work
// queue counter, the logarithm table and the per-binary set-up table (with its
// deferred-landing fields) for at most kNoAllocMax binaries, which is why a call is limited to that many.
//
// The array is shared by all calls: each call resets the queue counter and
// rewrites the set-up entries it uses, and calls whose GPU work overlaps (on
// different streams, or from different host threads) race on it.  The first
// call on each device looks up the array's device address, uploads the
// logarithm table and waits for the device, so that first call should come
// before any stream capture.

#include <cstring>
#include <mutex>
#include <string>

#include "pn_debug.h"
#include "pn_internal.h"

namespace {

constexpr int64_t kNoAllocMax = 16384;  // binaries per call
constexpr size_t kQueueOff = 0;         // unsigned long long work-queue counter
constexpr size_t kTabOff = 256;         // the logarithm table (pn::kLogTabBytes)
constexpr size_t kSetupOff = 256 + 4096;
constexpr size_t kNoAllocBytes = kSetupOff + (size_t)pn::kTableFields * kNoAllocMax * sizeof(double);
static_assert(kTabOff + pn::kLogTabBytes <= kSetupOff, "the logarithm table overlaps the set-up table");
static_assert(kSetupOff % 256 == 0, "the set-up table must start on a 256-byte boundary");

static __device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {};  // device address of g_scratch per device, once looked up
float g_host_tab[pn::kLogTabBytes / sizeof(float)];

int scratch_for_current_device(unsigned char** out, std::string* why) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return PN_E_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) { *why = "device index beyond the no-allocation table"; return PN_E_ARG; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) { *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); return PN_E_CUDA; }
    pn::fill_log_table(g_host_tab);
    e = cudaMemcpy((unsigned char*)p + kTabOff, g_host_tab, sizeof(g_host_tab), cudaMemcpyHostToDevice);
    // A copy from pageable memory may return before its DMA lands, and a caller's non-blocking
    // stream is not ordered after the legacy stream: wait for the table before any kernel reads it.
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { *why = std::string("log table upload: ") + cudaGetErrorString(e); return PN_E_CUDA; }
    g_ptr[dev] = (unsigned char*)p;
  }
  *out = g_ptr[dev];
  return PN_OK;
}

}  // namespace

// A debug build (-DPN_DEBUG) exports a wrapper (below) that waits for the work
// and reports the device bounds checks' flags (pn_debug.h).
#ifdef PN_DEBUG
static int pn_integrate_noalloc_body(int64_t n, const pn_params* p, const pn_inputs* in, pn_outputs* out,
                                     void* cuda_stream) {
#else
extern "C" int pn_integrate_noalloc(int64_t n, const pn_params* p, const pn_inputs* in, pn_outputs* out,
                                    void* cuda_stream) {
#endif
  std::string why;
  if (!p || !in || !out) return pn::set_thread_error(PN_E_ARG, "NULL params, inputs or outputs");
  if (n < 0) return pn::set_thread_error(PN_E_ARG, "n must be >= 0");
  if (n > kNoAllocMax)
    return pn::set_thread_error(PN_E_ARG, "n exceeds the no-allocation limit of 16384 binaries per call");
  if (!pn::check_params(p, &why)) return pn::set_thread_error(PN_E_ARG, why);
  if (!pn::check_io(in, out)) return pn::set_thread_error(PN_E_ARG, "NULL input or output pointer");
  unsigned char* base = nullptr;
  const int rc = scratch_for_current_device(&base, &why);
  if (rc != PN_OK) return pn::set_thread_error(rc, why);
  if (n == 0) return PN_OK;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  pn::KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.in = *in;
  a.out = *out;
  a.n = n;
  a.queue = (unsigned long long*)(base + kQueueOff);
  a.tabf = (const float*)(base + kTabOff);
  a.ctl = pn::ctl_from(*p);
  double* table = (double*)(base + kSetupOff);

  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = pn::prepare_integrate_kernels();
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 128;
  if (e == cudaSuccess) e = pn::integrate_occupancy(p->precision, true, block, &per_sm);
  if (e != cudaSuccess) return pn::set_thread_error(PN_E_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  if (per_sm < 1) per_sm = 1;
  const int64_t full = (n + block - 1) / block, cap = (int64_t)sms * per_sm;
  const int grid = (int)(full < cap ? full : cap);

  e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = pn::launch_setup(p->precision, a, table, kNoAllocMax, s);
  if (e == cudaSuccess) e = pn::launch_integrate(p->precision, true, block, grid, a, table, kNoAllocMax, s);
  if (e != cudaSuccess) return pn::set_thread_error(PN_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return PN_OK;
}

#ifdef PN_DEBUG
extern "C" int pn_integrate_noalloc(int64_t n, const pn_params* p, const pn_inputs* in, pn_outputs* out,
                                    void* cuda_stream) {
  const int rc = pn_integrate_noalloc_body(n, p, in, out, cuda_stream);
  if (rc != PN_OK) return rc;
  unsigned int site = 0u;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = pn::debug_take_kernels(&site);
  if (e != cudaSuccess) return pn::set_thread_error(PN_E_CUDA, std::string("pn_integrate_noalloc: ") + cudaGetErrorString(e));
  if (site)
    return pn::set_thread_error(PN_E_CHECK, "pn_integrate_noalloc: debug bounds check at site " + std::to_string(site) +
                                                " failed");
  return PN_OK;
}
#endif
