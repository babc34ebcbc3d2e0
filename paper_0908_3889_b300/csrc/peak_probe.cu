// peak_probe.cu -- measured FP64 and FP32 FMA throughput of the current GPU.
//
// The integrator is bound by the FP64 pipe (plain) or the FP64 pipe plus the
// FP32 pipe (mixed); its roofline denominators are these measured rates.  Each
// thread runs 8 independent FMA chains; the grid fills every SM several times
// over; the result is FLOP/s counting an FMA as 2 operations, the best launch of
// about half a second of launches per precision.
// Used by bench.py (not part of the integrator's C ABI).

#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; c++) x[c] = (T)(threadIdx.x * 1e-3) + (T)c;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; c++) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
double measure(int iters, int sms) {
  const int block = 256, grid = sms * 8;
  T* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * block * sizeof(T)) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<grid, block>>>(out, iters / 10, (T)1.0000001, (T)1e-9);
  // Best of at least 3 launches, repeated for about half a second so that clock samples taken
  // by the caller while the probe runs see it (at most 400 launches).
  float best = 1e30f, total = 0.f;
  for (int r = 0; r < 400 && (r < 3 || total < 500.f); r++) {
    cudaEventRecord(e0);
    fma_chains<T><<<grid, block>>>(out, iters, (T)1.0000001, (T)1e-9);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
    total += ms;
  }
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (!ok) return -1.0;
  return 2.0 * (double)grid * block * iters * 8 / (best * 1e-3);
}

}  // namespace

// Writes FP64 and FP32 FMA throughput in FLOP/s; returns 0, or -1 on a CUDA error.
extern "C" int pn_peak_probe(double* fp64_flops, double* fp32_flops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const double f64 = measure<double>(2000, sms);
  const double f32 = measure<float>(20000, sms);
  if (fp64_flops) *fp64_flops = f64;
  if (fp32_flops) *fp32_flops = f32;
  return (f64 > 0 && f32 > 0) ? 0 : -1;
}
