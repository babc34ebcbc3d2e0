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

// The same with packed pairs of FP32 (fma.rn.f32x2): each of the 8 chains is a
// pair, so an instruction carries 4 flops.
__global__ void fma2_chains(float* out, int iters, float a, float b) {
  unsigned long long x[8];
  unsigned long long aa, bb;
  asm("mov.b64 %0, {%1, %2};" : "=l"(aa) : "f"(a), "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
#pragma unroll
  for (int c = 0; c < 8; c++) {
    const float lo = threadIdx.x * 1e-3f + c, hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
  }
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < 8; c++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(aa), "l"(bb));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; c++) s += __uint_as_float((unsigned)x[c]) + __uint_as_float((unsigned)(x[c] >> 32));
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

double measure_f32x2(int iters, int sms) {
  const int block = 256, grid = sms * 8;
  float* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * block * sizeof(float)) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma2_chains<<<grid, block>>>(out, iters / 10, 1.0000001f, 1e-9f);
  float best = 1e30f;
  for (int r = 0; r < 5; r++) {
    cudaEventRecord(e0);
    fma2_chains<<<grid, block>>>(out, iters, 1.0000001f, 1e-9f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (!ok) return -1.0;
  return 4.0 * (double)grid * block * iters * 8 / (best * 1e-3);
}

// Dependent-chain latency in SM cycles: one warp, one chain of `iters` FMAs
// (scalar FP32, packed FP32 pair, FP64), timed with the SM's cycle counter.
__global__ void fma_latency(long long* cycles, int iters, float a, float b, double da, double db) {
  float x = threadIdx.x * 1e-3f;
  unsigned long long y, aa, bb;
  asm("mov.b64 %0, {%1, %2};" : "=l"(aa) : "f"(a), "f"(a));
  asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(x), "f"(x));
  double z = x;
  long long t0 = clock64();
  for (int i = 0; i < iters; i++) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x) : "f"(a), "f"(b));
  long long t1 = clock64();
  for (int i = 0; i < iters; i++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(y) : "l"(aa), "l"(bb));
  long long t2 = clock64();
  for (int i = 0; i < iters; i++) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(z) : "d"(da), "d"(db));
  long long t3 = clock64();
  if (threadIdx.x == 0) {
    cycles[0] = t1 - t0;
    cycles[1] = t2 - t1;
    cycles[2] = t3 - t2;
    cycles[3] = (long long)(x + __uint_as_float((unsigned)y) + (float)z);  // keeps the chains live
  }
}

}  // namespace

// Packed FP32 pair (f32x2) FMA throughput in FLOP/s, and the dependent-chain
// latencies of scalar FP32, packed FP32 and FP64 FMAs in cycles per operation.
// Returns 0, or -1 on a CUDA error.
extern "C" int pn_peak_probe_packed(double* f32x2_flops, double* lat_f32, double* lat_f32x2, double* lat_f64) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const double f2 = measure_f32x2(20000, sms);
  long long* d = nullptr;
  if (cudaMalloc(&d, 4 * sizeof(long long)) != cudaSuccess) return -1;
  const int iters = 4096;
  fma_latency<<<1, 32>>>(d, iters, 0.999f, 1e-3f, 0.999, 1e-3);
  long long h[4] = {0, 0, 0, 0};
  const bool ok = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(d);
  if (!ok || f2 <= 0) return -1;
  if (f32x2_flops) *f32x2_flops = f2;
  if (lat_f32) *lat_f32 = (double)h[0] / iters;
  if (lat_f32x2) *lat_f32x2 = (double)h[1] / iters;
  if (lat_f64) *lat_f64 = (double)h[2] / iters;
  return 0;
}

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
