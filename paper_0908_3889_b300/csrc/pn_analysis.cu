// pn_analysis.cu -- device statistics of the paper's analysis (Sec. V):
// histograms of the final (and initial) scalar products, the 79 x 79 initial
// vs final histogram, and the Gaussian kernel density estimate with the
// bandwidth h = 1.06 sigma N^(-1/5) (Silverman 1986) that Sec. V A uses.
//
// Only binaries with status PN_ST_OK and a finite value take part.  Binning
// rule (both axes): a value x in [lo, hi] goes to bin
//   k = min(nbins - 1, (int) floor((x - lo) * (nbins / (hi - lo)))),
// values outside [lo, hi] are not counted (numpy.histogram's convention).

#include <cmath>

#include "pn_analysis.h"
#include "pn_debug.h"

namespace pn {

// Value of a quantity for binary i (NaN if the binary does not take part).
__device__ __forceinline__ double quantity(int q, const pn_inputs& in, const pn_outputs& out, int64_t i) {
  if (out.status[i] != PN_ST_OK) return dnan();
  switch (q) {
    case PN_Q_FINAL_S1S2: return out.dot_s1s2[i];
    case PN_Q_FINAL_LS1: return out.dot_ls1[i];
    case PN_Q_FINAL_LS2: return out.dot_ls2[i];
    default: break;
  }
  const double ax = in.s1x[i], ay = in.s1y[i], az = in.s1z[i];
  const double bx = in.s2x[i], by = in.s2y[i], bz = in.s2z[i];
  const double lx = in.lx[i], ly = in.ly[i], lz = in.lz[i];
  const double na = sqrt(ax * ax + ay * ay + az * az), nb = sqrt(bx * bx + by * by + bz * bz);
  const double nl = sqrt(lx * lx + ly * ly + lz * lz);
  switch (q) {
    case PN_Q_INIT_S1S2: return (ax * bx + ay * by + az * bz) / (na * nb);
    case PN_Q_INIT_LS1: return (lx * ax + ly * ay + lz * az) / (nl * na);
    case PN_Q_INIT_LS2: return (lx * bx + ly * by + lz * bz) / (nl * nb);
    default: return dnan();
  }
}

__device__ __forceinline__ int bin_of(double x, double lo, double hi, double norm, int nb) {
  if (!(x >= lo && x <= hi)) return -1;  // outside, or NaN
  int k = (int)floor(__dmul_rn(__dsub_rn(x, lo), norm));
  return k < nb ? k : nb - 1;
}

// 1-D (ny = 1) or 2-D histogram; counts in shared memory per block, then one
// atomicAdd per bin per block.  nx * ny <= kMaxHistBins.
__global__ void __launch_bounds__(256) k_histogram(pn_inputs in, pn_outputs out, int64_t n, pn_hist_spec sp,
                                                   unsigned long long* counts) {
  extern __shared__ unsigned int h[];
  const int nbins = sp.nx * sp.ny;
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) h[k] = 0u;
  __syncthreads();
  const double nx_norm = (double)sp.nx / (sp.x_hi - sp.x_lo);
  const double ny_norm = sp.ny > 1 ? (double)sp.ny / (sp.y_hi - sp.y_lo) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = bin_of(quantity(sp.quantity_x, in, out, i), sp.x_lo, sp.x_hi, nx_norm, sp.nx);
    if (kx < 0) continue;
    int k = kx;
    if (sp.ny > 1) {
      const int ky = bin_of(quantity(sp.quantity_y, in, out, i), sp.y_lo, sp.y_hi, ny_norm, sp.ny);
      if (ky < 0) continue;
      k = kx * sp.ny + ky;
    }
    if (PN_DCHECK(k < nbins, 30)) atomicAdd(&h[k], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nbins; k += blockDim.x)
    if (h[k]) atomicAdd(&counts[k], (unsigned long long)h[k]);
}

// The same histogram with the counts directly in global memory, for bin counts
// beyond the shared-memory copy (up to kMaxHistBinsGlobal).  Lanes of a warp
// that fall in the same bin add their count once (match_any).
__global__ void __launch_bounds__(256) k_histogram_global(pn_inputs in, pn_outputs out, int64_t n, pn_hist_spec sp,
                                                          unsigned long long* counts) {
  const double nx_norm = (double)sp.nx / (sp.x_hi - sp.x_lo);
  const double ny_norm = sp.ny > 1 ? (double)sp.ny / (sp.y_hi - sp.y_lo) : 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t rounds = (n + stride - 1) / stride;  // every lane of a warp runs the same rounds
  const unsigned lane = threadIdx.x & 31u;
  for (int64_t r = 0; r < rounds; r++) {
    const int64_t i = r * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = -1;
    if (i < n) {
      k = bin_of(quantity(sp.quantity_x, in, out, i), sp.x_lo, sp.x_hi, nx_norm, sp.nx);
      if (k >= 0 && sp.ny > 1) {
        const int ky = bin_of(quantity(sp.quantity_y, in, out, i), sp.y_lo, sp.y_hi, ny_norm, sp.ny);
        k = ky < 0 ? -1 : k * sp.ny + ky;
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    if (k >= 0 && (int)lane == __ffs(peers) - 1 && PN_DCHECK(k < sp.nx * sp.ny, 31))
      atomicAdd(&counts[k], (unsigned long long)__popc(peers));
  }
}

// Sum and sum of squares (for the bandwidth) and count of one quantity.
__global__ void __launch_bounds__(256) k_moments(pn_inputs in, pn_outputs out, int64_t n, int q, double* part) {
  __shared__ double sh[3][8];
  double s = 0.0, s2 = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = quantity(q, in, out, i);
    if (!isfinite(x)) continue;
    s += x;
    s2 += x * x;
    c += 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s; sh[1][threadIdx.x >> 5] = s2; sh[2][threadIdx.x >> 5] = c; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += sh[threadIdx.x][w];
    part[(size_t)blockIdx.x * 3 + threadIdx.x] = v;
  }
}

// Gaussian KDE at grid point m: p(x_m) = 1/(N h) sum_j exp(-(x_m - x_j)^2 / (2 h^2)) / sqrt(2 pi).
// One block per grid point; deterministic block reduction.
__global__ void __launch_bounds__(256) k_kde(pn_inputs in, pn_outputs out, int64_t n, int q, const double* grid,
                                             double h, double count, double* density) {
  __shared__ double sh[8];
  const double x = grid[blockIdx.x];
  const double inv_h = 1.0 / h;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double xi = quantity(q, in, out, i);
    if (!isfinite(xi)) continue;
    const double u = (x - xi) * inv_h;
    s += exp(-0.5 * u * u);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += sh[w];
    density[blockIdx.x] = v * (0.3989422804014327 / (count * h));  // 1/sqrt(2 pi)
  }
}

cudaError_t launch_histogram(const pn_inputs& in, const pn_outputs& out, int64_t n, const pn_hist_spec& sp,
                             unsigned long long* counts, cudaStream_t s) {
  const int nbins = sp.nx * sp.ny;
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nbins * sizeof(unsigned long long), s);
  if (e != cudaSuccess || n <= 0) return e;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1184) blocks = 1184;
  if (nbins <= kMaxHistBins)
    k_histogram<<<(unsigned)blocks, 256, (size_t)nbins * sizeof(unsigned int), s>>>(in, out, n, sp, counts);
  else
    k_histogram_global<<<(unsigned)blocks, 256, 0, s>>>(in, out, n, sp, counts);
  return cudaGetLastError();
}

cudaError_t launch_moments(const pn_inputs& in, const pn_outputs& out, int64_t n, int q, double* part, int blocks,
                           cudaStream_t s) {
  k_moments<<<blocks, 256, 0, s>>>(in, out, n, q, part);
  return cudaGetLastError();
}

cudaError_t launch_kde(const pn_inputs& in, const pn_outputs& out, int64_t n, int q, const double* grid, int64_t m,
                       double h, double count, double* density, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_kde<<<(unsigned)m, 256, 0, s>>>(in, out, n, q, grid, h, count, density);
  return cudaGetLastError();
}

// SplitMix64's finaliser (Steele, Lea & Flood 2014) as a mixing function.
__device__ __forceinline__ unsigned long long fp_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Sum over binaries i and fields f of mix(bits(f, i) ^ mix(f * n + i)) (mod 2^64): the sum makes the
// result independent of the reduction's order, the position inside the mix makes it depend on the
// inputs' order.  One 64-bit atomic add per warp.
__global__ void __launch_bounds__(256) k_input_fingerprint(pn_inputs in, int64_t n, unsigned long long* acc) {
  const double* const f[15] = {in.m1, in.m2, in.chi1, in.chi2, in.s1x, in.s1y, in.s1z, in.s2x, in.s2y,
                               in.s2z, in.lx, in.ly, in.lz, in.omega0, in.omega_f};
  unsigned long long h = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 15; k++) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(f[k][i]);
      h += fp_mix(bits ^ fp_mix((unsigned long long)k * (unsigned long long)n + (unsigned long long)i));
    }
  }
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31u) == 0u) atomicAdd(acc, h);
}

cudaError_t launch_input_fingerprint(const pn_inputs& in, int64_t n, unsigned long long* acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_input_fingerprint<<<(unsigned)(blocks < 1184 ? blocks : 1184), 256, 0, s>>>(in, n, acc);
  return cudaGetLastError();
}

#ifdef PN_DEBUG
cudaError_t debug_take_analysis(unsigned int* site) { return debug_take_local(site); }
#else
cudaError_t debug_take_analysis(unsigned int* site) {
  *site = 0u;
  return cudaSuccess;
}
#endif

}  // namespace pn

// ---------------------------------------------------------------------------
// One-sample Kolmogorov-Smirnov test against the uniform distribution on
// [lo, hi], from binned counts (Sec. V B tests the final S1-hat.S2-hat for
// uniformity this way).  The empirical CDF F_n is known exactly at the bin
// edges e_k, so d_lo = max_k |F_n(e_k) - F(e_k)| <= D; inside bin k, F_n lies
// between F_n(e_k) and F_n(e_k+1) and F between F(e_k) and F(e_k+1), so
// D <= d_hi = max_k max(F(e_k+1) - F_n(e_k), F_n(e_k+1) - F(e_k)).  The
// p-values use the limiting Kolmogorov distribution,
// Q(t) = 2 sum_{j>=1} (-1)^(j-1) exp(-2 j^2 t^2), at t = (sqrt(N) + 0.12 +
// 0.11/sqrt(N)) D (Stephens' small-sample correction).
// ---------------------------------------------------------------------------
static double kolmogorov_q(double t) {
  if (t < 0.2) return 1.0;  // the series converges slowly there; Q is 1 to 1e-20
  double s = 0.0, sign = 1.0;
  for (int j = 1; j <= 200; j++) {
    const double term = std::exp(-2.0 * j * j * t * t);
    s += sign * term;
    if (term < 1e-300 || term < 1e-17 * std::fabs(s)) break;
    sign = -sign;
  }
  const double q = 2.0 * s;
  return q < 0.0 ? 0.0 : (q > 1.0 ? 1.0 : q);
}

extern "C" int pn_ks_uniform(const int64_t* counts, int32_t n_bins, double lo, double hi, pn_ks_result* res) {
  if (!counts || !res) return pn::set_thread_error(PN_E_ARG, "NULL pointer");
  if (n_bins < 1) return pn::set_thread_error(PN_E_ARG, "n_bins must be >= 1");
  if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi)) return pn::set_thread_error(PN_E_ARG, "need lo < hi");
  int64_t n = 0;
  for (int32_t k = 0; k < n_bins; k++) {
    if (counts[k] < 0) return pn::set_thread_error(PN_E_ARG, "negative count");
    n += counts[k];
  }
  res->n = n;
  res->d_lo = res->d_hi = 0.0;
  res->p_at_d_lo = res->p_at_d_hi = 1.0;
  if (n == 0) return PN_OK;
  const double inv_n = 1.0 / (double)n;
  int64_t cum = 0;
  double d_lo = 0.0, d_hi = 0.0;
  for (int32_t k = 0; k < n_bins; k++) {
    const double f0 = (double)k / n_bins, f1 = (double)(k + 1) / n_bins;  // F at the bin's edges
    const double g0 = cum * inv_n;
    cum += counts[k];
    const double g1 = cum * inv_n;  // F_n at the bin's edges
    d_lo = std::fmax(d_lo, std::fmax(std::fabs(g0 - f0), std::fabs(g1 - f1)));
    d_hi = std::fmax(d_hi, std::fmax(f1 - g0, g1 - f0));
  }
  const double sn = std::sqrt((double)n), corr = sn + 0.12 + 0.11 / sn;
  res->d_lo = d_lo;
  res->d_hi = d_hi;
  res->p_at_d_lo = kolmogorov_q(corr * d_lo);
  res->p_at_d_hi = kolmogorov_q(corr * d_hi);
  return PN_OK;
}
