// chym_energy.cu -- Ising readout, Ising energy and ground-state statistics.
//
// Readout s_p = sign(x_{p,0}) (ties to +1) and E = -sum_{p,q} J_pq s_p s_q
// (Eq. 3 with Ising spins); for +-1/0 couplings the sum is exact in integers.
// The statistics kernel counts ground-state hits per pump value (P_Ising(h)),
// bins the energy histogram H_E and finds the best run, i.e. the inputs of the
// figures of merit (i)-(iii) that follow Fig. 3 of arXiv 2308.02329.
#include <math.h>

#include "chym_internal.cuh"

namespace chym {
namespace {

constexpr int kEnergyThreads = 256;

// Deterministic block sum (fixed shuffle tree, then warp 0 over the partials).
template <typename V>
__device__ V block_sum(V v, V* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  V t = V(0);
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : V(0);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// One CTA per run.  J is symmetric, so thread p reads J[q][p] (coalesced).
template <typename T, bool PM1>
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(
    const T* __restrict__ X, int N, int D, const int8_t* __restrict__ J8,
    const double* __restrict__ J64, double* __restrict__ E, uint64_t* __restrict__ spins) {
  extern __shared__ int8_t s[];
  __shared__ int bad;
  __shared__ long long red_i[32];
  __shared__ double red_d[32];
  const int run = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  const T* x = X + (size_t)run * N * D;
  int my_bad = 0;
  for (int p = tid; p < N; p += blockDim.x) {
    const T v = x[(size_t)p * D];
    s[p] = (v >= T(0)) ? 1 : -1;
    for (int mu = 0; mu < D; ++mu) my_bad |= !isfinite((double)x[(size_t)p * D + mu]);
  }
  if (my_bad) atomicOr(&bad, 1);
  __syncthreads();
  if (spins) {
    const int words = (N + 63) / 64;
    for (int w = tid; w < words; w += blockDim.x) {
      uint64_t bits = 0;
      for (int b = 0; b < 64 && 64 * w + b < N; ++b)
        if (s[64 * w + b] > 0) bits |= (1ull << b);
      spins[(size_t)run * words + w] = bits;
    }
  }
  if (PM1) {
    long long acc = 0;
    for (int p = tid; p < N; p += blockDim.x) {
      int f = 0;
      for (int q = 0; q < N; ++q) f += (int)J8[(size_t)q * N + p] * (int)s[q];
      acc += (long long)s[p] * f;
    }
    const long long tot = block_sum<long long>(acc, red_i);
    if (tid == 0) E[run] = bad ? (double)NAN : -(double)tot;
  } else {
    double acc = 0.0;
    for (int p = tid; p < N; p += blockDim.x) {
      double f = 0.0;
      for (int q = 0; q < N; ++q) f += J64[(size_t)q * N + p] * (double)s[q];
      acc += (double)s[p] * f;
    }
    const double tot = block_sum<double>(acc, red_d);
    if (tid == 0) E[run] = bad ? (double)NAN : -tot;
  }
}

// Single CTA, deterministic: per-h hits, histogram, best run, finite count,
// sum of (E - E_gs) over finite runs.  out layout (see StatsOut).
struct StatsOut {
  double sum_dE;
  double best_E;
  long long best_run;
  long long n_finite;
  long long n_hits;
  long long pad[3];
  // followed by hits[n_h] and hist[n_bins] (long long)
};

constexpr int kStatsThreads = 1024;

__global__ void __launch_bounds__(kStatsThreads) stats_kernel(const double* __restrict__ E,
                                                              int n_runs, int replicas, int n_h,
                                                              double E_gs, double tol,
                                                              double bin_w, int n_bins,
                                                              StatsOut* out) {
  extern __shared__ unsigned long long sh_hits[];  // n_h counters
  __shared__ double red_d[32];
  __shared__ long long red_i[32];
  __shared__ double best_e[kStatsThreads / 32];
  __shared__ long long best_r[kStatsThreads / 32];
  long long* hits_out = reinterpret_cast<long long*>(out + 1);
  unsigned long long* hist_out = reinterpret_cast<unsigned long long*>(hits_out + n_h);
  const int tid = threadIdx.x;
  for (int i = tid; i < n_h; i += blockDim.x) sh_hits[i] = 0ull;
  for (int i = tid; i < n_bins; i += blockDim.x) hist_out[i] = 0ull;
  __syncthreads();
  double sum = 0.0, be = INFINITY;
  long long br = -1, nf = 0, nh = 0;
  for (int r = tid; r < n_runs; r += blockDim.x) {
    const double e = E[r];
    if (!isfinite(e)) continue;
    ++nf;
    sum += e - E_gs;
    const bool hit = fabs(e - E_gs) <= tol;
    if (hit) {
      atomicAdd(&sh_hits[r / replicas], 1ull);
      ++nh;
    }
    if (e < be || (e == be && r < br)) { be = e; br = r; }
    if (n_bins > 0) {
      double b = floor((e - E_gs) / bin_w + 0.5);
      int bi = b < 0.0 ? 0 : (b >= (double)n_bins ? n_bins - 1 : (int)b);
      atomicAdd(&hist_out[bi], 1ull);
    }
  }
  const double tsum = block_sum<double>(sum, red_d);
  __syncthreads();
  const long long tnf = block_sum<long long>(nf, red_i);
  __syncthreads();
  const long long tnh = block_sum<long long>(nh, red_i);
  // best (E, run): warp argmin then block argmin, ties to the lowest run
  for (int o = 16; o > 0; o >>= 1) {
    const double oe = __shfl_down_sync(0xffffffffu, be, o);
    const long long orr = __shfl_down_sync(0xffffffffu, br, o);
    if (orr >= 0 && (oe < be || (oe == be && (br < 0 || orr < br)))) { be = oe; br = orr; }
  }
  if ((tid & 31) == 0) { best_e[tid >> 5] = be; best_r[tid >> 5] = br; }
  __syncthreads();
  if (tid == 0) {
    double e0 = INFINITY;
    long long r0 = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (best_r[w] >= 0 && (best_e[w] < e0 || (best_e[w] == e0 && best_r[w] < r0))) {
        e0 = best_e[w];
        r0 = best_r[w];
      }
    out->sum_dE = tsum;
    out->best_E = e0;
    out->best_run = r0;
    out->n_finite = tnf;
    out->n_hits = tnh;
  }
  for (int i = tid; i < n_h; i += blockDim.x) hits_out[i] = (long long)sh_hits[i];
}

template <typename T>
cudaError_t launch_energy_typed(chym_ctx* c, double* d_E, uint64_t* d_spins, cudaStream_t st) {
  const T* X = (const T*)c->d_X;
  const size_t smem = (size_t)c->N;
  if (c->kind == CHYM_J_PM1)
    energy_kernel<T, true><<<c->n_runs, kEnergyThreads, smem, st>>>(X, c->N, c->D, c->d_J8,
                                                                     c->d_J64, d_E, d_spins);
  else
    energy_kernel<T, false><<<c->n_runs, kEnergyThreads, smem, st>>>(X, c->N, c->D, c->d_J8,
                                                                      c->d_J64, d_E, d_spins);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_energy(chym_ctx* c, double* d_E, uint64_t* d_spins, cudaStream_t st) {
  if (c->n_runs <= 0) return cudaSuccess;
  if (c->prec == CHYM_PREC_FP64) return launch_energy_typed<double>(c, d_E, d_spins, st);
  return launch_energy_typed<float>(c, d_E, d_spins, st);
}

size_t stats_out_bytes(int n_h, int n_bins) {
  return sizeof(StatsOut) + sizeof(long long) * ((size_t)n_h + (size_t)n_bins);
}

cudaError_t launch_stats(chym_ctx* c, const double* d_E, double E_gs, double tol, double bin_w,
                         int n_bins, void* d_out, cudaStream_t st) {
  const size_t smem = sizeof(unsigned long long) * (size_t)c->n_h;
  auto kern = stats_kernel;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<1, kStatsThreads, smem, st>>>(d_E, c->n_runs, c->n_runs / c->n_h, c->n_h, E_gs, tol,
                                       bin_w, n_bins, (StatsOut*)d_out);
  return cudaGetLastError();
}

}  // namespace chym
