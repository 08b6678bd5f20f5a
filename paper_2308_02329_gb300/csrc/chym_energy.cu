// chym_energy.cu -- Ising readout, Ising energy and ground-state statistics.
//
// Readout s_p = sign(x_{p,0}) (ties to +1) and E = -sum_{p,q} J_pq s_p s_q
// (Eq. 3 with Ising spins); for +-1/0 couplings the sum is exact in integers.
// The statistics kernel counts ground-state hits per pump value (P_Ising(h)),
// bins the energy histogram H_E and finds the best run, i.e. the inputs of the
// figures of merit (i)-(iii) that follow Fig. 3 of arXiv 2308.02329.
#include <math.h>

#include <algorithm>
#include <mutex>

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

// One CTA per run.  Real J: thread p reads J[q][p] (J symmetric: coalesced), FP64.
// +-1 J: bit planes of J, plane[w][p] = the bits of row p's columns 64 w .. 64 w + 63
// where J = +1 (Jpos) or -1 (Jneg), word-major so that consecutive rows are coalesced.
// With d_p = the spins that differ from s_p (one xor of the spin words),
//   sum_q J_pq s_p s_q = deg_p - 2 (popc(Jpos_p & d_p) - popc(Jneg_p & d_p)),
// deg_p = (#J = +1) - (#J = -1) in row p: an exact integer from N/64 words a row.
constexpr int kMaxSpinWords = 64;  // N <= 4096
template <typename T, bool PM1>
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(
    const T* __restrict__ X, int N, int D, const uint64_t* __restrict__ Jpos,
    const uint64_t* __restrict__ Jneg, const int32_t* __restrict__ deg,
    const double* __restrict__ J64, double* __restrict__ E, uint64_t* __restrict__ spins) {
  extern __shared__ int8_t s[];
  __shared__ int bad;
  __shared__ long long red_i[32];
  __shared__ double red_d[32];
  __shared__ uint64_t sw[kMaxSpinWords];
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
  const int words = (N + 63) / 64;
  for (int w = tid; w < words; w += blockDim.x) {
    uint64_t bits = 0;
    for (int b = 0; b < 64 && 64 * w + b < N; ++b)
      if (s[64 * w + b] > 0) bits |= (1ull << b);
    sw[w] = bits;
    if (spins) spins[(size_t)run * words + w] = bits;
  }
  __syncthreads();
  if (PM1) {
    long long acc = 0;
    for (int p = tid; p < N; p += blockDim.x) {
      const uint64_t flip = s[p] > 0 ? ~0ull : 0ull;  // d = spins unlike s_p (padding bits meet no J)
      int c = 0;
      for (int w = 0; w < words; ++w) {
        const uint64_t d = sw[w] ^ flip;
        c += __popcll(__ldg(Jpos + (size_t)w * N + p) & d) - __popcll(__ldg(Jneg + (size_t)w * N + p) & d);
      }
      acc += (long long)(deg[p] - 2 * c);
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

// One CTA per (run, segment): the Ising energy of the segment's spins alone,
// E_i = -sum_{p,q in i} J_pq s_p s_q (the energy of one graph of a block-diagonal
// packing); NaN when a state value of the segment is not finite.
template <typename T, bool PM1>
__global__ void __launch_bounds__(kEnergyThreads) energy_segments_kernel(
    const T* __restrict__ X, int N, int D, const int8_t* __restrict__ J8,
    const double* __restrict__ J64, SegTable t, double* __restrict__ E) {
  extern __shared__ int8_t s[];
  __shared__ int bad;
  __shared__ long long red_i[32];
  __shared__ double red_d[32];
  const int run = blockIdx.x, seg = blockIdx.y, tid = threadIdx.x;
  const int b = t.begin[seg], n = t.begin[seg + 1] - b;
  if (tid == 0) bad = 0;
  __syncthreads();
  const T* x = X + ((size_t)run * N + b) * D;
  int my_bad = 0;
  for (int p = tid; p < n; p += blockDim.x) {
    s[p] = (x[(size_t)p * D] >= T(0)) ? 1 : -1;
    for (int mu = 0; mu < D; ++mu) my_bad |= !isfinite((double)x[(size_t)p * D + mu]);
  }
  if (my_bad) atomicOr(&bad, 1);
  __syncthreads();
  double* out = E + (size_t)run * t.n + seg;
  if (PM1) {
    long long acc = 0;
    for (int p = tid; p < n; p += blockDim.x) {
      int f = 0;
      for (int q = 0; q < n; ++q) f += (int)J8[(size_t)(b + q) * N + b + p] * (int)s[q];
      acc += (long long)s[p] * f;
    }
    const long long tot = block_sum<long long>(acc, red_i);
    if (tid == 0) *out = bad ? (double)NAN : -(double)tot;
  } else {
    double acc = 0.0;
    for (int p = tid; p < n; p += blockDim.x) {
      double f = 0.0;
      for (int q = 0; q < n; ++q) f += J64[(size_t)(b + q) * N + b + p] * (double)s[q];
      acc += (double)s[p] * f;
    }
    const double tot = block_sum<double>(acc, red_d);
    if (tid == 0) *out = bad ? (double)NAN : -tot;
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
                                                              const int32_t* __restrict__ hidx,
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
      atomicAdd(&sh_hits[hidx ? hidx[r] : r / replicas], 1ull);
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
  if (c->N > 64 * kMaxSpinWords) return cudaErrorInvalidValue;
  const int W = (c->N + 63) / 64;
  if (c->kind == CHYM_J_PM1)
    energy_kernel<T, true><<<c->n_runs, kEnergyThreads, smem, st>>>(
        X, c->N, c->D, c->d_Jbits, c->d_Jbits + (size_t)W * c->N, c->d_jdeg, c->d_J64, d_E, d_spins);
  else
    energy_kernel<T, false><<<c->n_runs, kEnergyThreads, smem, st>>>(
        X, c->N, c->D, nullptr, nullptr, nullptr, c->d_J64, d_E, d_spins);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_energy(chym_ctx* c, double* d_E, uint64_t* d_spins, cudaStream_t st) {
  if (c->n_runs <= 0) return cudaSuccess;
  if (c->prec == CHYM_PREC_FP64) return launch_energy_typed<double>(c, d_E, d_spins, st);
  return launch_energy_typed<float>(c, d_E, d_spins, st);
}

cudaError_t launch_energy_segments(chym_ctx* c, const SegTable& t, double* d_E, cudaStream_t st) {
  if (c->n_runs <= 0) return cudaSuccess;
  int longest = 0;
  for (int i = 0; i < t.n; ++i) longest = std::max(longest, t.begin[i + 1] - t.begin[i]);
  const dim3 grid((unsigned)c->n_runs, (unsigned)t.n);
  const size_t smem = (size_t)longest;
  const bool pm1 = c->kind == CHYM_J_PM1;
  if (c->prec == CHYM_PREC_FP64) {
    const double* X = (const double*)c->d_X;
    if (pm1) energy_segments_kernel<double, true><<<grid, kEnergyThreads, smem, st>>>(X, c->N, c->D, c->d_J8, c->d_J64, t, d_E);
    else energy_segments_kernel<double, false><<<grid, kEnergyThreads, smem, st>>>(X, c->N, c->D, c->d_J8, c->d_J64, t, d_E);
  } else {
    const float* X = (const float*)c->d_X;
    if (pm1) energy_segments_kernel<float, true><<<grid, kEnergyThreads, smem, st>>>(X, c->N, c->D, c->d_J8, c->d_J64, t, d_E);
    else energy_segments_kernel<float, false><<<grid, kEnergyThreads, smem, st>>>(X, c->N, c->D, c->d_J8, c->d_J64, t, d_E);
  }
  return cudaGetLastError();
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
  kern<<<1, kStatsThreads, smem, st>>>(d_E, c->d_hidx, c->n_runs, c->n_runs / c->n_h, c->n_h, E_gs, tol,
                                       bin_w, n_bins, (StatsOut*)d_out);
  return cudaGetLastError();
}



// ---------------------------------------------------------------------------
// Allocation-free statistics.
//
// Some callers cannot allocate device memory when they need the statistics:
// code running under a memory manager that owns the whole device pool, callers
// that must not trigger the device-wide synchronisation cudaMalloc/cudaFree can
// imply, or real-time loops with a fixed memory budget.  For them the statistics
// kernel writes its result block into this file-scope device array instead of a
// context buffer.  Every GPU that loads the library holds the array until exit.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocMaxH = 4096;      // pump values
constexpr int kNoAllocMaxBins = 65536;  // histogram bins
constexpr size_t kNoAllocBytes =
    sizeof(StatsOut) + sizeof(long long) * ((size_t)kNoAllocMaxH + kNoAllocMaxBins);
static __device__ __align__(256) unsigned char g_stats_noalloc_scratch[kNoAllocBytes];

// Device address of the array on each device, looked up once per device with that
// device current (host code must not pass the array's name to a kernel).
constexpr int kMaxDevices = 64;
void* g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

cudaError_t noalloc_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stats_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace chym

extern "C" CHYM_API chym_status chym_stats_noalloc(const double* d_E, int n_runs, int n_h,
                                                   chym_jkind kind, double E_gs,
                                                   chym_stats_t* out, int64_t* hits_per_h,
                                                   int64_t* hist, int n_bins,
                                                   void* cuda_stream) {
  using namespace chym;
  if (!d_E || !out) return fail(CHYM_EINVAL, "NULL argument");
  if (n_h < 1 || n_runs < 1 || n_runs % n_h)
    return fail(CHYM_EINVAL, "n_runs must be a positive multiple of n_h");
  if (n_h > kNoAllocMaxH)
    return fail(CHYM_EINVAL, "chym_stats_noalloc: n_h exceeds the fixed limit of 4096");
  if (n_bins < 0 || n_bins > kNoAllocMaxBins || (hist && n_bins < 1))
    return fail(CHYM_EINVAL, "chym_stats_noalloc: n_bins must be in [1, 65536] with a histogram");
  if (kind != CHYM_J_PM1 && kind != CHYM_J_REAL) return fail(CHYM_EINVAL, "unknown J kind");
  if (!isfinite(E_gs)) return fail(CHYM_EINVAL, "E_gs must be finite");
  if (!hist) n_bins = 0;
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch_address(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(stats scratch)");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool pm1 = kind == CHYM_J_PM1;
  const double tol = pm1 ? 0.0 : 1e-9 * fabs(E_gs);
  double bin_w = pm1 ? 4.0 : 1e-3 * fabs(E_gs);
  if (!(bin_w > 0.0)) bin_w = 1.0;
  // the kernel initialises every word it reports (hits, bins, totals), so the
  // previous call's contents never leak into this one
  stats_kernel<<<1, kStatsThreads, sizeof(unsigned long long) * (size_t)n_h, st>>>(
      d_E, nullptr, n_runs, n_runs / n_h, n_h, E_gs, tol, bin_w, n_bins, (StatsOut*)scratch);
  CHYM_CUDA_TRY(cudaGetLastError());
  StatsOut head;
  CHYM_CUDA_TRY(cudaMemcpyAsync(&head, scratch, sizeof(head), cudaMemcpyDeviceToHost, st));
  const long long* d_hits = reinterpret_cast<const long long*>((const StatsOut*)scratch + 1);
  // per-pump counts are needed for P_max and W; without a caller buffer they go to a
  // fixed per-thread host array of the maximum size.  Every copy is ordered on st and
  // one synchronisation of st ends the call, so no other stream is waited for.
  static thread_local long long hits_tmp[kNoAllocMaxH];
  long long* hits = hits_per_h ? reinterpret_cast<long long*>(hits_per_h) : hits_tmp;
  CHYM_CUDA_TRY(cudaMemcpyAsync(hits, d_hits, sizeof(long long) * n_h, cudaMemcpyDeviceToHost, st));
  if (hist && n_bins)
    CHYM_CUDA_TRY(cudaMemcpyAsync(hist, d_hits + n_h, sizeof(long long) * n_bins,
                                  cudaMemcpyDeviceToHost, st));
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  const int reps = n_runs / n_h;
  double pmax = 0.0, psum = 0.0;
  int nz = 0;
  for (int i = 0; i < n_h; ++i) {
    const double P = (double)hits[i] / reps;
    pmax = std::max(pmax, P);
    psum += P;
    if (hits[i] > 0) ++nz;
  }
  out->P_max = pmax;
  out->W_range = nz ? psum / nz : 0.0;
  out->W_scan = psum / n_h;
  out->dE_mean = head.n_finite ? head.sum_dE / (double)head.n_finite : NAN;
  out->best_E = head.best_E;
  out->best_run = head.best_run;
  out->n_finite = head.n_finite;
  out->n_hits = head.n_hits;
  return CHYM_OK;
}

