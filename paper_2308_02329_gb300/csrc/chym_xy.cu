// chym_xy.cu -- readout of XY (D = 2) runs by best-axis rounding.
//
// The XY machine (D = 2 without annealing, text after Fig. 2) leaves every
// hyperspin as a planar vector; reading only its first component, as the Ising
// readout does, fixes the axis arbitrarily.  Best-axis rounding tries every axis
// u = (cos phi, sin phi): the pattern s_p = sign(x_p . u) changes only where u is
// perpendicular to a spin, at phi_p = theta_p + pi/2 (mod pi), so sweeping phi
// over [0, pi) flips one spin per critical angle.  One CTA per run:
//   1. critical angles (FP64 atan2, so that their order matches the oracle) and
//      the pattern of an axis inside the interval that wraps through pi;
//   2. bitonic sort of (angle, spin) in shared memory;
//   3. local fields h_q = sum_p J_qp s_p (N^2 multiply-adds) and E = -sum s h;
//   4. the sweep: per critical angle, E += 4 s_p h_p, s_p = -s_p and every h_q
//      moves by 2 J_qp s_p; after the last spin of a group of equal angles the
//      energy is a candidate; the lowest one (first in sweep order) wins;
//   5. the winning pattern is rebuilt and bit-packed.
// A run whose state holds a non-finite value (a diverged run) gets E = NaN, as in
// the Ising readout, and no sweep; its spins are then unspecified.
#include <math.h>

#include "chym_internal.cuh"

namespace chym {
namespace {

constexpr int kXyThreads = 256;
constexpr int kXyMaxN = 4096;

template <typename T, bool PM1>
__global__ void __launch_bounds__(kXyThreads) round_xy_kernel(const T* __restrict__ X, int N, int P2,
                                                              const int8_t* __restrict__ J8,
                                                              const double* __restrict__ J64,
                                                              double* __restrict__ E_out,
                                                              uint64_t* __restrict__ spins_out) {
  extern __shared__ __align__(16) unsigned char xy_smem[];
  double* key = reinterpret_cast<double*>(xy_smem);         // P2 critical angles
  double* h = key + P2;                                      // N local fields
  int* idx = reinterpret_cast<int*>(h + N);                  // P2 spin indices
  int8_t* s = reinterpret_cast<int8_t*>(idx + P2);           // N spins
  __shared__ double red[kXyThreads / 32];
  __shared__ double s_phi0;
  __shared__ int s_live, s_bad;
  const int run = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  const T* x = X + (size_t)run * N * 2;
  const double pi = 3.14159265358979323846;
  // 1. critical angles; spins of zero length never flip (key +inf)
  for (int i = tid; i < P2; i += blockDim.x) {
    double k = INFINITY;
    if (i < N) {
      const double a = (double)x[2 * (size_t)i], b = (double)x[2 * (size_t)i + 1];
      if (!isfinite(a) || !isfinite(b)) s_bad = 1;
      else if (a != 0.0 || b != 0.0) {
        k = fmod(atan2(b, a) + 0.5 * pi, pi);
        if (k < 0.0) k += pi;
      }
    }
    key[i] = k;
    idx[i] = i;
  }
  __syncthreads();
  // 2. bitonic sort by angle (ties by spin index)
  for (int kk = 2; kk <= P2; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const double a = key[i], b = key[l];
          const int ia = idx[i], ib = idx[l];
          const bool gt = a > b || (a == b && ia > ib);
          const bool up = (i & kk) == 0;
          if (gt == up) {
            key[i] = b;
            key[l] = a;
            idx[i] = ib;
            idx[l] = ia;
          }
        }
      }
      __syncthreads();
    }
  if (tid == 0) {
    int live = 0;
    while (live < N && key[live] < INFINITY) ++live;
    if (s_bad) live = 0;
    s_live = live;
    // an axis inside the interval that wraps from the last critical angle through pi
    s_phi0 = live > 0 ? 0.5 * (key[live - 1] + key[0] + pi) : 0.0;
  }
  __syncthreads();
  const int live = s_live;
  const double u0 = cos(s_phi0), u1 = sin(s_phi0);
  for (int p = tid; p < N; p += blockDim.x)
    s[p] = ((double)x[2 * (size_t)p] * u0 + (double)x[2 * (size_t)p + 1] * u1 >= 0.0) ? 1 : -1;
  __syncthreads();
  // 3. local fields and the energy of the starting pattern
  double part = 0.0;
  for (int q = tid; q < N; q += blockDim.x) {
    double f = 0.0;
    for (int p = 0; p < N; ++p)
      f += (PM1 ? (double)J8[(size_t)q * N + p] : J64[(size_t)q * N + p]) * (double)s[p];
    h[q] = f;
    part += (double)s[q] * f;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  double E = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) E -= red[w];
  // 4. the sweep over the critical angles (every thread keeps the same E)
  double best = E;
  int best_i = -1;
  for (int i = 0; i < live; ++i) {
    const int p = idx[i];
    const double sp = (double)s[p];
    E += 4.0 * sp * h[p];
    __syncthreads();  // every thread has read h[p] and s[p]
    const double ns = -sp;
    if (tid == 0) s[p] = (int8_t)ns;
    for (int q = tid; q < N; q += blockDim.x)
      h[q] += 2.0 * ns * (PM1 ? (double)J8[(size_t)q * N + p] : J64[(size_t)q * N + p]);
    __syncthreads();
    if ((i + 1 == live || key[i + 1] != key[i]) && E < best) {
      best = E;
      best_i = i;
    }
  }
  // 5. the winning pattern: the starting one with the first best_i + 1 spins flipped
  for (int p = tid; p < N; p += blockDim.x)
    s[p] = ((double)x[2 * (size_t)p] * u0 + (double)x[2 * (size_t)p + 1] * u1 >= 0.0) ? 1 : -1;
  __syncthreads();
  for (int i = tid; i <= best_i; i += blockDim.x) s[idx[i]] = (int8_t)(-s[idx[i]]);
  __syncthreads();
  if (tid == 0) E_out[run] = s_bad ? (double)NAN : best;
  if (spins_out) {
    const int words = (N + 63) / 64;
    for (int wd = tid; wd < words; wd += blockDim.x) {
      uint64_t bits = 0;
      for (int b = 0; b < 64 && wd * 64 + b < N; ++b)
        if (s[wd * 64 + b] > 0) bits |= (uint64_t)1 << b;
      spins_out[(size_t)run * words + wd] = bits;
    }
  }
}

template <typename T>
cudaError_t launch_round_xy_typed(chym_ctx* c, double* d_E, uint64_t* d_spins, cudaStream_t st) {
  int P2 = 1;
  while (P2 < c->N) P2 <<= 1;
  const size_t smem = (size_t)P2 * (sizeof(double) + sizeof(int)) + (size_t)c->N * (sizeof(double) + 1);
  auto kern = c->kind == CHYM_J_PM1 ? round_xy_kernel<T, true> : round_xy_kernel<T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<c->n_runs, kXyThreads, smem, st>>>((const T*)c->d_X, c->N, P2, c->d_J8, c->d_J64, d_E, d_spins);
  return cudaGetLastError();
}

cudaError_t launch_round_xy(chym_ctx* c, double* d_E, uint64_t* d_spins, cudaStream_t st) {
  if (c->n_runs <= 0) return cudaSuccess;
  if (c->prec == CHYM_PREC_FP64) return launch_round_xy_typed<double>(c, d_E, d_spins, st);
  return launch_round_xy_typed<float>(c, d_E, d_spins, st);
}

chym_status check_xy(const chym_ctx* c) {
  if (c->D != 2) return fail(CHYM_EINVAL, "best-axis rounding needs D = 2");
  if (c->N > kXyMaxN) return fail(CHYM_EINVAL, "best-axis rounding supports N <= 4096");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state: call chym_run first");
  return CHYM_OK;
}

}  // namespace
}  // namespace chym

using namespace chym;

extern "C" {

CHYM_API chym_status chym_readout_xy_device(chym_ctx* c, double* d_E, uint64_t* d_spins, void* stream) {
  chym::TraceRange trace_("chym_readout_xy_device");
  if (!c || !d_E) return fail(CHYM_EINVAL, "NULL argument");
  const chym_status ok = check_xy(c);
  if (ok != CHYM_OK) return ok;
  CHYM_CUDA_TRY(launch_round_xy(c, d_E, d_spins, (cudaStream_t)stream));
  return CHYM_OK;
}

CHYM_API chym_status chym_readout_xy(chym_ctx* c, double* E_out, uint64_t* spins_out, void* stream) {
  chym::TraceRange trace_("chym_readout_xy");
  if (!c || !E_out) return fail(CHYM_EINVAL, "NULL argument");
  const chym_status ok = check_xy(c);
  if (ok != CHYM_OK) return ok;
  cudaStream_t st = (cudaStream_t)stream;
  // the context's energy buffers hold the result; the cached Ising energies are gone
  CHYM_CUDA_TRY(launch_round_xy(c, c->d_E, c->d_spins, st));
  c->have_energy = false;
  CHYM_CUDA_TRY(cudaMemcpyAsync(E_out, c->d_E, sizeof(double) * c->n_runs, cudaMemcpyDeviceToHost, st));
  if (spins_out) {
    const size_t words = (size_t)(c->N + 63) / 64;
    CHYM_CUDA_TRY(cudaMemcpyAsync(spins_out, c->d_spins, sizeof(uint64_t) * c->n_runs * words,
                                  cudaMemcpyDeviceToHost, st));
  }
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  return CHYM_OK;
}

}  // extern "C"
