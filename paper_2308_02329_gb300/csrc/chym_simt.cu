// chym_simt.cu -- SIMT step kernels (FP64 oracle-comparison mode and the plain
// FP32 form) and the initial-state kernel.
//
// One CTA owns RC runs for the whole launch and keeps their state in shared
// memory across all steps; J (N x N) is staged in shared memory when it fits
// and read through L1/L2 otherwise.  A sparse J (N > 128, at most N^2 / 16
// nonzeros) is read as compressed rows instead, so the product costs 2 nnz D flops
// per run and step rather than 2 N^2 D.  Per step:
//   phase A  y_{p,mu} = sum_q J_pq x_{q,mu}  (C = J_N (x) 1_D, Eq. 1), J symmetric
//            so thread p reads column p of row q (consecutive p: no bank conflict);
//            each thread blocks RB runs so one J load feeds RB*D FMAs;
//   phase B  x <- x + dt [(h-1) x - kappa x^3 - gamma x |x_p|^2 + eps alpha_mu y]
//            + sigma sqrt(dt) xi  with xi from Philox4x32-10 + Box-Muller.
#include <algorithm>

#include "chym_internal.cuh"

namespace chym {
namespace {

template <typename T>
struct SimtTraits;
template <>
struct SimtTraits<double> {
  static constexpr int RB = 1;
};
template <>
struct SimtTraits<float> {
  static constexpr int RB = 4;
};

// Normal numbers of spin p for components 0..D-1 at step k (tag 0 or 1).
// For D <= 2 the 4/D spins with the same p / (4/D) share one Philox block: spin p
// takes the normals (p % (4/D)) * D .. + D - 1 of it (one Box-Muller pair).
template <typename T, int D>
__device__ __forceinline__ void spin_normals(uint64_t seed, uint32_t tag, uint64_t k, int p,
                                             T scale, T z[D]) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if constexpr (D <= 2) {
    constexpr uint32_t per = 4u / D;
    const uint4 w = philox4x32_10(noise_counter((uint32_t)p / per, 0u, tag, k), k0, k1);
    const uint32_t j0 = ((uint32_t)p % per) * D;  // first normal of this spin in the block
    const uint32_t wr = j0 >= 2u ? w.z : w.x, wa = j0 >= 2u ? w.w : w.y;
    T c, sn;
    if constexpr (sizeof(T) == 8) {
      double d0, d1;
      box_muller_f64(wr, wa, d0, d1);
      c = (T)(d0 * (double)scale);
      sn = (T)(d1 * (double)scale);
    } else {
      box_muller_f32(wr, wa, (float)scale, c, sn);
    }
    z[0] = (j0 & 1u) ? sn : c;
    if constexpr (D == 2) z[1] = sn;
  } else {
#pragma unroll
  for (int blk = 0; blk < (D + 3) / 4; ++blk) {
    const uint4 w = philox4x32_10(noise_counter((uint32_t)p, (uint32_t)blk, tag, k), k0, k1);
    T zz[4];
    if constexpr (sizeof(T) == 8) {
      double d[4];
      box_muller_f64(w.x, w.y, d[0], d[1]);
      if (D - 4 * blk > 2) box_muller_f64(w.z, w.w, d[2], d[3]);
      else d[2] = d[3] = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) zz[j] = (T)(d[j] * (double)scale);
    } else {
      box_muller_f32(w.x, w.y, (float)scale, zz[0], zz[1]);
      if (D - 4 * blk > 2) box_muller_f32(w.z, w.w, (float)scale, zz[2], zz[3]);
      else zz[2] = zz[3] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (4 * blk + j < D) z[4 * blk + j] = zz[j];
  }
  }
}

template <typename T, int D>
__global__ void init_kernel(T* __restrict__ X, const uint64_t* __restrict__ seeds, int N,
                            int n_runs, T init_std) {
  const int64_t pairs = (int64_t)N * n_runs;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < pairs;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int run = (int)(s / N), p = (int)(s % N);
    T z[D];
    spin_normals<T, D>(seeds[run], 1u, 0ull, p, init_std, z);
#pragma unroll
    for (int mu = 0; mu < D; ++mu) X[s * D + mu] = z[mu];
  }
}

// Compressed rows of a sparse J: row p holds the nonzeros rp[p] .. rp[p + 1] - 1.
template <typename T>
struct CsrRows {
  const int32_t* rp;
  const int32_t* ci;
  const T* cv;
};

template <typename T, int D, bool J_SMEM, bool CSR>
__global__ void __launch_bounds__(CSR && sizeof(T) == 4 ? 1024 : 512) step_simt_kernel(const T* __restrict__ Jg,
                                                        T* __restrict__ Xg,
                                                        const double* __restrict__ hg,
                                                        const uint64_t* __restrict__ seeds,
                                                        StepConsts sc, int RC, CsrRows<T> csr) {
  constexpr int RB = CSR ? 1 : SimtTraits<T>::RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = sc.N;
  T* Js = reinterpret_cast<T*>(smem_raw);
  T* Xs = J_SMEM ? Js + (size_t)N * N : Js;
  T* Ys = Xs + (size_t)RC * N * D;
  const int run0 = blockIdx.x * RC;
  const int nr = min(RC, sc.n_runs - run0);
  const int tid = threadIdx.x, nt = blockDim.x;

  if (J_SMEM)
    for (int i = tid; i < N * N; i += nt) Js[i] = Jg[i];
  for (int i = tid; i < RC * N * D; i += nt)
    Xs[i] = (i < nr * N * D) ? Xg[(size_t)run0 * N * D + i] : T(0);
  __syncthreads();
  const T* Jsrc = J_SMEM ? Js : Jg;

  const T dt = (T)sc.dt, gamma = (T)sc.gamma, kappa = (T)sc.kappa;
  const T inv_ramp = sc.sched_kind == 1 ? T(1) / (T)(sc.k_total - sc.k_anneal) : T(0);
  const int n_groups = RC / RB;
  for (int64_t k = sc.k0; k < sc.k0 + sc.steps; ++k) {
    // ---- phase A: coupling product, RB runs per thread ----
    for (int slot = tid; slot < N * n_groups; slot += nt) {
      const int p = slot % N, g = slot / N;
      T acc[RB][D];
#pragma unroll
      for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int mu = 0; mu < D; ++mu) acc[b][mu] = T(0);
      const T* xg = Xs + (size_t)(g * RB) * N * D;
      if constexpr (CSR) {
        const int e1 = __ldg(csr.rp + p + 1);
        for (int e = __ldg(csr.rp + p); e < e1; ++e) {
          const T j = __ldg(csr.cv + e);
          const int q = __ldg(csr.ci + e);
#pragma unroll
          for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int mu = 0; mu < D; ++mu) acc[b][mu] = fma(j, xg[((size_t)b * N + q) * D + mu], acc[b][mu]);
        }
      } else {
        for (int q = 0; q < N; ++q) {
          const T j = J_SMEM ? Jsrc[q * N + p] : __ldg(Jsrc + (size_t)q * N + p);
#pragma unroll
          for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int mu = 0; mu < D; ++mu) acc[b][mu] = fma(j, xg[((size_t)b * N + q) * D + mu], acc[b][mu]);
        }
      }
#pragma unroll
      for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int mu = 0; mu < D; ++mu) Ys[((size_t)(g * RB + b) * N + p) * D + mu] = acc[b][mu];
    }
    __syncthreads();
    // ---- phase B: local drift, annealing and noise (at each run's local step) ----
    for (int s = tid; s < nr * N; s += nt) {
      const int rl = s / N, p = s % N, run = run0 + rl;
      const int64_t kl = k - sc.koff[run];
      T ramp = T(1);  // alpha_mu(kl) for mu >= 1; mu = 0 keeps alpha = 1
      if (sc.sched_kind == 1 && kl >= sc.k_anneal)
        ramp = kl >= sc.k_total ? T(0) : T(1) - (T)(kl - sc.k_anneal) * inv_ramp;
      const T wp = sc.w ? (T)sc.w[p] : T(1);  // this spin's coupling weight
      T ea[D];
#pragma unroll
      for (int mu = 0; mu < D; ++mu) ea[mu] = (T)sc.eps * wp * (mu == 0 ? T(1) : ramp);
      const T hm1 = (T)(hg[sc.hidx[run]] - 1.0);
      T* x = Xs + (size_t)s * D;
      const T* y = Ys + (size_t)s * D;
      T n2 = T(0);
#pragma unroll
      for (int mu = 0; mu < D; ++mu) n2 = fma(x[mu], x[mu], n2);
      T z[D];
      spin_normals<T, D>(seeds[run], 0u, (uint64_t)kl, p, (T)sc.noise_scale, z);
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        const T xm = x[mu];
        const T f = hm1 * xm - kappa * xm * xm * xm - gamma * xm * n2 + ea[mu] * y[mu];
        x[mu] = xm + dt * f + z[mu];
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < nr * N * D; i += nt) Xg[(size_t)run0 * N * D + i] = Xs[i];
}

template <typename T, int D>
cudaError_t launch_simt_typed(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  const bool csr = c->sparse;  // the SIMT kernels use the compressed rows whenever they exist
  const int RB = csr ? 1 : SimtTraits<T>::RB;
  const int N = c->N;
  const size_t budget = kSimtSmemBudget;
  const size_t j_bytes = (size_t)N * N * sizeof(T);
  const bool j_smem = !csr && j_bytes <= budget / 2;
  const size_t per_run = (size_t)2 * N * D * sizeof(T);
  const size_t avail = budget - (j_smem ? j_bytes : 0);
  int RC = (int)std::min<size_t>(avail / per_run, 64);
  RC = std::max(RB, RC / RB * RB);
  if ((size_t)RC * per_run > avail) return cudaErrorInvalidConfiguration;  // N too large
  // do not make CTAs larger than needed to fill the GPU
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  while (RC > RB && (int64_t)((sc.n_runs + RC - 1) / RC) < sms) RC -= RB;
  const size_t smem = (j_smem ? j_bytes : 0) + (size_t)RC * per_run;
  // the FP32 compressed-row form needs few registers: twice the warps hide its gathers
  const int threads = std::min(csr && sizeof(T) == 4 ? 1024 : 512, std::max(64, ((N * (RC / RB) + 31) / 32) * 32));
  const int grid = (sc.n_runs + RC - 1) / RC;
  const T* J = sizeof(T) == 8 ? (const T*)c->d_J64 : (const T*)c->d_J32;
  T* X = (T*)c->d_X;
  const CsrRows<T> rows{c->d_rp, c->d_ci, sizeof(T) == 8 ? (const T*)c->d_cv64 : (const T*)c->d_cv32};
  auto kern = csr ? step_simt_kernel<T, D, false, true>
                  : j_smem ? step_simt_kernel<T, D, true, false> : step_simt_kernel<T, D, false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(J, X, c->d_h, c->d_seeds, sc, RC, rows);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_simt_D(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  switch (c->D) {
    case 1: return launch_simt_typed<T, 1>(c, sc, st);
    case 2: return launch_simt_typed<T, 2>(c, sc, st);
    case 3: return launch_simt_typed<T, 3>(c, sc, st);
    case 4: return launch_simt_typed<T, 4>(c, sc, st);
    case 5: return launch_simt_typed<T, 5>(c, sc, st);
    case 6: return launch_simt_typed<T, 6>(c, sc, st);
    case 7: return launch_simt_typed<T, 7>(c, sc, st);
    case 8: return launch_simt_typed<T, 8>(c, sc, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_init_typed(chym_ctx* c, cudaStream_t st, double init_std) {
  const int64_t pairs = (int64_t)c->N * c->n_runs;
  const int threads = 256;
  const int grid = (int)std::min<int64_t>((pairs + threads - 1) / threads, 152 * 32);
  T* X = (T*)c->d_X;
  switch (c->D) {
#define CHYM_INIT_CASE(DD) \
  case DD: init_kernel<T, DD><<<grid, threads, 0, st>>>(X, c->d_seeds, c->N, c->n_runs, (T)init_std); break;
    CHYM_INIT_CASE(1) CHYM_INIT_CASE(2) CHYM_INIT_CASE(3) CHYM_INIT_CASE(4)
    CHYM_INIT_CASE(5) CHYM_INIT_CASE(6) CHYM_INIT_CASE(7) CHYM_INIT_CASE(8)
#undef CHYM_INIT_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Reinitialise the listed runs from new seeds at local step 0 (offset = current k).
__global__ void fill_hidx_kernel(int32_t* hidx, int n_runs, int replicas) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_runs; r += gridDim.x * blockDim.x)
    hidx[r] = r / replicas;
}

template <typename T, int D>
__global__ void reseed_kernel(T* __restrict__ X, uint64_t* __restrict__ seeds, int64_t* __restrict__ koff,
                              int32_t* __restrict__ hidx, const int32_t* __restrict__ runs, int n,
                              const uint64_t* __restrict__ new_seeds, const int32_t* __restrict__ new_hidx,
                              int N, int64_t k_now, T init_std) {
  const int64_t total = (int64_t)n * N;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(s / N), p = (int)(s % N);
    const int run = runs[i];
    const uint64_t sd = new_seeds[i];
    T z[D];
    spin_normals<T, D>(sd, 1u, 0ull, p, init_std, z);
#pragma unroll
    for (int mu = 0; mu < D; ++mu) X[((int64_t)run * N + p) * D + mu] = z[mu];
    if (p == 0) {
      seeds[run] = sd;
      koff[run] = k_now;
      if (new_hidx) hidx[run] = new_hidx[i];
    }
  }
}

template <typename T>
cudaError_t launch_reseed_typed(chym_ctx* c, const int32_t* runs, int n, const uint64_t* ns,
                                const int32_t* nh, double init_std, cudaStream_t st) {
  const int threads = 256;
  const int grid = (int)std::min<int64_t>(((int64_t)n * c->N + threads - 1) / threads, 152 * 16);
  T* X = (T*)c->d_X;
  switch (c->D) {
#define CHYM_RESEED_CASE(DD)                                                                       \
  case DD:                                                                                        \
    reseed_kernel<T, DD><<<grid, threads, 0, st>>>(X, c->d_seeds, c->d_koff, c->d_hidx, runs, n, ns, nh, \
                                                  c->N, c->k, (T)init_std);                        \
    break;
    CHYM_RESEED_CASE(1) CHYM_RESEED_CASE(2) CHYM_RESEED_CASE(3) CHYM_RESEED_CASE(4)
    CHYM_RESEED_CASE(5) CHYM_RESEED_CASE(6) CHYM_RESEED_CASE(7) CHYM_RESEED_CASE(8)
#undef CHYM_RESEED_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_reseed(chym_ctx* c, const int32_t* d_runs, int n, const uint64_t* d_new_seeds,
                          const int32_t* d_new_hidx, double init_std, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (c->prec == CHYM_PREC_FP64)
    return launch_reseed_typed<double>(c, d_runs, n, d_new_seeds, d_new_hidx, init_std, st);
  return launch_reseed_typed<float>(c, d_runs, n, d_new_seeds, d_new_hidx, init_std, st);
}

cudaError_t launch_fill_hidx(int32_t* hidx, int n_runs, int replicas, cudaStream_t st) {
  if (n_runs <= 0) return cudaSuccess;
  fill_hidx_kernel<<<(n_runs + 255) / 256, 256, 0, st>>>(hidx, n_runs, replicas);
  return cudaGetLastError();
}

cudaError_t launch_step_simt(chym_ctx* c, const StepConsts& sc, int32_t prec, cudaStream_t st) {
  if (sc.steps <= 0 || sc.n_runs <= 0) return cudaSuccess;
  if (prec == CHYM_PREC_FP64) return launch_simt_D<double>(c, sc, st);
  return launch_simt_D<float>(c, sc, st);
}

cudaError_t launch_init(chym_ctx* c, int32_t prec, cudaStream_t st, double init_std) {
  if (c->n_runs <= 0) return cudaSuccess;
  if (prec == CHYM_PREC_FP64) return launch_init_typed<double>(c, st, init_std);
  return launch_init_typed<float>(c, st, init_std);
}

}  // namespace chym
