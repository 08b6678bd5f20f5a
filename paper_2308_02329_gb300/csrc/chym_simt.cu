// chym_simt.cu -- SIMT step kernels (FP64 oracle-comparison mode and the plain
// FP32 form) and the initial-state kernel.
//
// Every step kernel owns RC runs per CTA for the whole launch and keeps their state
// in shared memory across all steps.  A sparse J (at most N^2 / 16 nonzeros) is read
// as compressed rows, so the product costs 2 nnz D flops per run and step rather
// than 2 N^2 D.  Per step:
//   phase A  y_{p,mu} = sum_q J_pq x_{q,mu}  (C = J_N (x) 1_D, Eq. 1);
//   phase B  x <- x + dt [(h-1) x - kappa x^3 - gamma x |x_p|^2 + eps alpha_mu y]
//            + sigma sqrt(dt) xi  with xi from Philox4x32-10 + Box-Muller.
// FP32 runs on the register-tiled kernel (step_simt_tiled_kernel, below), whose
// threads each own 4 spins x RB runs through both phases; FP64, and FP32 where a
// tile's state does not fit, run on the per-spin kernel (step_simt_kernel), whose
// threads each take one (spin, run group) in phase A and one (spin, run) in phase B,
// with J staged in shared memory when it fits and read through L1/L2 otherwise.
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

// FP32 Box-Muller on the SFU approximations with denormals flushed (no argument or
// result of the transform is denormal): u = (w + 1/2) 2^-32, r = scale sqrt(-2 ln u_r),
// angle 2 pi u_a - pi, and the pair negated back (cos t = -cos(t - pi), likewise sin).
__device__ __forceinline__ void box_muller_sfu(uint32_t wr, uint32_t wa, float scale, float& z0,
                                               float& z1) {
  const float ur = __fmaf_rn((float)wr, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float ua = __fmaf_rn((float)wa, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  float l2, r, s, c;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(ur));
  const float r2 = l2 * (-1.3862943611198906f * scale * scale);  // -2 ln 2 scale^2 log2 u
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
  const float t = __fmaf_rn(ua, 6.2831853071795865f, -3.1415926535897932f);
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(t));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(t));
  z0 = -r * c;
  z1 = -r * s;
}

// Philox4x32-10 with the ten round keys precomputed (two rounds per uint4).
__device__ __forceinline__ uint4 philox_rounds(uint4 c, const uint4* rk) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint4 kk = rk[i];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t k0 = h ? kk.z : kk.x, k1 = h ? kk.w : kk.y;
      const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
      const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
      c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
  }
  return c;
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

// ---------------------------------------------------------------------------
// Register-tiled FP32 form (the plain FP32 form: dense J, or the nonzeros of a sparse J).
// The CTA keeps its RC runs in shared memory as Xs[q][r][DP] (spin-major, the runs of
// one spin contiguous, components padded to DP).  Thread (tp, rg) owns the tile of
// spins 4 tp .. 4 tp + 3 and runs RB rg .. RB rg + RB - 1.  Dense J: per q it loads the
// four couplings J_{q, 4tp..4tp+3} (J symmetric, rows zero padded to NP; one 16-byte
// read-only load that stays in L1) and the RB x DP state values of its runs (16-byte
// shared loads) for 4 RB D FMAs.  Sparse J: per nonzero J_pq of each of its spins the
// same RB x DP state values for RB D FMAs.  The thread then updates its own tile, so the
// coupling product never leaves registers, and its noise follows the counter layout of
// the other kernels; a tile of four spins holds whole Philox blocks for D <= 2.
// (J in shared memory instead of L1 measured slower: it leaves fewer CTAs per SM.)
template <int D, bool CSR>
struct TileCfg {
  static constexpr int DP = D == 3 ? 4 : (D > 4 ? 8 : D);
  static constexpr int RB = D == 1 ? 8 : D <= 4 ? 4 : 2;
  static_assert(RB * DP <= 2 || (RB * DP) % 4 == 0, "state loads are 4, 8 or 16k bytes");
};

// The n = RB DP consecutive state values of one spin and run group (n = 1, 2 or 4k).
template <int n>
__device__ __forceinline__ void load_x(const float* src, float (&xv)[n]) {
  if constexpr (n == 1) {
    xv[0] = src[0];
  } else if constexpr (n == 2) {
    const float2 t = *reinterpret_cast<const float2*>(src);
    xv[0] = t.x;
    xv[1] = t.y;
  } else {
#pragma unroll
    for (int v = 0; v < n / 4; ++v) {
      const float4 t = reinterpret_cast<const float4*>(src)[v];
      xv[4 * v] = t.x;
      xv[4 * v + 1] = t.y;
      xv[4 * v + 2] = t.z;
      xv[4 * v + 3] = t.w;
    }
  }
}

template <int D, bool CSR>
__global__ void __launch_bounds__(512) step_simt_tiled_kernel(const float* __restrict__ Jp,
                                                              float* __restrict__ Xg,
                                                              const double* __restrict__ hg,
                                                              const uint64_t* __restrict__ seeds,
                                                              StepConsts sc, int RC, int NP,
                                                              CsrRows<float> csr) {
  using Cfg = TileCfg<D, CSR>;
  constexpr int DP = Cfg::DP, RB = Cfg::RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = sc.N;
  float* Xs = reinterpret_cast<float*>(smem_raw);                     // NP x RC x DP
  uint4* s_rk = reinterpret_cast<uint4*>(Xs + (size_t)NP * RC * DP);  // RC x 5 round keys
  int64_t* s_koff = reinterpret_cast<int64_t*>(s_rk + (size_t)RC * 5);
  float* s_hm1 = reinterpret_cast<float*>(s_koff + RC);
  const int run0 = blockIdx.x * RC;
  const int nr = min(RC, sc.n_runs - run0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tiles_p = NP / 4;
  const int tp = tid % tiles_p, rg = tid / tiles_p;
  const int p0 = 4 * tp, r0 = RB * rg;
  const bool active = rg < RC / RB;

  for (int i = tid; i < NP * RC * DP; i += nt) {
    const int mu = i % DP, r = (i / DP) % RC, p = i / (DP * RC);
    Xs[i] = (mu < D && p < N && r < nr) ? Xg[((size_t)(run0 + r) * N + p) * D + mu] : 0.f;
  }
  for (int r = tid; r < RC; r += nt) {
    uint32_t k0 = 0u, k1 = 0u;
    float hm1 = 0.f;
    int64_t ko = 0;
    if (r < nr) {
      const int run = run0 + r;
      k0 = (uint32_t)seeds[run];
      k1 = (uint32_t)(seeds[run] >> 32);
      hm1 = (float)(hg[sc.hidx[run]] - 1.0);
      ko = sc.koff[run];
    }
    for (int i = 0; i < 5; ++i)  // Weyl key schedule: round j uses key + j (W0, W1)
      s_rk[r * 5 + i] = make_uint4(k0 + (2u * i) * kPhiloxW0, k1 + (2u * i) * kPhiloxW1,
                                   k0 + (2u * i + 1u) * kPhiloxW0, k1 + (2u * i + 1u) * kPhiloxW1);
    s_koff[r] = ko;
    s_hm1[r] = hm1;
  }
  __syncthreads();

  const float dt = (float)sc.dt, gamma = (float)sc.gamma, kappa = (float)sc.kappa;
  const float nscale = (float)sc.noise_scale;
  const float inv_ramp = sc.sched_kind == 1 ? 1.f / (float)(sc.k_total - sc.k_anneal) : 0.f;
  float edt[4];  // dt eps w_p of the tile's spins
  int e_beg[4], e_end[4];  // the tile's compressed rows
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = p0 + i;
    edt[i] = (float)(sc.dt * sc.eps) * ((sc.w && p < N) ? (float)sc.w[p] : 1.f);
    e_beg[i] = e_end[i] = 0;
    if (CSR && p < N) {
      e_beg[i] = __ldg(csr.rp + p);
      e_end[i] = __ldg(csr.rp + p + 1);
    }
  }
  const float* xcol = Xs + (size_t)r0 * DP;
  for (int64_t k = sc.k0; k < sc.k0 + sc.steps; ++k) {
    float acc[4][RB][D];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int b = 0; b < RB; ++b)
#pragma unroll
        for (int mu = 0; mu < D; ++mu) acc[i][b][mu] = 0.f;
    // ---- coupling product y = (J (x) 1_D) x of the tile, in registers ----
    if (active) {
      if constexpr (CSR) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          for (int e = e_beg[i]; e < e_end[i]; ++e) {
            const float j = __ldg(csr.cv + e);
            float xv[RB * DP];
            load_x<RB * DP>(xcol + (size_t)__ldg(csr.ci + e) * RC * DP, xv);
#pragma unroll
            for (int b = 0; b < RB; ++b)
#pragma unroll
              for (int mu = 0; mu < D; ++mu) acc[i][b][mu] = fmaf(j, xv[b * DP + mu], acc[i][b][mu]);
          }
        }
      } else {
#pragma unroll 2
        for (int q = 0; q < N; ++q) {
          const float4 jv = __ldg(reinterpret_cast<const float4*>(Jp + (size_t)q * NP + p0));
          const float jq[4] = {jv.x, jv.y, jv.z, jv.w};
          float xv[RB * DP];
          load_x<RB * DP>(xcol + (size_t)q * RC * DP, xv);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int b = 0; b < RB; ++b)
#pragma unroll
              for (int mu = 0; mu < D; ++mu) acc[i][b][mu] = fmaf(jq[i], xv[b * DP + mu], acc[i][b][mu]);
        }
      }
    }
    __syncthreads();  // every read of the old state precedes the first update
    // ---- drift, annealing scale and noise of the tile ----
    if (active) {
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int r = r0 + b;
        if (r >= nr) continue;
        const int64_t kl = k - s_koff[r];
        float ramp = 1.f;  // alpha_mu(kl) for mu >= 1
        if (sc.sched_kind == 1 && kl >= sc.k_anneal)
          ramp = kl >= sc.k_total ? 0.f : fmaxf(0.f, 1.f - (float)(kl - sc.k_anneal) * inv_ramp);
        const float a1 = 1.f + dt * s_hm1[r];
        const uint4* rk = s_rk + r * 5;
        float z[4][D];
        if constexpr (D == 1) {
          const uint4 w = philox_rounds(noise_counter((uint32_t)tp, 0u, 0u, (uint64_t)kl), rk);
          box_muller_sfu(w.x, w.y, nscale, z[0][0], z[1][0]);
          box_muller_sfu(w.z, w.w, nscale, z[2][0], z[3][0]);
        } else if constexpr (D == 2) {
#pragma unroll
          for (int hb = 0; hb < 2; ++hb) {
            const uint4 w = philox_rounds(noise_counter((uint32_t)(2 * tp + hb), 0u, 0u, (uint64_t)kl), rk);
            box_muller_sfu(w.x, w.y, nscale, z[2 * hb][0], z[2 * hb][1]);
            box_muller_sfu(w.z, w.w, nscale, z[2 * hb + 1][0], z[2 * hb + 1][1]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int blk = 0; blk < (D + 3) / 4; ++blk) {
              const uint4 w = philox_rounds(noise_counter((uint32_t)(p0 + i), (uint32_t)blk, 0u, (uint64_t)kl), rk);
              float zz[4];
              box_muller_sfu(w.x, w.y, nscale, zz[0], zz[1]);
              if (D - 4 * blk > 2) box_muller_sfu(w.z, w.w, nscale, zz[2], zz[3]);
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (4 * blk + j < D) z[i][4 * blk + j] = zz[j];
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int p = p0 + i;
          if (p >= N) continue;
          float* x = Xs + ((size_t)p * RC + r) * DP;
          float xv[D];
          float n2 = 0.f;
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            xv[mu] = x[mu];
            n2 = fmaf(xv[mu], xv[mu], n2);
          }
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            const float xm = xv[mu];
            // x + dt [(h-1) x - kappa x^3 - gamma x |x_p|^2 + eps w_p alpha_mu y] + noise
            const float lin = a1 - dt * (kappa * xm * xm + gamma * n2);
            const float ea = mu == 0 ? edt[i] : edt[i] * ramp;
            x[mu] = fmaf(xm, lin, fmaf(ea, acc[i][b][mu], z[i][mu]));
          }
        }
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < nr * N * D; i += nt) {
    const int mu = i % D, p = (i / D) % N, r = i / (D * N);
    Xg[(size_t)run0 * N * D + i] = Xs[((size_t)p * RC + r) * DP + mu];
  }
}

// Launch of the tiled FP32 form; InvalidConfiguration when a run group does not fit its
// shared memory (the caller then takes the per-spin kernel).
template <int D, bool CSR>
cudaError_t launch_simt_tiled(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  using Cfg = TileCfg<D, CSR>;
  const int N = c->N, NP = c->j32p_ld;
  const bool csr = CSR;
  if (!csr && (!c->d_J32p || NP < N)) return cudaErrorInvalidConfiguration;
  const size_t per_run = (size_t)NP * Cfg::DP * sizeof(float) + 5 * sizeof(uint4) + sizeof(int64_t) + sizeof(float);
  if (Cfg::RB * per_run > kSimtSmemBudget) return cudaErrorInvalidConfiguration;
  // sparse J with long rows of state (N of about 1000 and more): the per-spin kernel,
  // whose 1024-thread CTAs measured faster there than CTAs of a few run groups
  if (CSR && kSimtSmemBudget / per_run < (size_t)(4 * Cfg::RB)) return cudaErrorInvalidConfiguration;
  int RC = (int)std::min<size_t>(kSimtSmemBudget / per_run, 512);
  RC = RC / Cfg::RB * Cfg::RB;
  // at most 512 threads, and no larger CTAs than it takes to fill the GPU
  while (RC > Cfg::RB && (NP / 4) * (RC / Cfg::RB) > 512) RC -= Cfg::RB;
  if ((NP / 4) * (RC / Cfg::RB) > 512) return cudaErrorInvalidConfiguration;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  while (RC > Cfg::RB && (int64_t)((sc.n_runs + RC - 1) / RC) < sms) RC -= Cfg::RB;
  const int threads = std::max(32, ((NP / 4) * (RC / Cfg::RB) + 31) / 32 * 32);
  const size_t smem = (size_t)RC * per_run;
  const int grid = (sc.n_runs + RC - 1) / RC;
  const CsrRows<float> rows{c->d_rp, c->d_ci, c->d_cv32};
  auto kern = step_simt_tiled_kernel<D, CSR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, smem, st>>>(c->d_J32p, (float*)c->d_X, c->d_h, c->d_seeds, sc, RC, NP, rows);
  return cudaGetLastError();
}

template <typename T, int D>
cudaError_t launch_simt_typed(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  const bool csr = c->sparse;  // the SIMT kernels use the compressed rows whenever they exist
  if constexpr (sizeof(T) == 4) {
    const cudaError_t e = csr ? launch_simt_tiled<D, true>(c, sc, st) : launch_simt_tiled<D, false>(c, sc, st);
    if (e != cudaErrorInvalidConfiguration) return e;
  }
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
