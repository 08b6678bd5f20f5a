// chym_k2.cu -- large-N step: tcgen05 GEMM Y = J X with the CHYM update fused
// into its epilogue, one launch per Euler-Maruyama step (N > 128).
//
// Layouts (device, internal to this path):
//   Xm[c][p]      FP32 master state, column c = r * D + mu, spin p contiguous,
//                 leading dimension KP = 128 * MT (MT = ceil(N / 128));
//   Xt[b][t][ct][kc]  BF16 hi (t = 0) / lo (t = 1) split of Xm, double buffered
//                 (b), stored as ready-made B-operand blocks: column tile ct
//                 (n columns) x K chunk kc (64 spins), K-major canonical layout
//                 without swizzle: core matrix = 8 columns x 16 bytes, core
//                 (col/8, k/8) at (col/8) * kSboB + (k/8) * kLboB (padded strides
//                 keep the epilogue's shared-memory stores free of bank conflicts);
//   Aimg[t][mt][kc]  J (t = 0) and, for real couplings, its BF16 residual (t = 1)
//                 as A-operand blocks of 128 rows x 64 K, core (row/8, k/8) at
//                 (row/8) * 1024 + (k/8) * 128.
// CTA (mt, ct) computes rows [128 mt, 128 mt + 128) of Y for columns of tile ct:
//   warp 0  producer: TMA bulk copies of the A / B_hi / B_lo blocks of each K
//           chunk into a two-stage ring (mbarrier expect_tx);
//   warp 1  MMA issuer: tcgen05.mma (M = 128, N = n, K = 16), J_hi X_hi + J_hi X_lo
//           (+ J_lo X_hi), FP32 accumulator in TMEM;
//   warps 2-9  epilogue: thread = spin (TMEM lane) x column half; reads Y
//           (tcgen05.ld) and x (global), applies drift, loss, annealing and
//           Philox noise (text after Eq. 1 and after Fig. 2), writes x back and
//           stages the new BF16 hi/lo blocks of its 128 spins, which are then
//           bulk-stored into the other buffer (next step's B operand).
// All waits are bounded; a timeout raises the status word and the CTA returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "chym_internal.cuh"

namespace chym {
namespace {

constexpr uint32_t kLboB = 144;          // K-direction core stride of a B block (padded)
constexpr uint32_t kSboB = 8 * kLboB;    // column-group stride (8 K cores per 64 K)
constexpr uint32_t kABlock = 128 * 64 * 2;  // bytes of an A block
constexpr int kStages = 2;
constexpr int kThreads = 320;            // 10 warps
constexpr int kTimeoutNs = 2000000000;

__host__ __device__ constexpr int k2_cols(int D) {  // column tile width n
  return D == 3 ? 96 : D == 5 ? 80 : D == 6 ? 96 : D == 7 ? 112 : 128;
}
__host__ __device__ constexpr uint32_t b_block_bytes(int n) { return (uint32_t)(n / 8) * kSboB; }

struct K2Args {
  int N, KP, MT, KC, CT, n_runs, C;  // C = n_runs * D columns
  int a_terms;
  int64_t k;                          // step index of this launch
  float gdt, kdt, edt_mu0, edt_mu, neg2ln2s2;
  const float* ar;                    // per run: 1 + dt (h - 1)
  const uint4* rk;                    // per run: Philox round keys [5]
  unsigned* status;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 0u) {
      const uint64_t t = global_timer();
      if (it == 0) t0 = t;
      else if (t - t0 > (uint64_t)kTimeoutNs) return false;
    }
  }
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void philox_round(uint4& c, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x, p1 = (uint64_t)kPhiloxM1 * c.z;
  c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                 (uint32_t)p0);
}
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint4* __restrict__ rk) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint4 kk = __ldg(rk + i);
    philox_round(c, kk.x, kk.y);
    philox_round(c, kk.z, kk.w);
  }
  return c;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// Box-Muller on one pair of words (see box_muller_f32 in chym_internal.cuh).
__device__ __forceinline__ void box_muller(uint32_t wr, uint32_t wa, float neg2ln2s2, float& z0,
                                           float& z1) {
  const float ur = __fmaf_rn((float)wr, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float th = __fmaf_rn((float)wa, 1.4629180792671596e-09f, -3.1415926528582302f);
  const float r = -sqrt_approx(neg2ln2s2 * __log2f(ur));
  float s, c;
  __sincosf(th, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

template <int D>
__global__ void __launch_bounds__(kThreads, 2) step_k2_kernel(const uint8_t* __restrict__ Aimg,
                                                              float* __restrict__ Xm,
                                                              const uint8_t* __restrict__ Xt_cur,
                                                              uint8_t* __restrict__ Xt_next,
                                                              K2Args a) {
  constexpr int n = k2_cols(D);
  constexpr uint32_t BB = b_block_bytes(n);
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, ct = blockIdx.y;
  const uint32_t stage_bytes = (uint32_t)a.a_terms * kABlock + 2u * BB;
  const uint32_t blocks_per_buf = (uint32_t)a.CT * a.KC;  // blocks of one (hi or lo) buffer

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&s_tmem)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    s_abort = 0;
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&acc_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      for (int kc = 0; kc < a.KC; ++kc) {
        const int s = kc % kStages;
        if (kc >= kStages && !mbar_wait(smem_addr(&empty_bar[s]), (uint32_t)((kc / kStages - 1) & 1))) {
          atomicOr(a.status, STATUS_TIMEOUT);
          s_abort = 1;
          break;
        }
        const uint32_t base = smem_addr(smem) + (uint32_t)s * stage_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         smem_addr(&full_bar[s])), "r"(stage_bytes) : "memory");
        for (int t = 0; t < a.a_terms; ++t)
          bulk_g2s(base + (uint32_t)t * kABlock,
                   Aimg + ((size_t)(t * a.MT + mt) * a.KC + kc) * kABlock, kABlock,
                   smem_addr(&full_bar[s]));
        const size_t blk = (size_t)ct * a.KC + kc;
        bulk_g2s(base + (uint32_t)a.a_terms * kABlock, Xt_cur + blk * BB, BB, smem_addr(&full_bar[s]));
        bulk_g2s(base + (uint32_t)a.a_terms * kABlock + BB, Xt_cur + (blocks_per_buf + blk) * BB, BB,
                 smem_addr(&full_bar[s]));
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      bool ok = true;
      for (int kc = 0; kc < a.KC && ok; ++kc) {
        const int s = kc % kStages;
        if (!mbar_wait(smem_addr(&full_bar[s]), (uint32_t)((kc / kStages) & 1))) {
          atomicOr(a.status, STATUS_TIMEOUT);
          s_abort = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_addr(smem) + (uint32_t)s * stage_bytes;
        const uint32_t bhi = base + (uint32_t)a.a_terms * kABlock, blo = bhi + BB;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t da = smem_desc(base + (uint32_t)ks * 256u, 128u, 1024u);
          mma_bf16(tmem, da, smem_desc(bhi + (uint32_t)ks * 2u * kLboB, kLboB, kSboB), idesc,
                   (kc > 0 || ks > 0) ? 1u : 0u);
          mma_bf16(tmem, da, smem_desc(blo + (uint32_t)ks * 2u * kLboB, kLboB, kSboB), idesc, 1u);
          if (a.a_terms > 1)
            mma_bf16(tmem, smem_desc(base + kABlock + (uint32_t)ks * 256u, 128u, 1024u),
                     smem_desc(bhi + (uint32_t)ks * 2u * kLboB, kLboB, kSboB), idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&empty_bar[s])) : "memory");
      }
      if (ok)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&acc_bar)) : "memory");
      else
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acc_bar)) : "memory");
    }
  } else {
    // ---------------- epilogue: 8 warps ----------------
    const int q = warp & 3;                     // TMEM lane quarter
    const int half = (warp - 2) >> 2;           // column half
    const int i_loc = q * 32 + lane;            // row within the M tile
    const int p = mt * 128 + i_loc;             // spin
    const bool live = p < a.N;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&acc_bar), 0u)) && !s_abort;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // staging: the tile's new hi/lo blocks, K chunks 2 mt (rows 0-63) and 2 mt + 1
    // (rows 64-127); they reuse the pipeline stages, free once the accumulator is ready
    uint8_t* stg_hi = smem + (size_t)(i_loc >> 6) * BB;
    uint8_t* stg_lo = smem + (size_t)(2 + (i_loc >> 6)) * BB;
    const int kl = i_loc & 63;
    const uint32_t k_off = (uint32_t)(kl & 7) * 2u + (uint32_t)(kl >> 3) * kLboB;
    const int c_begin = half * (n / 2);
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    float e_mu[D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) e_mu[mu] = mu == 0 ? a.edt_mu0 : a.edt_mu;
    if (ok) {
      for (int c0 = c_begin; c0 < c_begin + n / 2; c0 += D) {
        const int c_glob = ct * n + c0;
        const int run = c_glob / D;
        // TMEM loads and their wait in one asm statement per column (see tmem_ld_wait)
        uint32_t yr[D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\t"
              "tcgen05.wait::ld.sync.aligned;"
              : "=r"(yr[mu])
              : "r"(trow + (uint32_t)(c0 + mu))
              : "memory");
        float xn[D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu) xn[mu] = 0.f;
        if (live && run < a.n_runs) {
          float x[D], n2 = 0.f;
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            x[mu] = Xm[(size_t)(c_glob + mu) * a.KP + p];
            n2 = fmaf(x[mu], x[mu], n2);
          }
          const float t = fmaf(-a.gdt, n2, __ldg(a.ar + run));
          float z[4 * ((D + 3) / 4)];
#pragma unroll
          for (int blk = 0; blk < (D + 3) / 4; ++blk) {
            const uint4 w = philox_rk(noise_counter((uint32_t)p, (uint32_t)blk, 0u, (uint64_t)a.k),
                                      a.rk + (size_t)run * 5);
            box_muller(w.x, w.y, a.neg2ln2s2, z[4 * blk], z[4 * blk + 1]);
            if (D - 4 * blk > 2) box_muller(w.z, w.w, a.neg2ln2s2, z[4 * blk + 2], z[4 * blk + 3]);
          }
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            const float s = fmaf(-a.kdt * x[mu], x[mu], t);
            xn[mu] = fmaf(x[mu], s, fmaf(e_mu[mu], __uint_as_float(yr[mu]), z[mu]));
            Xm[(size_t)(c_glob + mu) * a.KP + p] = xn[mu];
          }
        }
        // staged B blocks (zeros for padding spins and padding runs)
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
          const int c = c0 + mu;
          const uint32_t off = (uint32_t)(c >> 3) * kSboB + (uint32_t)(c & 7) * 16u + k_off;
          const __nv_bfloat16 hi = __float2bfloat16_rn(xn[mu]);
          const __nv_bfloat16 lo = __float2bfloat16_rn(xn[mu] - __bfloat162float(hi));
          *reinterpret_cast<__nv_bfloat16*>(stg_hi + off) = hi;
          *reinterpret_cast<__nv_bfloat16*>(stg_lo + off) = lo;
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (warp == 2 && lane == 0 && ok) {
      for (int t = 0; t < 2; ++t)
        for (int hh = 0; hh < 2; ++hh) {
          const size_t blk = (size_t)t * blocks_per_buf + (size_t)ct * a.KC + (2 * mt + hh);
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                           Xt_next + blk * BB),
                       "r"(smem_addr(smem + (size_t)(2 * t + hh) * BB)), "r"(BB) : "memory");
        }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
}

// X[run][p][mu] (float) -> Xm[c][p] and the hi/lo blocks of buffer 0 (zeros in padding).
template <int D>
__global__ void k2_pack_kernel(const float* __restrict__ X, float* __restrict__ Xm,
                               uint8_t* __restrict__ Xt, int N, int KP, int KC, int CT,
                               int n_runs) {
  constexpr int n = k2_cols(D);
  constexpr uint32_t BB = b_block_bytes(n);
  const size_t total = (size_t)CT * n * KP;
  const size_t per_buf = (size_t)CT * KC * BB;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % KP);
    const size_t c = e / KP;
    const size_t run = c / D;
    const int mu = (int)(c % D);
    float v = 0.f;
    if (p < N && run < (size_t)n_runs) v = X[(run * N + p) * D + mu];
    if (run < (size_t)n_runs) Xm[c * KP + p] = v;
    const int ct = (int)(c / n), cl = (int)(c % n), kc = p / 64, kl = p % 64;
    const size_t off = ((size_t)ct * KC + kc) * BB + (size_t)(cl >> 3) * kSboB + (cl & 7) * 16 +
                       (kl & 7) * 2 + (size_t)(kl >> 3) * kLboB;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    *reinterpret_cast<__nv_bfloat16*>(Xt + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(Xt + per_buf + off) = lo;
  }
}

__global__ void k2_unpack_kernel(const float* __restrict__ Xm, float* __restrict__ X, int N, int D,
                                 int KP, int n_runs) {
  const size_t total = (size_t)n_runs * N * D;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int mu = (int)(e % D);
    const size_t rp = e / D;
    const int p = (int)(rp % N);
    const size_t run = rp / N;
    X[e] = Xm[(run * D + mu) * KP + p];
  }
}

// per-run constants: 1 + dt (h - 1) and the ten Philox round keys
__global__ void k2_runconst_kernel(const double* __restrict__ h, const uint64_t* __restrict__ seeds,
                                   int n_runs, int replicas, double dt, float* ar, uint4* rk) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_runs; r += gridDim.x * blockDim.x) {
    ar[r] = (float)(1.0 + dt * (h[r / replicas] - 1.0));
    const uint32_t k0 = (uint32_t)seeds[r], k1 = (uint32_t)(seeds[r] >> 32);
    for (int i = 0; i < 5; ++i)
      rk[(size_t)r * 5 + i] = make_uint4(k0 + (2u * i) * kPhiloxW0, k1 + (2u * i) * kPhiloxW1,
                                         k0 + (2u * i + 1u) * kPhiloxW0, k1 + (2u * i + 1u) * kPhiloxW1);
  }
}

uint16_t bf16_bits_host(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)((u >> 16) | ((u & 0xFFFFu) ? 0x40u : 0u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_float_host(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

template <int D>
cudaError_t k2_run_typed(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  constexpr int n = k2_cols(D);
  const int N = c->N, MT = (N + 127) / 128, KP = MT * 128, KC = KP / 64;
  const int C = sc.n_runs * D, CT = (C + n - 1) / n;
  const int terms = c->kind == CHYM_J_PM1 ? 1 : 2;
  const size_t BB = b_block_bytes(n);
  // workspace: Xm, Xt (2 buffers x hi/lo), per-run constants
  const size_t xm_bytes = (size_t)CT * n * KP * 4;
  const size_t xt_bytes = (size_t)2 * 2 * CT * KC * BB;
  const size_t ar_bytes = ((size_t)sc.n_runs * 4 + 255) / 256 * 256;
  const size_t rk_bytes = (size_t)sc.n_runs * 5 * 16;
  const size_t need = xm_bytes + xt_bytes + ar_bytes + rk_bytes;
  if (need > c->k2_ws_bytes) {
    if (c->d_k2_ws) cudaFree(c->d_k2_ws);
    c->d_k2_ws = nullptr;
    c->k2_ws_bytes = 0;
    cudaError_t e = cudaMalloc(&c->d_k2_ws, need);
    if (e != cudaSuccess) return e;
    c->k2_ws_bytes = need;
  }
  uint8_t* ws = (uint8_t*)c->d_k2_ws;
  float* Xm = (float*)ws;
  uint8_t* Xt = ws + xm_bytes;
  float* ar = (float*)(Xt + xt_bytes);
  uint4* rk = (uint4*)((uint8_t*)ar + ar_bytes);
  cudaError_t e = cudaMemsetAsync(Xt, 0, xt_bytes, st);
  if (e != cudaSuccess) return e;
  k2_runconst_kernel<<<(sc.n_runs + 255) / 256, 256, 0, st>>>(c->d_h, c->d_seeds, sc.n_runs,
                                                             sc.replicas, sc.dt, ar, rk);
  k2_pack_kernel<D><<<152 * 8, 256, 0, st>>>((const float*)c->d_X, Xm, Xt, N, KP, KC, CT, sc.n_runs);
  K2Args a;
  a.N = N;
  a.KP = KP;
  a.MT = MT;
  a.KC = KC;
  a.CT = CT;
  a.n_runs = sc.n_runs;
  a.C = C;
  a.a_terms = terms;
  a.gdt = (float)(sc.dt * sc.gamma);
  a.kdt = (float)(sc.dt * sc.kappa);
  a.edt_mu0 = (float)(sc.dt * sc.eps);
  a.neg2ln2s2 = (float)(-2.0 * 0.69314718055994531 * sc.noise_scale * sc.noise_scale);
  a.ar = ar;
  a.rk = rk;
  a.status = c->d_status;
  const size_t stage_bytes = (size_t)terms * kABlock + 2 * BB;
  const size_t smem = std::max<size_t>(kStages * stage_bytes, 4 * BB);
  auto kern = step_k2_kernel<D>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const size_t buf = (size_t)2 * CT * KC * BB;  // one (hi + lo) buffer
  for (int64_t s = 0; s < sc.steps; ++s) {
    const int64_t k = sc.k0 + s;
    a.k = k;
    const double alpha = alpha_of(sc.sched_kind, k, sc.k_anneal, sc.k_total, 1);
    a.edt_mu = (float)(sc.dt * sc.eps * alpha);
    const uint8_t* cur = Xt + (size_t)(s & 1) * buf;
    uint8_t* nxt = Xt + (size_t)((s + 1) & 1) * buf;
    kern<<<dim3(MT, CT), kThreads, smem, st>>>((const uint8_t*)c->d_Ak2, Xm, cur, nxt, a);
  }
  k2_unpack_kernel<<<152 * 8, 256, 0, st>>>(Xm, (float*)c->d_X, N, D, KP, sc.n_runs);
  return cudaGetLastError();
}

}  // namespace

// A-operand blocks of J (and of its BF16 residual for real couplings).
cudaError_t prepare_k2_operand(chym_ctx* c) {
  if (c->d_Ak2) return cudaSuccess;
  const int N = c->N, MT = (N + 127) / 128, KP = MT * 128, KC = KP / 64;
  const int terms = c->kind == CHYM_J_PM1 ? 1 : 2;
  const size_t per_block = 128 * 64;
  std::vector<uint16_t> img((size_t)terms * MT * KC * per_block, 0);
  for (int m = 0; m < MT * 128; ++m)
    for (int k = 0; k < KP; ++k) {
      const double v = (m < N && k < N) ? c->h_J[(size_t)m * N + k] : 0.0;
      const uint16_t hi = bf16_bits_host((float)v);
      const uint16_t lo = bf16_bits_host((float)(v - (double)bf16_float_host(hi)));
      const int mt = m / 128, r = m % 128, kc = k / 64, kk = k % 64;
      const size_t off = ((size_t)mt * KC + kc) * per_block + (size_t)(r / 8) * 512 +
                         (size_t)(kk / 8) * 64 + (r % 8) * 8 + (kk % 8);  // in elements
      img[off] = hi;
      if (terms > 1) img[(size_t)MT * KC * per_block + off] = lo;
    }
  cudaError_t e = cudaMalloc(&c->d_Ak2, img.size() * 2);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(c->d_Ak2, img.data(), img.size() * 2, cudaMemcpyHostToDevice);
}

cudaError_t launch_step_k2(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  cudaError_t e = prepare_k2_operand(c);
  if (e != cudaSuccess) return e;
  switch (c->D) {
    case 1: return k2_run_typed<1>(c, sc, st);
    case 2: return k2_run_typed<2>(c, sc, st);
    case 3: return k2_run_typed<3>(c, sc, st);
    case 4: return k2_run_typed<4>(c, sc, st);
    case 5: return k2_run_typed<5>(c, sc, st);
    case 6: return k2_run_typed<6>(c, sc, st);
    case 7: return k2_run_typed<7>(c, sc, st);
    case 8: return k2_run_typed<8>(c, sc, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace chym
