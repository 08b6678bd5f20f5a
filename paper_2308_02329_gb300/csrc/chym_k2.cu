// chym_k2.cu -- large-N step: tcgen05 GEMM Y = J X with the CHYM update fused
// into its epilogue, one grouped launch per Euler-Maruyama step (N > 128).
//
// Layouts (device, internal to this path), per context:
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
// One launch covers a table of tiles (context, M tile mt, column tile ct) that may
// span many contexts of the same D.  CTA = one tile, rows [128 mt, 128 mt + 128):
//   warp 0  producer: TMA bulk copies of the A / B_hi / B_lo blocks of each K
//           chunk into a two-stage ring (mbarrier expect_tx);
//   warp 1  MMA issuer: tcgen05.mma (M = 128, N = n, K = 16), J_hi X_hi + J_hi X_lo
//           (+ J_lo X_hi), FP32 accumulator in TMEM;
//   warps 2-9  epilogue: thread = spin (TMEM lane) x column half; prefetches its
//           runs' x (global) while the MMAs run, then reads Y (tcgen05.ld), applies
//           drift, loss, annealing and Philox noise (text after Eq. 1 and after
//           Fig. 2), writes x back and stages the new BF16 hi/lo blocks of its 128
//           spins, which are bulk-stored into the other buffer (the next step's B).
// The step index comes from a device counter plus a per-launch offset, so a chunk
// of steps is captured once as a CUDA graph and replayed.  All waits are bounded;
// a timeout raises the status word and the CTA returns.
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
constexpr int kGraphSteps = 16;          // steps per captured graph

__host__ __device__ constexpr int k2_cols(int D) {  // column tile width n
  return D == 3 ? 96 : D == 5 ? 80 : D == 6 ? 96 : D == 7 ? 112 : 128;
}
__host__ __device__ constexpr uint32_t b_block_bytes(int n) { return (uint32_t)(n / 8) * kSboB; }

// One large-N context of a launch.
struct K2Desc {
  const uint8_t* Aimg;
  float* Xm;
  uint8_t* Xt;           // both buffers; buffer b at Xt + b * buf_bytes
  const float* ar;       // per run: 1 + dt (h - 1)
  const uint4* rk;       // per run: Philox round keys [5]
  const int64_t* koff;   // per run: global step of its (re)seeding
  unsigned long long buf_bytes;
  int N, KP, MT, KC, CT, n_runs, a_terms, sched_kind;
  int64_t k0, k_anneal, k_total;  // k0: step of the context when the call began
  float gdt, kdt, edt, neg2ln2s2, inv_ramp;
};

struct K2Tile {
  int desc, mt, ct, pad;
};

struct K2Launch {
  const K2Desc* descs;
  const K2Tile* tiles;
  const int64_t* done;   // steps already taken in this call (device counter)
  int k_off;             // this launch's offset within the captured chunk
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

// The D accumulator columns of one run and their wait, in one asm statement each
// (tcgen05.ld fills its registers asynchronously until tcgen05.wait::ld).
template <int D>
__device__ __forceinline__ void load_y(uint32_t taddr, float (&y)[D]) {
  uint32_t r[8];
  if constexpr (D == 1) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]) : "r"(taddr) : "memory");
  } else if constexpr (D == 2) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(taddr) : "memory");
  } else if constexpr (D == 3) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%3];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%2}, [%4];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]) : "r"(taddr), "r"(taddr + 2) : "memory");
  } else if constexpr (D == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr) : "memory");
  } else if constexpr (D == 5) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%5];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%4}, [%6];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]) : "r"(taddr), "r"(taddr + 4)
        : "memory");
  } else if constexpr (D == 6) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%6];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4,%5}, [%7];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5])
        : "r"(taddr), "r"(taddr + 4) : "memory");
  } else if constexpr (D == 7) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%7];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4,%5}, [%8];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%6}, [%9];\n\ttcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6])
        : "r"(taddr), "r"(taddr + 4), "r"(taddr + 6) : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr) : "memory");
  }
#pragma unroll
  for (int mu = 0; mu < D; ++mu) y[mu] = __uint_as_float(r[mu]);
}

template <int D>
__device__ __forceinline__ void load_x(const K2Desc& d, int c_glob, int p, bool valid, float (&x)[D]) {
#pragma unroll
  for (int mu = 0; mu < D; ++mu) x[mu] = valid ? d.Xm[(size_t)(c_glob + mu) * d.KP + p] : 0.f;
}

template <int D>
__global__ void __launch_bounds__(kThreads, 2) step_k2_kernel(K2Launch L) {
  constexpr int n = k2_cols(D);
  constexpr uint32_t BB = b_block_bytes(n);
  constexpr int runs_half = n / 2 / D;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const K2Tile tile = L.tiles[blockIdx.x];
  const K2Desc& d = L.descs[tile.desc];
  const int mt = tile.mt, ct = tile.ct;
  const int64_t step = *L.done + L.k_off;      // steps taken in this call before this one
  const int64_t k = d.k0 + step;
  const uint8_t* Xt_cur = d.Xt + (size_t)(step & 1) * d.buf_bytes;
  uint8_t* Xt_next = d.Xt + (size_t)((step + 1) & 1) * d.buf_bytes;
  const uint32_t stage_bytes = (uint32_t)d.a_terms * kABlock + 2u * BB;
  const uint32_t blocks_per_buf = (uint32_t)d.CT * d.KC;  // blocks of one (hi or lo) buffer

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
      for (int kc = 0; kc < d.KC; ++kc) {
        const int s = kc % kStages;
        if (kc >= kStages && !mbar_wait(smem_addr(&empty_bar[s]), (uint32_t)((kc / kStages - 1) & 1))) {
          atomicOr(L.status, STATUS_TIMEOUT);
          s_abort = 1;
          break;
        }
        const uint32_t base = smem_addr(smem) + (uint32_t)s * stage_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         smem_addr(&full_bar[s])), "r"(stage_bytes) : "memory");
        for (int t = 0; t < d.a_terms; ++t)
          bulk_g2s(base + (uint32_t)t * kABlock,
                   d.Aimg + ((size_t)(t * d.MT + mt) * d.KC + kc) * kABlock, kABlock,
                   smem_addr(&full_bar[s]));
        const size_t blk = (size_t)ct * d.KC + kc;
        bulk_g2s(base + (uint32_t)d.a_terms * kABlock, Xt_cur + blk * BB, BB, smem_addr(&full_bar[s]));
        bulk_g2s(base + (uint32_t)d.a_terms * kABlock + BB, Xt_cur + (blocks_per_buf + blk) * BB, BB,
                 smem_addr(&full_bar[s]));
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      bool ok = true;
      for (int kc = 0; kc < d.KC && ok; ++kc) {
        const int s = kc % kStages;
        if (!mbar_wait(smem_addr(&full_bar[s]), (uint32_t)((kc / kStages) & 1))) {
          atomicOr(L.status, STATUS_TIMEOUT);
          s_abort = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_addr(smem) + (uint32_t)s * stage_bytes;
        const uint32_t bhi = base + (uint32_t)d.a_terms * kABlock, blo = bhi + BB;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t da = smem_desc(base + (uint32_t)ks * 256u, 128u, 1024u);
          mma_bf16(tmem, da, smem_desc(bhi + (uint32_t)ks * 2u * kLboB, kLboB, kSboB), idesc,
                   (kc > 0 || ks > 0) ? 1u : 0u);
          mma_bf16(tmem, da, smem_desc(blo + (uint32_t)ks * 2u * kLboB, kLboB, kSboB), idesc, 1u);
          if (d.a_terms > 1)
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
    const bool live = p < d.N;
    const int c_begin = half * (n / 2);
    const int run_begin = (ct * n + c_begin) / D;
    // prefetch the first two runs' state while the tensor core works
    float xa[D], xb[D];
    load_x<D>(d, ct * n + c_begin, p, live && run_begin < d.n_runs, xa);
    load_x<D>(d, ct * n + c_begin + D, p, live && runs_half > 1 && run_begin + 1 < d.n_runs, xb);
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&acc_bar), 0u)) && !s_abort;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // staging: the tile's new hi/lo blocks, K chunks 2 mt (rows 0-63) and 2 mt + 1
    // (rows 64-127); they reuse the pipeline stages, free once the accumulator is ready
    uint8_t* stg_hi = smem + (size_t)(i_loc >> 6) * BB;
    uint8_t* stg_lo = smem + (size_t)(2 + (i_loc >> 6)) * BB;
    const int kl = i_loc & 63;
    const uint32_t k_off = (uint32_t)(kl & 7) * 2u + (uint32_t)(kl >> 3) * kLboB;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    if (ok) {
      for (int i = 0; i < runs_half; ++i) {
        const int c0 = c_begin + i * D;
        const int c_glob = ct * n + c0;
        const int run = c_glob / D;
        // keep two runs of state in flight ahead of the arithmetic
        float xc[D];
        load_x<D>(d, c_glob + 2 * D, p, live && i + 2 < runs_half && run + 2 < d.n_runs, xc);
        float y[D];
        load_y<D>(trow + (uint32_t)c0, y);
        float xn[D];
#pragma unroll
        for (int mu = 0; mu < D; ++mu) xn[mu] = 0.f;
        if (live && run < d.n_runs) {
          // the run's local step: noise counter and annealing scale alpha_mu
          const int64_t kl = k - __ldg(d.koff + run);
          float ramp = 1.f;
          if (d.sched_kind == 1 && kl >= d.k_anneal)
            ramp = kl >= d.k_total ? 0.f : fmaxf(0.f, 1.f - (float)(kl - d.k_anneal) * d.inv_ramp);
          float n2 = 0.f;
#pragma unroll
          for (int mu = 0; mu < D; ++mu) n2 = fmaf(xa[mu], xa[mu], n2);
          const float t = fmaf(-d.gdt, n2, __ldg(d.ar + run));
          float z[4 * ((D + 3) / 4)];
#pragma unroll
          for (int blk = 0; blk < (D + 3) / 4; ++blk) {
            const uint4 w = philox_rk(noise_counter((uint32_t)p, (uint32_t)blk, 0u, (uint64_t)kl),
                                      d.rk + (size_t)run * 5);
            box_muller(w.x, w.y, d.neg2ln2s2, z[4 * blk], z[4 * blk + 1]);
            if (D - 4 * blk > 2) box_muller(w.z, w.w, d.neg2ln2s2, z[4 * blk + 2], z[4 * blk + 3]);
          }
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            const float s = fmaf(-d.kdt * xa[mu], xa[mu], t);
            xn[mu] = fmaf(xa[mu], s, fmaf(d.edt * (mu == 0 ? 1.f : ramp), y[mu], z[mu]));
            d.Xm[(size_t)(c_glob + mu) * d.KP + p] = xn[mu];
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
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
          xa[mu] = xb[mu];
          xb[mu] = xc[mu];
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (warp == 2 && lane == 0 && ok) {
      for (int t = 0; t < 2; ++t)
        for (int hh = 0; hh < 2; ++hh) {
          const size_t blk = (size_t)t * blocks_per_buf + (size_t)ct * d.KC + (2 * mt + hh);
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

__global__ void k2_advance_kernel(int64_t* done, int64_t by) { *done += by; }

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
__global__ void k2_runconst_kernel(const double* __restrict__ h, const int32_t* __restrict__ hidx,
                                   const uint64_t* __restrict__ seeds, int n_runs, double dt, float* ar,
                                   uint4* rk) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_runs; r += gridDim.x * blockDim.x) {
    ar[r] = (float)(1.0 + dt * (h[hidx[r]] - 1.0));
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

// Workspace, per-run constants and buffer 0 of one context; fills its descriptor.
template <int D>
cudaError_t k2_prepare_typed(chym_ctx* c, const StepConsts& sc, cudaStream_t st, K2Desc& d) {
  constexpr int n = k2_cols(D);
  const int N = c->N, MT = (N + 127) / 128, KP = MT * 128, KC = KP / 64;
  const int C = sc.n_runs * D, CT = (C + n - 1) / n;
  const size_t BB = b_block_bytes(n);
  const size_t xm_bytes = ((size_t)CT * n * KP * 4 + 255) / 256 * 256;
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
  k2_runconst_kernel<<<(sc.n_runs + 255) / 256, 256, 0, st>>>(c->d_h, c->d_hidx, c->d_seeds,
                                                             sc.n_runs, sc.dt, ar, rk);
  k2_pack_kernel<D><<<152 * 8, 256, 0, st>>>((const float*)c->d_X, Xm, Xt, N, KP, KC, CT, sc.n_runs);
  d.Aimg = (const uint8_t*)c->d_Ak2;
  d.Xm = Xm;
  d.Xt = Xt;
  d.ar = ar;
  d.rk = rk;
  d.koff = c->d_koff;
  d.buf_bytes = (unsigned long long)(2 * CT * KC * BB);
  d.N = N;
  d.KP = KP;
  d.MT = MT;
  d.KC = KC;
  d.CT = CT;
  d.n_runs = sc.n_runs;
  d.a_terms = c->kind == CHYM_J_PM1 ? 1 : 2;
  d.sched_kind = sc.sched_kind;
  d.k0 = sc.k0;
  d.k_anneal = sc.k_anneal;
  d.k_total = sc.k_total;
  d.gdt = (float)(sc.dt * sc.gamma);
  d.kdt = (float)(sc.dt * sc.kappa);
  d.edt = (float)(sc.dt * sc.eps);
  d.neg2ln2s2 = (float)(-2.0 * 0.69314718055994531 * sc.noise_scale * sc.noise_scale);
  d.inv_ramp = sc.sched_kind == 1 ? (float)(1.0 / (double)(sc.k_total - sc.k_anneal)) : 0.f;
  return cudaGetLastError();
}

template <int D>
cudaError_t k2_launch_typed(const K2Launch& L, int n_tiles, int terms_max, cudaStream_t st) {
  constexpr int n = k2_cols(D);
  const size_t BB = b_block_bytes(n);
  const size_t smem = std::max<size_t>(kStages * ((size_t)terms_max * kABlock + 2 * BB), 4 * BB);
  auto kern = step_k2_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_tiles, kThreads, smem, st>>>(L);
  return cudaGetLastError();
}

cudaError_t k2_launch(int D, const K2Launch& L, int n_tiles, int terms_max, cudaStream_t st) {
  switch (D) {
    case 1: return k2_launch_typed<1>(L, n_tiles, terms_max, st);
    case 2: return k2_launch_typed<2>(L, n_tiles, terms_max, st);
    case 3: return k2_launch_typed<3>(L, n_tiles, terms_max, st);
    case 4: return k2_launch_typed<4>(L, n_tiles, terms_max, st);
    case 5: return k2_launch_typed<5>(L, n_tiles, terms_max, st);
    case 6: return k2_launch_typed<6>(L, n_tiles, terms_max, st);
    case 7: return k2_launch_typed<7>(L, n_tiles, terms_max, st);
    case 8: return k2_launch_typed<8>(L, n_tiles, terms_max, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

long long k2_work_units(int N, int D, int n_runs) {
  if (D < 1 || D > 8) return 0;
  static const int cols[9] = {0, k2_cols(1), k2_cols(2), k2_cols(3), k2_cols(4),
                              k2_cols(5), k2_cols(6), k2_cols(7), k2_cols(8)};
  const long long MT = (N + 127) / 128, KC = 2 * MT;
  const long long CT = ((long long)n_runs * D + cols[D] - 1) / cols[D];
  return MT * CT * KC;
}

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

// ---------------------------------------------------------------------------
// Runner: a set of large-N contexts integrated together for `steps` steps.
// ---------------------------------------------------------------------------
cudaError_t k2_prepare(chym_ctx* c, const StepConsts& sc, cudaStream_t st, void* desc_out) {
  cudaError_t e = prepare_k2_operand(c);
  if (e != cudaSuccess) return e;
  K2Desc& d = *reinterpret_cast<K2Desc*>(desc_out);
  switch (c->D) {
    case 1: return k2_prepare_typed<1>(c, sc, st, d);
    case 2: return k2_prepare_typed<2>(c, sc, st, d);
    case 3: return k2_prepare_typed<3>(c, sc, st, d);
    case 4: return k2_prepare_typed<4>(c, sc, st, d);
    case 5: return k2_prepare_typed<5>(c, sc, st, d);
    case 6: return k2_prepare_typed<6>(c, sc, st, d);
    case 7: return k2_prepare_typed<7>(c, sc, st, d);
    case 8: return k2_prepare_typed<8>(c, sc, st, d);
  }
  return cudaErrorInvalidValue;
}

size_t k2_desc_bytes() { return sizeof(K2Desc); }

cudaError_t k2_finish(chym_ctx* c, const void* desc, cudaStream_t st) {
  const K2Desc& d = *reinterpret_cast<const K2Desc*>(desc);
  k2_unpack_kernel<<<152 * 8, 256, 0, st>>>(d.Xm, (float*)c->d_X, c->N, c->D, d.KP, d.n_runs);
  return cudaGetLastError();
}

// Integrate the contexts whose descriptors are in `descs` (host copies, dims[i] =
// their D) for `steps` steps on stream st: one grouped launch per dimension per
// step, chunks of kGraphSteps steps captured once into a CUDA graph and replayed.
cudaError_t k2_integrate(K2Runner& R, const std::vector<unsigned char>& descs,
                         const std::vector<int>& dims, int64_t steps, unsigned* status,
                         cudaStream_t st) {
  const size_t db = sizeof(K2Desc);
  const int n_desc = (int)dims.size();
  // tile tables per dimension
  std::vector<K2Tile> tiles;
  std::vector<int> dim_first(9, 0), dim_count(9, 0), dim_terms(9, 1);
  for (int D = 1; D <= 8; ++D) {
    dim_first[D] = (int)tiles.size();
    for (int i = 0; i < n_desc; ++i) {
      if (dims[i] != D) continue;
      const K2Desc& d = *reinterpret_cast<const K2Desc*>(descs.data() + i * db);
      dim_terms[D] = std::max(dim_terms[D], d.a_terms);
      for (int ct = 0; ct < d.CT; ++ct)
        for (int mt = 0; mt < d.MT; ++mt) tiles.push_back(K2Tile{i, mt, ct, 0});  // mt fastest
    }
    dim_count[D] = (int)tiles.size() - dim_first[D];
  }
  const size_t bytes = 64 + descs.size() + tiles.size() * sizeof(K2Tile);
  cudaError_t e = cudaSuccess;
  if (bytes > R.bytes) {
    if (R.exec) cudaGraphExecDestroy(R.exec);
    R.exec = nullptr;
    if (R.d_buf) cudaFree(R.d_buf);
    R.d_buf = nullptr;
    R.bytes = 0;
    e = cudaMalloc(&R.d_buf, bytes);
    if (e != cudaSuccess) return e;
    R.bytes = bytes;
  }
  if (!R.stream) {
    e = cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  unsigned char* base = (unsigned char*)R.d_buf;
  int64_t* d_done = (int64_t*)base;
  const K2Desc* d_descs = (const K2Desc*)(base + 64);
  const K2Tile* d_tiles = (const K2Tile*)(base + 64 + descs.size());
  std::vector<unsigned char> blob(bytes, 0);
  memcpy(blob.data() + 64, descs.data(), descs.size());
  memcpy(blob.data() + 64 + descs.size(), tiles.data(), tiles.size() * sizeof(K2Tile));
  e = cudaMemcpyAsync(base, blob.data(), bytes, cudaMemcpyHostToDevice, st);  // also zeroes *done
  if (e != cudaSuccess) return e;

  auto issue = [&](int k_off, cudaStream_t s) -> cudaError_t {
    for (int D = 1; D <= 8; ++D) {
      if (!dim_count[D]) continue;
      K2Launch L{d_descs, d_tiles + dim_first[D], d_done, k_off, status};
      cudaError_t r = k2_launch(D, L, dim_count[D], dim_terms[D], s);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  };
  const int64_t chunks = steps / kGraphSteps, rem = steps % kGraphSteps;
  if (chunks > 0) {
    // the graph stays valid while the tile table keeps its shape; the descriptor
    // contents are refreshed in place above
    const bool reuse = R.exec && R.sig_tiles == tiles.size() && R.sig_dims == dim_count &&
                       R.sig_buf == R.d_buf;
    if (!reuse) {
      if (R.exec) cudaGraphExecDestroy(R.exec);
      R.exec = nullptr;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(R.stream, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return e;
      for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) e = issue(s, R.stream);
      if (e == cudaSuccess) {
        k2_advance_kernel<<<1, 1, 0, R.stream>>>(d_done, kGraphSteps);
        e = cudaGetLastError();
      }
      cudaError_t e2 = cudaStreamEndCapture(R.stream, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&R.exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
      R.sig_tiles = tiles.size();
      R.sig_dims = dim_count;
      R.sig_buf = R.d_buf;
    }
    for (int64_t c = 0; c < chunks; ++c) {
      e = cudaGraphLaunch(R.exec, st);
      if (e != cudaSuccess) return e;
    }
  }
  for (int s = 0; s < rem; ++s) {
    e = issue(s, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void k2_runner_release(K2Runner& R) {
  if (R.exec) cudaGraphExecDestroy(R.exec);
  if (R.d_buf) cudaFree(R.d_buf);
  if (R.stream) cudaStreamDestroy(R.stream);
  R = K2Runner();
}

cudaError_t launch_step_k2(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  std::vector<unsigned char> desc(sizeof(K2Desc));
  cudaError_t e = k2_prepare(c, sc, st, desc.data());
  if (e != cudaSuccess) return e;
  e = k2_integrate(c->k2_runner, desc, std::vector<int>{c->D}, sc.steps, c->d_status, st);
  if (e != cudaSuccess) return e;
  return k2_finish(c, desc.data(), st);
}

}  // namespace chym
