// chym_tc.cu -- fused tensor-core step kernel for N <= 128 (BF16 hi+lo coupling,
// FP32 state), persistent over all steps of a launch.
//
// Per step, for every group of runs (one warpgroup of 128 threads, thread = spin
// p = TMEM lane):
//   1. one thread issues tcgen05.mma:  Y (128 x C, FP32 in TMEM) =
//        J_hi X_hi + J_hi X_lo (+ J_lo X_hi for real J)            (C = J_N (x) 1_D, Eq. 1)
//      A = J (BF16, K-major canonical layout, staged once by a TMA bulk copy),
//      B = X split into BF16 hi + lo (MN-major canonical layout in shared memory),
//      columns ordered c = mu * R + r so a thread's 8 consecutive runs of one
//      component are 8 consecutive columns;
//   2. the warpgroup reads its rows of Y (tcgen05.ld) and the FP32 master state
//      (kept in TMEM beside the accumulator), applies the local drift, the
//      non-local loss, the annealing scale alpha_mu(k) (text after Fig. 2) and the
//      Philox4x32-10 / Box-Muller noise:
//        x <- x (1 + dt(h-1) - dt gamma |x_p|^2 - dt kappa x^2) + dt eps alpha_mu y
//             + sigma sqrt(dt) xi,
//      writes x back to TMEM and its BF16 hi/lo split into the B operand.
// Up to four groups share an SM and interleave their tensor-core and ALU phases.
// Every wait is bounded (%globaltimer); on timeout the kernel raises a status bit,
// drains its own tensor-core work with another bounded wait, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "chym_internal.cuh"

namespace chym {
namespace {

// One context of a launch: its J image, state, pumps, seeds and step constants.
struct TcDesc {
  const uint8_t* Aimg;
  float* X;
  const double* h;
  const uint64_t* seeds;
  const int64_t* koff;  // per run: global step of its (re)seeding
  const int32_t* hidx;  // per run: index of its pump value
  const double* w;      // per spin: coupling weight (nullable: all 1)
  int N, KP, n_runs, replicas, a_terms, sched_kind;
  int stall;            // CHYM_FLAG_TEST_STALL: completion of the products withheld
  int64_t k0, k_anneal, k_total;
  float dt, noise_scale, gdt, kdt, edt, inv_ramp;
};

// A block of consecutive runs of one context, integrated by one CTA: its G
// groups take RG runs each.
struct TcItem {
  int desc, run_begin, run_count, pad;
};

struct TcLaunch {
  const TcDesc* descs;
  const TcItem* items;
  const int* cta_begin;  // items of CTA b: [cta_begin[b], cta_begin[b + 1])
  int64_t steps;
  uint32_t a_region;     // bytes reserved for the largest J image of the launch
  int kp_max;            // largest K (rows of B) of the launch
  unsigned* status;
  unsigned long long wait_ns;  // limit of every bounded wait
};

// CH_ = 0: the default runs per epilogue chunk (8 for D <= 4, else 4); the batch
// autotuner may choose 4 for D <= 4.
template <int D, int CH_ = 0>
struct TcCfg {
  static constexpr int RG = D == 1 ? 64 : D == 2 ? 32 : (D == 6 || D == 8) ? 8 : 16;
  static constexpr int CG = D * RG;        // MMA N: columns of one group
  static constexpr int CH = CH_ ? CH_ : D <= 4 ? 8 : 4;  // runs per epilogue chunk
  static constexpr int G = std::min(4, 512 / (2 * CG));
  static_assert(CG % 16 == 0 && CG <= 256, "MMA N must be a multiple of 16 in [16, 256]");
  static_assert(RG % CH == 0, "chunk must divide the group");
};


__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of phase `parity` of an mbarrier, for at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 0u) {
      const uint64_t t = global_timer();
      if (it == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

// Shared-memory matrix descriptor, no swizzle: start address, byte offset between
// core matrices along K (lbo) and along M/N (sbo), descriptor version 1.
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

// Loads of the accumulator (ya) and master state (xa) columns followed by the wait
// in ONE asm statement: tcgen05.ld fills its registers asynchronously, so the
// compiler must not see (and possibly spill) them before tcgen05.wait::ld.
template <int CH>
__device__ __forceinline__ void tmem_ld2_wait(uint32_t ya, uint32_t xa, float (&y)[CH], float (&x)[CH]) {
  uint32_t r[2 * CH];
  if constexpr (CH == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(ya), "r"(xa)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%8];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%9];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(ya), "r"(xa)
        : "memory");
  }
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    y[j] = __uint_as_float(r[j]);
    x[j] = __uint_as_float(r[CH + j]);
  }
}

// Load of one group of columns followed by its wait, in one asm statement.
template <int CH>
__device__ __forceinline__ void tmem_ld_wait(uint32_t taddr, float (&v)[CH]) {
  uint32_t r[CH];
  if constexpr (CH == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(taddr)
        : "memory");
  }
#pragma unroll
  for (int j = 0; j < CH; ++j) v[j] = __uint_as_float(r[j]);
}

template <int CH>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const float (&v)[CH]) {
  if constexpr (CH == 8) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])));
  } else {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                 "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])));
  }
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Named barrier of one warpgroup; returns the OR of `flag` over its 128 threads.
__device__ __forceinline__ int group_bar_or(int id, int flag) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, 128, p;\n\tselp.s32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(flag), "r"(id)
      : "memory");
  return r;
}

// Split 2*n FP32 values into packed BF16 hi words and BF16 lo words (lo = x - hi).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
  const float ah = __low2float(h2), bh = __high2float(h2);
  const __nv_bfloat162 l2 = __floats2bfloat162_rn(a - ah, b - bh);
  hi = *reinterpret_cast<const uint32_t*>(&h2);
  lo = *reinterpret_cast<const uint32_t*>(&l2);
}

// Write CH consecutive B columns (n0 .. n0+CH-1) of row k = spin p, hi and lo.
template <int CH>
__device__ __forceinline__ void store_b(uint8_t* Bhi, uint8_t* Blo, uint32_t off, const float (&v)[CH]) {
  uint32_t h[CH / 2], l[CH / 2];
#pragma unroll
  for (int j = 0; j < CH / 2; ++j) split_pair(v[2 * j], v[2 * j + 1], h[j], l[j]);
  if constexpr (CH == 8) {
    *reinterpret_cast<uint4*>(Bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(Blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  } else {
    *reinterpret_cast<uint2*>(Bhi + off) = make_uint2(h[0], h[1]);
    *reinterpret_cast<uint2*>(Blo + off) = make_uint2(l[0], l[1]);
  }
}

// One Philox4x32 round with round key (k0, k1).
__device__ __forceinline__ void philox_round(uint4& c, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x, p1 = (uint64_t)kPhiloxM1 * c.z;
  c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                 (uint32_t)p0);
}

// Philox4x32-10 with the ten round keys precomputed (two rounds per uint4):
// the key schedule depends on the run only, so it is built once per launch.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint4* __restrict__ rk) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint4 kk = rk[i];
    philox_round(c, kk.x, kk.y);
    philox_round(c, kk.z, kk.w);
  }
  return c;
}

// SFU approximations with denormals flushed: no argument or result of the noise
// transform is denormal, so they equal the non-flushing forms there, in fewer
// instructions.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void sincos_approx(float x, float& s, float& c) {
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// Box-Muller for two runs at once: words (wr, wa) of run A and of run B give
// zc = (-r_A cos t_A, -r_B cos t_B), zs = (-r sin t) with u = (w + 1/2) 2^-32,
// r = sqrt(-2 ln u_r) * scale, t = 2 pi u_a - pi (the negation restores the
// angle 2 pi u_a).  neg2ln2s2 = -2 ln(2) scale^2 folds the radius scaling.
__device__ __forceinline__ void box_muller_x2(uint32_t wrA, uint32_t waA, uint32_t wrB,
                                              uint32_t waB, float neg2ln2s2, float2& zc,
                                              float2& zs) {
  const float2 two32 = make_float2(2.3283064365386963e-10f, 2.3283064365386963e-10f);
  const float2 half32 = make_float2(1.1641532182693481e-10f, 1.1641532182693481e-10f);
  const float2 ang_m = make_float2(1.4629180792671596e-09f, 1.4629180792671596e-09f);
  const float2 ang_c = make_float2(-3.1415926528582302f, -3.1415926528582302f);
  const float2 ur = __ffma2_rn(make_float2((float)wrA, (float)wrB), two32, half32);
  const float2 th = __ffma2_rn(make_float2((float)waA, (float)waB), ang_m, ang_c);
  const float2 r2 = __fmul2_rn(make_float2(lg2_approx(ur.x), lg2_approx(ur.y)),
                               make_float2(neg2ln2s2, neg2ln2s2));
  const float2 r = make_float2(-sqrt_approx(r2.x), -sqrt_approx(r2.y));
  float sA, cA, sB, cB;
  sincos_approx(th.x, sA, cA);
  sincos_approx(th.y, sB, cB);
  zc = __fmul2_rn(r, make_float2(cA, cB));
  zs = __fmul2_rn(r, make_float2(sA, sB));
}

// The four lanes of a quad hold the rows of a 4 x 4 matrix (lane m: a[m][0..3]);
// afterwards lane m holds column m (b[i] = a[i][m]).  Two exchange stages: with
// lane m ^ 1 the columns of the other parity, then with lane m ^ 2 the other half
// of the lane's own column.
__device__ __forceinline__ void quad_transpose(float v0, float v1, float v2, float v3, int m, float (&b)[4]) {
  const bool odd = (m & 1) != 0, high = (m & 2) != 0;
  const float s0 = odd ? v0 : v1, s1 = odd ? v2 : v3;  // columns of the other parity
  const float k0 = odd ? v1 : v0, k1 = odd ? v3 : v2;  // columns c0 = m & 1, c1 = c0 + 2
  const float r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
  // rows 2h and 2h + 1 (h = m / 2) of columns c0 and c1
  const float a00 = odd ? r0 : k0, a10 = odd ? k0 : r0, a01 = odd ? r1 : k1, a11 = odd ? k1 : r1;
  const float se = high ? a00 : a01, so = high ? a10 : a11;  // the column lane m ^ 2 needs
  const float ke = high ? a01 : a00, ko = high ? a11 : a10;  // column m
  const float re = __shfl_xor_sync(0xffffffffu, se, 2), ro = __shfl_xor_sync(0xffffffffu, so, 2);
  b[0] = high ? re : ke;
  b[1] = high ? ro : ko;
  b[2] = high ? ke : re;
  b[3] = high ? ko : ro;
}

template <int D, int CH_>
__global__ void __launch_bounds__(512, 1) step_tc_kernel(TcLaunch L) {
  using Cfg = TcCfg<D, CH_>;
  constexpr int RG = Cfg::RG, CG = Cfg::CG, CH = Cfg::CH, G = Cfg::G;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ __align__(8) uint64_t s_mbar[G];
  __shared__ __align__(8) uint64_t s_abar;
  __shared__ __align__(8) uint64_t s_wh[G];  // CHYM_FLAG_TEST_STALL: where the completion goes instead
  __shared__ __align__(8) float s_ar[G][RG];
  __shared__ uint4 s_rk[G][RG][5];  // Philox round keys of each run
  __shared__ int64_t s_koff[G][RG];  // each run's (re)seeding step
  __shared__ int s_kuni[G];           // 1 when all runs of the group share one offset
  // when they do not: each run's local step and annealing scale at the current step,
  // double buffered by step parity (written one step ahead by the run's own thread)
  __shared__ __align__(16) int64_t s_kl[2][G][RG];
  __shared__ __align__(8) float s_rp[2][G][RG];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 2, wq = warp & 3;
  const int p = wq * 32 + lane;  // spin = TMEM lane
  const uint32_t b_bytes = (uint32_t)L.kp_max * CG * 2u;
  uint8_t* Bhi = smem + L.a_region + (size_t)g * 2 * b_bytes;
  uint8_t* Blo = Bhi + b_bytes;
  const uint32_t lbo_b = (CG / 8) * 128u;  // B: core-matrix stride along K

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&s_tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_abar)));
    for (int q = 0; q < G; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_mbar[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_wh[q])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t t_lane = tmem + ((uint32_t)(wq * 32) << 16);
  const uint32_t acc_col = (uint32_t)(g * CG);
  const uint32_t mst_col = (uint32_t)(G * CG + g * CG);
  // B store offset of row k = p: (p % 8) * 16 + (p / 8) * lbo_b; column block adds n0/8*128 + n0%8*2
  const uint32_t b_row_off = (uint32_t)(p & 7) * 16u + (uint32_t)(p >> 3) * lbo_b;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) |
                         ((uint32_t)(CG >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const uint32_t a_base = smem_addr(smem);
  const uint32_t bhi_base = smem_addr(Bhi), blo_base = smem_addr(Blo);
  uint32_t phase = 0, a_phase = 0;
  int a_desc = -1;
  bool aborted = false;

  for (int it = L.cta_begin[blockIdx.x]; it < L.cta_begin[blockIdx.x + 1] && !aborted; ++it) {
    const TcItem item = L.items[it];
    const TcDesc d = L.descs[item.desc];
    const int N = d.N, KP = d.KP;
    const uint32_t a_bytes = 128u * (uint32_t)KP * 2u;
    // the item's runs are spread evenly over the groups in whole chunks
    const int per_g = min(RG, ((item.run_count + G - 1) / G + CH - 1) / CH * CH);
    const int run0 = item.run_begin + g * per_g;
    const int nr = max(0, min(per_g, item.run_begin + item.run_count - run0));
    const bool new_a = item.desc != a_desc;  // CTA-uniform
    if (new_a && tid == 0) {                 // TMA bulk copy of the context's J image
      const uint32_t bytes = (uint32_t)d.a_terms * a_bytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&s_abar)),
                   "r"(bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(smem)),
          "l"(d.Aimg), "r"(bytes), "r"(smem_addr(&s_abar))
          : "memory");
    }
    // per-run constants of this group: 1 + dt (h - 1) and the Philox round keys
    if (p < RG) {
      const int run = run0 + p;
      float ar = 0.f;
      uint32_t k0 = 0u, k1 = 0u;
      if (p < nr) {
        ar = (float)(1.0 + (double)d.dt * (d.h[d.hidx[run]] - 1.0));
        const uint64_t sd = d.seeds[run];
        k0 = (uint32_t)sd;
        k1 = (uint32_t)(sd >> 32);
      }
      s_ar[g][p] = ar;
      s_koff[g][p] = p < nr ? d.koff[run] : 0;
      for (int i = 0; i < 5; ++i) {  // Weyl key schedule: round r uses key + r * (W0, W1)
        s_rk[g][p][i] = make_uint4(k0 + (2u * i) * kPhiloxW0, k1 + (2u * i) * kPhiloxW1,
                                   k0 + (2u * i + 1u) * kPhiloxW0, k1 + (2u * i + 1u) * kPhiloxW1);
      }
    }
    if (p == 0) s_kuni[g] = 1;
    // zero the B operands (K padding rows and unused runs must stay finite zeros)
    for (uint32_t o = (uint32_t)(tid & 127) * 16u; o < 2u * b_bytes; o += 128u * 16u)
      *reinterpret_cast<uint4*>(Bhi + o) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();  // every zero must land before any thread writes its state into B
    if (p < nr && s_koff[g][p] != s_koff[g][0]) s_kuni[g] = 0;
    // run p's local step at step kk (noise counter) and its annealing scale alpha_mu
    // (mu >= 1), for the per-run path
    auto put_step = [&](int64_t kk) {
      if (p < RG) {
        const int64_t kl = kk - s_koff[g][p];
        float rp = 1.f;
        if (d.sched_kind == 1 && kl >= d.k_anneal)
          rp = kl >= d.k_total ? 0.f : fmaxf(0.f, 1.f - (float)(kl - d.k_anneal) * d.inv_ramp);
        s_kl[kk & 1][g][p] = kl;
        s_rp[kk & 1][g][p] = rp;
      }
    };
    put_step(d.k0);  // read after the barrier below
    const bool live = p < N;
    const float edt_p = d.edt * ((d.w && live) ? (float)d.w[p] : 1.f);  // dt eps times the spin's weight
    // ---- load the state: X[run][p][mu] -> TMEM master + BF16 hi/lo B ----
    for (int r0 = 0; r0 < nr; r0 += CH) {
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        float v[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int r = r0 + j;
          v[j] = (live && r < nr) ? d.X[((size_t)(run0 + r) * N + p) * D + mu] : 0.f;
        }
        tmem_st<CH>(t_lane + mst_col + (uint32_t)(mu * RG + r0), v);
        const uint32_t n0 = (uint32_t)(mu * RG + r0);
        if (live) store_b<CH>(Bhi, Blo, b_row_off + (n0 >> 3) * 128u + (n0 & 7u) * 2u, v);
      }
    }
    tmem_wait_st();
    fence_async_smem();
    tc_fence_before();
    __syncthreads();

    // ---- step loop (each group independently) ----
    const bool k_uniform = s_kuni[g] != 0;
    const int64_t koff_u = s_koff[g][0];
    const uint32_t a_sbo = (uint32_t)(KP / 8) * 128u;
    const int ksteps = KP / 16;
    const float neg2ln2s2 = -1.3862943611198906f * d.noise_scale * d.noise_scale;
    const float2 ngdt = make_float2(-d.gdt, -d.gdt), nkdt = make_float2(-d.kdt, -d.kdt);
    bool timed_out = false, a_pending = new_a;
    if (nr > 0) {
      for (int64_t k = d.k0; k < d.k0 + L.steps; ++k) {
        if (wq == 0 && lane == 0) {
          bool ok = true;
          if (a_pending) ok = mbar_wait(smem_addr(&s_abar), a_phase, L.wait_ns);
          a_pending = false;
          tc_fence_after();
          if (ok) {
            // a K step moves only the 14-bit start-address field of each descriptor
            // (shared addresses stay below 256 KB, so the field never carries)
            const uint64_t da0 = smem_desc(a_base, 128u, a_sbo), dj0 = smem_desc(a_base + a_bytes, 128u, a_sbo);
            const uint64_t dh0 = smem_desc(bhi_base, lbo_b, 128u), dl0 = smem_desc(blo_base, lbo_b, 128u);
            const uint64_t sa = 256u >> 4, sb = (2u * lbo_b) >> 4;
            for (int ks = 0; ks < ksteps; ++ks)
              mma_bf16(tmem + acc_col, da0 + ks * sa, dh0 + ks * sb, idesc, ks > 0);
            for (int ks = 0; ks < ksteps; ++ks)
              mma_bf16(tmem + acc_col, da0 + ks * sa, dl0 + ks * sb, idesc, 1u);
            if (d.a_terms > 1) {
              for (int ks = 0; ks < ksteps; ++ks)
                mma_bf16(tmem + acc_col, dj0 + ks * sa, dh0 + ks * sb, idesc, 1u);
            }
            // (test of the timeout path: the completion signal goes elsewhere, so the
            // group's wait below runs out; the drain after the loop waits for it)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(d.stall ? &s_wh[g] : &s_mbar[g]))
                : "memory");
          } else {
            atomicOr(L.status, STATUS_TIMEOUT);
            s_abort = 1;
            // nothing was issued: complete the phase so the group does not wait
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_mbar[g])) : "memory");
          }
        }
        // warp-uniform outcome: the TMEM loads below are warp-collective
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&s_mbar[g]), phase, L.wait_ns));
        phase ^= 1u;
        if (!ok) {
          timed_out = true;
          atomicOr(L.status, STATUS_TIMEOUT);
          s_abort = 1;
        }
        tc_fence_after();
        // annealing scale when every run of the group shares one local step
        float ramp_u = 1.f;
        const int64_t kl_u = k - koff_u;
        if (d.sched_kind == 1 && kl_u >= d.k_anneal)
          ramp_u = kl_u >= d.k_total ? 0.f : fmaxf(0.f, 1.f - (float)(kl_u - d.k_anneal) * d.inv_ramp);
        if (ok) {
          for (int r0 = 0; r0 < nr; r0 += CH) {
            float x[D][CH], y[D][CH];
#pragma unroll
            for (int mu = 0; mu < D; ++mu)
              tmem_ld2_wait<CH>(t_lane + acc_col + (uint32_t)(mu * RG + r0),
                                t_lane + mst_col + (uint32_t)(mu * RG + r0), y[mu], x[mu]);
            // D <= 2: every lane takes part in the noise (lanes exchange normals)
            if (live || D <= 2) {
              float nq[4];  // D = 1: this spin's normals of four consecutive runs
#pragma unroll
              for (int j = 0; j < CH; j += 2) {  // two runs at once, FP32x2 arithmetic
                const int r = r0 + j;
                const float2 ar = *reinterpret_cast<const float2*>(&s_ar[g][r]);
                // each run's local step: noise counter and annealing scale alpha_mu
                int64_t klA = kl_u, klB = kl_u;
                float rA = ramp_u, rB = ramp_u;
                if (!k_uniform) {
                  const longlong2 kl2 = *reinterpret_cast<const longlong2*>(&s_kl[k & 1][g][r]);
                  const float2 rp2 = *reinterpret_cast<const float2*>(&s_rp[k & 1][g][r]);
                  klA = kl2.x;
                  klB = kl2.y;
                  rA = rp2.x;
                  rB = rp2.y;
                }
                const float2 e0 = make_float2(edt_p, edt_p), e1 = make_float2(edt_p * rA, edt_p * rB);
                float2 z[4 * ((D + 3) / 4)];
                if constexpr (D == 2) {
                  // spins p and p ^ 1 share one Philox block per run (pair 0: the even
                  // spin, pair 1: the odd one): each lane draws the block of one of the
                  // two runs and hands the partner spin's pair to the partner lane
                  const bool odd = (p & 1) != 0;
                  const uint4 w = philox_rk(noise_counter((uint32_t)p >> 1, 0u, 0u, (uint64_t)(odd ? klB : klA)),
                                            s_rk[g][odd ? r + 1 : r]);
                  float2 zc, zs;
                  box_muller_x2(w.x, w.y, w.z, w.w, neg2ln2s2, zc, zs);
                  const float kc = odd ? zc.y : zc.x, ks = odd ? zs.y : zs.x;  // own spin, own run
                  const float rc = __shfl_xor_sync(0xffffffffu, odd ? zc.x : zc.y, 1);
                  const float rs = __shfl_xor_sync(0xffffffffu, odd ? zs.x : zs.y, 1);  // own spin, other run
                  z[0] = odd ? make_float2(rc, kc) : make_float2(kc, rc);
                  z[1] = odd ? make_float2(rs, ks) : make_float2(ks, rs);
                  if (!live) continue;
                } else if constexpr (D == 1) {
                  // four spins share one block (spin p takes normal p % 4 of it): at every
                  // fourth run each lane of a quad draws the block of one of the four runs
                  // and the quad transposes the normals
                  if ((j & 3) == 0) {
                    const int m = p & 3, rm = r + m;
                    const int64_t klm = k_uniform ? kl_u : s_kl[k & 1][g][rm];
                    const uint4 w = philox_rk(noise_counter((uint32_t)p >> 2, 0u, 0u, (uint64_t)klm), s_rk[g][rm]);
                    float2 zc, zs;  // normals (0, 2) and (1, 3) of the block
                    box_muller_x2(w.x, w.y, w.z, w.w, neg2ln2s2, zc, zs);
                    quad_transpose(zc.x, zs.x, zc.y, zs.y, m, nq);
                  }
                  z[0] = (j & 3) == 0 ? make_float2(nq[0], nq[1]) : make_float2(nq[2], nq[3]);
                  if (!live) continue;
                } else {
#pragma unroll
                  for (int blk = 0; blk < (D + 3) / 4; ++blk) {
                    const uint4 wA = philox_rk(noise_counter((uint32_t)p, (uint32_t)blk, 0u, (uint64_t)klA),
                                               s_rk[g][r]);
                    const uint4 wB = philox_rk(noise_counter((uint32_t)p, (uint32_t)blk, 0u, (uint64_t)klB),
                                               s_rk[g][r + 1]);
                    box_muller_x2(wA.x, wA.y, wB.x, wB.y, neg2ln2s2, z[4 * blk], z[4 * blk + 1]);
                    if (D - 4 * blk > 2)
                      box_muller_x2(wA.z, wA.w, wB.z, wB.w, neg2ln2s2, z[4 * blk + 2], z[4 * blk + 3]);
                  }
                }
                float2 xx[D], n2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                  xx[mu] = make_float2(x[mu][j], x[mu][j + 1]);
                  n2 = __ffma2_rn(xx[mu], xx[mu], n2);
                }
                const float2 t = __ffma2_rn(ngdt, n2, ar);
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                  const float2 q = __fmul2_rn(nkdt, xx[mu]);
                  const float2 sfac = __ffma2_rn(q, xx[mu], t);
                  const float2 inner = __ffma2_rn(mu == 0 ? e0 : e1, make_float2(y[mu][j], y[mu][j + 1]), z[mu]);
                  const float2 xn = __ffma2_rn(xx[mu], sfac, inner);
                  x[mu][j] = xn.x;
                  x[mu][j + 1] = xn.y;
                }
              }
            }
#pragma unroll
            for (int mu = 0; mu < D; ++mu) {
              tmem_st<CH>(t_lane + mst_col + (uint32_t)(mu * RG + r0), x[mu]);
              const uint32_t n0 = (uint32_t)(mu * RG + r0);
              if (live) store_b<CH>(Bhi, Blo, b_row_off + (n0 >> 3) * 128u + (n0 & 7u) * 2u, x[mu]);
            }
          }
        }
        if (!k_uniform) put_step(k + 1);  // the other parity: nobody reads it in this step
        tmem_wait_st();
        fence_async_smem();
        tc_fence_before();
        if (group_bar_or(1 + g, s_abort)) break;
      }
    }
    if (wq == 0 && lane == 0) {
      // the J copy must have landed before the next item may overwrite it
      if (a_pending) mbar_wait(smem_addr(&s_abar), a_phase, L.wait_ns);
      // the tensor core may still own this group's accumulator: wait once more (bounded)
      // for the completion of the products of the step that timed out
      if (timed_out) {
        if (d.stall) mbar_wait(smem_addr(&s_wh[g]), 0u, L.wait_ns);  // the one step issued
        else mbar_wait(smem_addr(&s_mbar[g]), phase ^ 1u, L.wait_ns);
      }
    }
    if (new_a) {
      a_phase ^= 1u;
      a_desc = item.desc;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    aborted = s_abort != 0;
    // ---- store the state back (skipped after a timeout: the status reports it) ----
    if (!aborted) {
      for (int r0 = 0; r0 < nr; r0 += CH) {
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
          float v[CH];
          tmem_ld_wait<CH>(t_lane + mst_col + (uint32_t)(mu * RG + r0), v);
          if (live) {
#pragma unroll
            for (int j = 0; j < CH; ++j)
              if (r0 + j < nr) d.X[((size_t)(run0 + r0 + j) * N + p) * D + mu] = v[j];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // the next item reuses B, TMEM and (possibly) the J region
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Host: IEEE round-to-nearest-even of an FP32 value to BF16 (bit pattern).
uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)((u >> 16) | ((u & 0xFFFFu) ? 0x40u : 0u));
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

template <int D, int CH_>
cudaError_t launch_tc_plan(const TcLaunch& L, int n_cta, cudaStream_t st) {
  using Cfg = TcCfg<D, CH_>;
  const size_t b_bytes = (size_t)L.kp_max * Cfg::CG * 2u;
  // at least 128 KB: one CTA owns all 512 TMEM columns of its SM, so neither a
  // second CTA of this kernel nor a large-N step CTA (>= 104 KB) may be placed
  // beside it (it would wait in tcgen05.alloc until this CTA exits)
  const size_t smem = std::max<size_t>(L.a_region + (size_t)Cfg::G * 2 * b_bytes, 128 * 1024);
  auto kern = step_tc_kernel<D, CH_>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_cta, 128 * Cfg::G, smem, st>>>(L);
  return cudaGetLastError();
}

}  // namespace

int tc_runs_per_item(int D) {
  switch (D) {
    case 1: return TcCfg<1>::G * TcCfg<1>::RG;
    case 2: return TcCfg<2>::G * TcCfg<2>::RG;
    case 3: return TcCfg<3>::G * TcCfg<3>::RG;
    case 4: return TcCfg<4>::G * TcCfg<4>::RG;
    case 5: return TcCfg<5>::G * TcCfg<5>::RG;
    case 6: return TcCfg<6>::G * TcCfg<6>::RG;
    case 7: return TcCfg<7>::G * TcCfg<7>::RG;
    case 8: return TcCfg<8>::G * TcCfg<8>::RG;
  }
  return 0;
}

int tc_chunk_runs(int D) { return D <= 4 ? 8 : 4; }

size_t tc_desc_bytes() { return sizeof(TcDesc); }
size_t tc_item_bytes() { return sizeof(TcItem); }

// Fill the descriptor of one context for a launch starting at sc.k0.
void tc_fill_desc(const chym_ctx* c, const StepConsts& sc, void* out) {
  TcDesc& d = *reinterpret_cast<TcDesc*>(out);
  d.Aimg = (const uint8_t*)c->d_Jbf16;
  d.X = (float*)c->d_X;
  d.h = c->d_h;
  d.seeds = c->d_seeds;
  d.koff = c->d_koff;
  d.hidx = c->d_hidx;
  d.w = sc.w;
  d.N = c->N;
  d.KP = (c->N + 15) / 16 * 16;
  d.n_runs = sc.n_runs;
  d.replicas = sc.replicas;
  d.a_terms = c->kind == CHYM_J_PM1 ? 1 : 2;
  d.stall = sc.test_stall;
  d.sched_kind = sc.sched_kind;
  d.k0 = sc.k0;
  d.k_anneal = sc.k_anneal;
  d.k_total = sc.k_total;
  d.dt = (float)sc.dt;
  d.noise_scale = (float)sc.noise_scale;
  d.gdt = (float)(sc.dt * sc.gamma);
  d.kdt = (float)(sc.dt * sc.kappa);
  d.edt = (float)(sc.dt * sc.eps);
  d.inv_ramp = sc.sched_kind == 1 ? (float)(1.0 / (double)(sc.k_total - sc.k_anneal)) : 0.f;
}

void tc_fill_item(void* out, int desc, int run_begin, int run_count) {
  TcItem& it = *reinterpret_cast<TcItem*>(out);
  it.desc = desc;
  it.run_begin = run_begin;
  it.run_count = run_count;
  it.pad = 0;
}

// Launch the small-N tensor-core kernel of dimension D on a prepared plan in
// device memory: descs, items and the per-CTA item ranges.
cudaError_t launch_tc_items(int D, const void* d_descs, const void* d_items, const int* d_cta_begin,
                            int n_cta, int64_t steps, int kp_max, int terms_max, unsigned* status,
                            cudaStream_t st, bool test_stall, int chunk) {
  TcLaunch L;
  L.wait_ns = test_stall ? kTestWaitLimitNs : kWaitLimitNs;
  L.descs = (const TcDesc*)d_descs;
  L.items = (const TcItem*)d_items;
  L.cta_begin = d_cta_begin;
  L.steps = steps;
  L.kp_max = kp_max;
  L.a_region = (uint32_t)(terms_max * 128 * kp_max * 2);
  L.status = status;
  switch (D) {
    case 1: return chunk == 4 ? launch_tc_plan<1, 4>(L, n_cta, st) : launch_tc_plan<1, 0>(L, n_cta, st);
    case 2: return chunk == 4 ? launch_tc_plan<2, 4>(L, n_cta, st) : launch_tc_plan<2, 0>(L, n_cta, st);
    case 3: return chunk == 4 ? launch_tc_plan<3, 4>(L, n_cta, st) : launch_tc_plan<3, 0>(L, n_cta, st);
    case 4: return chunk == 4 ? launch_tc_plan<4, 4>(L, n_cta, st) : launch_tc_plan<4, 0>(L, n_cta, st);
    case 5: return launch_tc_plan<5, 0>(L, n_cta, st);
    case 6: return launch_tc_plan<6, 0>(L, n_cta, st);
    case 7: return launch_tc_plan<7, 0>(L, n_cta, st);
    case 8: return launch_tc_plan<8, 0>(L, n_cta, st);
  }
  return cudaErrorInvalidValue;
}


// Canonical K-major, no-swizzle image of J for the A operand: 128 rows (M) x KP
// (K) BF16, core matrices of 8 rows x 16 bytes; element (m, k) at byte
// (m%8)*16 + (k%8)*2 + (m/8)*(KP/8)*128 + (k/8)*128.  Real J gets a second
// image holding the BF16 residual J - bf16(J).
cudaError_t prepare_tc_operand(chym_ctx* c) {
  if (c->d_Jbf16) return cudaSuccess;
  const int N = c->N, KP = (N + 15) / 16 * 16;
  const int terms = c->kind == CHYM_J_PM1 ? 1 : 2;
  const size_t img = 128u * (size_t)KP;  // elements per term
  std::vector<uint16_t> h(terms * img, 0);
  for (int m = 0; m < 128; ++m)
    for (int k = 0; k < KP; ++k) {
      const double v = (m < N && k < N) ? c->h_J[(size_t)m * N + k] : 0.0;
      const uint16_t hi = bf16_bits((float)v);
      const uint16_t lo = bf16_bits((float)(v - (double)bf16_value(hi)));
      const size_t off = (size_t)(m % 8) * 8 + (k % 8) + (size_t)(m / 8) * (KP / 8) * 64 +
                         (size_t)(k / 8) * 64;  // in elements
      h[off] = hi;
      if (terms > 1) h[img + off] = lo;
    }
  cudaError_t e = cudaMalloc(&c->d_Jbf16, h.size() * sizeof(uint16_t));
  if (e != cudaSuccess) return e;
  c->jbf16_ld = KP;
  return cudaMemcpy(c->d_Jbf16, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
}

cudaError_t launch_step_tc(chym_ctx* c, const StepConsts& sc, cudaStream_t st) {
  if (c->N > 128) return cudaErrorNotSupported;
  cudaError_t e = prepare_tc_operand(c);
  if (e != cudaSuccess) return e;
  // one item (one CTA's worth of runs) per CTA
  const int per_item = tc_runs_per_item(c->D);
  const int n_items = (sc.n_runs + per_item - 1) / per_item;
  const size_t bytes = sizeof(TcDesc) + sizeof(TcItem) * n_items + sizeof(int) * (n_items + 1);
  std::vector<unsigned char> plan(bytes);
  tc_fill_desc(c, sc, plan.data());
  TcItem* items = reinterpret_cast<TcItem*>(plan.data() + sizeof(TcDesc));
  int* cta = reinterpret_cast<int*>(plan.data() + sizeof(TcDesc) + sizeof(TcItem) * n_items);
  for (int i = 0; i < n_items; ++i) {
    tc_fill_item(&items[i], 0, i * per_item, std::min(per_item, sc.n_runs - i * per_item));
    cta[i] = i;
  }
  cta[n_items] = n_items;
  if (bytes > c->plan_bytes) {
    if (c->d_plan) cudaFree(c->d_plan);
    c->d_plan = nullptr;
    c->plan_bytes = 0;
    e = cudaMalloc(&c->d_plan, bytes);
    if (e != cudaSuccess) return e;
    c->plan_bytes = bytes;
  }
  e = cudaMemcpyAsync(c->d_plan, plan.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const unsigned char* base = (const unsigned char*)c->d_plan;
  return launch_tc_items(c->D, base, base + sizeof(TcDesc),
                         (const int*)(base + sizeof(TcDesc) + sizeof(TcItem) * n_items), n_items,
                         sc.steps, (c->N + 15) / 16 * 16, c->kind == CHYM_J_PM1 ? 1 : 2,
                         c->d_status, st, sc.test_stall != 0);
}

}  // namespace chym
