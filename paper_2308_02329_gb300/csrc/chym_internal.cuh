// chym_internal.cuh -- shared declarations of the CHYM CUDA library.
//
// Context layout, error plumbing, the per-step constant block and the device
// helpers every kernel uses: the Philox4x32-10 generator (Salmon et al., SC'11)
// and the Box-Muller transform that draw the additive noise of the
// Euler-Maruyama step, and the dimensional-annealing schedule alpha_mu(k)
// (C -> alpha_mu C, text after Fig. 2 of arXiv 2308.02329).
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/chym.h"

namespace chym {

// ---------------------------------------------------------------- errors ---
void set_error(const std::string& msg);
chym_status fail(chym_status st, const std::string& msg);
chym_status cuda_fail(cudaError_t e, const char* what);

#define CHYM_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::chym::cuda_fail(_e, #expr); \
  } while (0)

// ---------------------------------------------------------- step constants ---
// Everything a step kernel needs besides pointers.  Built on the host from
// chym_params / chym_schedule for each chym_run call.
struct StepConsts {
  int N, D, n_runs, replicas;
  int64_t k0, steps;          // first step and number of steps of this launch
  double dt, noise_scale;     // noise_scale = sigma * sqrt(dt)
  double gamma, kappa, eps;
  int sched_kind;             // 0 none, 1 linear
  int64_t k_anneal, k_total;
  const int64_t* koff;        // per run: global step at which the run was (re)seeded
  const int32_t* hidx;        // per run: index of its pump value in h
  const double* w;            // per spin: weight of its coupling term (nullable: all 1)
  int fp8;                    // CHYM_PREC_FP8: e4m3 lo operands on the large-N path
  int test_stall;             // CHYM_FLAG_TEST_STALL: withhold the product completion signal
};

// Limit of every bounded device-side wait, and the short one of CHYM_FLAG_TEST_STALL.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
constexpr unsigned long long kTestWaitLimitNs = 2000000ull;

// Contiguous spin ranges [begin[i], begin[i + 1]) whose Ising energies are read
// out separately (independent graphs packed into one block-diagonal J).
constexpr int kMaxSegments = 128;
struct SegTable {
  int n;
  int begin[kMaxSegments + 1];
};

// Shared-memory budget of the SIMT step kernels, which keep every run of a CTA in
// shared memory for a whole launch (state and coupling product: 2 N D values a run).
constexpr size_t kSimtSmemBudget = 200 * 1024;

// Device status word: bit flags raised by kernels, read back by the host.
enum : unsigned { STATUS_TIMEOUT = 1u, STATUS_BAD_LAUNCH = 2u };

#if defined(__CUDACC__)
// ------------------------------------------------------------------ Philox ---
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Ten Philox4x32 rounds: two 32x32->64 products, xor with the other half and
// the round key, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// Counter of the noise of spin p, Philox block `blk` (components 4 blk .. 4 blk
// + 3), stream tag (0 step noise, 1 initial state), step k.
__device__ __forceinline__ uint4 noise_counter(uint32_t p, uint32_t blk, uint32_t tag,
                                               uint64_t k) {
  return make_uint4(p, (tag << 8) | blk, (uint32_t)k, (uint32_t)(k >> 32));
}

// Box-Muller on one pair of 32-bit words, FP64: u = (w + 1/2) 2^-32,
// (r cos 2 pi u_a, r sin 2 pi u_a) with r = sqrt(-2 ln u_r).
__device__ __forceinline__ void box_muller_f64(uint32_t wr, uint32_t wa, double& z0,
                                               double& z1) {
  const double ur = ((double)wr + 0.5) * 2.3283064365386963e-10;
  const double ua = ((double)wa + 0.5) * 2.3283064365386963e-10;
  const double r = sqrt(-2.0 * log(ur));
  double s, c;
  sincospi(2.0 * ua, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// FP32 Box-Muller with the SFU approximations; the angle is taken in
// (-pi, pi] where the hardware sine/cosine are accurate, and the pair is
// negated back: cos(t) = -cos(t - pi), sin(t) = -sin(t - pi).  `scale`
// multiplies both outputs (folded into the radius).
__device__ __forceinline__ void box_muller_f32(uint32_t wr, uint32_t wa, float scale,
                                               float& z0, float& z1) {
  const float ur = __fmaf_rn((float)wr, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float ua = __fmaf_rn((float)wa, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float r = sqrtf(-2.0f * scale * scale * __logf(ur));
  float s, c;
  __sincosf(__fmaf_rn(ua, 6.2831853071795865f, -3.1415926535897932f), &s, &c);
  z0 = -r * c;
  z1 = -r * s;
}

// Normal number j (0..3) of a Philox block in FP64.
__device__ __forceinline__ void block_normals_f64(uint4 w, double z[4]) {
  box_muller_f64(w.x, w.y, z[0], z[1]);
  box_muller_f64(w.z, w.w, z[2], z[3]);
}

#endif  // __CUDACC__

// ------------------------------------------------------- annealing schedule ---
// alpha_mu(k): 1 for mu = 0 or before k_anneal, then linear down to 0 at k_total.
__host__ __device__ __forceinline__ double alpha_of(int kind, int64_t k, int64_t k_anneal,
                                                    int64_t k_total, int mu) {
  if (kind == 0 || mu == 0 || k < k_anneal) return 1.0;
  if (k >= k_total) return 0.0;
  const double a = 1.0 - (double)(k - k_anneal) / (double)(k_total - k_anneal);
  return a < 0.0 ? 0.0 : a;
}

}  // namespace chym

namespace chym {
// NVTX range over one ABI call, visible in Nsight Systems timelines; without an
// attached tool the push and pop return at once.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace chym

namespace chym {
// Launch state of the large-N path: device tables, a private capture stream and the
// CUDA graph of a chunk of steps (re-captured when the tile table changes shape).
struct K2Runner {
  void* d_buf = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t sig_tiles = 0;
  std::vector<int> sig_dims;
  void* sig_buf = nullptr;
  int sig_cap = 0;
  bool sig_stall = false;
  std::vector<int> sig_stages;
  int sms = 0;
};
}  // namespace chym

// ------------------------------------------------------------------ context ---
struct chym_ctx {
  int N = 0, D = 0;
  chym_jkind kind = CHYM_J_PM1;
  int device = 0;
  double* h_J = nullptr;      // host copy, row-major FP64
  // device copies of J
  double* d_J64 = nullptr;    // FP64 N x N
  float* d_J32 = nullptr;     // FP32 N x N
  float* d_J32p = nullptr;    // FP32 N x j32p_ld, rows zero padded to a multiple of 4
  int j32p_ld = 0;
  int8_t* d_J8 = nullptr;     // int8 N x N (+-1/0 couplings only)
  // +-1 couplings: bit planes for the Ising energy, [plane][word w][row p] (plane 0: J = +1,
  // plane 1: J = -1; word w holds columns 64 w .. 64 w + 63), and per row (#+1) - (#-1)
  uint64_t* d_Jbits = nullptr;
  int32_t* d_jdeg = nullptr;
  // J in compressed rows when it is sparse (at most N^2 / 16 nonzeros): the coupling
  // product then runs on the CUDA cores over the nonzeros only
  bool sparse = false;
  bool csr_bf16 = false;      // the compressed rows also replace the BF16 tensor-core product
  int nnz = 0;
  int32_t* d_rp = nullptr;    // row starts, N + 1
  int32_t* d_ci = nullptr;    // column of each nonzero
  float* d_cv32 = nullptr;    // value of each nonzero, FP32 and FP64
  double* d_cv64 = nullptr;
  void* d_Jbf16 = nullptr;    // BF16, padded for the tensor-core kernels (lazily built)
  int jbf16_ld = 0;           // leading dimension of d_Jbf16 in elements
  // batch
  int n_runs = 0, n_h = 0, cap_runs = 0, cap_h = 0;
  int64_t k = 0;
  int32_t prec = -1;          // precision the state is stored in (-1: no state)
  void* d_X = nullptr;        // state X[run][p][mu], double (FP64) or float
  size_t x_bytes = 0;
  double* d_h = nullptr;
  uint64_t* d_seeds = nullptr;
  int64_t* d_koff = nullptr;  // per run: global step of its (re)seeding; local step = k - koff
  int32_t* d_hidx = nullptr;  // per run: index of its pump value (run / replicas unless reseeded)
  double* d_E = nullptr;      // energies of the last chym_energy*
  uint64_t* d_spins = nullptr;
  bool have_energy = false;
  double* d_w = nullptr;      // per spin coupling weights (nullable: all 1)
  double* d_Eseg = nullptr;   // energies of the last chym_energy_segments, [run][segment]
  size_t eseg_cap = 0;        // doubles
  unsigned* d_status = nullptr;
  void* d_scratch = nullptr;  // stats scratch
  size_t scratch_bytes = 0;
  void* d_plan = nullptr;     // launch plan of the small-N tensor-core kernel
  size_t plan_bytes = 0;
  void* d_Ak2 = nullptr;      // J as A-operand blocks of the large-N path (lazily built)
  void* d_k2_ws = nullptr;    // large-N workspace: column-major master state, BF16 blocks
  size_t k2_ws_bytes = 0;
  chym::K2Runner k2_runner;
};

namespace chym {
// Whether a step of context c at precision prec runs its coupling over the compressed
// rows on the CUDA cores: always for a sparse J in FP32/FP64 (against the dense SIMT
// product), and in place of the BF16 tensor-core product only where that measured
// slower and a run's state fits the SIMT kernel's shared memory: N >= 1024, D >= 3,
// on average at most N / 256 nonzeros per row (nnz <= N^2 / 256) and
// 2 N D sizeof(float) <= kSimtSmemBudget.
// Precisions whose coupling product runs on the tensor cores (FP32 state, BF16 hi
// part; FP8 mode differs from BF16X2 only in the lo operands of the large-N path).
inline bool is_tc_prec(int32_t prec) { return prec == CHYM_PREC_BF16X2 || prec == CHYM_PREC_FP8; }
inline bool uses_csr(const chym_ctx* c, int32_t prec) {
  return c->sparse && (!is_tc_prec(prec) || c->csr_bf16);
}
// kernel launchers (implemented in the .cu files)
cudaError_t launch_init(chym_ctx* c, int32_t prec, cudaStream_t st, double init_std);
cudaError_t launch_reseed(chym_ctx* c, const int32_t* d_runs, int n, const uint64_t* d_new_seeds,
                          const int32_t* d_new_hidx, double init_std, cudaStream_t st);
cudaError_t launch_fill_hidx(int32_t* hidx, int n_runs, int replicas, cudaStream_t st);
cudaError_t launch_step_simt(chym_ctx* c, const StepConsts& sc, int32_t prec, cudaStream_t st);
cudaError_t launch_step_tc(chym_ctx* c, const StepConsts& sc, cudaStream_t st);
cudaError_t launch_step_k2(chym_ctx* c, const StepConsts& sc, cudaStream_t st);
// large-N path over several contexts (chym_k2.cu)
cudaError_t k2_prepare(chym_ctx* c, const StepConsts& sc, cudaStream_t st, void* desc_out, int rt = 0);
// most ring stages of the large-N kernel for a context of dimension D with rt runs per
// column tile (0: the default), real J (terms 2) or FP8 lo, within its shared memory
int k2_max_stages(int D, int rt, int n_runs, int a_terms, int lo8);
size_t k2_desc_bytes();
// tiles x K chunks of one step of a large-N context (the planner's work unit)
long long k2_work_units(int N, int D, int n_runs, int rt = 0);
cudaError_t k2_finish(chym_ctx* c, const void* desc, cudaStream_t st);
// max_ctas > 0 caps the persistent grid (the SMs left to the large-N path when the
// small-N kernels of a batch occupy the others).
cudaError_t k2_integrate(K2Runner& R, const std::vector<unsigned char>& descs,
                         const std::vector<int>& dims, int64_t steps, unsigned* status,
                         cudaStream_t st, int max_ctas = 0, const int* stages = nullptr);
void k2_runner_release(K2Runner& R);
// small-N tensor-core kernel over an item plan (chym_tc.cu)
cudaError_t prepare_tc_operand(chym_ctx* c);
int tc_runs_per_item(int D);
int tc_chunk_runs(int D);
int tc_groups(int D);  // warpgroups of a CTA: the chunks it advances side by side
size_t tc_desc_bytes();
size_t tc_item_bytes();
void tc_fill_desc(const chym_ctx* c, const StepConsts& sc, void* out);
void tc_fill_item(void* out, int desc, int run_begin, int run_count);
cudaError_t launch_tc_items(int D, const void* d_descs, const void* d_items, const int* d_cta_begin,
                            int n_cta, int64_t steps, int kp_max, int terms_max, unsigned* status,
                            cudaStream_t st, bool test_stall = false, int chunk = 0);
// Tile shapes the batch autotuner may choose (0: the kernels' defaults).
struct TileShapes {
  int rt[9] = {};      // large-N path: runs per column tile, per D
  int stages[9] = {};  // large-N path: depth of the operand ring, per D
  int ch[9] = {};      // small-N path: runs per epilogue chunk, per D (4 or 8 for D <= 4)
};
// valid choices of the large-N runs per column tile for dimension D (a multiple of 32,
// D RT <= 256 and a multiple of 16)
inline bool k2_rt_valid(int D, int rt) {
  return rt >= 32 && rt % 32 == 0 && D * rt <= 256 && (D * rt) % 16 == 0;
}
cudaError_t launch_energy(chym_ctx* c, double* d_E, uint64_t* d_spins, cudaStream_t st);
cudaError_t launch_energy_segments(chym_ctx* c, const SegTable& t, double* d_E, cudaStream_t st);
cudaError_t launch_stats(chym_ctx* c, const double* d_E, double E_gs, double tol, double bin_w,
                         int n_bins, void* d_out, cudaStream_t st);
double host_lambda_max(const double* J, int N);
}  // namespace chym
