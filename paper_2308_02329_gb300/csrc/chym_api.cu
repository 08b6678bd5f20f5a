// chym_api.cu -- the C ABI of include/chym.h: argument checks, device buffers,
// kernel dispatch and the host side of the figures of merit.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "chym_internal.cuh"

namespace chym {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

chym_status fail(chym_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

chym_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return CHYM_ECUDA;
}

size_t stats_out_bytes(int n_h, int n_bins);
cudaError_t launch_step(chym_ctx* c, const StepConsts& sc, int32_t prec, cudaStream_t st);

namespace {

template <typename P>
void free_dev(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

chym_status check_params(const chym_params* prm) {
  if (!prm) return fail(CHYM_EINVAL, "params is NULL");
  if (!(prm->dt > 0.0) || !isfinite(prm->dt)) return fail(CHYM_EINVAL, "dt must be > 0");
  if (!(prm->sigma >= 0.0) || !isfinite(prm->sigma)) return fail(CHYM_EINVAL, "sigma must be >= 0");
  if (!(prm->init_std >= 0.0) || !isfinite(prm->init_std))
    return fail(CHYM_EINVAL, "init_std must be >= 0");
  if (!isfinite(prm->gamma) || !isfinite(prm->kappa) || !isfinite(prm->eps))
    return fail(CHYM_EINVAL, "gamma, kappa, eps must be finite");
  if (prm->prec < CHYM_PREC_FP64 || prm->prec > CHYM_PREC_FP8)
    return fail(CHYM_EINVAL, "unknown precision");
  if (prm->flags != 0 && prm->flags != CHYM_FLAG_TEST_STALL)
    return fail(CHYM_EINVAL, "params.flags must be 0 or CHYM_FLAG_TEST_STALL");
  return CHYM_OK;
}

chym_status check_schedule(const chym_schedule* s) {
  if (!s) return fail(CHYM_EINVAL, "schedule is NULL");
  if (s->kind != 0 && s->kind != 1) return fail(CHYM_EINVAL, "schedule.kind must be 0 or 1");
  if (s->reserved != 0) return fail(CHYM_EINVAL, "schedule.reserved must be 0");
  if (s->kind == 1 && (s->k_anneal < 0 || s->k_total <= s->k_anneal))
    return fail(CHYM_EINVAL, "linear schedule needs 0 <= k_anneal < k_total");
  return CHYM_OK;
}


// Make room for n_runs runs and n_h pumps.
chym_status ensure_batch(chym_ctx* c, int n_runs, int n_h) {
  if (n_runs > c->cap_runs) {
    free_dev(c->d_X);
    free_dev(c->d_seeds);
    free_dev(c->d_koff);
    free_dev(c->d_hidx);
    free_dev(c->d_E);
    free_dev(c->d_spins);
    c->cap_runs = 0;
    const size_t xb = (size_t)n_runs * c->N * c->D * sizeof(double);
    const int words = (c->N + 63) / 64;
    CHYM_CUDA_TRY(cudaMalloc(&c->d_X, xb));
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_seeds, sizeof(uint64_t) * n_runs));
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_koff, sizeof(int64_t) * n_runs));
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_hidx, sizeof(int32_t) * n_runs));
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_E, sizeof(double) * n_runs));
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_spins, sizeof(uint64_t) * (size_t)n_runs * words));
    c->x_bytes = xb;
    c->cap_runs = n_runs;
  }
  if (n_h > c->cap_h) {
    free_dev(c->d_h);
    c->cap_h = 0;
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_h, sizeof(double) * n_h));
    c->cap_h = n_h;
  }
  return CHYM_OK;
}

}  // namespace

StepConsts make_step_consts(const chym_ctx* c, const chym_params* prm, const chym_schedule* s,
                            int64_t k0, int64_t steps) {
  StepConsts sc;
  sc.N = c->N;
  sc.D = c->D;
  sc.n_runs = c->n_runs;
  sc.replicas = c->n_runs / c->n_h;
  sc.k0 = k0;
  sc.steps = steps;
  sc.dt = prm->dt;
  sc.noise_scale = prm->sigma * sqrt(prm->dt);
  sc.gamma = prm->gamma;
  sc.kappa = prm->kappa;
  sc.eps = prm->eps;
  sc.sched_kind = s->kind;
  sc.k_anneal = s->k_anneal;
  sc.k_total = s->k_total;
  sc.koff = c->d_koff;
  sc.hidx = c->d_hidx;
  sc.w = c->d_w;
  sc.fp8 = prm->prec == CHYM_PREC_FP8 ? 1 : 0;
  sc.test_stall = (prm->flags & CHYM_FLAG_TEST_STALL) ? 1 : 0;
  return sc;
}

namespace {

// Shared body of chym_run / chym_run_device once h and seeds sit on the device.
chym_status run_on_device(chym_ctx* c, const chym_params* prm, bool init, int64_t steps,
                          const chym_schedule* sched, cudaStream_t st) {
  if (init) {
    c->prec = prm->prec;
    c->k = 0;
    CHYM_CUDA_TRY(cudaMemsetAsync(c->d_koff, 0, sizeof(int64_t) * c->n_runs, st));
    CHYM_CUDA_TRY(launch_fill_hidx(c->d_hidx, c->n_runs, c->n_runs / c->n_h, st));
    CHYM_CUDA_TRY(launch_init(c, c->prec, st, prm->init_std));
  } else if (prm->prec != c->prec) {
    // FP32 and BF16X2 share FP32 storage; FP64 storage cannot be continued in
    // another precision (re-initialise, or reload it with chym_set_state)
    if ((c->prec == CHYM_PREC_FP64) != (prm->prec == CHYM_PREC_FP64))
      return fail(CHYM_EINVAL, "cannot continue an FP64 state in FP32 storage or back");
    c->prec = prm->prec;
  }
  c->have_energy = false;
  if (steps > 0 && c->d_w && c->N > 128 && is_tc_prec(c->prec) && !uses_csr(c, c->prec))
    return fail(CHYM_ENOTSUP, "coupling weights need N <= 128 on the tensor-core path");
  if (steps > 0) {
    const StepConsts sc = make_step_consts(c, prm, sched, c->k, steps);
    cudaError_t e = launch_step(c, sc, c->prec, st);
    if (e == cudaErrorInvalidConfiguration)
      return fail(CHYM_ENOTSUP, "problem too large for the selected kernel (N*D per run)");
    if (e == cudaErrorNotSupported)
      return fail(CHYM_ENOTSUP, "no kernel for this precision and size");
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    c->k += steps;
  }
  return CHYM_OK;
}

// Read and clear the device status word after the stream has been synchronised.
chym_status check_device_status(chym_ctx* c) {
  unsigned st = 0;
  CHYM_CUDA_TRY(cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st) {
    CHYM_CUDA_TRY(cudaMemset(c->d_status, 0, sizeof(unsigned)));
    if (st & STATUS_TIMEOUT) return fail(CHYM_ETIMEOUT, "a device-side wait timed out; state not updated");
    return fail(CHYM_ECUDA, "device status word set");
  }
  return CHYM_OK;
}

chym_status check_run_args(chym_ctx* c, const chym_params* prm, int n_h, int n_runs,
                           int64_t steps, const chym_schedule* sched, bool have_seeds) {
  if (!c) return fail(CHYM_EINVAL, "ctx is NULL");
  chym_status s = check_params(prm);
  if (s != CHYM_OK) return s;
  s = check_schedule(sched);
  if (s != CHYM_OK) return s;
  if (steps < 0) return fail(CHYM_EINVAL, "steps must be >= 0");
  if (n_h < 1) return fail(CHYM_EINVAL, "n_h must be >= 1");
  if (n_runs < 1) return fail(CHYM_EINVAL, "n_runs must be >= 1");
  if (n_runs % n_h != 0) return fail(CHYM_EINVAL, "n_runs must be a multiple of n_h");
  if (!have_seeds) {
    if (c->prec < 0) return fail(CHYM_ESTATE, "no state to continue: pass seeds first");
    if (n_runs != c->n_runs) return fail(CHYM_EINVAL, "n_runs differs from the running batch");
  }
  return CHYM_OK;
}

}  // namespace

cudaError_t launch_step(chym_ctx* c, const StepConsts& sc, int32_t prec, cudaStream_t st) {
  // sparse J: the coupling over the nonzeros on the CUDA cores, FP32 state unless FP64
  if (uses_csr(c, prec)) return launch_step_simt(c, sc, prec == CHYM_PREC_FP64 ? prec : CHYM_PREC_FP32, st);
  if (prec == CHYM_PREC_FP64 || prec == CHYM_PREC_FP32) return launch_step_simt(c, sc, prec, st);
  if (is_tc_prec(prec))
    return c->N <= 128 ? launch_step_tc(c, sc, st) : launch_step_k2(c, sc, st);
  return cudaErrorNotSupported;
}

}  // namespace chym

using namespace chym;

extern "C" {

const char* chym_last_error(void) { return g_last_error.c_str(); }

chym_status chym_create(const double* J, int N, int D, chym_jkind kind, chym_ctx** out) {
  chym::TraceRange trace_("chym_create");
  if (!out) return fail(CHYM_EINVAL, "out is NULL");
  if (!J) return fail(CHYM_EINVAL, "J is NULL");
  if (N < 1 || N > 4096) return fail(CHYM_EINVAL, "N must be in [1, 4096]");
  if (D < 1 || D > 8) return fail(CHYM_EINVAL, "D must be in [1, 8]");
  if (kind != CHYM_J_PM1 && kind != CHYM_J_REAL) return fail(CHYM_EINVAL, "unknown J kind");
  for (int i = 0; i < N; ++i) {
    if (J[(size_t)i * N + i] != 0.0) return fail(CHYM_EINVAL, "J must have a zero diagonal");
    for (int j = 0; j < N; ++j) {
      const double v = J[(size_t)i * N + j];
      if (!isfinite(v)) return fail(CHYM_EINVAL, "J has a non-finite entry");
      if (v != J[(size_t)j * N + i]) return fail(CHYM_EINVAL, "J must be symmetric");
      if (kind == CHYM_J_PM1 && v != 0.0 && v != 1.0 && v != -1.0)
        return fail(CHYM_EINVAL, "CHYM_J_PM1 needs entries in {-1, 0, 1}");
    }
  }
  chym_ctx* c = new (std::nothrow) chym_ctx();
  if (!c) return fail(CHYM_ENOMEM, "host allocation failed");
  c->N = N;
  c->D = D;
  c->kind = kind;
  cudaError_t e = cudaGetDevice(&c->device);
  const size_t nn = (size_t)N * N;
  c->h_J = new (std::nothrow) double[nn];
  if (!c->h_J) {
    delete c;
    return fail(CHYM_ENOMEM, "host allocation failed");
  }
  memcpy(c->h_J, J, nn * sizeof(double));
  std::vector<float> j32(nn);
  std::vector<int8_t> j8(nn);
  for (size_t i = 0; i < nn; ++i) {
    j32[i] = (float)J[i];
    j8[i] = (int8_t)(kind == CHYM_J_PM1 ? (int)J[i] : 0);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_J64, nn * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_J32, nn * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_J8, nn);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_J64, J, nn * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_J32, j32.data(), nn * sizeof(float), cudaMemcpyHostToDevice);
  {  // rows padded to 16 bytes for the vector loads of the tiled FP32 kernel
    const int ld = (N + 3) / 4 * 4;
    std::vector<float> jp((size_t)N * ld, 0.f);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) jp[(size_t)i * ld + j] = j32[(size_t)i * N + j];
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_J32p, jp.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_J32p, jp.data(), jp.size() * sizeof(float), cudaMemcpyHostToDevice);
    c->j32p_ld = ld;
  }
  if (e == cudaSuccess) e = cudaMemcpy(c->d_J8, j8.data(), nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
  if (e == cudaSuccess && kind == CHYM_J_PM1) {  // bit planes of the Ising energy
    const int W = (N + 63) / 64;
    std::vector<uint64_t> planes((size_t)2 * W * N, 0ull);
    std::vector<int32_t> deg(N, 0);
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < N; ++q) {
        const double v = J[(size_t)p * N + q];
        if (v == 0.0) continue;
        const size_t at = (size_t)(v > 0.0 ? 0 : W) * N + (size_t)(q / 64) * N + p;
        planes[at] |= 1ull << (q % 64);
        deg[p] += v > 0.0 ? 1 : -1;
      }
    e = cudaMalloc((void**)&c->d_Jbits, planes.size() * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_jdeg, sizeof(int32_t) * N);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_Jbits, planes.data(), planes.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_jdeg, deg.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
  }
  // sparse J: compressed rows for the CUDA-core product
  size_t nz = 0;
  for (size_t i = 0; i < nn; ++i) nz += J[i] != 0.0;
  if (e == cudaSuccess && nz * 16 <= nn) {
    std::vector<int32_t> rp(N + 1, 0), ci;
    std::vector<float> v32;
    std::vector<double> v64;
    ci.reserve(nz);
    v32.reserve(nz);
    v64.reserve(nz);
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j) {
        const double v = J[(size_t)i * N + j];
        if (v != 0.0) {
          ci.push_back(j);
          v32.push_back((float)v);
          v64.push_back(v);
        }
      }
      rp[i + 1] = (int32_t)ci.size();
    }
    c->sparse = true;
    c->csr_bf16 = N >= 1024 && D >= 3 && nz * 256 <= nn &&
                  (size_t)2 * N * D * sizeof(float) <= kSimtSmemBudget;
    c->nnz = (int)nz;
    const size_t nzb = std::max<size_t>(nz, 1);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_rp, sizeof(int32_t) * (N + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ci, sizeof(int32_t) * nzb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_cv32, sizeof(float) * nzb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_cv64, sizeof(double) * nzb);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_rp, rp.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nz) e = cudaMemcpy(c->d_ci, ci.data(), sizeof(int32_t) * nz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nz) e = cudaMemcpy(c->d_cv32, v32.data(), sizeof(float) * nz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nz) e = cudaMemcpy(c->d_cv64, v64.data(), sizeof(double) * nz, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    chym_status st = cuda_fail(e, "chym_create device setup");
    chym_destroy(c);
    return st;
  }
  *out = c;
  return CHYM_OK;
}

chym_status chym_destroy(chym_ctx* c) {
  if (!c) return CHYM_OK;
  free_dev(c->d_J64);
  free_dev(c->d_J32);
  free_dev(c->d_J32p);
  free_dev(c->d_J8);
  free_dev(c->d_Jbits);
  free_dev(c->d_jdeg);
  free_dev(c->d_Jbf16);
  free_dev(c->d_X);
  free_dev(c->d_h);
  free_dev(c->d_seeds);
  free_dev(c->d_koff);
  free_dev(c->d_hidx);
  free_dev(c->d_E);
  free_dev(c->d_spins);
  free_dev(c->d_w);
  free_dev(c->d_Eseg);
  free_dev(c->d_rp);
  free_dev(c->d_ci);
  free_dev(c->d_cv32);
  free_dev(c->d_cv64);
  free_dev(c->d_status);
  free_dev(c->d_scratch);
  free_dev(c->d_Ak2);
  free_dev(c->d_plan);
  k2_runner_release(c->k2_runner);
  free_dev(c->d_k2_ws);
  delete[] c->h_J;
  delete c;
  return CHYM_OK;
}

chym_status chym_lambda_max(chym_ctx* c, double* out) {
  if (!c || !out) return fail(CHYM_EINVAL, "NULL argument");
  *out = host_lambda_max(c->h_J, c->N);
  return CHYM_OK;
}

chym_status chym_reseed_device(chym_ctx* c, const int32_t* d_runs, int n, const uint64_t* d_new_seeds,
                               const int32_t* d_new_pump, double init_std, void* stream) {
  chym::TraceRange trace_("chym_reseed_device");
  if (!c) return fail(CHYM_EINVAL, "ctx is NULL");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state: call chym_run first");
  if (n < 0 || (n > 0 && (!d_runs || !d_new_seeds))) return fail(CHYM_EINVAL, "bad run list");
  if (!(init_std >= 0.0) || !isfinite(init_std)) return fail(CHYM_EINVAL, "init_std must be >= 0");
  if (n == 0) return CHYM_OK;
  CHYM_CUDA_TRY(launch_reseed(c, d_runs, n, d_new_seeds, d_new_pump, init_std, (cudaStream_t)stream));
  c->have_energy = false;
  return CHYM_OK;
}

chym_status chym_get_offsets_device(chym_ctx* c, int64_t* d_koff_out, void* stream) {
  if (!c || !d_koff_out) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state");
  CHYM_CUDA_TRY(cudaMemcpyAsync(d_koff_out, c->d_koff, sizeof(int64_t) * c->n_runs,
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return CHYM_OK;
}

chym_status chym_info(chym_ctx* c, int* n_runs, int* n_h, int64_t* k) {
  if (!c) return fail(CHYM_EINVAL, "ctx is NULL");
  if (n_runs) *n_runs = c->n_runs;
  if (n_h) *n_h = c->n_h;
  if (k) *k = c->k;
  return CHYM_OK;
}

chym_status chym_run(chym_ctx* c, const chym_params* prm, const double* h, int n_h,
                     const uint64_t* seeds, int n_runs, int64_t steps,
                     const chym_schedule* sched, void* stream) {
  chym::TraceRange trace_("chym_run");
  chym_status s = check_run_args(c, prm, n_h, n_runs, steps, sched, seeds != nullptr);
  if (s != CHYM_OK) return s;
  if (!h && seeds) return fail(CHYM_EINVAL, "h is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (seeds) {
    s = ensure_batch(c, n_runs, n_h);
    if (s != CHYM_OK) return s;
    c->n_runs = n_runs;
    c->n_h = n_h;
    CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_seeds, seeds, sizeof(uint64_t) * n_runs,
                                  cudaMemcpyHostToDevice, st));
  } else if (n_h != c->n_h) {
    return fail(CHYM_EINVAL, "n_h differs from the running batch");
  }
  if (h) CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_h, h, sizeof(double) * n_h, cudaMemcpyHostToDevice, st));
  return run_on_device(c, prm, seeds != nullptr, steps, sched, st);
}

chym_status chym_run_device(chym_ctx* c, const chym_params* prm, const double* d_h, int n_h,
                            const uint64_t* d_seeds, int n_runs, int64_t steps,
                            const chym_schedule* sched, void* stream) {
  chym::TraceRange trace_("chym_run_device");
  chym_status s = check_run_args(c, prm, n_h, n_runs, steps, sched, d_seeds != nullptr);
  if (s != CHYM_OK) return s;
  if (!d_h && d_seeds) return fail(CHYM_EINVAL, "d_h is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (d_seeds) {
    s = ensure_batch(c, n_runs, n_h);
    if (s != CHYM_OK) return s;
    c->n_runs = n_runs;
    c->n_h = n_h;
    CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_seeds, d_seeds, sizeof(uint64_t) * n_runs,
                                  cudaMemcpyDeviceToDevice, st));
  } else if (n_h != c->n_h) {
    return fail(CHYM_EINVAL, "n_h differs from the running batch");
  }
  if (d_h)
    CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_h, d_h, sizeof(double) * n_h, cudaMemcpyDeviceToDevice, st));
  return run_on_device(c, prm, d_seeds != nullptr, steps, sched, st);
}

chym_status chym_energy_device(chym_ctx* c, double* d_E, uint64_t* d_spins, void* stream) {
  chym::TraceRange trace_("chym_energy_device");
  if (!c || !d_E) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state: call chym_run first");
  cudaStream_t st = (cudaStream_t)stream;
  CHYM_CUDA_TRY(launch_energy(c, d_E, d_spins, st));
  if (d_E != c->d_E)
    CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_E, d_E, sizeof(double) * c->n_runs, cudaMemcpyDeviceToDevice, st));
  c->have_energy = true;
  return CHYM_OK;
}

chym_status chym_energy(chym_ctx* c, double* E_out, uint64_t* spins_out, void* stream) {
  chym::TraceRange trace_("chym_energy");
  if (!c || !E_out) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state: call chym_run first");
  cudaStream_t st = (cudaStream_t)stream;
  CHYM_CUDA_TRY(launch_energy(c, c->d_E, c->d_spins, st));
  c->have_energy = true;
  CHYM_CUDA_TRY(cudaMemcpyAsync(E_out, c->d_E, sizeof(double) * c->n_runs, cudaMemcpyDeviceToHost, st));
  if (spins_out) {
    const size_t words = (size_t)(c->N + 63) / 64;
    CHYM_CUDA_TRY(cudaMemcpyAsync(spins_out, c->d_spins, sizeof(uint64_t) * c->n_runs * words,
                                  cudaMemcpyDeviceToHost, st));
  }
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  return check_device_status(c);
}

chym_status chym_set_coupling_weights(chym_ctx* c, const double* w) {
  if (!c) return fail(CHYM_EINVAL, "ctx is NULL");
  if (!w) {
    free_dev(c->d_w);
    return CHYM_OK;
  }
  for (int p = 0; p < c->N; ++p)
    if (!isfinite(w[p])) return fail(CHYM_EINVAL, "coupling weights must be finite");
  if (!c->d_w) CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_w, sizeof(double) * c->N));
  CHYM_CUDA_TRY(cudaMemcpy(c->d_w, w, sizeof(double) * c->N, cudaMemcpyHostToDevice));
  return CHYM_OK;
}

chym_status chym_energy_segments(chym_ctx* c, int n_seg, const int* seg_begin, double* E_out,
                                 void* stream) {
  chym::TraceRange trace_("chym_energy_segments");
  if (!c || !seg_begin || !E_out) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state: call chym_run first");
  if (n_seg < 1 || n_seg > kMaxSegments) return fail(CHYM_EINVAL, "n_seg must be in [1, 128]");
  if (seg_begin[0] != 0 || seg_begin[n_seg] != c->N)
    return fail(CHYM_EINVAL, "segments must start at spin 0 and end at spin N");
  SegTable t;
  t.n = n_seg;
  for (int i = 0; i <= n_seg; ++i) {
    if (i > 0 && seg_begin[i] <= seg_begin[i - 1]) return fail(CHYM_EINVAL, "segments must be non-empty and ordered");
    t.begin[i] = seg_begin[i];
  }
  const size_t need = (size_t)c->n_runs * n_seg;
  if (need > c->eseg_cap) {
    free_dev(c->d_Eseg);
    c->eseg_cap = 0;
    CHYM_CUDA_TRY(cudaMalloc((void**)&c->d_Eseg, sizeof(double) * need));
    c->eseg_cap = need;
  }
  cudaStream_t st = (cudaStream_t)stream;
  CHYM_CUDA_TRY(launch_energy_segments(c, t, c->d_Eseg, st));
  CHYM_CUDA_TRY(cudaMemcpyAsync(E_out, c->d_Eseg, sizeof(double) * need, cudaMemcpyDeviceToHost, st));
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  return check_device_status(c);
}

chym_status chym_stats(chym_ctx* c, double E_gs, chym_stats_t* out, int64_t* hits_per_h,
                       int64_t* hist, int n_bins, void* stream) {
  chym::TraceRange trace_("chym_stats");
  if (!c || !out) return fail(CHYM_EINVAL, "NULL argument");
  if (!c->have_energy) return fail(CHYM_ESTATE, "call chym_energy first");
  if (n_bins < 0 || (hist && n_bins < 1)) return fail(CHYM_EINVAL, "bad n_bins");
  if (!isfinite(E_gs)) return fail(CHYM_EINVAL, "E_gs must be finite");
  if (!hist) n_bins = 0;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = stats_out_bytes(c->n_h, n_bins);
  if (need > c->scratch_bytes) {
    free_dev(c->d_scratch);
    c->scratch_bytes = 0;
    CHYM_CUDA_TRY(cudaMalloc(&c->d_scratch, need));
    c->scratch_bytes = need;
  }
  const bool pm1 = c->kind == CHYM_J_PM1;
  const double tol = pm1 ? 0.0 : 1e-9 * fabs(E_gs);
  double bin_w = pm1 ? 4.0 : 1e-3 * fabs(E_gs);
  if (!(bin_w > 0.0)) bin_w = 1.0;
  CHYM_CUDA_TRY(launch_stats(c, c->d_E, E_gs, tol, bin_w, n_bins, c->d_scratch, st));  // per-run pumps
  std::vector<unsigned char> buf(need);
  CHYM_CUDA_TRY(cudaMemcpyAsync(buf.data(), c->d_scratch, need, cudaMemcpyDeviceToHost, st));
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  struct Head {
    double sum_dE, best_E;
    long long best_run, n_finite, n_hits, pad[3];
  } head;
  memcpy(&head, buf.data(), sizeof(head));
  std::vector<long long> hits(c->n_h);
  memcpy(hits.data(), buf.data() + sizeof(head), sizeof(long long) * c->n_h);
  const int reps = c->n_runs / c->n_h;
  double pmax = 0.0, psum = 0.0;
  int nz = 0;
  for (int i = 0; i < c->n_h; ++i) {
    const double P = (double)hits[i] / reps;
    pmax = std::max(pmax, P);
    psum += P;
    if (hits[i] > 0) ++nz;
    if (hits_per_h) hits_per_h[i] = hits[i];
  }
  if (hist)
    memcpy(hist, buf.data() + sizeof(head) + sizeof(long long) * c->n_h, sizeof(long long) * n_bins);
  out->P_max = pmax;
  out->W_range = nz ? psum / nz : 0.0;
  out->W_scan = psum / c->n_h;
  out->dE_mean = head.n_finite ? head.sum_dE / (double)head.n_finite : NAN;
  out->best_E = head.best_E;
  out->best_run = head.best_run;
  out->n_finite = head.n_finite;
  out->n_hits = head.n_hits;
  return CHYM_OK;
}

chym_status chym_get_state(chym_ctx* c, double* X_out, int64_t* k_out, void* stream) {
  chym::TraceRange trace_("chym_get_state");
  if (!c || !X_out) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)c->n_runs * c->N * c->D;
  if (c->prec == CHYM_PREC_FP64) {
    CHYM_CUDA_TRY(cudaMemcpyAsync(X_out, c->d_X, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    std::vector<float> tmp(n);
    CHYM_CUDA_TRY(cudaMemcpyAsync(tmp.data(), c->d_X, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    CHYM_CUDA_TRY(cudaStreamSynchronize(st));
    for (size_t i = 0; i < n; ++i) X_out[i] = tmp[i];
  }
  if (k_out) *k_out = c->k;
  return check_device_status(c);
}

chym_status chym_set_state(chym_ctx* c, const double* X, int n_runs, const double* h, int n_h,
                           const uint64_t* seeds, int64_t k, int32_t prec, void* stream) {
  chym::TraceRange trace_("chym_set_state");
  if (!c || !X || !h || !seeds) return fail(CHYM_EINVAL, "NULL argument");
  if (n_h < 1 || n_runs < 1 || n_runs % n_h) return fail(CHYM_EINVAL, "bad n_runs / n_h");
  if (k < 0) return fail(CHYM_EINVAL, "k must be >= 0");
  if (prec < CHYM_PREC_FP64 || prec > CHYM_PREC_FP8) return fail(CHYM_EINVAL, "bad prec");
  chym_status s = ensure_batch(c, n_runs, n_h);
  if (s != CHYM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  c->n_runs = n_runs;
  c->n_h = n_h;
  const size_t n = (size_t)n_runs * c->N * c->D;
  if (prec == CHYM_PREC_FP64) {
    CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_X, X, n * sizeof(double), cudaMemcpyHostToDevice, st));
  } else {
    std::vector<float> tmp(n);
    for (size_t i = 0; i < n; ++i) tmp[i] = (float)X[i];
    CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_X, tmp.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_h, h, sizeof(double) * n_h, cudaMemcpyHostToDevice, st));
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_seeds, seeds, sizeof(uint64_t) * n_runs,
                                cudaMemcpyHostToDevice, st));
  CHYM_CUDA_TRY(cudaMemsetAsync(c->d_koff, 0, sizeof(int64_t) * n_runs, st));
  CHYM_CUDA_TRY(launch_fill_hidx(c->d_hidx, n_runs, n_runs / n_h, st));
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  c->prec = prec;
  c->k = k;
  c->have_energy = false;
  return CHYM_OK;
}

// ---- checkpoint / restore: the complete run state in one host buffer ----
namespace {
struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t N, D, n_runs, n_h, prec;
  int64_t k;
  uint64_t x_bytes;
};
constexpr char kCkptMagic[8] = {'C', 'H', 'Y', 'M', 'C', 'K', 'P', 'T'};
size_t ckpt_bytes(int n_runs, int n_h, size_t x_bytes) {
  return sizeof(CkptHeader) + x_bytes + sizeof(double) * n_h +
         (sizeof(uint64_t) + sizeof(int64_t) + sizeof(int32_t)) * (size_t)n_runs;
}
}  // namespace

chym_status chym_checkpoint(chym_ctx* c, void* buf, size_t* len, void* stream) {
  chym::TraceRange trace_("chym_checkpoint");
  if (!c || !len) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state");
  const size_t xb = (size_t)c->n_runs * c->N * c->D * (c->prec == CHYM_PREC_FP64 ? 8 : 4);
  const size_t need = ckpt_bytes(c->n_runs, c->n_h, xb);
  if (!buf) {
    *len = need;
    return CHYM_OK;
  }
  if (*len < need) return fail(CHYM_EINVAL, "checkpoint buffer too small");
  cudaStream_t st = (cudaStream_t)stream;
  CkptHeader hd;
  memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.N = c->N;
  hd.D = c->D;
  hd.n_runs = c->n_runs;
  hd.n_h = c->n_h;
  hd.prec = c->prec;
  hd.k = c->k;
  hd.x_bytes = xb;
  unsigned char* b = (unsigned char*)buf;
  memcpy(b, &hd, sizeof(hd));
  unsigned char* o = b + sizeof(hd);
  CHYM_CUDA_TRY(cudaMemcpyAsync(o, c->d_X, xb, cudaMemcpyDeviceToHost, st));
  o += xb;
  CHYM_CUDA_TRY(cudaMemcpyAsync(o, c->d_h, sizeof(double) * c->n_h, cudaMemcpyDeviceToHost, st));
  o += sizeof(double) * c->n_h;
  CHYM_CUDA_TRY(cudaMemcpyAsync(o, c->d_seeds, sizeof(uint64_t) * c->n_runs, cudaMemcpyDeviceToHost, st));
  o += sizeof(uint64_t) * c->n_runs;
  CHYM_CUDA_TRY(cudaMemcpyAsync(o, c->d_koff, sizeof(int64_t) * c->n_runs, cudaMemcpyDeviceToHost, st));
  o += sizeof(int64_t) * c->n_runs;
  CHYM_CUDA_TRY(cudaMemcpyAsync(o, c->d_hidx, sizeof(int32_t) * c->n_runs, cudaMemcpyDeviceToHost, st));
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  *len = need;
  return check_device_status(c);
}

chym_status chym_restore(chym_ctx* c, const void* buf, size_t len, void* stream) {
  chym::TraceRange trace_("chym_restore");
  if (!c || !buf) return fail(CHYM_EINVAL, "NULL argument");
  CkptHeader hd;
  if (len < sizeof(hd)) return fail(CHYM_EINVAL, "checkpoint too short");
  memcpy(&hd, buf, sizeof(hd));
  if (memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1)
    return fail(CHYM_EINVAL, "not a checkpoint of this library");
  if (hd.N != c->N || hd.D != c->D) return fail(CHYM_EINVAL, "checkpoint of another N or D");
  if (hd.n_h < 1 || hd.n_runs < 1 || hd.n_runs % hd.n_h || hd.k < 0 || hd.prec < CHYM_PREC_FP64 ||
      hd.prec > CHYM_PREC_FP8)
    return fail(CHYM_EINVAL, "corrupt checkpoint header");
  const size_t xb = (size_t)hd.n_runs * c->N * c->D * (hd.prec == CHYM_PREC_FP64 ? 8 : 4);
  if (hd.x_bytes != xb || len < ckpt_bytes(hd.n_runs, hd.n_h, xb))
    return fail(CHYM_EINVAL, "checkpoint size does not match its header");
  chym_status s = ensure_batch(c, hd.n_runs, hd.n_h);
  if (s != CHYM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned char* o = (const unsigned char*)buf + sizeof(hd);
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_X, o, xb, cudaMemcpyHostToDevice, st));
  o += xb;
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_h, o, sizeof(double) * hd.n_h, cudaMemcpyHostToDevice, st));
  o += sizeof(double) * hd.n_h;
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_seeds, o, sizeof(uint64_t) * hd.n_runs, cudaMemcpyHostToDevice, st));
  o += sizeof(uint64_t) * hd.n_runs;
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_koff, o, sizeof(int64_t) * hd.n_runs, cudaMemcpyHostToDevice, st));
  o += sizeof(int64_t) * hd.n_runs;
  CHYM_CUDA_TRY(cudaMemcpyAsync(c->d_hidx, o, sizeof(int32_t) * hd.n_runs, cudaMemcpyHostToDevice, st));
  CHYM_CUDA_TRY(cudaStreamSynchronize(st));
  c->n_runs = hd.n_runs;
  c->n_h = hd.n_h;
  c->prec = hd.prec;
  c->k = hd.k;
  c->have_energy = false;
  return CHYM_OK;
}

}  // extern "C"
