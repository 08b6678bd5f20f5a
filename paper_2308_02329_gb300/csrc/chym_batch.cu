// chym_batch.cu -- batched integration of many contexts (instances x D) at once.
//
// Contexts on the small-N tensor-core path (N <= 128) are integrated by one
// persistent launch per hyperspin dimension D.  Every CTA of such a launch walks a
// host-built list of items (a run range of one context).  The planner spreads each
// dimension's runs over its CTAs in near-equal numbers of 8-run chunks, so no SM
// idles while another finishes a whole extra item.  The SMs are shared between the
// dimensions in proportion to their estimated cost.  Contexts on the large-N path
// run their per-step GEMM launches on forked streams, captured once into a CUDA graph
// per chunk of steps and replayed.  Contexts in FP32/FP64 run the SIMT kernels on
// forked streams.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "chym_internal.cuh"

namespace chym {
StepConsts make_step_consts(const chym_ctx* c, const chym_params* prm, const chym_schedule* s,
                            int64_t k0, int64_t steps);
cudaError_t launch_step(chym_ctx* c, const StepConsts& sc, int32_t prec, cudaStream_t st);
}  // namespace chym

struct chym_batch {
  std::vector<chym_ctx*> ctxs;
  std::vector<cudaStream_t> streams;  // one per context (forked work)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  void* d_plan = nullptr;
  size_t plan_bytes = 0;
  unsigned* d_status = nullptr;
  int sms = 0;
  chym::K2Runner k2;
  // Cost model of the planner, in SM-microseconds: one 8- or 4-run chunk advanced
  // one step on the small-N path, per dimension D; and one (128-row tile x K chunk
  // of 64) advanced one step on the large-N path.  The defaults were measured on a
  // GB300; chym_batch_tune re-measures them for the batch's own contexts.
  double chunk_cost[9] = {0, 1.10, 0.555, 0.89, 1.07, 1.27, 1.43, 1.60, 1.76};
  double k2_cost = 1.05;
  bool tuned = false;
  // Tile shapes (0: the kernels' defaults), chosen by chym_batch_tune's search or set by
  // the caller: large-N runs per column tile and ring depth, small-N epilogue chunk.
  chym::TileShapes shapes;
  // Timing of the parts of a run (used by the tuner): index D = 1..8 for the small-N
  // launch of dimension D, 0 for the large-N launches; their CTAs and work units.
  bool timing = false;
  cudaEvent_t t_begin[9] = {}, t_end[9] = {};
  bool timed[9] = {};
  int part_ctas[9] = {};
  double part_units[9] = {};
};

namespace chym {
namespace {

struct PlanJob {
  int desc, n_runs;
};

// Split the runs of `jobs` (all of one dimension) over P CTAs in near-equal chunk
// counts; items never cross a context and hold at most `per_item` runs.
void plan_dimension(const std::vector<PlanJob>& jobs, int CH, int per_item, int P,
                    std::vector<unsigned char>& items, std::vector<int>& cta_begin) {
  long long C = 0;
  for (const auto& j : jobs) C += (j.n_runs + CH - 1) / CH;
  if (P > C) P = (int)std::max(1LL, C);
  const size_t ib = tc_item_bytes();
  cta_begin.assign(1, 0);
  int cta = 0;
  long long acc = 0;
  auto bound = [&](int b) { return (long long)llround((double)(b + 1) * (double)C / P); };
  int n_items = 0;
  for (const auto& j : jobs) {
    int run = 0;
    while (run < j.n_runs) {
      long long cap = bound(cta) - acc;
      if (cap <= 0 && cta + 1 < P) {
        cta_begin.push_back(n_items);
        ++cta;
        continue;
      }
      if (cap <= 0) cap = (j.n_runs - run + CH - 1) / CH;  // last CTA takes the rest
      const int left_chunks = (j.n_runs - run + CH - 1) / CH;
      const int take = (int)std::min<long long>({cap, (long long)(per_item / CH), (long long)left_chunks});
      const int runs = std::min(take * CH, j.n_runs - run);
      items.resize(items.size() + ib);
      tc_fill_item(items.data() + items.size() - ib, j.desc, run, runs);
      ++n_items;
      run += runs;
      acc += take;
    }
  }
  while ((int)cta_begin.size() < P + 1) cta_begin.push_back(n_items);
}

}  // namespace
}  // namespace chym

using namespace chym;

extern "C" {

CHYM_API chym_status chym_batch_create(chym_ctx* const* ctxs, int n_ctx, chym_batch** out) {
  if (!ctxs || !out || n_ctx < 1) return fail(CHYM_EINVAL, "need at least one context");
  for (int i = 0; i < n_ctx; ++i)
    if (!ctxs[i]) return fail(CHYM_EINVAL, "NULL context in the batch");
  chym_batch* b = new (std::nothrow) chym_batch();
  if (!b) return fail(CHYM_ENOMEM, "host allocation failed");
  b->ctxs.assign(ctxs, ctxs + n_ctx);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n_ctx && e == cudaSuccess; ++i) {
    cudaStream_t s;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->streams.push_back(s);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->joins.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    chym_status st = cuda_fail(e, "chym_batch_create");
    chym_batch_destroy(b);
    return st;
  }
  *out = b;
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_destroy(chym_batch* b) {
  if (!b) return CHYM_OK;
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_plan) cudaFree(b->d_plan);
  if (b->d_status) cudaFree(b->d_status);
  for (int p = 0; p <= 8; ++p) {
    if (b->t_begin[p]) cudaEventDestroy(b->t_begin[p]);
    if (b->t_end[p]) cudaEventDestroy(b->t_end[p]);
  }
  k2_runner_release(b->k2);
  delete b;
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_run(chym_batch* b, const chym_params* params,
                                    const chym_schedule* schedules, int64_t steps,
                                    void* cuda_stream) {
  chym::TraceRange trace_("chym_batch_run");
  if (!b || !params || !schedules) return fail(CHYM_EINVAL, "NULL argument");
  if (steps < 0) return fail(CHYM_EINVAL, "steps must be >= 0");
  const int n = (int)b->ctxs.size();
  for (int i = 0; i < n; ++i) {
    const chym_ctx* c = b->ctxs[i];
    const chym_params& p = params[i];
    const chym_schedule& s = schedules[i];
    if (c->prec < 0) return fail(CHYM_ESTATE, "every context needs a state (chym_run with seeds first)");
    if (!(p.dt > 0.0) || !(p.sigma >= 0.0) || (p.flags != 0 && p.flags != CHYM_FLAG_TEST_STALL) ||
        p.prec < CHYM_PREC_FP64 ||
        p.prec > CHYM_PREC_FP8 || !isfinite(p.gamma) || !isfinite(p.kappa) || !isfinite(p.eps))
      return fail(CHYM_EINVAL, "bad params in the batch");
    if ((c->prec == CHYM_PREC_FP64) != (p.prec == CHYM_PREC_FP64))
      return fail(CHYM_EINVAL, "a context cannot change between FP64 and FP32 storage");
    if (c->d_w && c->N > 128 && is_tc_prec(p.prec) && !uses_csr(c, p.prec))
      return fail(CHYM_ENOTSUP, "coupling weights need N <= 128 on the tensor-core path");
    if ((s.kind != 0 && s.kind != 1) || s.reserved != 0 ||
        (s.kind == 1 && (s.k_anneal < 0 || s.k_total <= s.k_anneal)))
      return fail(CHYM_EINVAL, "bad schedule in the batch");
  }
  if (steps == 0) return CHYM_OK;
  cudaStream_t main = (cudaStream_t)cuda_stream;
  CHYM_CUDA_TRY(cudaEventRecord(b->fork, main));

  // ---- small-N tensor-core contexts: one persistent launch per dimension ----
  std::vector<int> by_dim[9];
  for (int i = 0; i < n; ++i) {
    chym_ctx* c = b->ctxs[i];
    if (is_tc_prec(params[i].prec) && c->N <= 128) {
      c->prec = params[i].prec;
      by_dim[c->D].push_back(i);
      cudaError_t e = prepare_tc_operand(c);
      if (e != cudaSuccess) return cuda_fail(e, "J operand image");
    }
  }
  // work in SM-microseconds per step: each small-N dimension and the large-N group.
  // The SMs are split in proportion, so that all parts finish together; the
  // large-N launches take the SMs that the persistent small-N CTAs leave free.
  double cost[9] = {0};
  double total = 0.0;
  for (int D = 1; D <= 8; ++D) {
    for (int i : by_dim[D]) {
      const int CH = tc_chunk_runs(D);
      cost[D] += b->chunk_cost[D] * ((b->ctxs[i]->n_runs + CH - 1) / CH);
    }
    total += cost[D];
  }
  double small_total = total;
  for (int i = 0; i < n; ++i) {
    const chym_ctx* c = b->ctxs[i];
    if (is_tc_prec(params[i].prec) && c->N > 128 && !uses_csr(c, params[i].prec))
      total += b->k2_cost * (double)k2_work_units(c->N, c->D, c->n_runs, b->shapes.rt[c->D]);
  }
  // SMs for the small-N dimensions (all of them when there is no large-N work)
  const int sms_small = small_total > 0.0
                            ? std::min(b->sms, std::max(1, (int)llround(b->sms * small_total / total)))
                            : 0;
  // plan: descriptors of all small-N contexts, then per dimension its items and CTA ranges
  std::vector<unsigned char> blob;
  const size_t db = tc_desc_bytes();
  std::vector<int> desc_of(n, -1);
  int n_desc = 0;
  for (int D = 1; D <= 8; ++D)
    for (int i : by_dim[D]) {
      blob.resize(blob.size() + db);
      const StepConsts sc = make_step_consts(b->ctxs[i], &params[i], &schedules[i], b->ctxs[i]->k, steps);
      tc_fill_desc(b->ctxs[i], sc, blob.data() + blob.size() - db);
      desc_of[i] = n_desc++;
    }
  struct DimLaunch {
    int D, P, kp_max, terms_max;
    size_t items_off, cta_off;
    bool stall;
  };
  std::vector<DimLaunch> dl;
  int dims_left = 0;
  for (int D = 1; D <= 8; ++D) dims_left += by_dim[D].empty() ? 0 : 1;
  int sms_left = std::max(sms_small, dims_left);
  for (int D = 1; D <= 8; ++D) {
    if (by_dim[D].empty()) continue;
    int P = std::max(1, (int)llround(sms_left * cost[D] / small_total));
    small_total -= cost[D];
    P = std::min(P, sms_left - (dims_left - 1));
    P = std::max(P, 1);
    sms_left -= P;
    --dims_left;
    std::vector<PlanJob> jobs;
    int kp_max = 16, terms_max = 1;
    bool stall = false;
    for (int i : by_dim[D]) {
      jobs.push_back({desc_of[i], b->ctxs[i]->n_runs});
      stall = stall || (params[i].flags & CHYM_FLAG_TEST_STALL);
      kp_max = std::max(kp_max, (b->ctxs[i]->N + 15) / 16 * 16);
      terms_max = std::max(terms_max, b->ctxs[i]->kind == CHYM_J_PM1 ? 1 : 2);
    }
    std::vector<unsigned char> items;
    std::vector<int> cta;
    plan_dimension(jobs, tc_chunk_runs(D), tc_runs_per_item(D), P, items, cta);
    DimLaunch L{D, (int)cta.size() - 1, kp_max, terms_max, 0, 0, stall};
    b->part_ctas[D] = L.P;
    b->part_units[D] = 0.0;
    for (const auto& jj : jobs) b->part_units[D] += (double)((jj.n_runs + tc_chunk_runs(D) - 1) / tc_chunk_runs(D));
    blob.resize((blob.size() + 15) / 16 * 16);
    L.items_off = blob.size();
    blob.insert(blob.end(), items.begin(), items.end());
    blob.resize((blob.size() + 15) / 16 * 16);
    L.cta_off = blob.size();
    const unsigned char* cp = reinterpret_cast<const unsigned char*>(cta.data());
    blob.insert(blob.end(), cp, cp + cta.size() * sizeof(int));
    dl.push_back(L);
  }
  if (!blob.empty()) {
    if (blob.size() > b->plan_bytes) {
      if (b->d_plan) cudaFree(b->d_plan);
      b->d_plan = nullptr;
      b->plan_bytes = 0;
      CHYM_CUDA_TRY(cudaMalloc(&b->d_plan, blob.size()));
      b->plan_bytes = blob.size();
    }
    CHYM_CUDA_TRY(cudaMemcpyAsync(b->d_plan, blob.data(), blob.size(), cudaMemcpyHostToDevice, main));
    CHYM_CUDA_TRY(cudaEventRecord(b->fork, main));
  }
  std::vector<bool> used(n, false);
  int si = 0;
  const unsigned char* base = (const unsigned char*)b->d_plan;
  for (int D = 0; D <= 8; ++D) b->timed[D] = false;
  for (const auto& L : dl) {
    cudaStream_t s = b->streams[si];
    CHYM_CUDA_TRY(cudaStreamWaitEvent(s, b->fork, 0));
    if (b->timing) CHYM_CUDA_TRY(cudaEventRecord(b->t_begin[L.D], s));
    CHYM_CUDA_TRY(launch_tc_items(L.D, base, base + L.items_off, (const int*)(base + L.cta_off), L.P,
                                  steps, L.kp_max, L.terms_max, b->d_status, s, L.stall,
                                  b->shapes.ch[L.D]));
    if (b->timing) {
      CHYM_CUDA_TRY(cudaEventRecord(b->t_end[L.D], s));
      b->timed[L.D] = true;
    }
    CHYM_CUDA_TRY(cudaEventRecord(b->joins[si], s));
    used[si++] = true;
  }
  // ---- large-N tensor-core contexts: grouped per-step launches, graph replay ----
  {
    std::vector<unsigned char> descs;
    std::vector<int> dims, idx;
    const size_t kb = k2_desc_bytes();
    const int sidx = si < n ? si++ : 0;
    cudaStream_t s = b->streams[sidx];
    for (int i = 0; i < n; ++i) {
      chym_ctx* c = b->ctxs[i];
      if (desc_of[i] >= 0 || !is_tc_prec(params[i].prec) || uses_csr(c, params[i].prec)) continue;
      if (idx.empty()) CHYM_CUDA_TRY(cudaStreamWaitEvent(s, b->fork, 0));
      c->prec = params[i].prec;
      descs.resize(descs.size() + kb);
      const StepConsts sc = make_step_consts(c, &params[i], &schedules[i], c->k, steps);
      cudaError_t e = k2_prepare(c, sc, s, descs.data() + descs.size() - kb, b->shapes.rt[c->D]);
      if (e != cudaSuccess) return cuda_fail(e, "large-N preparation");
      dims.push_back(c->D);
      idx.push_back(i);
    }
    if (!idx.empty()) {
      // the persistent large-N grid takes the SMs the small-N CTAs leave free
      int small_ctas = 0;
      for (const auto& L : dl) small_ctas += L.P;
      const int cap = small_ctas > 0 ? std::max(1, b->sms - small_ctas) : 0;
      b->part_ctas[0] = cap > 0 ? cap : b->sms;
      b->part_units[0] = 0.0;
      for (int i : idx)
        b->part_units[0] += (double)k2_work_units(b->ctxs[i]->N, b->ctxs[i]->D, b->ctxs[i]->n_runs,
                                                  b->shapes.rt[b->ctxs[i]->D]);
      if (b->timing) CHYM_CUDA_TRY(cudaEventRecord(b->t_begin[0], s));
      cudaError_t e = k2_integrate(b->k2, descs, dims, steps, b->d_status, s, cap, b->shapes.stages);
      if (b->timing && e == cudaSuccess) {
        CHYM_CUDA_TRY(cudaEventRecord(b->t_end[0], s));
        b->timed[0] = true;
      }
      if (e != cudaSuccess) return cuda_fail(e, "large-N batched integration");
      for (size_t t = 0; t < idx.size(); ++t) {
        chym_ctx* c = b->ctxs[idx[t]];
        e = k2_finish(c, descs.data() + t * kb, s);
        if (e != cudaSuccess) return cuda_fail(e, "large-N state unpack");
        c->k += steps;
        c->have_energy = false;
        desc_of[idx[t]] = -2;  // handled
      }
      CHYM_CUDA_TRY(cudaEventRecord(b->joins[sidx], s));
      used[sidx] = true;
    }
  }
  // ---- every other context (FP32/FP64): its own launches on its own stream ----
  for (int i = 0; i < n; ++i) {
    chym_ctx* c = b->ctxs[i];
    if (desc_of[i] >= 0) {
      c->k += steps;
      c->have_energy = false;
      continue;
    }
    if (desc_of[i] == -2) continue;
    const int sidx = si < n ? si++ : (i % n);
    cudaStream_t s = b->streams[sidx];
    CHYM_CUDA_TRY(cudaStreamWaitEvent(s, b->fork, 0));
    c->prec = params[i].prec;
    const StepConsts sc = make_step_consts(c, &params[i], &schedules[i], c->k, steps);
    cudaError_t e = launch_step(c, sc, c->prec, s);
    if (e == cudaErrorInvalidConfiguration || e == cudaErrorNotSupported)
      return fail(CHYM_ENOTSUP, "no kernel for a context of this batch (size or precision)");
    if (e != cudaSuccess) return cuda_fail(e, "batched step launch");
    CHYM_CUDA_TRY(cudaEventRecord(b->joins[sidx], s));
    used[sidx] = true;
    c->k += steps;
    c->have_energy = false;
  }
  for (int i = 0; i < n; ++i)
    if (used[i]) CHYM_CUDA_TRY(cudaStreamWaitEvent(main, b->joins[i], 0));
  return CHYM_OK;
}

// Autotuner: measure the planner's cost model on this device, for the batch's own
// contexts and at the split it will run with.  The whole batch runs for probe_steps
// steps (once untimed to warm up, then a few rounds timed per part with CUDA events,
// each part's time the shorter of two runs, so that one slow run does not decide);
// after each round every part's cost is re-estimated from its measured time at
// its CTA count (SM-microseconds per unit of work), which moves the next split
// towards equal finish times.  The split with the shortest slowest part is kept.
// The states, steps and energies of the contexts are saved before and restored after.
CHYM_API chym_status chym_batch_tune(chym_batch* b, const chym_params* params,
                                     const chym_schedule* schedules, int64_t probe_steps,
                                     void* cuda_stream) {
  chym::TraceRange trace_("chym_batch_tune");
  if (!b || !params || !schedules) return fail(CHYM_EINVAL, "NULL argument");
  if (probe_steps < 1) return fail(CHYM_EINVAL, "probe_steps must be >= 1");
  const int n = (int)b->ctxs.size();
  for (int i = 0; i < n; ++i)
    if (b->ctxs[i]->prec < 0) return fail(CHYM_ESTATE, "every context needs a state (chym_run with seeds first)");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  struct Saved {
    void* d = nullptr;
    size_t bytes = 0;
    int64_t k = 0;
    bool have_energy = false;
  };
  std::vector<Saved> saved(n);
  auto release = [&]() {
    for (auto& sv : saved)
      if (sv.d) cudaFree(sv.d);
  };
  for (int i = 0; i < n; ++i) {
    chym_ctx* c = b->ctxs[i];
    Saved& sv = saved[i];
    sv.bytes = (size_t)c->n_runs * c->N * c->D * (c->prec == CHYM_PREC_FP64 ? 8 : 4);
    sv.k = c->k;
    sv.have_energy = c->have_energy;
    cudaError_t e = cudaMalloc(&sv.d, sv.bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv.d, c->d_X, sv.bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(e, "chym_batch_tune: state snapshot");
    }
  }
  chym_status status = CHYM_OK;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p <= 8 && e == cudaSuccess; ++p) {
    if (!b->t_begin[p]) e = cudaEventCreate(&b->t_begin[p]);
    if (e == cudaSuccess && !b->t_end[p]) e = cudaEventCreate(&b->t_end[p]);
  }
  if (e != cudaSuccess) status = cuda_fail(e, "chym_batch_tune: events");
  double best_chunk[9], best_k2 = b->k2_cost, best_T = INFINITY;
  for (int D = 0; D <= 8; ++D) best_chunk[D] = b->chunk_cost[D];
  constexpr int kRounds = 4, kReps = 2;
  for (int round = -1; round < kRounds && status == CHYM_OK; ++round) {
    double T[9];
    bool seen[9] = {};
    for (int p = 0; p <= 8; ++p) T[p] = INFINITY;
    for (int rep = 0; rep < (round < 0 ? 1 : kReps) && status == CHYM_OK; ++rep) {
      b->timing = round >= 0;
      status = chym_batch_run(b, params, schedules, probe_steps, st);
      if (status != CHYM_OK) break;
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        status = cuda_fail(e, "chym_batch_tune: probe");
        break;
      }
      status = chym_batch_status(b);
      if (status != CHYM_OK || round < 0) break;
      for (int p = 0; p <= 8; ++p) {
        if (!b->timed[p]) continue;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, b->t_begin[p], b->t_end[p]);
        if (e != cudaSuccess) break;
        T[p] = std::min(T[p], 1e3 * (double)ms);
        seen[p] = true;
      }
      if (e != cudaSuccess) status = cuda_fail(e, "chym_batch_tune: timing");
    }
    if (status != CHYM_OK || round < 0) continue;
    double T_max = 0.0;
    for (int p = 0; p <= 8; ++p)
      if (seen[p]) T_max = std::max(T_max, T[p]);
    if (T_max < best_T) {  // the split of this round is the best so far
      best_T = T_max;
      for (int D = 0; D <= 8; ++D) best_chunk[D] = b->chunk_cost[D];
      best_k2 = b->k2_cost;
    }
    // re-estimate each part's cost at its operating point
    for (int p = 0; p <= 8; ++p) {
      if (!seen[p] || b->part_units[p] <= 0.0) continue;
      const double c = T[p] * (double)b->part_ctas[p] / (b->part_units[p] * (double)probe_steps);
      if (p == 0) b->k2_cost = c;
      else b->chunk_cost[p] = c;
    }
  }
  // ---- tile shapes: coordinate search, one part at a time, at the tuned split ----
  // Each candidate runs the whole batch for probe_steps steps (timed per part); a part
  // keeps the candidate under which its own time was shortest.  Large-N parts (one per
  // dimension, timed together): runs per column tile, then ring depth; small-N parts:
  // the epilogue chunk.  Changing one part's shape leaves the others' work unchanged.
  if (status == CHYM_OK) {
    for (int D = 0; D <= 8; ++D) b->chunk_cost[D] = best_chunk[D];
    b->k2_cost = best_k2;
    auto probe = [&](int part, double* t_out) -> chym_status {
      *t_out = INFINITY;
      for (int rep = 0; rep < kReps; ++rep) {  // the shorter of two runs
        chym_status r = chym_batch_run(b, params, schedules, probe_steps, st);
        if (r != CHYM_OK) return r;
        cudaError_t ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_fail(ce, "chym_batch_tune: shape probe");
        r = chym_batch_status(b);
        if (r != CHYM_OK) return r;
        float ms = 0.f;
        if (!b->timed[part]) return fail(CHYM_ESTATE, "chym_batch_tune: part not timed");
        ce = cudaEventElapsedTime(&ms, b->t_begin[part], b->t_end[part]);
        if (ce != cudaSuccess) return cuda_fail(ce, "chym_batch_tune: timing");
        *t_out = std::min(*t_out, (double)ms);
      }
      return CHYM_OK;
    };
    bool large[9] = {}, small[9] = {};
    int terms[9] = {}, lo8[9] = {}, runs[9] = {};
    for (int i = 0; i < n; ++i) {
      const chym_ctx* c = b->ctxs[i];
      if (!is_tc_prec(params[i].prec) || uses_csr(c, params[i].prec)) continue;
      if (c->N <= 128) {
        small[c->D] = true;
      } else {
        large[c->D] = true;
        terms[c->D] = std::max(terms[c->D], c->kind == CHYM_J_PM1 ? 1 : 2);
        lo8[c->D] = lo8[c->D] || (params[i].prec == CHYM_PREC_FP8 && c->kind == CHYM_J_PM1);
        runs[c->D] = std::max(runs[c->D], c->n_runs);
      }
    }
    b->timing = true;
    for (int D = 1; D <= 8 && status == CHYM_OK; ++D) {
      if (!large[D]) continue;
      double best = INFINITY;
      int best_rt = b->shapes.rt[D];
      for (int rt = 32; rt <= 256 && status == CHYM_OK; rt *= 2) {
        if (!k2_rt_valid(D, rt) || (rt > 32 && rt / 2 >= runs[D])) continue;
        b->shapes.rt[D] = rt;
        double t = 0.0;
        status = probe(0, &t);
        if (status == CHYM_OK && t < best) {
          best = t;
          best_rt = rt;
        }
      }
      b->shapes.rt[D] = best_rt;
      const int smax = k2_max_stages(D, best_rt, runs[D], terms[D], lo8[D]);
      int best_s = 0;  // the most that fit
      for (int sg = smax - 1; sg >= std::max(2, smax - 3) && status == CHYM_OK; --sg) {
        b->shapes.stages[D] = sg;
        double t = 0.0;
        status = probe(0, &t);
        if (status == CHYM_OK && t < best) {
          best = t;
          best_s = sg;
        }
      }
      b->shapes.stages[D] = best_s;
    }
    for (int D = 1; D <= 4 && status == CHYM_OK; ++D) {
      if (!small[D]) continue;
      double t8 = 0.0, t4 = 0.0;
      b->shapes.ch[D] = 8;
      status = probe(D, &t8);
      if (status != CHYM_OK) break;
      b->shapes.ch[D] = 4;
      status = probe(D, &t4);
      b->shapes.ch[D] = t4 < t8 ? 4 : 8;
    }
  }
  b->timing = false;
  // restore the states
  for (int i = 0; i < n; ++i) {
    chym_ctx* c = b->ctxs[i];
    const Saved& sv = saved[i];
    if (!sv.d) continue;
    e = cudaMemcpyAsync(c->d_X, sv.d, sv.bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess && status == CHYM_OK) status = cuda_fail(e, "chym_batch_tune: state restore");
    c->k = sv.k;
    c->have_energy = sv.have_energy;
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && status == CHYM_OK) status = cuda_fail(e, "chym_batch_tune");
  release();
  for (int D = 0; D <= 8; ++D) b->chunk_cost[D] = best_chunk[D];
  b->k2_cost = best_k2;
  if (status != CHYM_OK) b->shapes = TileShapes();
  if (status != CHYM_OK) return status;
  b->tuned = true;
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_get_tuning(chym_batch* b, double* chunk_costs, double* k2_cost,
                                           int* tuned) {
  if (!b) return fail(CHYM_EINVAL, "NULL batch");
  if (chunk_costs)
    for (int D = 0; D < 8; ++D) chunk_costs[D] = b->chunk_cost[D + 1];
  if (k2_cost) *k2_cost = b->k2_cost;
  if (tuned) *tuned = b->tuned ? 1 : 0;
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_set_tuning(chym_batch* b, const double* chunk_costs, const double* k2_cost) {
  if (!b) return fail(CHYM_EINVAL, "NULL batch");
  if (chunk_costs)
    for (int D = 0; D < 8; ++D)
      if (!(chunk_costs[D] > 0.0) || !isfinite(chunk_costs[D]))
        return fail(CHYM_EINVAL, "costs must be positive and finite");
  if (k2_cost && (!(*k2_cost > 0.0) || !isfinite(*k2_cost)))
    return fail(CHYM_EINVAL, "costs must be positive and finite");
  if (chunk_costs)
    for (int D = 0; D < 8; ++D) b->chunk_cost[D + 1] = chunk_costs[D];
  if (k2_cost) b->k2_cost = *k2_cost;
  if (chunk_costs || k2_cost) b->tuned = true;
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_get_shapes(chym_batch* b, int* rt, int* stages, int* chunk) {
  if (!b) return fail(CHYM_EINVAL, "NULL batch");
  for (int D = 0; D < 8; ++D) {
    if (rt) rt[D] = b->shapes.rt[D + 1];
    if (stages) stages[D] = b->shapes.stages[D + 1];
    if (chunk) chunk[D] = b->shapes.ch[D + 1];
  }
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_set_shapes(chym_batch* b, const int* rt, const int* stages, const int* chunk) {
  if (!b) return fail(CHYM_EINVAL, "NULL batch");
  for (int D = 1; D <= 8; ++D) {
    if (rt && rt[D - 1] != 0 && !k2_rt_valid(D, rt[D - 1]))
      return fail(CHYM_EINVAL, "runs per column tile: 0, or a multiple of 32 with D rt <= 256");
    if (stages && stages[D - 1] != 0 && (stages[D - 1] < 2 || stages[D - 1] > 8))
      return fail(CHYM_EINVAL, "ring stages: 0, or 2..8");
    if (chunk && chunk[D - 1] != 0 && !(D <= 4 && (chunk[D - 1] == 4 || chunk[D - 1] == 8)))
      return fail(CHYM_EINVAL, "epilogue chunk: 0, or 4 or 8 for D <= 4");
  }
  for (int D = 1; D <= 8; ++D) {
    if (rt) b->shapes.rt[D] = rt[D - 1];
    if (stages) b->shapes.stages[D] = stages[D - 1];
    if (chunk) b->shapes.ch[D] = chunk[D - 1];
  }
  return CHYM_OK;
}

CHYM_API chym_status chym_batch_status(chym_batch* b) {
  if (!b) return fail(CHYM_EINVAL, "NULL batch");
  unsigned st = 0;
  CHYM_CUDA_TRY(cudaMemcpy(&st, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st) {
    CHYM_CUDA_TRY(cudaMemset(b->d_status, 0, sizeof(unsigned)));
    return fail(CHYM_ETIMEOUT, "a device-side wait of the batch timed out");
  }
  return CHYM_OK;
}

}  // extern "C"
