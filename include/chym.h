/*
 * chym.h -- C ABI of the GB300 simulator of the coherent hyperspin machine
 * (CHYM) of "Hyperscaling in the coherent hyperspin machine" (Calvanese
 * Strinati & Conti, arXiv 2308.02329).
 *
 * The library integrates many independent runs (replicas x pump values h) of
 * the CHYM equations for one coupling matrix J_N and one hyperspin dimension
 * D, then reads out the Ising spins, their Ising energy and the ground-state
 * hit statistics.  Plain C types only: pointers are host pointers unless the
 * name of the entry point ends in _device, sizes are element counts.
 *
 * Model (one run, hyperspin p = 0..N-1, component mu = 0..D-1, step k):
 *   y_{p,mu} = sum_q J_pq x_{q,mu}                      coupling C = J_N (x) 1_D (Eq. 1)
 *   n_p      = sum_nu x_{p,nu}^2                        non-local loss W = beta 1_N (x) I_D (Eq. 1)
 *   x_{p,mu} <- x_{p,mu} + dt [ (h-1) x_{p,mu} - kappa x_{p,mu}^3 - gamma x_{p,mu} n_p
 *                              + eps alpha_mu(k) y_{p,mu} ] + sigma sqrt(dt) xi
 * i.e. the round-trip map of Eq. 2 read as the Euler-Maruyama step of its
 * continuous-time limit (gamma stands for beta b^2, kappa for the local
 * kappa L), with dimensional annealing C -> alpha_mu C (text after Fig. 2)
 * and additive Gaussian noise xi drawn from Philox4x32-10 (key = run seed,
 * Box-Muller on the four words of a block; for D >= 3 component mu of spin p
 * takes normal mu mod 4 of the block with counter (p, tag << 8 | mu / 4, k lo,
 * k hi); for D <= 2 the 4/D spins with the same p / (4/D) share the block with
 * counter (p / (4/D), tag << 8, k lo, k hi) and spin p takes its normals
 * (p mod 4/D) D + mu; tag 0 for the step noise, 1 for the initial state; k is
 * the run's local step).  With per-spin coupling weights
 * (chym_set_coupling_weights) the coupling term of spin p is eps w_p alpha_mu y.
 * The Ising readout is s_p = sign(x_{p,0}) (ties to +1) and the energy is
 * E = -sum_{p,q} J_pq s_p s_q (Eq. 3 with Ising spins).
 *
 * Runs are h-major: run = ih * replicas + rep, replicas = n_runs / n_h.
 *
 * Errors: every entry point returns a chym_status and never aborts or throws;
 * on failure chym_last_error() returns a message (thread-local, valid until
 * the next call on the same thread).  Calls on one context are not
 * thread-safe; different contexts are independent.
 */
#ifndef CHYM_H
#define CHYM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CHYM_API __attribute__((visibility("default")))
#else
#define CHYM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chym_ctx chym_ctx; /* opaque; owns the device copies of J and the run state */

typedef enum {
  CHYM_OK = 0,
  CHYM_EINVAL = 1,   /* invalid argument; nothing was launched */
  CHYM_ENOMEM = 2,   /* host or device allocation failed */
  CHYM_ECUDA = 3,    /* a CUDA call failed; chym_last_error() has the CUDA message */
  CHYM_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  CHYM_ENOTSUP = 5,  /* valid request that the library does not implement */
  CHYM_ESTATE = 6    /* call out of order (e.g. energy before any run) */
} chym_status;

typedef enum {
  CHYM_J_PM1 = 0, /* entries in {-1, 0, +1}: energies are exact integers */
  CHYM_J_REAL = 1 /* arbitrary real couplings: energies accumulate in FP64 */
} chym_jkind;

typedef enum {
  CHYM_PREC_FP64 = 0,   /* FP64 state and arithmetic (oracle-comparison mode) */
  CHYM_PREC_FP32 = 1,   /* FP32 state, FP32 SIMT coupling product (plain form) */
  CHYM_PREC_BF16X2 = 2, /* FP32 state; J x on tcgen05 tensor cores with J in BF16 and
                           x split into BF16 hi + lo, FP32 accumulation (FP32 over
                           the nonzeros for very sparse large J, see chym_create) */
  CHYM_PREC_FP8 = 3     /* as BF16X2, except that on the large-N path (N > 128) with
                           +-1 couplings the lo half of x is held in FP8 e4m3 (both
                           halves scaled by 2^16) and multiplied by J in e4m3 (exact
                           for +-1) at twice the BF16 rate: x keeps about 13
                           significant bits in the product (|x - hi - lo| <= 2^-13 |x|)
                           instead of 17.  Elsewhere (N <= 128, real J) it runs as
                           BF16X2.  The FP8 e4m3 coupling image of the +-1 J of the
                           paper's SK instances is exact (text before Fig. 4). */
} chym_prec;

typedef struct {
  double dt;       /* Euler-Maruyama time step */
  double sigma;    /* diffusion coefficient; the per-step noise std is sigma*sqrt(dt) */
  double init_std; /* std of the initial amplitudes x(0) */
  double gamma;    /* non-local saturation (beta b^2) */
  double kappa;    /* local saturation (kappa L) */
  double eps;      /* feedback coupling strength */
  int32_t prec;    /* chym_prec */
  int32_t flags;   /* 0, or CHYM_FLAG_TEST_STALL (tests of the timeout path only) */
} chym_params;

/* Test of the failure path of the tensor-core kernels (BF16X2/FP8 steps), nothing
 * else: the thread that issues a step's tensor-core products withholds the signal
 * that they are complete, so the warps that wait for them give up after their
 * bounded wait (2 ms with this flag instead of the usual 2 s), raise the status
 * word, drain the products they issued and free their tensor memory.  The next
 * synchronising call (chym_energy, chym_get_state, chym_batch_status) returns
 * CHYM_ETIMEOUT and clears the word; the state of the affected runs is then
 * unspecified, and a following chym_run with seeds restarts them normally.  No
 * fault, trap or unbounded wait is involved.  Paths without tensor cores ignore it. */
#define CHYM_FLAG_TEST_STALL 1

typedef struct {
  int32_t kind;     /* 0: no annealing (alpha = 1); 1: linear */
  int32_t reserved; /* must be 0 */
  int64_t k_anneal; /* linear: alpha_mu = 1 for k < k_anneal (mu >= 1) ... */
  int64_t k_total;  /* ... then 1 - (k - k_anneal)/(k_total - k_anneal), 0 from k_total on */
} chym_schedule;

typedef struct {
  double P_max;     /* max over h of P_Ising(h) (figure of merit (i)) */
  double W_range;   /* figure of merit (ii) normalised by the number of h with P > 0 */
  double W_scan;    /* figure of merit (ii) normalised by the number of scanned h */
  double dE_mean;   /* figure of merit (iii): mean E - E_GS over finite runs */
  double best_E;    /* lowest final Ising energy over all runs */
  int64_t best_run; /* lowest run index reaching best_E */
  int64_t n_finite; /* runs whose state stayed finite */
  int64_t n_hits;   /* runs with E == E_GS */
} chym_stats_t;

/* Thread-local message describing the last failure on this thread. */
CHYM_API const char* chym_last_error(void);

/* Create a context for the N x N coupling matrix J (row-major FP64, copied)
 * and hyperspin dimension D.  J must be symmetric with a zero diagonal
 * (J_N is the symmetric adjacency matrix of the graph, text after Eq. 1);
 * kind CHYM_J_PM1 additionally requires entries in {-1,0,1}.
 * Limits: 1 <= N <= 4096, 1 <= D <= 8.  EINVAL otherwise; ECUDA/ENOMEM on
 * device failures.  *out is set only on success.  With at most N^2/16 nonzeros
 * the context also keeps J in compressed rows: steps in FP32/FP64 then sum the
 * coupling over the nonzeros on the CUDA cores, and so do steps in BF16X2 mode when
 * N >= 1024, D >= 3, J has on average at most N/256 nonzeros per row
 * (nnz <= N^2/256; where that was measured faster than the tensor-core product) and
 * 2 N D floats fit the SIMT kernel's 200 KiB of shared memory; the state stays FP32
 * there. */
CHYM_API chym_status chym_create(const double* J, int N, int D, chym_jkind kind, chym_ctx** out);

/* Release every device and host resource of ctx (NULL is accepted). */
CHYM_API chym_status chym_destroy(chym_ctx* ctx);

/* Largest eigenvalue of J (FP64 Lanczos on the host), used for the pump
 * threshold h_th = 1 - eps * lambda_max of the linearised equations. */
CHYM_API chym_status chym_lambda_max(chym_ctx* ctx, double* lambda_out);

/* Integrate n_runs runs for `steps` Euler-Maruyama steps on `cuda_stream`
 * (a cudaStream_t; NULL = default stream).  h: n_h pump values (host);
 * seeds: n_runs 64-bit noise keys (host).  With seeds != NULL every run is
 * (re)initialised from its seed at step 0 (x(0) = init_std * N(0,1), tag 1);
 * with seeds == NULL the existing runs continue from the context's current
 * step (checkpoint/resume: the noise is counter based, so two calls of K/2
 * steps equal one call of K) and n_runs must match.  The schedule refers to
 * absolute steps.  The call is asynchronous with respect to the host except
 * for the upload of h and seeds.
 * EINVAL: steps < 0, n_h < 1, n_runs not a multiple of n_h, bad params. */
CHYM_API chym_status chym_run(chym_ctx* ctx, const chym_params* params, const double* h, int n_h,
                     const uint64_t* seeds, int n_runs, int64_t steps,
                     const chym_schedule* schedule, void* cuda_stream);

/* Same as chym_run with h (n_h doubles) and seeds (n_runs uint64) already in
 * device memory; nothing is copied between host and device. */
CHYM_API chym_status chym_run_device(chym_ctx* ctx, const chym_params* params, const double* d_h,
                            int n_h, const uint64_t* d_seeds, int n_runs, int64_t steps,
                            const chym_schedule* schedule, void* cuda_stream);

/* Ising readout and energy of every run (Eq. 3 with s_p = sign x_{p,0}).
 * E_out: n_runs doubles (host), exact integers for CHYM_J_PM1, NaN for a run
 * whose state is not finite.  spins_out: nullable, n_runs * ceil(N/64) words,
 * bit p of word p/64 set when s_p = +1.  Synchronises the stream. */
CHYM_API chym_status chym_energy(chym_ctx* ctx, double* E_out, uint64_t* spins_out, void* cuda_stream);

/* Device-memory variant of chym_energy: d_E (n_runs doubles) and nullable
 * d_spins are device pointers; asynchronous. */
CHYM_API chym_status chym_energy_device(chym_ctx* ctx, double* d_E, uint64_t* d_spins, void* cuda_stream);

/* Readout of XY runs (D = 2, the XY machine of the text after Fig. 2) by
 * best-axis rounding: instead of the first component, the Ising pattern
 * s_p = sign(x_p . u) along the axis u = (cos phi, sin phi) whose pattern has the
 * lowest energy E = -sum_{p,q} J_pq s_p s_q, over all axes (the pattern changes
 * only where u is perpendicular to a spin; phi and phi + pi give opposite patterns
 * of equal energy).  A spin of zero length reads +1.  Same outputs and layouts as
 * chym_energy (E = NaN for a run whose state is not finite, its spins then
 * unspecified); the lowest energy is unique, its pattern is the first reached when
 * the axis turns from inside the interval that wraps through pi.  EINVAL unless
 * D = 2 and N <= 4096; ESTATE without a state.  chym_readout_xy writes into the
 * context's energy buffers (the cached Ising energies of chym_energy are dropped)
 * and synchronises the stream; the device variant writes d_E (n_runs doubles)
 * and nullable d_spins and is asynchronous. */
CHYM_API chym_status chym_readout_xy(chym_ctx* ctx, double* E_out, uint64_t* spins_out, void* cuda_stream);
CHYM_API chym_status chym_readout_xy_device(chym_ctx* ctx, double* d_E, uint64_t* d_spins,
                                            void* cuda_stream);

/* Ground-state statistics of the last energies (figures of merit (i)-(iii)
 * after Fig. 3): hits_per_h (nullable, n_h int64) counts replicas with
 * E == E_gs (|E - E_gs| <= 1e-9 |E_gs| for real J); hist (nullable, n_bins
 * int64) is H_E binned by (E - E_gs) / bin_width (4 for +-1 couplings, whose
 * energies move in steps of 4; 1e-3 |E_gs| otherwise), energies past the last
 * bin counted in it.  Requires chym_energy or chym_energy_device first.
 * Synchronises the stream. */
CHYM_API chym_status chym_stats(chym_ctx* ctx, double E_gs, chym_stats_t* out, int64_t* hits_per_h,
                       int64_t* hist, int n_bins, void* cuda_stream);

/* Per-spin weights of the coupling term: spin p's term eps alpha_mu y_p becomes
 * eps w_p alpha_mu y_p in every following step (w: N finite doubles, host, copied;
 * NULL restores w = 1).  This lets independent graphs share one context as the
 * blocks of a block-diagonal J, each with its own eps_i = eps w_p (the text after
 * Eq. 1 fixes the coupling per graph, and eps = eps_hat / lambda_max differs
 * between graphs); the noise counters of a packed graph use its spins' indices in
 * the packed J.  Weights are supported on the FP64/FP32 paths and on the tensor-core
 * path up to N = 128 (chym_run and chym_batch_run return ENOTSUP beyond). */
CHYM_API chym_status chym_set_coupling_weights(chym_ctx* ctx, const double* w);

/* Ising energies of contiguous spin segments [seg_begin[i], seg_begin[i+1]),
 * i < n_seg (seg_begin: n_seg + 1 ints, host, 0 first and N last, strictly
 * increasing, 1 <= n_seg <= 128): E_out[run * n_seg + i] = -sum_{p,q in segment i}
 * J_pq s_p s_q with s_p = sign x_{p,0} (Eq. 3 restricted to one block of a packed
 * block-diagonal J); exact integers for CHYM_J_PM1, NaN for a segment whose state
 * is not finite.  E_out: n_runs * n_seg doubles (host).  Does not touch the
 * energies chym_stats uses.  Synchronises the stream. */
CHYM_API chym_status chym_energy_segments(chym_ctx* ctx, int n_seg, const int* seg_begin,
                                          double* E_out, void* cuda_stream);

/* Copy the run state to the host as FP64, layout X[run][p][mu] (n_runs*N*D
 * doubles), and the current step.  Synchronises the stream. */
CHYM_API chym_status chym_get_state(chym_ctx* ctx, double* X_out, int64_t* k_out, void* cuda_stream);

/* Replace the run state (X[run][p][mu], FP64 host) and the step counter,
 * e.g. to resume from a checkpoint; the precision of the following chym_run
 * decides how it is stored.  seeds: n_runs noise keys; h: n_h pumps. */
CHYM_API chym_status chym_set_state(chym_ctx* ctx, const double* X, int n_runs, const double* h,
                           int n_h, const uint64_t* seeds, int64_t k, int32_t prec,
                           void* cuda_stream);

/* Checkpoint of the complete run state of ctx into a host buffer: the state in its
 * storage precision (bit-exact), the step k, the pumps h, and per run its noise key,
 * (re)seeding step and pump index, behind a header (format version 1, N, D, n_runs,
 * n_h, precision).  The noise is counter based, so restoring and continuing equals
 * continuing the original, reseeded runs included (the paper's runs are integrated over
 * up to 1.5e5 round trips each, text before Fig. 4).  With buf NULL, *len gets the size
 * needed; otherwise *len is the buffer's size (EINVAL if too small) and gets the size
 * written.  ESTATE without a state.  Synchronises the stream. */
CHYM_API chym_status chym_checkpoint(chym_ctx* ctx, void* buf, size_t* len, void* cuda_stream);

/* Restore a checkpoint written by chym_checkpoint into ctx, which must have the same N
 * and D (EINVAL otherwise, and for a buffer whose header or size does not match); the
 * context then continues exactly where the checkpointed one was.  Synchronises. */
CHYM_API chym_status chym_restore(chym_ctx* ctx, const void* buf, size_t len, void* cuda_stream);

/* Retire-and-reseed: the n runs listed in d_runs (device int32) restart from the
 * new seeds d_new_seeds (device, n keys) at their local step 0 while the other
 * runs continue: x(0) = init_std * N(0,1) from the new key (tag 1), and from then
 * on the run's noise counter and annealing schedule use its local step
 * k - k_reseed (k_reseed = the context's current step).  A reseeded run therefore
 * follows exactly the trajectory of a fresh run with that seed.  d_new_pump
 * (device int32, nullable) gives each restarted run a new index into h (default:
 * keep its pump); chym_stats counts every run under its current pump.
 * Asynchronous; listed runs must be distinct and < n_runs. */
CHYM_API chym_status chym_reseed_device(chym_ctx* ctx, const int32_t* d_runs, int n,
                                        const uint64_t* d_new_seeds, const int32_t* d_new_pump,
                                        double init_std, void* cuda_stream);

/* Per-run (re)seeding steps (device int64, n_runs): the local step of run r at the
 * context's step k is k - offsets[r].  Asynchronous. */
CHYM_API chym_status chym_get_offsets_device(chym_ctx* ctx, int64_t* d_offsets_out, void* cuda_stream);

/* Shape of the current batch: n_runs, n_h and the current step (any may be NULL). */
CHYM_API chym_status chym_info(chym_ctx* ctx, int* n_runs, int* n_h, int64_t* k);

/* ---- Ground-state references (host; E_GS of the success probability
 * P_Ising, which counts the runs that end at the Ising ground-state energy,
 * text before Fig. 4).  Energies use E = -sum_{p,q} J_pq s_p s_q. ---- */

/* Exact E_GS of ctx's J by exhaustive Gray-code enumeration of the 2^{N-1}
 * states (spin N-1 fixed by the global flip symmetry).  N <= 34, EINVAL
 * otherwise.  spins_out: nullable, ceil(N/64) words, bit p set for s_p = +1. */
CHYM_API chym_status chym_ground_state_exact(chym_ctx* ctx, double* E_out, uint64_t* spins_out);

/* Exact E_GS of the Moebius ladder (ring bonds j_ring between i and i+1 mod N,
 * rungs j_rung between i and i+N/2) by a minimisation over rung states along
 * the ladder.  N even, >= 6. */
CHYM_API chym_status chym_ground_state_mobius(int N, double j_ring, double j_rung, double* E_out);

/* Best-known E_GS of ctx's J by simulated annealing (restarts x sweeps
 * single-spin Metropolis sweeps, geometric inverse-temperature ramp, then
 * greedy descent), deterministic for a given seed.  An upper bound on E_GS. */
CHYM_API chym_status chym_ground_state_search(chym_ctx* ctx, int restarts, int sweeps, uint64_t seed,
                                              double* E_out, uint64_t* spins_out);

/* ---- Batched integration of many contexts (instances x hyperspin dimensions) ----
 * The runs of every context are independent (the statistics of the text before
 * Fig. 4 are averages over replicas, pump values and graphs), so a batch spreads
 * them over the whole GPU: contexts on the small-N tensor-core path (BF16X2,
 * N <= 128) are integrated by one persistent launch per dimension D whose CTAs walk
 * a host-planned list of run ranges, balanced in whole 8-run chunks across the SMs;
 * the other contexts run their own launches concurrently on forked streams.  The
 * batch keeps the contexts (not owned) and its streams, events and plan buffer. */
typedef struct chym_batch chym_batch;

/* ctxs: n_ctx contexts (pointers copied; the contexts must outlive the batch). */
CHYM_API chym_status chym_batch_create(chym_ctx* const* ctxs, int n_ctx, chym_batch** out);

/* Advance every context by `steps` steps from its own current step, with
 * params[i] and schedules[i] (arrays of n_ctx).  Every context must already hold
 * a state (chym_run/chym_run_device with seeds, possibly with steps = 0, or
 * chym_set_state); the result equals integrating each context alone.  Work is
 * ordered after prior work on cuda_stream and the stream waits for all of it.
 * EINVAL on bad params, ESTATE on a context without state, ENOTSUP when no kernel
 * covers a context. */
CHYM_API chym_status chym_batch_run(chym_batch* b, const chym_params* params,
                                    const chym_schedule* schedules, int64_t steps, void* cuda_stream);

/* Read and clear the batch's device status word (synchronous): CHYM_ETIMEOUT when a
 * bounded device-side wait of a batched launch gave up. */
CHYM_API chym_status chym_batch_status(chym_batch* b);

/* Autotuner of the batch planner.  The planner splits the SMs between the
 * small-N dimensions and the large-N launches in proportion to their estimated
 * work, from a cost model in SM-microseconds: per dimension D, one chunk of runs
 * (8 runs for D <= 4, 4 above) advanced one step on the small-N path; and one
 * unit of the large-N path (a 128-row output tile x one 64-wide K chunk) advanced
 * one step.  chym_batch_tune measures these costs on the current device for the
 * batch's own contexts at the split they run with: the whole batch is integrated
 * for probe_steps steps (once to warm up, then a few rounds timed per part with CUDA
 * events, each part's time the shorter of two runs); after each round every part's
 * cost is re-estimated from its measured
 * time and CTA count, which moves the next split towards equal finish times, and
 * the split whose slowest part was fastest is kept.  Every context's state, step
 * and energies are restored afterwards, so tuning does not change any result.
 * Synchronous; needs the contexts' states (ESTATE otherwise); probe_steps >= 1. */
CHYM_API chym_status chym_batch_tune(chym_batch* b, const chym_params* params,
                                     const chym_schedule* schedules, int64_t probe_steps,
                                     void* cuda_stream);
/* The cost model: chunk_costs[D-1] for D = 1..8 and k2_cost (SM-microseconds),
 * tuned = 1 once measured or set.  Outputs may be NULL.  With set, a caller
 * restores costs it cached from an earlier tuning (positive and finite values;
 * NULL keeps the current ones). */
CHYM_API chym_status chym_batch_get_tuning(chym_batch* b, double* chunk_costs, double* k2_cost,
                                           int* tuned);
CHYM_API chym_status chym_batch_set_tuning(chym_batch* b, const double* chunk_costs,
                                           const double* k2_cost);

/* Tile shapes of the batch's kernels, per hyperspin dimension D = 1..8 (arrays of 8,
 * entry D-1; 0 stands for the kernel's default): rt, the runs per column tile of the
 * large-N path (a multiple of 32 with D rt <= 256 and D rt a multiple of 16; default
 * 256 / 128 / 64 / 32 for D = 1 / 2 / 3-4 / 5-8, fewer for contexts with fewer runs);
 * stages, the depth of its operand ring (2..8, capped by what its shared memory holds;
 * default: the most that fit); chunk, the runs per epilogue chunk of the small-N path
 * (4 or 8 for D <= 4; default 8).  chym_batch_tune chooses them by measurement after
 * its cost-model rounds: for each D with large-N contexts every valid rt, then the
 * three ring depths below the largest; for each D <= 4 with small-N contexts both
 * chunks; each part keeps the shape under which it ran fastest (the whole batch runs
 * probe_steps steps per candidate; results are unchanged by the shapes except in the
 * order of floating-point sums).  get: outputs may be NULL; set: NULL keeps an array,
 * EINVAL for invalid values. */
CHYM_API chym_status chym_batch_get_shapes(chym_batch* b, int* rt, int* stages, int* chunk);
CHYM_API chym_status chym_batch_set_shapes(chym_batch* b, const int* rt, const int* stages,
                                           const int* chunk);

CHYM_API chym_status chym_batch_destroy(chym_batch* b);

/* ---- Learned early exit (no counterpart in the paper's method; a layer on top of
 * it): features of a run's early trajectory and a 24-64-64-1 GELU network with
 * BF16 weights and FP32 accumulation that predicts whether the run will end at
 * the Ising ground state, so that runs judged doomed can be retired and their
 * slots reseeded (chym_reseed_device). ---- */
typedef struct chym_mlp chym_mlp;

/* Copy the raw run state (the context's storage type: double for FP64, float
 * otherwise; n_runs * N * D values, layout X[run][p][mu]) to device memory, e.g.
 * to keep a snapshot for chym_features_device.  Asynchronous. */
CHYM_API chym_status chym_copy_state_device(chym_ctx* ctx, void* d_dst, void* cuda_stream);

/* 24 features per run into d_features (device float, n_runs x 24) from the current
 * state and a snapshot taken earlier with chym_copy_state_device:
 *  0-11  quantiles of |x_p0| / rms at levels j/11 (sorted order statistic
 *        floor(j (N-1)/11 + 1/2)), rms = sqrt(mean_p x_p0^2);
 *  12    E/N, Ising energy of the signs now (Eq. 3 with Ising spins);
 *  13    (E - E_snapshot)/N;  14  extra-dimension weight sum_{mu>=1} x^2 / sum x^2;
 *  15    its change since the snapshot;  16  fraction of spins whose sign flipped;
 *  17    E_hs/N (Eq. 3);  18  mean |x_p|;  19  the run's pump h;  20  D/8;
 *  21    ln N / ln 2048;  22  k_frac (fraction of the schedule reached);  23  rms.
 * N <= 4096.  Asynchronous. */
CHYM_API chym_status chym_features_device(chym_ctx* ctx, const void* d_snapshot, double k_frac,
                                          float* d_features, void* cuda_stream);

/* Network 24 -> 64 -> 64 -> 1: standardised input (f - mean) * istd, GELU hidden
 * layers, logit output; 5825 FP32 master parameters laid out W1[64][24], b1[64],
 * W2[64][64], b2[64], W3[64], b3, a BF16 copy of them used by the forward pass,
 * and Adam moments.  Initialised Glorot-uniform from `seed`; max_batch bounds the
 * training batch.  Synchronous. */
CHYM_API chym_status chym_mlp_create(uint64_t seed, int max_batch, chym_mlp** out);
CHYM_API chym_status chym_mlp_destroy(chym_mlp* net);
/* Host parameter vector (5825 floats) and standardisation (24 + 24); any may be
 * NULL to keep the current values.  Setting the parameters resets Adam. */
CHYM_API chym_status chym_mlp_set_params(chym_mlp* net, const float* theta, const float* mean,
                                         const float* istd);
CHYM_API chym_status chym_mlp_get_params(chym_mlp* net, float* theta_out);
/* Logits of B feature rows (device).  Asynchronous. */
CHYM_API chym_status chym_mlp_forward_device(chym_mlp* net, const float* d_features, int B,
                                             float* d_logits, void* cuda_stream);
/* Gradient of the mean binary cross-entropy-with-logits over B rows with labels
 * d_labels (device, 0 or 1) into d_grad (device, 5825, nullable) and the loss into
 * d_loss (device, nullable).  B <= max_batch.  Asynchronous. */
CHYM_API chym_status chym_mlp_grad_device(chym_mlp* net, const float* d_features, const float* d_labels,
                                          int B, float* d_grad, float* d_loss, void* cuda_stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that gradient with learning rate lr. */
CHYM_API chym_status chym_mlp_train_step_device(chym_mlp* net, const float* d_features,
                                                const float* d_labels, int B, float lr,
                                                float* d_loss, void* cuda_stream);

/* One decision pass of continuous operation with the learned early exit: for every run
 * at the context's current step k, with its local step l = k - offset (see
 * chym_reseed_device): done = l >= K; hit = done and |E - E_gs| <= 1e-9 max(1, |E_gs|)
 * (d_E: the runs' energies, device doubles, e.g. from chym_energy_device); at_dec = l ==
 * k_dec where d_logits (device float, nullable) is given; retire = at_dec and logit <
 * theta; restart = done or retire.  d_counts (device int64, 5): the numbers of at_dec,
 * retire, done, hit and restart runs.  d_order (device int32, n_runs): the restarted
 * runs in increasing order, then the others in increasing order (the first `restart`
 * entries are the list chym_reseed_device takes).  K >= 1.  Asynchronous. */
CHYM_API chym_status chym_exit_scan_device(chym_ctx* ctx, const double* d_E, double E_gs,
                                           const float* d_logits, float theta, int64_t K,
                                           int64_t k_dec, long long* d_counts, int32_t* d_order,
                                           void* cuda_stream);

/* ---- Statistics without device allocation ----
 * No counterpart in the paper: this entry point exists for callers that cannot
 * allocate device memory at the point where they need the statistics (a host
 * framework whose memory manager owns the whole device pool, a real-time loop
 * with a fixed budget, or code that must avoid the device-wide synchronisation
 * that cudaMalloc/cudaFree can cause).  It computes the same figures as
 * chym_stats from energies the caller already holds on the device, without a
 * context, and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * d_E: n_runs energies in device memory (h-major runs, as chym_energy_device
 * writes them); kind decides exact (CHYM_J_PM1) or relative-tolerance hits.
 * out, hits_per_h (nullable, n_h int64) and hist (nullable, n_bins int64) are
 * host memory, filled as by chym_stats.  The kernel's result block lives in a
 * fixed device array of about 545 KB compiled into the library, held by every
 * GPU that loads it until the process exits.  Limits: n_h <= 4096 and
 * n_bins <= 65536; larger sizes return CHYM_EINVAL.  The first call on a device
 * looks up that array's device address (once per device); make that first call
 * before any stream capture.  All calls share the one array: two calls whose
 * work overlaps on the GPU (different streams, or different host threads) race
 * and may return each other's numbers; serialise them.  Synchronises the stream. */
CHYM_API chym_status chym_stats_noalloc(const double* d_E, int n_runs, int n_h, chym_jkind kind,
                                        double E_gs, chym_stats_t* out, int64_t* hits_per_h,
                                        int64_t* hist, int n_bins, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CHYM_H */
