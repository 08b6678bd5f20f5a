/*
 * chym_oracle.c -- plain, slow, FP64 CPU oracle for the coherent hyperspin
 * machine (CHYM) of "Hyperscaling in the coherent hyperspin machine"
 * (Calvanese Strinati & Conti, arXiv 2308.02329).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent oracle that the
 * CUDA path is compared against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Everything is written in the order and notation of the paper, with no
 * blocking, fusion or reordering:
 *   - the hyperspin layout j = (p-1) D + mu of the D x N oscillator amplitudes
 *     (text before Eq. 1): here X[run][p][mu], p = 0..N-1, mu = 0..D-1;
 *   - the coupling C = J_N (x) 1_D (text after Eq. 1): every component mu is
 *     multiplied by the same N x N matrix J;
 *   - the non-local loss W = beta 1_N (x) I_D (text after Eq. 1): the
 *     saturation of oscillator (p, mu) is driven by the squared norm of
 *     hyperspin p, sum_nu x_{p,nu}^2;
 *   - dimensional annealing C_jl -> alpha_{mu,tau} C_jl (text after Fig. 2);
 *   - the Ising energy E = - sum_{p,q} J_pq s_p s_q of the signed spins and the
 *     hyperspin energy of Eq. 3.
 *
 * Readings where the paper is silent (the supplement holding K, alpha and the
 * noise model is not part of the text): the round-trip map of Eq. 2 is taken
 * as the Euler-Maruyama step of
 *   dx_{p,mu}/dt = (h-1) x - kappa x^3 - gamma x |x_p|^2
 *                  + eps alpha_mu(t) sum_q J_pq x_{q,mu} + sigma xi(t),
 * with gamma standing for beta b^2 and kappa for the local kappa L; the
 * annealing schedule is linear; the noise is additive Gaussian drawn from the
 * counter-based Philox4x32-10 generator with a Box-Muller transform.
 *
 * Parity status of each function is stated in its comment: every function
 * here is pinned by a CPU test against a closed form, an invariant, a
 * published known-answer vector or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Pinned by the     */
/* published known-answer vectors.                                           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: Weyl sequence bump between rounds */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Gaussian noise of the method (reading: additive Gaussian noise per PO).   */
/*                                                                           */
/* For run seed s, stream tag t (0: per-step noise, 1: initial state), step  */
/* k, spin p and component mu of a D-component hyperspin: key = (lo32 s,     */
/* hi32 s).  One Philox4x32-10 block gives four normals:                     */
/*   D >= 3: counter (p, (t << 8) | (mu / 4), lo32 k, hi32 k), normal mu % 4; */
/*   D <= 2: the 4/D spins p with the same p / (4/D) share one block,        */
/*           counter (p / (4/D), t << 8, lo32 k, hi32 k), normal number      */
/*           (p % (4/D)) * D + mu (so every normal of the block is used).    */
/* (For D = 4 the two rules coincide.)  The four 32-bit words become         */
/* uniforms u_j = (w_j + 1/2) 2^-32 in (0,1); Box-Muller turns (u0,u1) into   */
/* (r cos 2 pi u1, r sin 2 pi u1) with r = sqrt(-2 ln u0), likewise (u2,u3).  */
/* ------------------------------------------------------------------------ */
#define ORACLE_TWO_PI 6.283185307179586476925286766559

double oracle_normal(uint64_t seed, uint32_t tag, uint64_t k, uint32_t p,
                     uint32_t mu, uint32_t D) {
  uint32_t block, j;
  if (D <= 2u) {
    const uint32_t per = 4u / D; /* spins per block */
    block = p / per;
    j = (p % per) * D + mu;
  } else {
    block = p;
    j = mu % 4u;
  }
  uint32_t ctr[4] = {block, (tag << 8) | (D <= 2u ? 0u : mu / 4u), (uint32_t)k,
                     (uint32_t)(k >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  oracle_philox4x32_10(ctr, key, w);
  uint32_t pair = j / 2u; /* 0: words (0,1), 1: words (2,3) */
  double u_r = ((double)w[2 * pair] + 0.5) / 4294967296.0;
  double u_a = ((double)w[2 * pair + 1] + 0.5) / 4294967296.0;
  double r = sqrt(-2.0 * log(u_r));
  double angle = ORACLE_TWO_PI * u_a;
  return (j % 2u == 0u) ? r * cos(angle) : r * sin(angle);
}

/* ------------------------------------------------------------------------ */
/* Dimensional annealing schedule alpha_mu(k) (text after Fig. 2: C_jl ->    */
/* alpha_{mu,tau} C_jl).  Reading: component mu = 0 (the paper's mu = 1)     */
/* keeps alpha = 1; components mu >= 1 keep alpha = 1 until step k_anneal,   */
/* then fall linearly to 0 at step k_total.  kind 0: no annealing.           */
/* ------------------------------------------------------------------------ */
double oracle_alpha(int kind, int64_t k, int64_t k_anneal, int64_t k_total,
                    int mu) {
  if (kind == 0 || mu == 0) return 1.0;
  if (k < k_anneal) return 1.0;
  if (k >= k_total) return 0.0;
  double a = 1.0 - (double)(k - k_anneal) / (double)(k_total - k_anneal);
  return a < 0.0 ? 0.0 : a;
}

/* ------------------------------------------------------------------------ */
/* Initial amplitudes x_{p,mu}(0) = init_std * N(0,1), tag 1, step 0.        */
/* Layout X[run][p][mu].                                                     */
/* ------------------------------------------------------------------------ */
void oracle_init(int N, int D, int n_runs, const uint64_t* seeds,
                 double init_std, double* X) {
  for (int r = 0; r < n_runs; ++r)
    for (int p = 0; p < N; ++p)
      for (int mu = 0; mu < D; ++mu)
        X[((size_t)r * N + p) * D + mu] =
            init_std * oracle_normal(seeds[r], 1u, 0u, (uint32_t)p, (uint32_t)mu, (uint32_t)D);
}

/* ------------------------------------------------------------------------ */
/* Drift f of one run at step k (noise excluded).                            */
/*   y_{p,mu} = sum_q J_pq x_{q,mu}                     (C = J (x) 1_D, Eq. 1) */
/*   n_p      = sum_nu x_{p,nu}^2                       (W = beta 1 (x) I_D)   */
/*   f_{p,mu} = (h-1) x_{p,mu} - kappa x_{p,mu}^3 - gamma x_{p,mu} n_p        */
/*              + eps alpha_mu(k) y_{p,mu}                                    */
/* x: N*D values of one run, f: N*D output.                                  */
/* ------------------------------------------------------------------------ */
void oracle_drift(const double* J, int N, int D, const double* x, double h,
                  double gamma, double kappa, double eps, int sched_kind,
                  int64_t k, int64_t k_anneal, int64_t k_total, double* f) {
  for (int p = 0; p < N; ++p) {
    double n_p = 0.0;
    for (int nu = 0; nu < D; ++nu) {
      double v = x[(size_t)p * D + nu];
      n_p += v * v;
    }
    for (int mu = 0; mu < D; ++mu) {
      double y = 0.0;
      for (int q = 0; q < N; ++q) y += J[(size_t)p * N + q] * x[(size_t)q * D + mu];
      double xm = x[(size_t)p * D + mu];
      double alpha = oracle_alpha(sched_kind, k, k_anneal, k_total, mu);
      f[(size_t)p * D + mu] = (h - 1.0) * xm - kappa * xm * xm * xm -
                              gamma * xm * n_p + eps * alpha * y;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Euler-Maruyama integration of n_runs independent runs, steps k0 .. k0 +   */
/* steps - 1:  x <- x + dt f(x, k) + sigma sqrt(dt) xi_k, xi from tag 0.     */
/* h_run[r] is the pump of run r.  Runs are independent, so they are spread  */
/* over OpenMP threads; the arithmetic of each run is the sequential loop.   */
/* ------------------------------------------------------------------------ */
void oracle_integrate(const double* J, int N, int D, int n_runs,
                      const double* h_run, const uint64_t* seeds, double dt,
                      double sigma, double gamma, double kappa, double eps,
                      int sched_kind, int64_t k_anneal, int64_t k_total,
                      int64_t k0, int64_t steps, double* X, int n_threads) {
  double noise_scale = sigma * sqrt(dt);
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
  {
    double* f = (double*)malloc(sizeof(double) * (size_t)N * D);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int r = 0; r < n_runs; ++r) {
      double* x = X + (size_t)r * N * D;
      for (int64_t k = k0; k < k0 + steps; ++k) {
        oracle_drift(J, N, D, x, h_run[r], gamma, kappa, eps, sched_kind, k,
                     k_anneal, k_total, f);
        for (int p = 0; p < N; ++p)
          for (int mu = 0; mu < D; ++mu) {
            double xi = oracle_normal(seeds[r], 0u, (uint64_t)k, (uint32_t)p,
                                      (uint32_t)mu, (uint32_t)D);
            x[(size_t)p * D + mu] += dt * f[(size_t)p * D + mu] + noise_scale * xi;
          }
      }
    }
    free(f);
  }
}

/* ------------------------------------------------------------------------ */
/* Ising readout (reading: the sign of the surviving component mu = 0, ties  */
/* to +1) and Ising energy E = - sum_{p,q} J_pq s_p s_q (full double sum, as  */
/* in Eq. 3).                                                                */
/* ------------------------------------------------------------------------ */
void oracle_readout(int N, int D, int n_runs, const double* X, int8_t* s) {
  for (int r = 0; r < n_runs; ++r)
    for (int p = 0; p < N; ++p)
      s[(size_t)r * N + p] = (X[((size_t)r * N + p) * D] >= 0.0) ? 1 : -1;
}

double oracle_ising_energy(const double* J, int N, const int8_t* s) {
  double e = 0.0;
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) e += J[(size_t)p * N + q] * (double)s[p] * (double)s[q];
  return -e;
}

/* Best-axis rounding of a two-component (XY, D = 2) state: among all axes     */
/* u = (cos phi, sin phi), the Ising pattern s_p = +1 if x_p . u >= 0 else -1 */
/* with the lowest energy E = -sum J s s.  The pattern changes only where an  */
/* axis is perpendicular to a spin, at phi_p = theta_p + pi/2 (mod pi), so the */
/* candidates are one axis inside every interval between consecutive distinct */
/* critical angles (phi and phi + pi give opposite patterns of equal energy). */
/* Spins of zero length project to 0 and stay +1.  Written plainly: every     */
/* candidate's pattern and energy from scratch, O(N^3).  Returns the lowest   */
/* energy and the first pattern (in increasing phi) that reaches it.          */
/* ------------------------------------------------------------------------ */
static int cmp_double(const void* a, const void* b) {
  const double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

double oracle_round_xy(const double* J, int N, const double* x, int8_t* s_out) {
  const double pi = 3.14159265358979323846;
  double* crit = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  int8_t* s = (int8_t*)malloc((size_t)(N > 0 ? N : 1));
  int n_crit = 0;
  for (int p = 0; p < N; ++p) {
    const double a = x[2 * (size_t)p], b = x[2 * (size_t)p + 1];
    if (a == 0.0 && b == 0.0) continue;
    double c = fmod(atan2(b, a) + 0.5 * pi, pi);
    if (c < 0.0) c += pi;
    crit[n_crit++] = c;
  }
  qsort(crit, (size_t)n_crit, sizeof(double), cmp_double);
  int n_dist = 0;
  for (int i = 0; i < n_crit; ++i)
    if (n_dist == 0 || crit[i] != crit[n_dist - 1]) crit[n_dist++] = crit[i];
  double best = INFINITY;
  const int n_cand = n_dist > 0 ? n_dist : 1;
  for (int i = 0; i < n_cand; ++i) {
    /* the interval after critical angle i (the last one wraps around through pi) */
    double phi;
    if (n_dist == 0) phi = 0.0;
    else if (i + 1 < n_dist) phi = 0.5 * (crit[i] + crit[i + 1]);
    else phi = 0.5 * (crit[i] + crit[0] + pi);
    const double u0 = cos(phi), u1 = sin(phi);
    for (int p = 0; p < N; ++p)
      s[p] = (x[2 * (size_t)p] * u0 + x[2 * (size_t)p + 1] * u1 >= 0.0) ? 1 : -1;
    const double e = oracle_ising_energy(J, N, s);
    if (e < best) {
      best = e;
      if (s_out) memcpy(s_out, s, (size_t)N);
    }
  }
  free(crit);
  free(s);
  return best;
}

/* Hyperspin energy of Eq. 3 with sigma_p = x_p / |x_p| (zero vector if      */
/* x_p = 0).                                                                 */
double oracle_hyperspin_energy(const double* J, int N, int D, const double* x) {
  double* sig = (double*)malloc(sizeof(double) * (size_t)N * D);
  for (int p = 0; p < N; ++p) {
    double n2 = 0.0;
    for (int mu = 0; mu < D; ++mu) n2 += x[(size_t)p * D + mu] * x[(size_t)p * D + mu];
    double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    for (int mu = 0; mu < D; ++mu) sig[(size_t)p * D + mu] = x[(size_t)p * D + mu] * inv;
  }
  double e = 0.0;
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) {
      double dot = 0.0;
      for (int mu = 0; mu < D; ++mu) dot += sig[(size_t)p * D + mu] * sig[(size_t)q * D + mu];
      e += J[(size_t)p * N + q] * dot;
    }
  free(sig);
  return -e;
}

/* ------------------------------------------------------------------------ */
/* XY ground state (the reference of the XY machine, D = 2 without           */
/* annealing: the text after Fig. 2 and its footnote compare the machine's    */
/* energy with the XY ground state found by a numerical minimiser).  Planar   */
/* unit spins sigma_p = (cos theta_p, sin theta_p) turn Eq. 3 into            */
/*   E_XY(theta) = - sum_{p,q} J_pq cos(theta_p - theta_q).                   */
/* The terms that hold theta_p are -2 sum_q J_pq cos(theta_p - theta_q)       */
/* (J symmetric), i.e. minus twice the projection of sigma_p on the local     */
/* field f_p = sum_q J_pq sigma_q; with the others fixed the exact minimiser  */
/* over theta_p is the direction of f_p (kept when f_p = 0).  Coordinate      */
/* descent sweeps p = 0..N-1 with that update; each update can only lower E,  */
/* and a sweep that lowers E by at most tol |E| (or max_sweeps sweeps) ends a  */
/* start.  n_starts starts from the given initial angles theta0[start][p]     */
/* (drawn by the caller); the lowest energy is returned and its angles written */
/* to theta_out (nullable).  An upper bound on the true XY ground-state       */
/* energy, equal to it when one of the starts reaches the global minimum.     */
/* ------------------------------------------------------------------------ */
static double xy_energy(const double* J, int N, const double* th) {
  double e = 0.0;
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) e += J[(size_t)p * N + q] * cos(th[p] - th[q]);
  return -e;
}

double oracle_xy_energy(const double* J, int N, const double* theta) {
  return xy_energy(J, N, theta);
}

double oracle_xy_ground_state(const double* J, int N, int n_starts, const double* theta0,
                              int max_sweeps, double tol, double* theta_out) {
  double best = INFINITY;
  double* th = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  for (int st = 0; st < n_starts; ++st) {
    memcpy(th, theta0 + (size_t)st * N, sizeof(double) * (size_t)N);
    double e = xy_energy(J, N, th);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
      for (int p = 0; p < N; ++p) {
        double fx = 0.0, fy = 0.0;
        for (int q = 0; q < N; ++q) {
          fx += J[(size_t)p * N + q] * cos(th[q]);
          fy += J[(size_t)p * N + q] * sin(th[q]);
        }
        if (fx != 0.0 || fy != 0.0) th[p] = atan2(fy, fx);
      }
      const double e_new = xy_energy(J, N, th);
      const double drop = e - e_new;
      e = e_new;
      if (drop <= tol * fabs(e)) break;
    }
    if (e < best) {
      best = e;
      if (theta_out) memcpy(theta_out, th, sizeof(double) * (size_t)N);
    }
  }
  free(th);
  return best;
}

/* ------------------------------------------------------------------------ */
/* Ising ground state by exhaustive enumeration (the reference the paper's   */
/* success probability is measured against).  The global flip s -> -s keeps */
/* E, so s_{N-1} = +1 is fixed and the 2^{N-1} others are walked in Gray-code */
/* order: flipping spin p changes E by 4 s_p sum_{q != p} J_pq s_q (before    */
/* the flip), for symmetric J.  Returns E_GS and one minimiser in s_out.      */
/* ------------------------------------------------------------------------ */
double oracle_ground_state_bruteforce(const double* J, int N, int8_t* s_out) {
  int8_t* s = (int8_t*)malloc((size_t)N);
  double* field = (double*)malloc(sizeof(double) * (size_t)N);
  for (int p = 0; p < N; ++p) s[p] = 1;
  for (int p = 0; p < N; ++p) {
    field[p] = 0.0;
    for (int q = 0; q < N; ++q) if (q != p) field[p] += J[(size_t)p * N + q] * s[q];
  }
  double e = oracle_ising_energy(J, N, s);
  double best = e;
  memcpy(s_out, s, (size_t)N);
  uint64_t n_states = (N >= 1) ? (1ull << (N - 1)) : 1ull;
  for (uint64_t g = 1; g < n_states; ++g) {
    int p = __builtin_ctzll(g); /* Gray code: bit that changes at step g */
    /* E(s with p flipped) - E(s) = 4 s_p field_p (diagonal terms unchanged) */
    e += 4.0 * (double)s[p] * field[p];
    s[p] = (int8_t)-s[p];
    for (int q = 0; q < N; ++q)
      if (q != p) field[q] += 2.0 * J[(size_t)q * N + p] * (double)s[p];
    if (e < best) {
      best = e;
      memcpy(s_out, s, (size_t)N);
    }
  }
  free(s);
  free(field);
  return best;
}

/* ------------------------------------------------------------------------ */
/* Exact ground state of the Moebius ladder (ring of N = 2L sites with bond  */
/* Jr between i and i+1 mod N, plus rungs of bond Jg between i and i+L), by   */
/* a transfer-matrix minimisation over the L rungs (a_i, b_i) = (s_i,         */
/* s_{i+L}).  Consecutive rungs couple a_i-a_{i+1} and b_i-b_{i+1}; the last  */
/* rung closes with a twist: a_{L-1}-b_0 and b_{L-1}-a_0.  Each bond enters   */
/* E = -sum_{p,q} J s s twice.                                               */
/* ------------------------------------------------------------------------ */
static double mob_rung(double Jg, int a, int b) { return -2.0 * Jg * a * b; }
static double mob_link(double Jr, int a0, int b0, int a1, int b1) {
  return -2.0 * Jr * (a0 * a1 + b0 * b1);
}
static int mob_spin(int st, int which) { return ((st >> which) & 1) ? -1 : 1; }

double oracle_ground_state_mobius(int N, double Jr, double Jg) {
  int L = N / 2;
  double best = INFINITY;
  for (int first = 0; first < 4; ++first) {
    double cost[4];
    for (int st = 0; st < 4; ++st) cost[st] = INFINITY;
    cost[first] = mob_rung(Jg, mob_spin(first, 0), mob_spin(first, 1));
    for (int i = 1; i < L; ++i) {
      double next[4];
      for (int st = 0; st < 4; ++st) {
        next[st] = INFINITY;
        for (int prev = 0; prev < 4; ++prev) {
          if (cost[prev] == INFINITY) continue;
          double c = cost[prev] +
                     mob_link(Jr, mob_spin(prev, 0), mob_spin(prev, 1),
                              mob_spin(st, 0), mob_spin(st, 1)) +
                     mob_rung(Jg, mob_spin(st, 0), mob_spin(st, 1));
          if (c < next[st]) next[st] = c;
        }
      }
      for (int st = 0; st < 4; ++st) cost[st] = next[st];
    }
    int a0 = mob_spin(first, 0), b0 = mob_spin(first, 1);
    for (int st = 0; st < 4; ++st) {
      if (cost[st] == INFINITY) continue;
      int aL = mob_spin(st, 0), bL = mob_spin(st, 1);
      /* twisted closure: a_{L-1} - b_0 and b_{L-1} - a_0 */
      double c = cost[st] - 2.0 * Jr * (aL * b0 + bL * a0);
      if (c < best) best = c;
    }
  }
  return best;
}

/* Normals of one run and one step for all (p, mu), layout out[p][mu]. */
void oracle_normals(uint64_t seed, uint32_t tag, uint64_t k, int N, int D,
                    double* out) {
  for (int p = 0; p < N; ++p)
    for (int mu = 0; mu < D; ++mu)
      out[(size_t)p * D + mu] = oracle_normal(seed, tag, k, (uint32_t)p, (uint32_t)mu, (uint32_t)D);
}
