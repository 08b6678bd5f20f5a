// chym_groundstate.cpp -- host references for the Ising ground-state energy E_GS
// that the success probability P_Ising is measured against (text before
// Fig. 4 of arXiv 2308.02329: P_Ising counts the runs that reach E_GS).
//
//  * exact, small N: exhaustive walk over the 2^{N-1} states with spin N-1
//    fixed (global flip symmetry), in Gray-code order with incremental fields;
//  * exact, Moebius ladder: minimisation over rung states along the ladder
//    (4 states per rung, twisted closure);
//  * best known, any N: simulated annealing with restarts (the paper's
//    references were found with an unspecified Monte-Carlo algorithm).
// Energies use E = -sum_{p,q} J_pq s_p s_q.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chym_internal.cuh"

namespace chym {
namespace {

double energy_of(const double* J, int N, const int8_t* s) {
  double e = 0.0;
  for (int p = 0; p < N; ++p) {
    double f = 0.0;
    for (int q = 0; q < N; ++q) f += J[(size_t)p * N + q] * s[q];
    e += s[p] * f;
  }
  return -e;
}

void pack(const int8_t* s, int N, uint64_t* out) {
  const int words = (N + 63) / 64;
  for (int w = 0; w < words; ++w) out[w] = 0;
  for (int p = 0; p < N; ++p)
    if (s[p] > 0) out[p / 64] |= 1ull << (p % 64);
}

struct Xoshiro {  // xoshiro256** (Blackman & Vigna) for the annealer's proposals
  uint64_t s[4];
  explicit Xoshiro(uint64_t seed) {
    for (int i = 0; i < 4; ++i) {  // seeded through SplitMix64
      seed += 0x9E3779B97F4A7C15ull;
      uint64_t z = seed;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      s[i] = z ^ (z >> 31);
    }
  }
  static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  uint64_t next() {
    const uint64_t r = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return r;
  }
  double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
};

}  // namespace
}  // namespace chym

using namespace chym;

extern "C" {

CHYM_API chym_status chym_ground_state_exact(chym_ctx* c, double* E_out, uint64_t* spins_out) {
  if (!c || !E_out) return fail(CHYM_EINVAL, "NULL argument");
  const int N = c->N;
  if (N > 34) return fail(CHYM_EINVAL, "exhaustive search limited to N <= 34");
  const double* J = c->h_J;
  std::vector<int8_t> s(N, 1), best(N, 1);
  std::vector<double> field(N, 0.0);  // sum_{q != p} J_pq s_q
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) field[p] += J[(size_t)p * N + q] * s[q];
  double e = energy_of(J, N, s.data()), e_best = e;
  const uint64_t n_states = N >= 1 ? (1ull << (N - 1)) : 1ull;
  for (uint64_t g = 1; g < n_states; ++g) {
    const int p = __builtin_ctzll(g);
    e += 4.0 * s[p] * field[p];  // flipping s_p changes E by 4 s_p field_p
    s[p] = (int8_t)-s[p];
    const double d = 2.0 * s[p];
    const double* col = J + (size_t)p * N;  // J symmetric: column p = row p
    for (int q = 0; q < N; ++q) field[q] += d * col[q];
    if (e < e_best) {
      e_best = e;
      best = s;
    }
  }
  *E_out = energy_of(J, N, best.data());  // recomputed from the spins, no drift
  if (spins_out) pack(best.data(), N, spins_out);
  return CHYM_OK;
}

CHYM_API chym_status chym_ground_state_mobius(int N, double j_ring, double j_rung, double* E_out) {
  if (!E_out || N < 6 || N % 2) return fail(CHYM_EINVAL, "Moebius ladder needs even N >= 6");
  const int L = N / 2;
  auto spin = [](int st, int b) { return ((st >> b) & 1) ? -1.0 : 1.0; };
  double best = INFINITY;
  for (int s0 = 0; s0 < 4; ++s0) {
    double cost[4];
    for (int st = 0; st < 4; ++st) cost[st] = INFINITY;
    cost[s0] = -2.0 * j_rung * spin(s0, 0) * spin(s0, 1);
    for (int i = 1; i < L; ++i) {
      double nxt[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
      for (int prev = 0; prev < 4; ++prev) {
        if (!isfinite(cost[prev])) continue;
        for (int st = 0; st < 4; ++st) {
          const double link = -2.0 * j_ring * (spin(prev, 0) * spin(st, 0) + spin(prev, 1) * spin(st, 1));
          const double v = cost[prev] + link - 2.0 * j_rung * spin(st, 0) * spin(st, 1);
          nxt[st] = std::min(nxt[st], v);
        }
      }
      memcpy(cost, nxt, sizeof(cost));
    }
    for (int st = 0; st < 4; ++st) {
      if (!isfinite(cost[st])) continue;
      // closing bonds with the twist: top of the last rung to bottom of the first
      const double close = -2.0 * j_ring * (spin(st, 0) * spin(s0, 1) + spin(st, 1) * spin(s0, 0));
      best = std::min(best, cost[st] + close);
    }
  }
  *E_out = best;
  return CHYM_OK;
}

CHYM_API chym_status chym_ground_state_search(chym_ctx* c, int restarts, int sweeps,
                                              uint64_t seed, double* E_out, uint64_t* spins_out) {
  if (!c || !E_out || restarts < 1 || sweeps < 1) return fail(CHYM_EINVAL, "bad argument");
  const int N = c->N;
  const double* J = c->h_J;
  double jmax = 0.0;
  for (size_t i = 0; i < (size_t)N * N; ++i) jmax = std::max(jmax, fabs(J[i]));
  if (jmax == 0.0) jmax = 1.0;
  Xoshiro rng(seed);
  std::vector<int8_t> s(N), best(N);
  std::vector<double> field(N);
  double e_best = INFINITY;
  for (int r = 0; r < restarts; ++r) {
    for (int p = 0; p < N; ++p) s[p] = (rng.next() >> 63) ? 1 : -1;
    for (int p = 0; p < N; ++p) {
      field[p] = 0.0;
      for (int q = 0; q < N; ++q) field[p] += J[(size_t)p * N + q] * s[q];
    }
    double e = energy_of(J, N, s.data());
    // inverse temperature from 0.1/jmax to 10/jmax, geometric
    const double b0 = 0.1 / jmax, b1 = 10.0 / jmax;
    for (int sw = 0; sw < sweeps; ++sw) {
      const double beta = b0 * pow(b1 / b0, (double)sw / std::max(1, sweeps - 1));
      for (int p = 0; p < N; ++p) {
        const double dE = 4.0 * s[p] * field[p];
        if (dE <= 0.0 || rng.uniform() < exp(-beta * dE)) {
          s[p] = (int8_t)-s[p];
          e += dE;
          const double d = 2.0 * s[p];
          const double* col = J + (size_t)p * N;
          for (int q = 0; q < N; ++q) field[q] += d * col[q];
        }
      }
    }
    // greedy descent to the nearest local minimum
    bool moved = true;
    while (moved) {
      moved = false;
      for (int p = 0; p < N; ++p)
        if (4.0 * s[p] * field[p] < 0.0) {
          s[p] = (int8_t)-s[p];
          const double d = 2.0 * s[p];
          const double* col = J + (size_t)p * N;
          for (int q = 0; q < N; ++q) field[q] += d * col[q];
          moved = true;
        }
    }
    e = energy_of(J, N, s.data());
    if (e < e_best) {
      e_best = e;
      best = s;
    }
  }
  *E_out = e_best;
  if (spins_out) pack(best.data(), N, spins_out);
  return CHYM_OK;
}

}  // extern "C"
