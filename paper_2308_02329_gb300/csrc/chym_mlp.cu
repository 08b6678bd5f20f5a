// chym_mlp.cu -- learned early exit: run features and the 24-64-64-1 network.
//
// The paper has no learned component.  A run's early trajectory (its state at the
// decision step and an earlier snapshot) is reduced to 24 features; a small GELU
// network with BF16 weights and FP32 accumulation predicts whether the run will
// end at the Ising ground state, so that runs judged doomed can be retired and
// their slots reseeded.  Kernels:
//   features_kernel   one CTA per run: sorted |x_0|/rms quantiles (bitonic sort in
//                     shared memory), Ising energies of the signs now and at the
//                     snapshot (exact integers for +-1 couplings), extra-dimension
//                     weight, sign flips, hyperspin energy (Eq. 3), norms;
//   mlp_forward       one warp per sample, weights (BF16-rounded) in shared memory;
//   mlp_grad          4 warps per CTA, per-warp gradient buffers in shared memory,
//                     per-CTA partial gradients reduced by mlp_adam in a fixed order;
//   mlp_adam          reduction of the partials, Adam on the FP32 master weights,
//                     refresh of the BF16 copy used by the forward pass.
// Network sizes are SIMT-sized (5825 parameters, ~6 kFLOP per sample): a tensor-core
// tile would be mostly padding at these widths.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "chym_internal.cuh"

namespace chym {
namespace {

constexpr int kF = 24, kH = 64;
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH, kP = oB3 + 1;  // 5825 parameters
constexpr int kGradWarps = 4, kGradSamplesPerCta = 64;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * __expf(-0.5f * z * z) * 0.3989422804014327f;
}

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
template <typename V>
__device__ V block_sum(V v, V* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  V t = V(0);
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;  // valid in every thread
}

constexpr int kFeatThreads = 256;

template <typename T, bool PM1>
__global__ void __launch_bounds__(kFeatThreads) features_kernel(
    const T* __restrict__ X, const T* __restrict__ Xs, int N, int D, int P2,
    const int8_t* __restrict__ J8, const double* __restrict__ J64, const double* __restrict__ h,
    const int32_t* __restrict__ hidx, float k_frac, float* __restrict__ F) {
  extern __shared__ float sm[];
  float* buf = sm;                         // P2 floats: sort buffer, then sigma_mu
  float* inv = buf + P2;                   // N floats: 1/|x_p|
  int8_t* s = reinterpret_cast<int8_t*>(inv + N);
  int8_t* ss = s + N;
  __shared__ float red_f[32];
  __shared__ double red_d[32];
  __shared__ long long red_i[32];
  const int run = blockIdx.x, tid = threadIdx.x;
  const T* x = X + (size_t)run * N * D;
  const T* xs = Xs + (size_t)run * N * D;
  float sx0 = 0.f, snorm = 0.f, sextra = 0.f, snorm_s = 0.f, sextra_s = 0.f, sabs = 0.f, flips = 0.f;
  for (int p = tid; p < N; p += blockDim.x) {
    float n2 = 0.f, e2 = 0.f, n2s = 0.f, e2s = 0.f;
    for (int mu = 0; mu < D; ++mu) {
      const float v = (float)x[(size_t)p * D + mu], vs = (float)xs[(size_t)p * D + mu];
      n2 += v * v;
      n2s += vs * vs;
      if (mu > 0) {
        e2 += v * v;
        e2s += vs * vs;
      }
    }
    const float x0 = (float)x[(size_t)p * D];
    sx0 += x0 * x0;
    snorm += n2;
    sextra += e2;
    snorm_s += n2s;
    sextra_s += e2s;
    sabs += sqrtf(n2);
    inv[p] = n2 > 0.f ? rsqrtf(n2) : 0.f;
    s[p] = x[(size_t)p * D] >= T(0) ? 1 : -1;
    ss[p] = xs[(size_t)p * D] >= T(0) ? 1 : -1;
    flips += (s[p] != ss[p]) ? 1.f : 0.f;
  }
  sx0 = block_sum<float>(sx0, red_f);
  snorm = block_sum<float>(snorm, red_f);
  sextra = block_sum<float>(sextra, red_f);
  snorm_s = block_sum<float>(snorm_s, red_f);
  sextra_s = block_sum<float>(sextra_s, red_f);
  sabs = block_sum<float>(sabs, red_f);
  flips = block_sum<float>(flips, red_f);
  const float rms = sqrtf(sx0 / (float)N);
  // sorted |x_0| / rms (bitonic sort, padding +inf)
  for (int i = tid; i < P2; i += blockDim.x)
    buf[i] = i < N ? fabsf((float)x[(size_t)i * D]) / (rms + 1e-30f) : INFINITY;
  __syncthreads();
  for (int kk = 2; kk <= P2; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const float a = buf[i], b = buf[l];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) {
            buf[i] = b;
            buf[l] = a;
          }
        }
      }
      __syncthreads();
    }
  float q12[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) q12[j] = buf[(int)floorf(j * (N - 1) / 11.0f + 0.5f)];
  __syncthreads();
  // Ising energies of the signs now and at the snapshot: E = -sum_p s_p sum_q J_pq s_q
  double E = 0.0, Es = 0.0;
  if (PM1) {
    long long a = 0, b = 0;
    for (int p = tid; p < N; p += blockDim.x) {
      int f = 0, fs = 0;
      for (int q = 0; q < N; ++q) {
        const int j = J8[(size_t)q * N + p];
        f += j * s[q];
        fs += j * ss[q];
      }
      a += (long long)s[p] * f;
      b += (long long)ss[p] * fs;
    }
    E = -(double)block_sum<long long>(a, red_i);
    Es = -(double)block_sum<long long>(b, red_i);
  } else {
    double a = 0.0, b = 0.0;
    for (int p = tid; p < N; p += blockDim.x) {
      double f = 0.0, fs = 0.0;
      for (int q = 0; q < N; ++q) {
        const double j = J64[(size_t)q * N + p];
        f += j * s[q];
        fs += j * ss[q];
      }
      a += s[p] * f;
      b += ss[p] * fs;
    }
    E = -block_sum<double>(a, red_d);
    Es = -block_sum<double>(b, red_d);
  }
  // hyperspin energy (Eq. 3): -sum_mu sum_p sigma_p,mu sum_q J_pq sigma_q,mu
  float ehs = 0.f;
  for (int mu = 0; mu < D; ++mu) {
    __syncthreads();
    for (int q = tid; q < N; q += blockDim.x) buf[q] = (float)x[(size_t)q * D + mu] * inv[q];
    __syncthreads();
    for (int p = tid; p < N; p += blockDim.x) {
      float f = 0.f;
      if (PM1)
        for (int q = 0; q < N; ++q) f += (float)J8[(size_t)q * N + p] * buf[q];
      else
        for (int q = 0; q < N; ++q) f += (float)J64[(size_t)q * N + p] * buf[q];
      ehs += buf[p] * f;
    }
  }
  ehs = -block_sum<float>(ehs, red_f);
  if (tid == 0) {
    float* o = F + (size_t)run * kF;
    for (int j = 0; j < 12; ++j) o[j] = q12[j];
    o[12] = (float)(E / N);
    o[13] = (float)((E - Es) / N);
    const float w = (snorm > 0.f && D > 1) ? sextra / snorm : 0.f;
    const float ws = (snorm_s > 0.f && D > 1) ? sextra_s / snorm_s : 0.f;
    o[14] = w;
    o[15] = w - ws;
    o[16] = flips / (float)N;
    o[17] = ehs / (float)N;
    o[18] = sabs / (float)N;
    o[19] = (float)h[hidx[run]];
    o[20] = (float)D / 8.f;
    o[21] = logf((float)N) / logf(2048.f);
    o[22] = k_frac;
    o[23] = rms;
  }
}

// ---------------------------------------------------------------------------
// network
// ---------------------------------------------------------------------------
struct NetView {
  const float* theta;       // FP32 master
  const __nv_bfloat16* wb;  // BF16 copy of every parameter (biases included)
  const float* mean;
  const float* istd;
};

// Parameters into shared memory as floats rounded through BF16; W1 and W2 also
// transposed so that lane u reads consecutive addresses.
struct SmemNet {
  float W1t[kF * kH];  // [i][u]
  float W2[kH * kH];   // [u][k]
  float W2t[kH * kH];  // [k][u]
  float b1[kH], b2[kH], W3[kH], b3, mean[kF], istd[kF];
};

__device__ void load_net(const NetView& n, SmemNet& s) {
  for (int e = threadIdx.x; e < kH * kF; e += blockDim.x) {
    const int u = e / kF, i = e % kF;
    s.W1t[i * kH + u] = __bfloat162float(n.wb[oW1 + e]);
  }
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int u = e / kH, k = e % kH;
    const float w = __bfloat162float(n.wb[oW2 + e]);
    s.W2[e] = w;
    s.W2t[k * kH + u] = w;
  }
  for (int u = threadIdx.x; u < kH; u += blockDim.x) {
    s.b1[u] = __bfloat162float(n.wb[oB1 + u]);
    s.b2[u] = __bfloat162float(n.wb[oB2 + u]);
    s.W3[u] = __bfloat162float(n.wb[oW3 + u]);
  }
  for (int i = threadIdx.x; i < kF; i += blockDim.x) {
    s.mean[i] = n.mean[i];
    s.istd[i] = n.istd[i];
  }
  if (threadIdx.x == 0) s.b3 = __bfloat162float(n.wb[oB3]);
  __syncthreads();
}

struct WarpAct {
  float f[kF], z1[kH], h1[kH], z2[kH], h2[kH];
};

// Forward of one sample by one warp; lane l owns hidden units l and l + 32.
__device__ float warp_forward(const SmemNet& s, const float* __restrict__ feat, WarpAct& a) {
  const int l = threadIdx.x & 31;
  if (l < kF) a.f[l] = (feat[l] - s.mean[l]) * s.istd[l];
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int u = l + 32 * h;
    float z = s.b1[u];
#pragma unroll
    for (int i = 0; i < kF; ++i) z = fmaf(s.W1t[i * kH + u], a.f[i], z);
    a.z1[u] = z;
    a.h1[u] = gelu(z);
  }
  __syncwarp();
  float out = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int u = l + 32 * h;
    float z = s.b2[u];
    for (int k = 0; k < kH; ++k) z = fmaf(s.W2t[k * kH + u], a.h1[k], z);
    a.z2[u] = z;
    a.h2[u] = gelu(z);
    out = fmaf(s.W3[u], a.h2[u], out);
  }
  for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
  __syncwarp();
  return out + s.b3;
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(NetView n, const float* __restrict__ F, int B,
                                                          float* __restrict__ logits) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemNet& s = *reinterpret_cast<SmemNet*>(smem);
  WarpAct* act = reinterpret_cast<WarpAct*>(smem + sizeof(SmemNet));
  load_net(n, s);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = blockIdx.x * nw + w; b < B; b += gridDim.x * nw) {
    const float z = warp_forward(s, F + (size_t)b * kF, act[w]);
    if ((threadIdx.x & 31) == 0) logits[b] = z;
  }
}

// Partial gradient of the mean BCE-with-logits loss over this CTA's samples.  The
// warp buffers hold W1 as [i][u] and W2 as [k][u] (lane u walks consecutive
// addresses); the CTA partial is written in the parameter layout.
struct WarpGrad {
  float g[kP];
};

__global__ void __launch_bounds__(kGradWarps * 32) mlp_grad_kernel(NetView n, const float* __restrict__ F,
                                                                   const float* __restrict__ y, int B,
                                                                   float* __restrict__ partial,
                                                                   float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemNet& s = *reinterpret_cast<SmemNet*>(smem);
  WarpAct* act = reinterpret_cast<WarpAct*>(smem + sizeof(SmemNet));
  WarpGrad* wg = reinterpret_cast<WarpGrad*>(smem + sizeof(SmemNet) + kGradWarps * sizeof(WarpAct));
  __shared__ float s_dz2[kGradWarps][kH], s_dz1[kGradWarps][kH];
  __shared__ float s_loss[kGradWarps];
  load_net(n, s);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int e = l; e < kP; e += 32) wg[w].g[e] = 0.f;
  float lsum = 0.f;
  const float invB = 1.f / (float)B;
  const int b0 = blockIdx.x * kGradSamplesPerCta;
  const int b1 = min(B, b0 + kGradSamplesPerCta);
  for (int b = b0 + w; b < b1; b += kGradWarps) {
    WarpAct& a = act[w];
    const float logit = warp_forward(s, F + (size_t)b * kF, a);
    const float yb = y[b];
    if (l == 0) lsum += fmaxf(logit, 0.f) - logit * yb + log1pf(__expf(-fabsf(logit)));
    const float dl = (1.f / (1.f + __expf(-logit)) - yb) * invB;
    float* g = wg[w].g;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = l + 32 * h;
      g[oW3 + u] += dl * a.h2[u];
      s_dz2[w][u] = dl * s.W3[u] * gelu_grad(a.z2[u]);
    }
    if (l == 0) g[oB3] += dl;
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = l + 32 * h;
      const float dz2 = s_dz2[w][u];
      g[oB2 + u] += dz2;
      // dW2[u][k] += dz2[u] h1[k], buffer layout [k][u]
      for (int k = 0; k < kH; ++k) g[oW2 + k * kH + u] += dz2 * a.h1[k];
      // dh1[k] = sum_u W2[u][k] dz2[u], lane l owns k = u here
      float dh1 = 0.f;
      for (int v = 0; v < kH; ++v) dh1 = fmaf(s.W2[v * kH + u], s_dz2[w][v], dh1);
      s_dz1[w][u] = dh1 * gelu_grad(a.z1[u]);
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = l + 32 * h;
      const float dz1 = s_dz1[w][u];
      g[oB1 + u] += dz1;
#pragma unroll
      for (int i = 0; i < kF; ++i) g[oW1 + i * kH + u] += dz1 * a.f[i];
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (l == 0) s_loss[w] = lsum;
  __syncthreads();
  // fixed-order reduction of the warps' buffers into this CTA's partial
  for (int e = threadIdx.x; e < kP; e += blockDim.x) {
    int src = e;  // buffer index of parameter e
    if (e < oB1) src = oW1 + (e % kF) * kH + e / kF;
    else if (e >= oW2 && e < oB2) src = oW2 + ((e - oW2) % kH) * kH + (e - oW2) / kH;
    float t = 0.f;
    for (int q = 0; q < kGradWarps; ++q) t += wg[q].g[src];
    partial[(size_t)blockIdx.x * kP + e] = t;
  }
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int q = 0; q < kGradWarps; ++q) t += s_loss[q];
    loss_part[blockIdx.x] = t * invB;
  }
}

// Sum the CTA partials (fixed order), then optionally one Adam step.
__global__ void mlp_reduce_adam_kernel(const float* __restrict__ partial, int n_parts,
                                       const float* __restrict__ loss_part, float* __restrict__ grad,
                                       float* __restrict__ loss, float* theta, float* m, float* v,
                                       __nv_bfloat16* wb, int t, float lr, int do_adam) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kP; e += gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int c = 0; c < n_parts; ++c) g += partial[(size_t)c * kP + e];
    grad[e] = g;
    if (do_adam) {
      const float b1 = 0.9f, b2 = 0.999f;
      const float mm = b1 * m[e] + (1.f - b1) * g;
      const float vv = b2 * v[e] + (1.f - b2) * g * g;
      m[e] = mm;
      v[e] = vv;
      const float mh = mm / (1.f - powf(b1, (float)t)), vh = vv / (1.f - powf(b2, (float)t));
      const float th = theta[e] - lr * mh / (sqrtf(vh) + 1e-8f);
      theta[e] = th;
      wb[e] = __float2bfloat16_rn(th);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    float s = 0.f;
    for (int c = 0; c < n_parts; ++c) s += loss_part[c];
    *loss = s;
  }
}

__global__ void mlp_refresh_bf16_kernel(const float* theta, __nv_bfloat16* wb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kP; e += gridDim.x * blockDim.x)
    wb[e] = __float2bfloat16_rn(theta[e]);
}

template <typename T>
cudaError_t launch_features_typed(chym_ctx* c, const void* snap, double k_frac, float* F, cudaStream_t st) {
  int P2 = 1;
  while (P2 < c->N) P2 <<= 1;
  const size_t smem = sizeof(float) * ((size_t)P2 + c->N) + 2 * (size_t)c->N + 16;
  if (c->kind == CHYM_J_PM1) {
    auto kern = features_kernel<T, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<c->n_runs, kFeatThreads, smem, st>>>((const T*)c->d_X, (const T*)snap, c->N, c->D, P2,
                                                c->d_J8, c->d_J64, c->d_h, c->d_hidx, (float)k_frac, F);
  } else {
    auto kern = features_kernel<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<c->n_runs, kFeatThreads, smem, st>>>((const T*)c->d_X, (const T*)snap, c->N, c->D, P2,
                                                c->d_J8, c->d_J64, c->d_h, c->d_hidx, (float)k_frac, F);
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace chym

struct chym_mlp {
  float* theta = nullptr;         // FP32 master
  __nv_bfloat16* wb = nullptr;    // BF16 copy
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  float* mean = nullptr;
  float* istd = nullptr;
  float* loss = nullptr;
  float* partial = nullptr;       // per-CTA partial gradients
  float* loss_part = nullptr;
  int max_batch = 0;
  int t = 0;                      // Adam step
};

using namespace chym;

namespace {
NetView view(const chym_mlp* n) { return NetView{n->theta, n->wb, n->mean, n->istd}; }
size_t grad_smem() {
  return sizeof(SmemNet) + kGradWarps * (sizeof(WarpAct) + sizeof(WarpGrad));
}
}  // namespace

namespace chym {
namespace {
// One decision pass of continuous operation, one CTA: thread t owns the runs
// [t n / T, (t + 1) n / T) in order, so an exclusive scan of the per-thread restart counts
// gives every restarted run its place in the increasing list.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) exit_scan_kernel(
    const int64_t* __restrict__ koff, int n, int64_t k, const double* __restrict__ E, double E_gs,
    double tol, const float* __restrict__ logits, float theta, int64_t K, int64_t k_dec,
    long long* __restrict__ counts, int32_t* __restrict__ restart) {
  __shared__ int s_cnt[kScanThreads];
  __shared__ long long s_sum[5][32];
  const int t = threadIdx.x;
  const int b = (int)((int64_t)t * n / kScanThreads), e = (int)((int64_t)(t + 1) * n / kScanThreads);
  long long c_dec = 0, c_ret = 0, c_done = 0, c_hit = 0;
  int c_rs = 0;
  for (int r = b; r < e; ++r) {
    const int64_t l = k - koff[r];
    const bool done = l >= K;
    const bool at_dec = logits != nullptr && l == k_dec;
    const bool retire = at_dec && logits[r] < theta;
    c_dec += at_dec;
    c_ret += retire;
    c_done += done;
    c_hit += done && fabs(E[r] - E_gs) <= tol;
    c_rs += done || retire;
  }
  s_cnt[t] = c_rs;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // inclusive scan (Hillis-Steele)
    const int v = t >= o ? s_cnt[t - o] : 0;
    __syncthreads();
    s_cnt[t] += v;
    __syncthreads();
  }
  int at = s_cnt[t] - c_rs;  // exclusive prefix
  for (int r = b; r < e; ++r) {
    const int64_t l = k - koff[r];
    const bool restart_r = l >= K || (logits != nullptr && l == k_dec && logits[r] < theta);
    if (restart_r) restart[at++] = r;
  }
  // the other runs after the restarted ones, in increasing order (a full permutation)
  const int total = s_cnt[kScanThreads - 1];
  int keep = total + (b - (s_cnt[t] - c_rs));
  for (int r = b; r < e; ++r) {
    const int64_t l = k - koff[r];
    const bool restart_r = l >= K || (logits != nullptr && l == k_dec && logits[r] < theta);
    if (!restart_r) restart[keep++] = r;
  }
  long long v[5] = {c_dec, c_ret, c_done, c_hit, (long long)c_rs};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    long long x = v[i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((t & 31) == 0) s_sum[i][t >> 5] = x;
  }
  __syncthreads();
  if (t < 5) {
    long long x = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) x += s_sum[t][w];
    counts[t] = x;
  }
}
}  // namespace
}  // namespace chym

extern "C" {

CHYM_API chym_status chym_exit_scan_device(chym_ctx* c, const double* d_E, double E_gs,
                                           const float* d_logits, float theta, int64_t K,
                                           int64_t k_dec, long long* d_counts, int32_t* d_order,
                                           void* stream) {
  if (!c || !d_E || !d_counts || !d_order) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state");
  if (K < 1 || k_dec < 0 || !isfinite(E_gs)) return fail(CHYM_EINVAL, "bad K, k_dec or E_gs");
  const double tol = 1e-9 * fmax(1.0, fabs(E_gs));
  exit_scan_kernel<<<1, kScanThreads, 0, (cudaStream_t)stream>>>(
      c->d_koff, c->n_runs, c->k, d_E, E_gs, tol, d_logits, theta, K, k_dec, d_counts, d_order);
  CHYM_CUDA_TRY(cudaGetLastError());
  return CHYM_OK;
}

CHYM_API chym_status chym_copy_state_device(chym_ctx* c, void* d_dst, void* stream) {
  if (!c || !d_dst) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state");
  const size_t el = c->prec == CHYM_PREC_FP64 ? 8 : 4;
  CHYM_CUDA_TRY(cudaMemcpyAsync(d_dst, c->d_X, el * (size_t)c->n_runs * c->N * c->D,
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return CHYM_OK;
}

CHYM_API chym_status chym_features_device(chym_ctx* c, const void* d_snapshot, double k_frac,
                                          float* d_features, void* stream) {
  chym::TraceRange trace_("chym_features_device");
  if (!c || !d_snapshot || !d_features) return fail(CHYM_EINVAL, "NULL argument");
  if (c->prec < 0) return fail(CHYM_ESTATE, "no state");
  if (c->N > 4096) return fail(CHYM_EINVAL, "features need N <= 4096");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = c->prec == CHYM_PREC_FP64
                      ? launch_features_typed<double>(c, d_snapshot, k_frac, d_features, st)
                      : launch_features_typed<float>(c, d_snapshot, k_frac, d_features, st);
  if (e != cudaSuccess) return cuda_fail(e, "feature kernel");
  return CHYM_OK;
}

CHYM_API chym_status chym_mlp_create(uint64_t seed, int max_batch, chym_mlp** out) {
  if (!out || max_batch < 1) return fail(CHYM_EINVAL, "bad argument");
  chym_mlp* n = new (std::nothrow) chym_mlp();
  if (!n) return fail(CHYM_ENOMEM, "host allocation failed");
  n->max_batch = max_batch;
  const int parts = (max_batch + kGradSamplesPerCta - 1) / kGradSamplesPerCta;
  cudaError_t e = cudaSuccess;
  float** fl[] = {&n->theta, &n->m, &n->v, &n->grad};
  for (float** p : fl)
    if (e == cudaSuccess) e = cudaMalloc((void**)p, sizeof(float) * kP);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->wb, sizeof(__nv_bfloat16) * kP);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->mean, sizeof(float) * kF);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->istd, sizeof(float) * kF);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->partial, sizeof(float) * kP * parts);
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->loss_part, sizeof(float) * parts);
  // Glorot-uniform weights, zero biases, identity standardisation (SplitMix64 stream)
  std::vector<float> th(kP, 0.f), mean(kF, 0.f), istd(kF, 1.f);
  uint64_t z = seed;
  auto unif = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t r = z;
    r = (r ^ (r >> 30)) * 0xBF58476D1CE4E5B9ull;
    r = (r ^ (r >> 27)) * 0x94D049BB133111EBull;
    r ^= r >> 31;
    return (double)(r >> 11) * 0x1.0p-53 * 2.0 - 1.0;
  };
  const double a1 = sqrt(6.0 / (kF + kH)), a2 = sqrt(6.0 / (2 * kH)), a3 = sqrt(6.0 / (kH + 1));
  for (int i = 0; i < kH * kF; ++i) th[oW1 + i] = (float)(a1 * unif());
  for (int i = 0; i < kH * kH; ++i) th[oW2 + i] = (float)(a2 * unif());
  for (int i = 0; i < kH; ++i) th[oW3 + i] = (float)(a3 * unif());
  if (e == cudaSuccess) e = cudaMemcpy(n->theta, th.data(), sizeof(float) * kP, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->mean, mean.data(), sizeof(float) * kF, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(n->istd, istd.data(), sizeof(float) * kF, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * kP);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * kP);
  if (e == cudaSuccess) {
    mlp_refresh_bf16_kernel<<<23, 256>>>(n->theta, n->wb);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    chym_status s = cuda_fail(e, "chym_mlp_create");
    chym_mlp_destroy(n);
    return s;
  }
  *out = n;
  return CHYM_OK;
}

CHYM_API chym_status chym_mlp_destroy(chym_mlp* n) {
  if (!n) return CHYM_OK;
  void* ptrs[] = {n->theta, n->wb, n->m, n->v, n->grad, n->mean, n->istd, n->loss, n->partial, n->loss_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete n;
  return CHYM_OK;
}

CHYM_API chym_status chym_mlp_set_params(chym_mlp* n, const float* theta, const float* mean,
                                         const float* istd) {
  if (!n) return fail(CHYM_EINVAL, "NULL net");
  if (theta) CHYM_CUDA_TRY(cudaMemcpy(n->theta, theta, sizeof(float) * kP, cudaMemcpyHostToDevice));
  if (mean) CHYM_CUDA_TRY(cudaMemcpy(n->mean, mean, sizeof(float) * kF, cudaMemcpyHostToDevice));
  if (istd) CHYM_CUDA_TRY(cudaMemcpy(n->istd, istd, sizeof(float) * kF, cudaMemcpyHostToDevice));
  if (theta) {
    mlp_refresh_bf16_kernel<<<23, 256>>>(n->theta, n->wb);
    CHYM_CUDA_TRY(cudaGetLastError());
    CHYM_CUDA_TRY(cudaMemset(n->m, 0, sizeof(float) * kP));
    CHYM_CUDA_TRY(cudaMemset(n->v, 0, sizeof(float) * kP));
    n->t = 0;
  }
  CHYM_CUDA_TRY(cudaDeviceSynchronize());
  return CHYM_OK;
}

CHYM_API chym_status chym_mlp_get_params(chym_mlp* n, float* theta) {
  if (!n || !theta) return fail(CHYM_EINVAL, "NULL argument");
  CHYM_CUDA_TRY(cudaMemcpy(theta, n->theta, sizeof(float) * kP, cudaMemcpyDeviceToHost));
  return CHYM_OK;
}

CHYM_API chym_status chym_mlp_forward_device(chym_mlp* n, const float* d_F, int B, float* d_logits,
                                             void* stream) {
  chym::TraceRange trace_("chym_mlp_forward_device");
  if (!n || !d_F || !d_logits || B < 0) return fail(CHYM_EINVAL, "bad argument");
  if (B == 0) return CHYM_OK;
  const size_t smem = sizeof(SmemNet) + 8 * sizeof(WarpAct);
  CHYM_CUDA_TRY(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min((B + 7) / 8, 152 * 4);
  mlp_forward_kernel<<<grid, 256, smem, (cudaStream_t)stream>>>(view(n), d_F, B, d_logits);
  CHYM_CUDA_TRY(cudaGetLastError());
  return CHYM_OK;
}

// Gradient of the mean loss over the batch (and optionally one Adam step).
static chym_status mlp_grad_impl(chym_mlp* n, const float* d_F, const float* d_y, int B, float lr,
                                 bool adam, float* d_grad_out, float* d_loss_out, cudaStream_t st) {
  if (!n || !d_F || !d_y || B < 1) return fail(CHYM_EINVAL, "bad argument");
  if (B > n->max_batch) return fail(CHYM_EINVAL, "batch larger than the net's max_batch");
  const int parts = (B + kGradSamplesPerCta - 1) / kGradSamplesPerCta;
  const size_t smem = grad_smem();
  CHYM_CUDA_TRY(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  mlp_grad_kernel<<<parts, kGradWarps * 32, smem, st>>>(view(n), d_F, d_y, B, n->partial, n->loss_part);
  CHYM_CUDA_TRY(cudaGetLastError());
  if (adam) ++n->t;
  mlp_reduce_adam_kernel<<<23, 256, 0, st>>>(n->partial, parts, n->loss_part, n->grad, n->loss, n->theta,
                                             n->m, n->v, n->wb, n->t, lr, adam ? 1 : 0);
  CHYM_CUDA_TRY(cudaGetLastError());
  if (d_grad_out)
    CHYM_CUDA_TRY(cudaMemcpyAsync(d_grad_out, n->grad, sizeof(float) * kP, cudaMemcpyDeviceToDevice, st));
  if (d_loss_out)
    CHYM_CUDA_TRY(cudaMemcpyAsync(d_loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return CHYM_OK;
}

CHYM_API chym_status chym_mlp_grad_device(chym_mlp* n, const float* d_F, const float* d_y, int B,
                                          float* d_grad_out, float* d_loss_out, void* stream) {
  chym::TraceRange trace_("chym_mlp_grad_device");
  return mlp_grad_impl(n, d_F, d_y, B, 0.f, false, d_grad_out, d_loss_out, (cudaStream_t)stream);
}

CHYM_API chym_status chym_mlp_train_step_device(chym_mlp* n, const float* d_F, const float* d_y, int B,
                                                float lr, float* d_loss_out, void* stream) {
  chym::TraceRange trace_("chym_mlp_train_step_device");
  if (!(lr > 0.f)) return fail(CHYM_EINVAL, "lr must be > 0");
  return mlp_grad_impl(n, d_F, d_y, B, lr, true, nullptr, d_loss_out, (cudaStream_t)stream);
}

}  // extern "C"
