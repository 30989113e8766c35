// Chain plates: the autoregressive daily timeseries of App. F's Covid model
// as a plate whose elements are (region, day) pairs, element c T + d.  Day 0
// of a region takes the level's prior given the parent sample; day d >= 1
// takes N(z_{c,d-1}, b I) (b = prior_b).  Every day is its own latent with
// its own sample index, so Eq. mp_iw factorises along the chain, the
// previous day acting as the parent (Sec. 6's recursion):
//   forward (last day first), d >= 1:
//     beta_d[j] = log (1/K) sum_k exp( log N(z_d^k; z_{d-1}^j, b I) + h_d[k] + beta_{d+1}[k] ),
//   day 0, per parent sample p:
//     lt_0[p]   = log (1/K) sum_k exp( log p(z_0^k | z_par^p) + h_0[k] + beta_1[k] ),
//   adjoint (first day first, Eq. mmp with indicator moments):
//     w_0[k] = sum_p w_par[p] exp(S_0[p][k] - lt_0[p] - log K),
//     w_d[k] = sum_j w_{d-1}[j] exp(S_d[j][k] - beta_d[j] - log K).
// h = the relative local factor htil (the sampler's shift joins cst, which
// the plate sum adds for every day).  beta_d accumulates the evidence of all
// later days, so its size grows along the chain; each day's beta is stored
// relative to its maximum over j, the maximum kept in FP64 in the day's off
// (the parent's plate sum adds lt + off + cst of every element, and lt of
// days >= 1 is written 0), so every FP32 argument of an exponential stays near
// zero for the samples that carry weight.  The shifts are constant over each
// day's rows and columns, so the adjoint drops them and renormalises each
// day's weights to sum to one (exact: every row of P(k | j) sums to one).
// One block per region; each row (forward) or sample (adjoint) takes G lanes
// of a warp; a day's samples are staged whole in shared memory; K <= 1024.
#include <math.h>

#include "qem_internal.cuh"

namespace qem {

constexpr int kChainThreadsMax = 1024;

// Block-wide maximum / sum (every thread of the block calls; red holds 32).
__device__ __forceinline__ float chain_block_max(float x, float* red) {
  for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  float r = -INFINITY;
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) r = fmaxf(r, red[w]);
  __syncthreads();
  return r;
}
__device__ __forceinline__ float chain_block_sum(float x, float* red) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) r += red[w];
  __syncthreads();
  return r;
}

// Lanes per row (forward) or per sample (adjoint): G consecutive lanes of a
// warp split one row's columns (one sample's rows) and combine by shuffles,
// so a region's block holds up to 1024 threads (one warp per row would leave
// a scheduler with one warp, exposing every exponential's latency).
__host__ __device__ constexpr int chain_lanes(int K) {
  return K <= 128 ? 8 : K <= 256 ? 4 : K <= 512 ? 2 : 1;
}

template <int MAXD, int G>
__global__ void __launch_bounds__(kChainThreadsMax) k_chain_forward(LevelView v, LevelView par, int K) {
  constexpr int CH = 16;
  extern __shared__ float chain_sm[];
  float* zs = chain_sm;        // [K][MAXD] the day's samples (the columns)
  float* gs = zs + K * MAXD;   // [K]       htil + beta of the next day
  __shared__ float red[32];
  const int T = v.chain, D = v.D;
  const long long e0 = (long long)blockIdx.x * T;
  const long long p = v.parent[e0];
  const float lnK = logf((float)K);
  const float pp_step = -0.5f / v.prior_b;
  const float pc_step = -0.5f * (float)D * logf(6.283185307179586f * v.prior_b);
  const int j = threadIdx.x / G, g = threadIdx.x % G;  // row: sample j of the previous day (day 0: of the parent)
  const bool act = j < K;
  for (int d = T - 1; d >= 0; --d) {
    const long long e = e0 + d;
    __syncthreads();  // the previous day's readers are done; its beta is written
    for (int i = threadIdx.x; i < K * MAXD; i += blockDim.x) {
      const int kk = i / MAXD, dd = i % MAXD;
      zs[i] = dd < D ? v.z[(e * K + kk) * D + dd] : 0.f;
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x)
      gs[i] = v.htil[e * K + i] + (d + 1 < T ? v.beta[(e + 1) * K + i] : 0.f);
    float pm[MAXD], pp[MAXD], pc = 0.f;
#pragma unroll
    for (int dd = 0; dd < MAXD; ++dd) {
      pm[dd] = 0.f;
      pp[dd] = 0.f;
      if (act && dd < D) {
        if (d == 0) {
          pm[dd] = par.pm[(p * K + j) * D + dd];
          pp[dd] = par.pp[(p * K + j) * D + dd];
        } else {
          pm[dd] = v.z[((e - 1) * K + j) * D + dd];
          pp[dd] = pp_step;
        }
      }
    }
    if (act) pc = d == 0 ? par.pc[p * K + j] : pc_step;
    __syncthreads();
    float m = -INFINITY, s = 0.f;
    if (act) {
      for (int k0 = g; k0 < K; k0 += G * CH) {  // columns g, g + G, ...
        float val[CH];
        float cm = -INFINITY;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int k = k0 + c * G;
          float a = -INFINITY;
          if (k < K) {
            float a0 = gs[k], a1 = 0.f;
#pragma unroll
            for (int dd = 0; dd < MAXD; dd += 2) {
              float t0, t1, q0, q1;
              diff2(t0, t1, zs[k * MAXD + dd], zs[k * MAXD + dd + 1], pm[dd], pm[dd + 1]);
              mul2(q0, q1, t0, t1, t0, t1);
              fma2(a0, a1, pp[dd], pp[dd + 1], q0, q1);
            }
            a = a0 + a1;
          }
          val[c] = a;
          cm = fmaxf(cm, a);
        }
        if (cm == -INFINITY) continue;
        if (cm > m) {
          s *= expf(m - cm);
          m = cm;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) s += expf(val[c] - m);
      }
    }
    // the row's G partial sums (lanes of one group, all in one warp)
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const float m2 = __shfl_xor_sync(0xffffffffu, m, o);
      const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const float mm = fmaxf(m, m2);
      if (mm != -INFINITY) {
        s = s * expf(m - mm) + s2 * expf(m2 - mm);
        m = mm;
      }
    }
    const float r = act ? pc + (m + logf(s) - lnK) : -INFINITY;
    if (d > 0) {
      float c = chain_block_max(r, red);
      c = isfinite(c) ? c : 0.f;
      if (act && g == 0) {
        v.beta[e * K + j] = r - c;
        v.lt[e * K + j] = 0.f;
      }
      if (threadIdx.x == 0) v.off[e] = (double)c;
    } else {
      if (act && g == 0) v.lt[e * K + j] = r;
      if (threadIdx.x == 0) v.off[e] = 0.0;
    }
  }
}

template <int MAXD, int G>
__global__ void __launch_bounds__(kChainThreadsMax) k_chain_adjoint(LevelView v, LevelView par, int K) {
  extern __shared__ float chain_sm[];
  float* pms = chain_sm;        // [K][MAXD] row means (the previous day's samples, or the parent's)
  float* pps = pms + K * MAXD;  // [K][MAXD] row -1/(2 var)
  float* cfs = pps + K * MAXD;  // [K]       row coefficients ln w - ln K + pc - normaliser
  __shared__ float red[32];
  const int T = v.chain, D = v.D;
  const long long e0 = (long long)blockIdx.x * T;
  const long long p = v.parent[e0];
  const float lnK = logf((float)K);
  const float pp_step = -0.5f / v.prior_b;
  const float pc_step = -0.5f * (float)D * logf(6.283185307179586f * v.prior_b);
  const int k = threadIdx.x / G, g = threadIdx.x % G;  // sample k of the day; rows g, g + G, ...
  const bool act = k < K;
  for (int d = 0; d < T; ++d) {
    const long long e = e0 + d;
    __syncthreads();  // the previous day's readers are done; its weights are written
    for (int i = threadIdx.x; i < K * MAXD; i += blockDim.x) {
      const int jj = i / MAXD, dd = i % MAXD;
      const bool ok = dd < D;
      if (d == 0) {
        pms[i] = ok ? par.pm[(p * K + jj) * D + dd] : 0.f;
        pps[i] = ok ? par.pp[(p * K + jj) * D + dd] : 0.f;
      } else {
        pms[i] = ok ? v.z[((e - 1) * K + jj) * D + dd] : 0.f;
        pps[i] = ok ? pp_step : 0.f;
      }
    }
    for (int jj = threadIdx.x; jj < K; jj += blockDim.x) {
      const float wj = d == 0 ? par.w[p * K + jj] : v.w[(e - 1) * K + jj];
      cfs[jj] = wj > 0.f ? logf(wj) - lnK + (d == 0 ? par.pc[p * K + jj] - v.lt[e * K + jj]
                                                    : pc_step - v.beta[e * K + jj])
                         : -INFINITY;
    }
    float zr[MAXD];
#pragma unroll
    for (int dd = 0; dd < MAXD; ++dd) zr[dd] = (act && dd < D) ? v.z[(e * K + k) * D + dd] : 0.f;
    const float gk = act ? v.htil[e * K + k] + (d + 1 < T ? v.beta[(e + 1) * K + k] : 0.f) : 0.f;
    __syncthreads();
    float acc = 0.f;
    if (act) {
#pragma unroll 4
      for (int jj = g; jj < K; jj += G) {
        const float c = cfs[jj];
        if (c == -INFINITY) continue;
        float a0 = c + gk, a1 = 0.f;
#pragma unroll
        for (int dd = 0; dd < MAXD; dd += 2) {
          float t0, t1, q0, q1;
          diff2(t0, t1, zr[dd], zr[dd + 1], pms[jj * MAXD + dd], pms[jj * MAXD + dd + 1]);
          mul2(q0, q1, t0, t1, t0, t1);
          fma2(a0, a1, pps[jj * MAXD + dd], pps[jj * MAXD + dd + 1], q0, q1);
        }
        acc += expf(a0 + a1);
      }
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float tot = chain_block_sum(act && g == 0 ? acc : 0.f, red);
    if (act && g == 0) v.w[e * K + k] = tot > 0.f ? acc / tot : 0.f;
  }
}

size_t chain_smem(int D, int K, bool adjoint) {
  const int MAXD = D <= 2 ? 2 : 8;
  return sizeof(float) * (size_t)K * (adjoint ? 2 * MAXD + 1 : MAXD + 1);
}

template <int MAXD, int G>
static cudaError_t chain_cfg(size_t fwd, size_t adj) {
  cudaError_t e = opt_in_smem(k_chain_forward<MAXD, G>, fwd);
  if (e == cudaSuccess) e = opt_in_smem(k_chain_adjoint<MAXD, G>, adj);
  return e;
}

// Opt the chain kernels of (D, K) into their dynamic shared memory (plan time).
cudaError_t configure_chain(int D, int K) {
  if (K > kChainThreadsMax || D > 8) return cudaErrorInvalidValue;
  const size_t f = chain_smem(D, K, false), a = chain_smem(D, K, true);
  const int G = chain_lanes(K);
  if (D <= 2) {
    if (G == 8) return chain_cfg<2, 8>(f, a);
    if (G == 4) return chain_cfg<2, 4>(f, a);
    if (G == 2) return chain_cfg<2, 2>(f, a);
    return chain_cfg<2, 1>(f, a);
  }
  if (G == 8) return chain_cfg<8, 8>(f, a);
  if (G == 4) return chain_cfg<8, 4>(f, a);
  if (G == 2) return chain_cfg<8, 2>(f, a);
  return chain_cfg<8, 1>(f, a);
}

template <int MAXD, int G>
static void chain_launch(bool adjoint, unsigned n_ch, int thr, size_t sm, const LevelView& v, const LevelView& par,
                         int K, cudaStream_t s) {
  if (adjoint)
    k_chain_adjoint<MAXD, G><<<n_ch, thr, sm, s>>>(v, par, K);
  else
    k_chain_forward<MAXD, G><<<n_ch, thr, sm, s>>>(v, par, K);
}

static cudaError_t chain_dispatch(bool adjoint, const LevelView& v, const LevelView& par, int K, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  if (v.chain < 2 || v.n % v.chain || K > kChainThreadsMax || v.D > 8) return cudaErrorInvalidValue;
  const unsigned n_ch = (unsigned)(v.n / v.chain);
  const int G = chain_lanes(K);
  const int thr = ((K * G + 31) / 32) * 32;  // <= 1024 by the choice of G
  const size_t sm = chain_smem(v.D, K, adjoint);
  if (v.D <= 2) {
    if (G == 8) chain_launch<2, 8>(adjoint, n_ch, thr, sm, v, par, K, s);
    else if (G == 4) chain_launch<2, 4>(adjoint, n_ch, thr, sm, v, par, K, s);
    else if (G == 2) chain_launch<2, 2>(adjoint, n_ch, thr, sm, v, par, K, s);
    else chain_launch<2, 1>(adjoint, n_ch, thr, sm, v, par, K, s);
  } else {
    if (G == 8) chain_launch<8, 8>(adjoint, n_ch, thr, sm, v, par, K, s);
    else if (G == 4) chain_launch<8, 4>(adjoint, n_ch, thr, sm, v, par, K, s);
    else if (G == 2) chain_launch<8, 2>(adjoint, n_ch, thr, sm, v, par, K, s);
    else chain_launch<8, 1>(adjoint, n_ch, thr, sm, v, par, K, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_chain_forward(const LevelView& v, const LevelView& par, int K, cudaStream_t s) {
  return chain_dispatch(false, v, par, K, s);
}

cudaError_t launch_chain_adjoint(const LevelView& v, const LevelView& par, int K, cudaStream_t s) {
  return chain_dispatch(true, v, par, K, s);
}

}  // namespace qem
