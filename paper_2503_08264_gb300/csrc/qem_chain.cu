// Chain plates: the autoregressive daily timeseries of App. F's Covid model
// as a plate whose elements are (region, day) pairs, element c T + d.  Day 0
// of a region takes the level's prior given the parent sample; day d >= 1
// takes N(z_{c,d-1}, b I) (b = prior_b).  Every day is its own latent with
// its own sample index, so Eq. mp_iw factorises along the chain, the
// previous day acting as the parent (Sec. 7's recursion):
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
// One block per region, one thread per row (forward) or per sample
// (adjoint), K <= 1024; the column samples stream through shared memory.
#include <math.h>

#include "qem_internal.cuh"

namespace qem {

constexpr int kChainChunk = 32;
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

template <int MAXD>
__global__ void __launch_bounds__(kChainThreadsMax) k_chain_forward(LevelView v, LevelView par, int K) {
  constexpr int CH = MAXD > 2 ? 16 : kChainChunk;  // fits the 64 registers of a 1024-thread block
  __shared__ float zs[CH * MAXD];
  __shared__ float gs[CH];
  __shared__ float red[32];
  const int T = v.chain, D = v.D;
  const long long e0 = (long long)blockIdx.x * T;
  const long long p = v.parent[e0];
  const float lnK = logf((float)K);
  const float pp_step = -0.5f / v.prior_b;
  const float pc_step = -0.5f * (float)D * logf(6.283185307179586f * v.prior_b);
  const int j = threadIdx.x;  // row: sample j of the previous day (day 0: of the parent)
  const bool act = j < K;
  for (int d = T - 1; d >= 0; --d) {
    const long long e = e0 + d;
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
    float m = -INFINITY, s = 0.f;
    for (int k0 = 0; k0 < K; k0 += CH) {
      const int nk = min(CH, K - k0);
      __syncthreads();
      for (int i = threadIdx.x; i < CH * MAXD; i += blockDim.x) {
        const int jj = i / MAXD, dd = i % MAXD;
        zs[i] = (jj < nk && dd < D) ? v.z[(e * K + k0 + jj) * D + dd] : 0.f;
      }
      for (int i = threadIdx.x; i < nk; i += blockDim.x)
        gs[i] = v.htil[e * K + k0 + i] + (d + 1 < T ? v.beta[(e + 1) * K + k0 + i] : 0.f);
      __syncthreads();
      if (!act) continue;
      float val[CH];
      float cm = -INFINITY;
#pragma unroll
      for (int jj = 0; jj < CH; ++jj) {
        float a = -INFINITY;
        if (jj < nk) {
          float a0 = gs[jj], a1 = 0.f;
#pragma unroll
          for (int dd = 0; dd < MAXD; dd += 2) {
            float t0, t1, q0, q1;
            diff2(t0, t1, zs[jj * MAXD + dd], zs[jj * MAXD + dd + 1], pm[dd], pm[dd + 1]);
            mul2(q0, q1, t0, t1, t0, t1);
            fma2(a0, a1, pp[dd], pp[dd + 1], q0, q1);
          }
          a = a0 + a1;
        }
        val[jj] = a;
        cm = fmaxf(cm, a);
      }
      if (cm == -INFINITY) continue;
      if (cm > m) {
        s *= expf(m - cm);
        m = cm;
      }
#pragma unroll
      for (int jj = 0; jj < CH; ++jj) s += expf(val[jj] - m);
    }
    const float r = act ? pc + (m + logf(s) - lnK) : -INFINITY;
    if (d > 0) {
      float c = chain_block_max(r, red);
      c = isfinite(c) ? c : 0.f;
      if (act) {
        v.beta[e * K + j] = r - c;
        v.lt[e * K + j] = 0.f;
      }
      if (threadIdx.x == 0) v.off[e] = (double)c;
    } else {
      if (act) v.lt[e * K + j] = r;
      if (threadIdx.x == 0) v.off[e] = 0.0;
    }
    __syncthreads();  // beta of day d is complete before day d-1 stages it
  }
}

template <int MAXD>
__global__ void __launch_bounds__(kChainThreadsMax) k_chain_adjoint(LevelView v, LevelView par, int K) {
  __shared__ float pms[kChainChunk * MAXD];
  __shared__ float pps[kChainChunk * MAXD];
  __shared__ float cfs[kChainChunk];
  __shared__ float red[32];
  const int T = v.chain, D = v.D;
  const long long e0 = (long long)blockIdx.x * T;
  const long long p = v.parent[e0];
  const float lnK = logf((float)K);
  const float pp_step = -0.5f / v.prior_b;
  const float pc_step = -0.5f * (float)D * logf(6.283185307179586f * v.prior_b);
  const int k = threadIdx.x;  // sample of the current day
  const bool act = k < K;
  for (int d = 0; d < T; ++d) {
    const long long e = e0 + d;
    float zr[MAXD];
#pragma unroll
    for (int dd = 0; dd < MAXD; ++dd) zr[dd] = (act && dd < D) ? v.z[(e * K + k) * D + dd] : 0.f;
    const float gk = act ? v.htil[e * K + k] + (d + 1 < T ? v.beta[(e + 1) * K + k] : 0.f) : 0.f;
    float acc = 0.f;
    for (int j0 = 0; j0 < K; j0 += kChainChunk) {
      const int nj = min(kChainChunk, K - j0);
      __syncthreads();
      for (int i = threadIdx.x; i < kChainChunk * MAXD; i += blockDim.x) {
        const int jj = i / MAXD, dd = i % MAXD;
        const bool ok = jj < nj && dd < D;
        const int j = j0 + jj;
        if (d == 0) {
          pms[i] = ok ? par.pm[(p * K + j) * D + dd] : 0.f;
          pps[i] = ok ? par.pp[(p * K + j) * D + dd] : 0.f;
        } else {
          pms[i] = ok ? v.z[((e - 1) * K + j) * D + dd] : 0.f;
          pps[i] = ok ? pp_step : 0.f;
        }
      }
      for (int jj = threadIdx.x; jj < kChainChunk; jj += blockDim.x) {
        float cf = -INFINITY;
        if (jj < nj) {
          const int j = j0 + jj;
          const float wj = d == 0 ? par.w[p * K + j] : v.w[(e - 1) * K + j];
          if (wj > 0.f)
            cf = logf(wj) - lnK + (d == 0 ? par.pc[p * K + j] - v.lt[e * K + j] : pc_step - v.beta[e * K + j]);
        }
        cfs[jj] = cf;
      }
      __syncthreads();
      if (!act) continue;
#pragma unroll 4
      for (int jj = 0; jj < kChainChunk; ++jj) {
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
    const float tot = chain_block_sum(act ? acc : 0.f, red);
    if (act) v.w[e * K + k] = tot > 0.f ? acc / tot : 0.f;
    __syncthreads();  // day d's weights are complete before day d+1 stages them
  }
}

cudaError_t launch_chain_forward(const LevelView& v, const LevelView& par, int K, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  if (v.chain < 2 || v.n % v.chain || K > kChainThreadsMax || v.D > 8) return cudaErrorInvalidValue;
  const unsigned n_ch = (unsigned)(v.n / v.chain);
  const int thr = ((K + 31) / 32) * 32;
  if (v.D <= 2)
    k_chain_forward<2><<<n_ch, thr, 0, s>>>(v, par, K);
  else
    k_chain_forward<8><<<n_ch, thr, 0, s>>>(v, par, K);
  return cudaGetLastError();
}

cudaError_t launch_chain_adjoint(const LevelView& v, const LevelView& par, int K, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  if (v.chain < 2 || v.n % v.chain || K > kChainThreadsMax || v.D > 8) return cudaErrorInvalidValue;
  const unsigned n_ch = (unsigned)(v.n / v.chain);
  const int thr = ((K + 31) / 32) * 32;
  if (v.D <= 2)
    k_chain_adjoint<2><<<n_ch, thr, 0, s>>>(v, par, K);
  else
    k_chain_adjoint<8><<<n_ch, thr, 0, s>>>(v, par, K);
  return cudaGetLastError();
}

}  // namespace qem
