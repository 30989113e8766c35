// FP32 CUDA-core forward contraction of the K_parent x K_child log-factor
// tiles: the log-sum-exp over the child samples (Eq. Prmp).  The kernel
// template is instantiated by two translation units (qem_simt_fwd.cu: latent
// dimensions up to 32, qem_simt_fwd64.cu: up to 64) that compile in parallel.
#pragma once

#include <math.h>

#include "qem_internal.cuh"

namespace qem {

// ---------------------------------------------------------------------------
// K3 (FP32): forward contraction of one plate element (Eq. Prmp summed over
// the child index, Sec. 6):
//   lt[e][kp] = log (1/K) sum_k exp( log p(z_e^k | z_p^kp) + htil[e][k] )
// One thread per parent sample kp; the element's child samples stream
// through shared memory in chunks; online max-shifted sum per row.
// SPLIT: the parent's two halves (mean, log-variance) are separate latents
// with their own sample indices, so a row is a pair kp = a K + b: the
// child-prior mean of parent sample a and the precision and normaliser of
// parent sample b; lt then holds K^2 values per element.
constexpr int kFwdRowsMax = 256;

template <int MAXD, int CHUNK, bool SPLIT>
__global__ void __launch_bounds__(kFwdRowsMax) k_fwd_simt(LevelView v, LevelView par, int K, int n_rt) {
  __shared__ float zs[CHUNK * MAXD];
  __shared__ float hs[CHUNK];
  const int Kp = SPLIT ? K * K : K;  // rows per element
  const long long e = blockIdx.x / n_rt;
  const int kp = (blockIdx.x % n_rt) * blockDim.x + threadIdx.x;
  const int D = v.D;
  const long long p = v.parent[e];
  const bool act = kp < Kp;
  const int ka = SPLIT ? kp / K : kp, kb = SPLIT ? kp % K : kp;
  float pm[MAXD], pp[MAXD], pc = 0.f;
#pragma unroll
  for (int d = 0; d < MAXD; ++d) {
    pm[d] = 0.f;
    pp[d] = 0.f;
    if (act && d < D) {
      pm[d] = par.pm[(p * K + ka) * D + d];
      pp[d] = par.pp[(p * K + kb) * D + d];
    }
  }
  if (act) pc = par.pc[p * K + kb];
  float m = -INFINITY, s = 0.f;
  for (int k0 = 0; k0 < K; k0 += CHUNK) {
    const int nk = min(CHUNK, K - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < CHUNK * MAXD; i += blockDim.x) {
      const int j = i / MAXD, d = i % MAXD;
      zs[i] = (j < nk && d < D) ? v.z[(e * K + k0 + j) * D + d] : 0.f;
    }
    for (int i = threadIdx.x; i < nk; i += blockDim.x) hs[i] = v.htil[e * K + k0 + i];
    __syncthreads();
    if (!act) continue;
    float val[CHUNK];
    float cm = -INFINITY;
#pragma unroll
    for (int j = 0; j < CHUNK; ++j) {
      float a = -INFINITY;
      if (j < nk) {
        // dimensions in pairs (packed FP32): a += pp_d (z_d - pm_d)^2
        float a0 = hs[j], a1 = 0.f;
#pragma unroll
        for (int d = 0; d < MAXD; d += 2) {
          float t0, t1, q0, q1;
          diff2(t0, t1, zs[j * MAXD + d], zs[j * MAXD + d + 1], pm[d], pm[d + 1]);
          mul2(q0, q1, t0, t1, t0, t1);
          fma2(a0, a1, pp[d], pp[d + 1], q0, q1);
        }
        a = a0 + a1;
      }
      val[j] = a;
      cm = fmaxf(cm, a);
    }
    if (cm == -INFINITY) continue;
    if (cm > m) {
      s *= expf(m - cm);
      m = cm;
    }
#pragma unroll
    for (int j = 0; j < CHUNK; ++j) s += expf(val[j] - m);
  }
  if (act) v.lt[e * Kp + kp] = pc + (m + logf(s) - logf((float)K));
}

template <int MAXD, int CHUNK, bool SPLIT>
inline cudaError_t fwd_simt_launch(const LevelView& v, const LevelView& par, int K, int rows, cudaStream_t s) {
  const int Kp = SPLIT ? K * K : K;
  const int thr = Kp >= rows ? rows : ((Kp + 31) / 32) * 32;
  const long long n_rt = (Kp + thr - 1) / thr;
  if (v.n * n_rt > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_fwd_simt<MAXD, CHUNK, SPLIT><<<(unsigned)(v.n * n_rt), thr, 0, s>>>(v, par, K, (int)n_rt);
  return cudaGetLastError();
}

// (the split mode, K^2 rows per element, stages 32 child samples per round
// and takes dimensions up to 32)
template <int MAXD, bool SPLIT>
inline cudaError_t fwd_simt_dispatch(const LevelView& v, const LevelView& par, int K, int rows, int chunk,
                                     cudaStream_t s) {
  if (SPLIT) return fwd_simt_launch<MAXD, 32, SPLIT>(v, par, K, rows, s);
  if (chunk == 16) return fwd_simt_launch<MAXD, 16, SPLIT>(v, par, K, rows, s);
  if (chunk == 64 && MAXD <= 20) return fwd_simt_launch<MAXD, 64, SPLIT>(v, par, K, rows, s);
  return fwd_simt_launch<MAXD, 32, SPLIT>(v, par, K, rows, s);
}

// Dimensions 33..64 of the grouped mode (qem_simt_fwd64.cu).
cudaError_t fwd_simt_d64(const LevelView& v, const LevelView& par, int K, int rows, int chunk, cudaStream_t s);

}  // namespace qem
