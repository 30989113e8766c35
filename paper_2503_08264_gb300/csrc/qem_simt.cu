// libqem CUDA-core kernels: sampling and local factors, plate sums, the root,
// compaction, moments and the M-step (the FP32 log-factor contraction and its
// adjoint are in qem_simt_contract.cu).  Every kernel cites the passage of arXiv
// 2503.08264 it realises.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qem_internal.cuh"

namespace qem {

// ---------------------------------------------------------------------------
// Control block kernels (let a captured graph advance the iteration).
__global__ void k_set_ctl(Ctl* ctl, unsigned long long seed, unsigned long long iter, long long t,
                          long long trace_row) {
  ctl->seed = seed;
  ctl->iter = iter;
  ctl->t = t;
  ctl->trace_row = trace_row;
}

__global__ void k_advance_ctl(Ctl* ctl) {
  ctl->iter += 1;
  ctl->t += 1;
  if (ctl->trace_row >= 0) ctl->trace_row += 1;
}

cudaError_t launch_set_ctl(Ctl* ctl, unsigned long long seed, unsigned long long iter, long long t,
                           long long trace_row, cudaStream_t s) {
  k_set_ctl<<<1, 1, 0, s>>>(ctl, seed, iter, t, trace_row);
  return cudaGetLastError();
}

// Device-side iteration loop of qem_run: the body of a conditional (while)
// graph node ends with k_loop_next, which advances the iteration counters
// like k_advance_ctl, counts the iteration off and sets the node's condition;
// the loop also stops once an error bit is set.
__global__ void k_loop_begin(Ctl* ctl, long long iterations) { ctl->remaining = iterations; }

__global__ void k_loop_next(Ctl* ctl, cudaGraphConditionalHandle h) {
  ctl->iter += 1;
  ctl->t += 1;
  if (ctl->trace_row >= 0) ctl->trace_row += 1;
  const long long left = --ctl->remaining;
  cudaGraphSetConditional(h, (left > 0 && ctl->err == 0) ? 1u : 0u);
}

cudaError_t launch_loop_begin(Ctl* ctl, long long iterations, cudaStream_t s) {
  k_loop_begin<<<1, 1, 0, s>>>(ctl, iterations);
  return cudaGetLastError();
}

cudaError_t launch_loop_next(Ctl* ctl, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_loop_next<<<1, 1, 0, s>>>(ctl, h);
  return cudaGetLastError();
}

cudaError_t launch_advance_ctl(Ctl* ctl, long long, cudaStream_t s) {
  k_advance_ctl<<<1, 1, 0, s>>>(ctl);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gamma / Beta draws from noise (Marsaglia & Tsang 2000; Beta = G1/(G1+G2)).
// Accept/reject decisions are taken in FP64.
struct NoiseSrc {
  const float* eps;   // this sample's supplied noise, or nullptr
  unsigned long long seed, iter, sample;
  int level, qfam;
  __device__ float operator()(int idx) const {
    return eps ? eps[idx] : noise_at(seed, iter, level, sample, idx, qfam);
  }
};

__device__ double gamma_variate(double a, const NoiseSrc& ns, int base) {
  const double ab = a < 1.0 ? a + 1.0 : a;
  const double d = ab - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  double g = d;
  for (int t = 0; t < QEM_GAMMA_TRIES; ++t) {
    const double xn = ns(base + 2 * t), u = ns(base + 2 * t + 1);
    double v = 1.0 + c * xn;
    if (v <= 0.0) continue;
    v = v * v * v;
    if (log(u) < 0.5 * xn * xn + d - d * v + d * log(v)) {
      g = d * v;
      break;
    }
  }
  if (a < 1.0) g *= pow((double)ns(base + 2 * QEM_GAMMA_TRIES), 1.0 / a);
  return g;
}

// ---------------------------------------------------------------------------
// K1/K2: draw z ~ Q and evaluate the local factor of every sample
// (Alg. 1 "z ~ Q_t"; the P(x|z)/Q(z) part of r_k in Eq. rmp):
//   loc[e][k] = sum_n log p(y_en | z_e^k, x_en) - log q(z_e^k) (+ log p(z) at level 0),
// split into a sample-dependent FP32 part (loc, centred on its maximum) and a
// sample-independent FP64 part (cst, written by k_elem_const).  Leaf levels:
// one block per element, loc staged in shared memory and centred on its
// maximum before it is written (the contraction reads it in FP32 / BF16).
// Levels with children: their local factor is re-centred in FP64 by
// k_finalize (and the root's is summed in FP64), so no centring is needed and
// the K samples of an element are spread over several blocks (grid.y).
// Covariates in shared memory (rows padded to a multiple of 4 for 16-byte
// loads); each thread keeps its sample in registers; samples are staged
// through shared memory for coalesced stores.  No FP64 arithmetic runs per
// element here: single-lane FP64 work (GB300's FP64 rate is a small fraction
// of FP32) dominated the kernel.
constexpr int kSampleThreadsMax = 256;

// e^x - 1 - x without cancellation: for |x| < 1/2 the series
// x^2 (1/2! + x/3! + ... + x^7/9!) (truncation below 3e-9 relative), beyond
// it expm1(x) - x (no cancellation there: |expm1(x) - x| > 0.1 |x|).
__device__ __forceinline__ float expm1mx(float x) {
  if (fabsf(x) < 0.5f) {
    float p = 1.f / 362880.f;
    p = fmaf(p, x, 1.f / 40320.f);
    p = fmaf(p, x, 1.f / 5040.f);
    p = fmaf(p, x, 1.f / 720.f);
    p = fmaf(p, x, 1.f / 120.f);
    p = fmaf(p, x, 1.f / 24.f);
    p = fmaf(p, x, 1.f / 6.f);
    p = fmaf(p, x, 0.5f);
    return x * x * p;
  }
  return expm1f(x) - x;
}

// Poisson-log reference point s0 of an observation: the per-sample part of
// y s - e^s is then (y - e^s0)(s - s0) - e^s0 (e^(s-s0) - 1 - (s-s0)), and
// y s0 - e^s0 - lgamma(y + 1) joins the element's FP64 constant.  Its
// derivative y - e^s multiplies every rounding of s - s0, so s0 sits where
// the samples are: for Gaussian proposals the centre loc . x of the
// observation (FP64, capped so that e^s0 stays finite); otherwise (parent-
// conditioned or Gamma/Beta proposals) log max(y, 1) in FP32.  e^s0 is
// rounded to FP32 once and the same value enters both parts.  The sampler and
// the per-element constants call these functions, so both sides agree bit
// for bit.
constexpr double kPoisRefMax = 80.0;
__device__ __forceinline__ double loc_dot(const float* loc, const float* x, int D) {
  double c = 0.0;
  for (int d = 0; d < D; ++d) c = fma((double)loc[d], (double)x[d], c);
  return c;
}
__device__ __forceinline__ void pois_ref(float y, float& s0, float& ey0) {
  s0 = logf(fmaxf(y, 1.f));
  ey0 = expf(s0);
}
__device__ __forceinline__ float pois_exp_ref(double s0) { return (float)exp(s0); }

// lgamma(y + 1) of every count y < kCountTable (FP64).
__global__ void k_count_table(double* tab) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= kCountTable) return;
  tab[y] = lgamma((double)y + 1.0);
}

cudaError_t launch_count_table(double* tab, cudaStream_t s) {
  k_count_table<<<(kCountTable + 255) / 256, 256, 0, s>>>(tab);
  return cudaGetLastError();
}

// Sample-independent part of each element's local factor, one thread per
// element, in FP64 (all lanes busy): likelihood normalisers and count terms,
// the -log q normaliser sum_d log sigma_d + D/2 log 2 pi, the root prior's
// normaliser, and the maximum the sampler took out of loc.
__global__ void k_elem_const(LevelView v, const float* __restrict__ q) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= v.n) return;
  const int D = v.D, nobs = v.n_obs;
  const bool rel = v.qfam == QEM_Q_GAUSS && !v.qcond;  // the sampler's relative form
  double c = 0.0;
  for (int n = 0; n < nobs; ++n) {
    const float yv = v.y[e * nobs + n];
    switch (v.lik) {
      case QEM_LIK_GAUSS: c += -0.5 * log(2.0 * 3.141592653589793 * (double)v.lik_var); break;
      case QEM_LIK_POISSON_LOG: {
        const int yi = (int)yv;
        const double lg = (yv >= 0.f && yv < (float)kCountTable && (float)yi == yv && v.ltab)
                              ? v.ltab[yi] : lgamma((double)yv + 1.0);
        if (rel) {
          const double s0 = fmin(loc_dot(q + e * 2 * D, v.x + (e * nobs + n) * D, D), kPoisRefMax);
          c += (double)yv * s0 - (double)pois_exp_ref(s0) - lg;
        } else {
          float s0, ey0;
          pois_ref(yv, s0, ey0);
          c += (double)yv * s0 - (double)ey0 - lg;
        }
        break;
      }
      case QEM_LIK_POISSON_RATE: c += -lgamma((double)yv + 1.0); break;
      default: break;
    }
  }
  if (v.qfam == QEM_Q_GAUSS) {
    const float* sd = q + e * 2 * D + D;
    for (int d = 0; d < D; ++d) c += (double)logf(sd[d]);
    c += 0.5 * D * kLog2PiD;
  }
  if (v.level == 0) {
    const double a0 = v.prior_a, b0 = v.prior_b;
    if (v.prior == QEM_PRIOR_STD_NORMAL) c += -0.5 * D * log(2.0 * 3.141592653589793 * a0);
    if (v.prior == QEM_PRIOR_GAMMA) c += D * (a0 * log(b0) - lgamma(a0));
    if (v.prior == QEM_PRIOR_BETA) c += -D * (lgamma(a0) + lgamma(b0) - lgamma(a0 + b0));
  }
  v.cst[e] = c + (double)v.cshift[e];
}

cudaError_t launch_elem_const(const LevelView& v, const float* q, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  k_elem_const<<<(unsigned)((v.n + 255) / 256), 256, 0, s>>>(v, q);
  return cudaGetLastError();
}

__device__ __forceinline__ float softplusf(float s) { return fmaxf(s, 0.f) + log1p_small(__expf(-fabsf(s))); }

template <int MAXD>
__global__ void __launch_bounds__(kSampleThreadsMax) k_sample_local(LevelView v, int K, int kchunk,
                                                                  const float* __restrict__ q,
                                                                  const float* __restrict__ eps, const Ctl* ctl) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float fred[kSampleThreadsMax / 32];
  const long long e = blockIdx.x;
  const int D = v.D, nobs = v.n_obs, Dp = (D + 3) & ~3, zs_stride = D + 1;
  float* xs = sm;                       // [nobs][Dp]
  float* ys = xs + nobs * Dp;           // [nobs]
  float* s0s = ys + nobs;               // [nobs] reference point of the Poisson-log term
  float* ey0s = s0s + nobs;             // [nobs] exp(s0)
  float* qs = ey0s + nobs;              // [2][D]
  float* zs = qs + 2 * D;               // [blockDim][D+1]
  const bool centre = kchunk >= K;      // one block holds all K samples of the element
  float* ls = zs + blockDim.x * zs_stride;  // [K] loc before centring (centre only)
  for (int i = threadIdx.x; i < nobs * Dp; i += blockDim.x) {
    const int n = i / Dp, d = i % Dp;
    xs[i] = d < D ? v.x[(e * nobs + n) * D + d] : 0.f;
  }
  for (int i = threadIdx.x; i < 2 * D; i += blockDim.x) qs[i] = q[e * 2 * D + i];
  __syncthreads();
  // Gaussian proposals (not parent-conditioned) form s_n = loc . x_n + (scale eps) . x_n
  // with the first term per element in FP64, so the likelihood never sees the
  // FP32 rounding of z = loc + scale eps (a count y multiplies that rounding,
  // ~2^-24 |z|, by y).  s0s[n] holds the FP64 part the per-sample dot adds to:
  // loc . x_n less the Poisson-log reference point, or loc . x_n itself.
  const bool rel = v.qfam == QEM_Q_GAUSS && !v.qcond;
  for (int n = threadIdx.x; n < nobs; n += blockDim.x) {
    const float yv = v.y[e * nobs + n];
    ys[n] = yv;
    if (rel) {
      const double c = loc_dot(qs, xs + n * Dp, D);
      if (v.lik == QEM_LIK_POISSON_LOG) {
        const double s0 = fmin(c, kPoisRefMax);
        s0s[n] = (float)(c - s0);
        ey0s[n] = pois_exp_ref(s0);
      } else {
        s0s[n] = (float)c;
      }
    } else if (v.lik == QEM_LIK_POISSON_LOG) {
      pois_ref(yv, s0s[n], ey0s[n]);
    }
  }
  __syncthreads();
  if (rel) {
    // the per-sample dot then takes eps itself: (scale eps) . x_n = eps . (scale x_n)
    for (int i = threadIdx.x; i < nobs * Dp; i += blockDim.x) {
      const int d = i % Dp;
      if (d < D) xs[i] *= qs[D + d];
    }
    __syncthreads();
  }
  const unsigned long long seed = ctl->seed, iter = ctl->iter;
  const float4* xs4 = reinterpret_cast<const float4*>(xs);
  float lmax = -INFINITY;
  const int kbeg = blockIdx.y * kchunk, kend = min(K, kbeg + kchunk);

  for (int k0 = kbeg; k0 < kend; k0 += blockDim.x) {
    const int nk = min((int)blockDim.x, kend - k0);
    const int k = k0 + threadIdx.x;
    const bool act = threadIdx.x < nk;
    float z[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) z[d] = 0.f;
    if (act) {
      float lq = 0.f;  // sample-dependent part of log q
      if (v.qfam == QEM_Q_GAUSS) {
        if (eps) {
          const float* src = eps + (e * K + k) * (long long)D;
#pragma unroll
          for (int d = 0; d < MAXD; ++d)
            if (d < D) z[d] = src[d];
        } else {
          const unsigned long long sample = (unsigned long long)(e + v.ebase) * K + k;
#pragma unroll
          for (int d0 = 0; d0 < MAXD; d0 += 4) {
            if (d0 < D) {
              const float4 g = normal4(seed, iter, v.level, sample, (uint32_t)(d0 >> 2));
              z[d0] = g.x;
              if (d0 + 1 < MAXD) z[d0 + 1] = d0 + 1 < D ? g.y : 0.f;
              if (d0 + 2 < MAXD) z[d0 + 2] = d0 + 2 < D ? g.z : 0.f;
              if (d0 + 3 < MAXD) z[d0 + 3] = d0 + 3 < D ? g.w : 0.f;
            }
          }
        }
        float ss = 0.f;
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
          if (d < D) {
            const float ep = z[d];
            ss = fmaf(ep, ep, ss);
            if (!rel) z[d] = fmaf(qs[D + d], ep, qs[d]);  // rel: z stays eps until after the likelihood
          }
        }
        if (v.qcond) {
          // parent-conditioned proposal: copy k is centred on the parent's copy perm[k]
          // (clamped: a supplied permutation is caller data)
          const int pk = min(max(v.perm[e * K + k], 0), K - 1);
          const float* zp = v.pz + (v.parent[e] * K + pk) * (long long)v.pD;
#pragma unroll
          for (int d = 0; d < MAXD; ++d)
            if (d < D) z[d] += zp[d];
        }
        lq = -0.5f * ss;
      } else {
        const unsigned long long sample = (unsigned long long)(e + v.ebase) * K + k;
        NoiseSrc ns{eps ? eps + (e * K + k) * (long long)v.nps : nullptr, seed, iter, sample, v.level, v.qfam};
        const int blk = 2 * QEM_GAMMA_TRIES + 1;
        double lqd = 0.0;
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
          if (d < D) {
            const double a = qs[d], b = qs[D + d];
            double zz;
            if (v.qfam == QEM_Q_GAMMA) {
              zz = gamma_variate(a, ns, d * blk) / b;
              lqd += a * log(b) - lgamma(a) + (a - 1.0) * log(zz) - b * zz;
            } else {
              const double g1 = gamma_variate(a, ns, (2 * d) * blk), g2 = gamma_variate(b, ns, (2 * d + 1) * blk);
              zz = g1 / (g1 + g2);
              lqd += (a - 1.0) * log(zz) + (b - 1.0) * log1p(-zz) - (lgamma(a) + lgamma(b) - lgamma(a + b));
            }
            z[d] = (float)zz;
          }
        }
        lq = (float)lqd;
      }
      float ll = 0.f;
      for (int n = 0; n < nobs; ++n) {
        float s = rel ? s0s[n] : 0.f;
#pragma unroll
        for (int d4 = 0; d4 < MAXD / 4; ++d4) {
          if (4 * d4 < Dp) {
            const float4 xv = xs4[n * (Dp >> 2) + d4];
            s = fmaf(z[4 * d4], xv.x, s);
            s = fmaf(z[4 * d4 + 1], xv.y, s);
            s = fmaf(z[4 * d4 + 2], xv.z, s);
            s = fmaf(z[4 * d4 + 3], xv.w, s);
          }
        }
        const float yv = ys[n];
        switch (v.lik) {
          case QEM_LIK_GAUSS: {
            const float r = yv - s;
            ll += -r * r / (2.f * v.lik_var);
            break;
          }
          case QEM_LIK_BERNOULLI_LOGIT: ll += yv * s - softplusf(s); break;
          case QEM_LIK_POISSON_LOG: {
            // y dl - e^s0 expm1(dl) = (y - e^s0) dl - e^s0 (e^dl - 1 - dl): the
            // two large products of the first form (each ~ y |dl|) never appear;
            // dl = s - s0 is the scaled noise's dot (plus a rarely nonzero FP64
            // remainder) when s0 is the proposal centre
            const float dl = rel ? s : s - s0s[n];
            ll += fmaf(yv - ey0s[n], dl, -ey0s[n] * expm1mx(dl));
            break;
          }
          case QEM_LIK_POISSON_RATE: ll += yv * logf(z[0]) - z[0]; break;
          case QEM_LIK_BERNOULLI_PROB: ll += yv * logf(z[0]) + (1.f - yv) * log1pf(-z[0]); break;
          default: break;
        }
      }
      if (rel) {
#pragma unroll
        for (int d = 0; d < MAXD; ++d)
          if (d < D) z[d] = fmaf(qs[D + d], z[d], qs[d]);
      }
      float lp = 0.f;
      if (v.level == 0) {
        if (v.prior == QEM_PRIOR_STD_NORMAL) {
          float ss = 0.f;
#pragma unroll
          for (int d = 0; d < MAXD; ++d) ss = fmaf(z[d], z[d], ss);
          lp = -0.5f * ss / v.prior_a;
        } else if (v.prior == QEM_PRIOR_GAMMA) {
          const double a0 = v.prior_a, b0 = v.prior_b;
          double acc = 0.0;
          for (int d = 0; d < D && d < MAXD; ++d) acc += (a0 - 1.0) * log((double)z[d]) - b0 * z[d];
          lp = (float)acc;
        } else if (v.prior == QEM_PRIOR_BETA) {
          const double a0 = v.prior_a, b0 = v.prior_b;
          double acc = 0.0;
          for (int d = 0; d < D && d < MAXD; ++d)
            acc += (a0 - 1.0) * log((double)z[d]) + (b0 - 1.0) * log1p(-(double)z[d]);
          lp = (float)acc;
        }
      }
      const float lv = ll - lq + lp;
      if (centre)
        ls[k] = lv;
      else
        v.loc[e * K + k] = lv;
      lmax = fmaxf(lmax, lv);
      float* zr = zs + threadIdx.x * zs_stride;
#pragma unroll
      for (int d = 0; d < MAXD; ++d)
        if (d < D) zr[d] = z[d];
    }
    __syncthreads();
    // coalesced store of the block's samples (row and column of element i
    // advanced incrementally: no division per element)
    float* dst = v.z + (e * K + k0) * (long long)D;
    {
      const int step_r = blockDim.x / D, step_c = blockDim.x % D;
      int r = threadIdx.x / D, c = threadIdx.x % D;
      for (int i = threadIdx.x; i < nk * D; i += blockDim.x) {
        dst[i] = zs[r * zs_stride + c];
        r += step_r;
        c += step_c;
        if (c >= D) {
          c -= D;
          ++r;
        }
      }
    }
    __syncthreads();
  }
  if (!centre) {
    if (blockIdx.y == 0 && threadIdx.x == 0) v.cshift[e] = 0.f;
    return;
  }
  // Centre the element's sample-dependent factor on its maximum (the offset
  // joins the FP64 constant), so every later FP32 step works near zero for
  // the samples that carry weight.
  float mx = lmax;
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) fred[threadIdx.x >> 5] = mx;
  __syncthreads();
  float cmax = -INFINITY;
  for (int j = 0; j < (int)(blockDim.x >> 5); ++j) cmax = fmaxf(cmax, fred[j]);
  if (!isfinite(cmax)) cmax = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) v.loc[e * K + k] = ls[k] - cmax;
  if (threadIdx.x == 0) v.cshift[e] = cmax;
}

size_t sample_local_smem(const LevelView& v, int K, int threads) {
  const int Dp = (v.D + 3) & ~3;
  return sizeof(float) * (size_t)(v.n_obs * Dp + 3 * v.n_obs + 2 * v.D + threads * (v.D + 1) + K) + 16;
}

template <int MAXD>
static cudaError_t sample_cfg(size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return opt_in_smem(k_sample_local<MAXD>, smem);
}

cudaError_t configure_sample_local(size_t smem) {
  cudaError_t e = sample_cfg<4>(smem);
  if (e == cudaSuccess) e = sample_cfg<8>(smem);
  if (e == cudaSuccess) e = sample_cfg<12>(smem);
  if (e == cudaSuccess) e = sample_cfg<20>(smem);
  if (e == cudaSuccess) e = sample_cfg<40>(smem);
  if (e == cudaSuccess) e = sample_cfg<64>(smem);
  return e;
}

cudaError_t launch_sample_local(const LevelView& v, int K, int threads, const float* q, const float* eps, const Ctl* ctl,
                                cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  if (threads < 32 || threads > kSampleThreadsMax || threads % 32) return cudaErrorInvalidValue;
  const size_t smem = sample_local_smem(v, K, threads);
  // leaves: one block per element (centred); inner levels: K split over blocks
  const int kchunk = v.Dc == 0 ? K : threads;
  const dim3 grid((unsigned)v.n, (unsigned)((K + kchunk - 1) / kchunk));
  const int Dp = (v.D + 3) & ~3;
  if (Dp <= 4) k_sample_local<4><<<grid, threads, smem, s>>>(v, K, kchunk, q, eps, ctl);
  else if (Dp <= 8) k_sample_local<8><<<grid, threads, smem, s>>>(v, K, kchunk, q, eps, ctl);
  else if (Dp <= 12) k_sample_local<12><<<grid, threads, smem, s>>>(v, K, kchunk, q, eps, ctl);
  else if (Dp <= 20) k_sample_local<20><<<grid, threads, smem, s>>>(v, K, kchunk, q, eps, ctl);
  else if (Dp <= 40) k_sample_local<40><<<grid, threads, smem, s>>>(v, K, kchunk, q, eps, ctl);
  else k_sample_local<64><<<grid, threads, smem, s>>>(v, K, kchunk, q, eps, ctl);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conditional parameters of a child given each parent sample: the child prior
// p(z_c | z_p^kp) = N(mean, diag(1/prec)) written as
//   log p = pc + sum_d pp_d (z_d - pm_d)^2,  pp = -prec/2.
// (App. F: N(z_parent, v I) and N(mu, diag exp(psi)).)
__global__ void k_parent_params(LevelView par, int child_prior, float child_var, int Dc, int K) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // parent sample (p, kp)
  if (i >= par.n * K) return;
  const float* zp = par.z + i * par.D;
  float* pm = par.pm + i * Dc;
  float* pp = par.pp + i * Dc;
  if (child_prior == QEM_PRIOR_NORMAL_FIXED_VAR) {
    for (int d = 0; d < Dc; ++d) {
      pm[d] = zp[d];
      pp[d] = -0.5f / child_var;
    }
    par.pc[i] = -0.5f * Dc * logf(2.f * 3.14159265358979f * child_var);
  } else {
    float c = -0.5f * Dc * kLog2Pi;
    for (int d = 0; d < Dc; ++d) {
      const float lv = zp[Dc + d];
      pm[d] = zp[d];
      pp[d] = -0.5f * expf(-lv);
      c -= 0.5f * lv;
    }
    par.pc[i] = c;
  }
}

cudaError_t launch_parent_params(const LevelView& parent, const LevelView& child, int K, cudaStream_t s) {
  const long long tot = parent.n * K;
  if (tot == 0 || child.n == 0) return cudaSuccess;
  k_parent_params<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(parent, child.prior, child.prior_a, child.D, K);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Relative local factor of an element with children: htil = loc + H - c,
// c = max_k (loc + H)[k] kept in FP64 (off), so the FP32 contraction sees
// values near zero for the samples that matter; c re-enters at the parent's
// plate sum.
__global__ void k_finalize(LevelView v, int K) {
  const long long e = blockIdx.x;
  __shared__ double red[32];
  double mx = -INFINITY;
  for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, (double)v.loc[e * K + k] + v.hsum[e * K + k]);
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const double c = isfinite(red[0]) ? red[0] : 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) v.htil[e * K + k] = (float)((double)v.loc[e * K + k] + (v.hsum[e * K + k] - c));
  if (threadIdx.x == 0) v.off[e] = c;
}

cudaError_t launch_finalize(const LevelView& v, int K, bool has_children, cudaStream_t s) {
  if (v.n == 0 || !has_children) return cudaSuccess;
  k_finalize<<<(unsigned)v.n, 256, 0, s>>>(v, K);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plate sum (Sec. 6: the child's factor enters the parent's as a sum over the
// plate): hsum_p[kp] = sum_{e in children(p)} (lt[e][kp] + off[e] + cst[e]) in
// FP64, in a fixed order (deterministic).  Stage 1 sums chunks of at most 32
// consecutive children into partial[chunk][kp]; stage 2 adds a parent's
// chunks in order.
__global__ void k_plate_partial(LevelView ch, int K) {
  const long long i = blockIdx.x;
  const int kp = blockIdx.y * blockDim.x + threadIdx.x;
  if (kp >= K) return;
  double acc = 0.0;
  for (long long c = ch.chk_beg[i]; c < ch.chk_end[i]; ++c)
    acc += (double)ch.lt[c * K + kp] + (ch.off ? ch.off[c] : 0.0) + ch.cst[c];
  ch.partial[i * K + kp] = acc;
}

__global__ void k_plate_final(LevelView par, LevelView ch, int K) {
  const long long p = blockIdx.x;
  const int kp = blockIdx.y * blockDim.x + threadIdx.x;
  if (kp >= K) return;
  double acc = 0.0;
  for (long long i = par.chk_off[p]; i < par.chk_off[p + 1]; ++i) acc += ch.partial[i * K + kp];
  par.hsum[p * K + kp] = acc;
}

cudaError_t launch_plate_sum(const LevelView& parent, const LevelView& child, int K, cudaStream_t s) {
  if (parent.n == 0) return cudaSuccess;
  const unsigned ky = (unsigned)((K + 255) / 256);
  if (child.n_chunks > 0) k_plate_partial<<<dim3((unsigned)child.n_chunks, ky), 256, 0, s>>>(child, K);
  k_plate_final<<<dim3((unsigned)parent.n, ky), 256, 0, s>>>(parent, child, K);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K4: root of each instance (Eq. Prmp after all children are summed out):
//   a[k] = log p(z_0^k) + log lik - log q + H[k],
//   log P_MP = log (1/K) sum_k exp a[k],   w_0[k] = exp(a[k] - log sum exp a)   (FP64).
__global__ void k_root(LevelView v, int K, int has_children, double* log_pmp, double* user_out, double* trace,
                       Ctl* ctl) {
  const long long i = blockIdx.x;
  __shared__ double red[32];
  __shared__ double bc;
  auto a_of = [&](int k) -> double {
    return (double)v.loc[i * K + k] + v.cst[i] + (has_children ? v.hsum[i * K + k] : 0.0);
  };
  double mx = -INFINITY;
  for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, a_of(k));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = -INFINITY;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) m = fmax(m, red[j]);
    bc = m;
  }
  __syncthreads();
  const double m = bc;
  double sacc = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) sacc += exp(a_of(k) - m);
  for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += red[j];
    const double lse = m + log(t);
    bc = lse;
    const double lp = lse - log((double)K);
    log_pmp[i] = lp;
    if (user_out) user_out[i] = lp;
    if (trace && ctl->trace_row >= 0) trace[ctl->trace_row * gridDim.x + i] = lp;
    if (!isfinite(lp)) atomicOr(&ctl->err, ERR_NUMERIC);
  }
  __syncthreads();
  const double lse = bc;
  for (int k = threadIdx.x; k < K; k += blockDim.x) v.w[i * K + k] = (float)exp(a_of(k) - lse);
}

cudaError_t launch_root(const LevelView& v, int K, bool has_children, double* log_pmp, double* user_out,
                        double* trace, Ctl* ctl, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  k_root<<<(unsigned)v.n, 256, 0, s>>>(v, K, has_children ? 1 : 0, log_pmp, user_out, trace, ctl);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Compaction of the parent samples that carry weight: kept = w_p[kp] >
// rel * max_kp w_p, in index order.  The dropped samples change the marginal
// weights by less than K rel in total (the plan takes rel = 2^-40 for the FP32
// path, ~1e-9 at K = 1024, and 2^-24 for the mixed-precision paths, ~6e-5,
// both below the path's error).  cw = ln w_p - ln Kc of each kept
// sample (Kc = the child's sample count; K = the row length, K^2 for the
// pairs of a split parent); the list is padded to a multiple of 16 with
// cw = -inf.
__global__ void k_compact(LevelView par, int K, int Kc, float rel) {
  const long long p = blockIdx.x;
  __shared__ float red[32];
  __shared__ int scan[1024];
  const float* w = par.w + p * K;
  float mx = 0.f;
  for (int kp = threadIdx.x; kp < K; kp += blockDim.x) mx = fmaxf(mx, w[kp]);
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  float wmax = 0.f;
  for (int j = 0; j < (int)(blockDim.x >> 5); ++j) wmax = fmaxf(wmax, red[j]);
  const float thr = wmax * rel;
  const int per = (K + blockDim.x - 1) / blockDim.x;
  const int k0 = threadIdx.x * per, k1 = min(K, k0 + per);
  int cnt = 0;
  for (int kp = k0; kp < k1; ++kp) cnt += (w[kp] > thr && w[kp] > 0.f) ? 1 : 0;
  scan[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int add = threadIdx.x >= (unsigned)o ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += add;
    __syncthreads();
  }
  int pos = scan[threadIdx.x] - cnt;
  const int total = scan[blockDim.x - 1];
  const float lnK = logf((float)Kc);
  for (int kp = k0; kp < k1; ++kp) {
    if (w[kp] > thr && w[kp] > 0.f) {
      par.cidx[p * K + pos] = kp;
      par.cw[p * K + pos] = logf(w[kp]) - lnK;
      ++pos;
    }
  }
  const int npad = min(K, max(16, (total + 15) & ~15));
  for (int j = total + threadIdx.x; j < npad; j += blockDim.x) {
    par.cidx[p * K + j] = 0;
    par.cw[p * K + j] = -INFINITY;
  }
  if (threadIdx.x == 0) par.ccnt[p] = total;
}

cudaError_t launch_compact(const LevelView& parent, int K, float rel, cudaStream_t s, int Kc) {
  if (parent.n == 0) return cudaSuccess;
  k_compact<<<(unsigned)parent.n, 256, 0, s>>>(parent, K, Kc > 0 ? Kc : K, rel);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K6: moments m_e = sum_k w_e[k] T(z_e^k) (Eq. momone(z)).  Thread t of a
// block owns dimension t % D (consecutive threads read consecutive floats of
// z) and accumulates its share in FP32 with Kahan compensation; the shares of
// a dimension are then combined pairwise in a fixed tree with an error-free
// FP32 sum (TwoSum), so the result carries close to FP64 accuracy without
// per-element FP64 arithmetic (single-lane FP64 loops dominated this kernel).
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
// (s1 - c1) + (s2 - c2) -> (s1 - c1): TwoSum of the leading parts, the
// rounding error joins the compensation.
__device__ __forceinline__ void comp_merge(float& s1, float& c1, float s2, float c2) {
  const float t = s1 + s2;
  const float bp = t - s1;
  const float err = (s1 - (t - bp)) + (s2 - bp);
  s1 = t;
  c1 = (c1 + c2) - err;
}

__global__ void k_moments(LevelView v, int K, double* mom) {
  extern __shared__ float4 smf[];   // per thread: (s0, c0, s1, c1)
  const long long e = blockIdx.x;
  const int D = v.D;
  const int per = blockDim.x / D;
  const int t = threadIdx.x;
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
  if (t < per * D) {
    const int d = t % D;
    int k = t / D;
    // eight samples' loads in flight before their accumulation (the Kahan
    // chain would otherwise wait for every load in turn)
    for (; k + 7 * per < K; k += 8 * per) {
      float wk[8], zv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        wk[u] = v.w[e * K + k + u * per];
        zv[u] = v.z[(e * K + k + u * per) * D + d];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float t0, t1;
        if (v.qfam == QEM_Q_GAUSS) {
          t0 = zv[u];
          t1 = zv[u] * zv[u];
        } else if (v.qfam == QEM_Q_GAMMA) {
          t0 = zv[u];
          t1 = logf(zv[u]);
        } else {
          t0 = logf(zv[u]);
          t1 = log1pf(-zv[u]);
        }
        kahan_add(s0, c0, wk[u] * t0);
        kahan_add(s1, c1, wk[u] * t1);
      }
    }
    for (; k < K; k += per) {
      const float wk = v.w[e * K + k];
      const float zv = v.z[(e * K + k) * D + d];
      float t0, t1;
      if (v.qfam == QEM_Q_GAUSS) {
        t0 = zv;
        t1 = zv * zv;
      } else if (v.qfam == QEM_Q_GAMMA) {
        t0 = zv;
        t1 = logf(zv);
      } else {
        t0 = logf(zv);
        t1 = log1pf(-zv);
      }
      kahan_add(s0, c0, wk * t0);
      kahan_add(s1, c1, wk * t1);
    }
  }
  smf[t] = make_float4(s0, c0, s1, c1);
  __syncthreads();
  // share j of dimension d sits at j * D + d; merge j and j + h for h = 1, 2, 4, ...
  const int j = t / D;
  for (int h = 1; h < per; h <<= 1) {
    if (t < per * D && (j & (2 * h - 1)) == 0 && j + h < per) {
      float4 a = smf[t];
      const float4 b = smf[t + h * D];
      comp_merge(a.x, a.y, b.x, b.y);
      comp_merge(a.z, a.w, b.z, b.w);
      smf[t] = a;
    }
    __syncthreads();
  }
  if (t < D) {
    const float4 a = smf[t];
    mom[(e * 2) * D + t] = (double)a.x - (double)a.y;
    mom[(e * 2 + 1) * D + t] = (double)a.z - (double)a.w;
  }
}

cudaError_t launch_moments(const LevelView& v, int K, int threads, double* mom, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  if (threads < v.D || threads > 1024) threads = v.D > 256 ? v.D : 256;
  const int per = threads / v.D > 0 ? threads / v.D : 1;
  const int thr = per * v.D;
  k_moments<<<(unsigned)v.n, thr, sizeof(float4) * thr, s>>>(v, K, mom);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Special functions for the Gamma/Beta M-steps: digamma and trigamma from
// their recurrences (psi(x) = psi(x+1) - 1/x, psi'(x) = psi'(x+1) + 1/x^2)
// and asymptotic expansions in 1/x^2 with Bernoulli-number coefficients.
// Both are defined here for finite x > 0 only and return NaN otherwise (the
// recurrence would not terminate for x = -inf or x below -2^53).
__device__ double dev_digamma(double x) {
  if (!(x > 0.0) || !isfinite(x)) return nan("");
  double r = 0.0;
  for (; x < 8.0; x += 1.0) r -= 1.0 / x;
  const double x2 = 1.0 / (x * x);
  // -sum B_2n/(2n x^2n): B2/2=1/12, B4/4=-1/120, B6/6=1/252, B8/8=-1/240, B10/10=1/132, B12/12=-691/32760
  const double ser = x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132 - x2 * (691.0 / 32760))))));
  return r + log(x) - 0.5 / x - ser;
}

__device__ double dev_trigamma(double x) {
  if (!(x > 0.0) || !isfinite(x)) return nan("");
  double r = 0.0;
  for (; x < 8.0; x += 1.0) r += 1.0 / (x * x);
  const double x2 = 1.0 / (x * x);
  // 1/x + 1/(2x^2) + sum B_2n / x^(2n+1)
  const double ser = (x2 / x) * (1.0 / 6 - x2 * (1.0 / 30 - x2 * (1.0 / 42 - x2 * (1.0 / 30 - x2 * (5.0 / 66 - x2 * (691.0 / 2730))))));
  return r + 1.0 / x + 0.5 * x2 + ser;
}

// K7: EMA of the mean parameters and the moment-matching M-step (Alg. 1,
// Eq. ema, App. B): Gaussian mean/variance from (E z, E z^2) with a floor;
// Gamma shape from log a - psi(a) = log E z - E log z (Newton from Minka's
// closed-form start), rate = a / E z; Beta from psi(a) - psi(a+b) = E log z,
// psi(b) - psi(a+b) = E log(1-z) (2-D Newton).  Statistics that no Gamma or
// Beta matches (non-finite; E log z >= log E z for the Gamma; e^{E log z} +
// e^{E log(1-z)} >= 1 for the Beta, reachable through rounding when the
// weights collapse) and a Newton run that fails to reach a finite positive
// solution keep the element's previous parameters and raise ERR_NUMERIC;
// every loop is bounded.
__global__ void k_mstep(LevelView v, const double* __restrict__ mom, double* m, float* q, double lambda,
                        double sched_p, double var_floor, long long t_host, Ctl* ctl) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int D = v.D;
  if (i >= v.n * D) return;
  const long long e = i / D;
  const int d = (int)(i % D);
  const long long i0 = (e * 2) * D + d, i1 = (e * 2 + 1) * D + d;
  double m0 = m[i0], m1 = m[i1];
  if (mom) {
    const double tt = (double)(t_host > 0 ? t_host : ctl->t);
    const double lam = sched_p > 0.0 ? pow(tt, -sched_p) : lambda;
    m0 = (1.0 - lam) * m0 + lam * mom[i0];
    m1 = (1.0 - lam) * m1 + lam * mom[i1];
    m[i0] = m0;
    m[i1] = m1;
  }
  double qa, qb;
  if (v.qfam == QEM_Q_GAUSS) {
    double var = m1 - m0 * m0;
    const double fl = var_floor * fmax(1.0, m0 * m0);
    if (!(var > fl)) var = fl;
    qa = m0;
    qb = sqrt(var);
  } else if (v.qfam == QEM_Q_GAMMA) {
    const double s = log(m0) - m1;
    if (!(m0 > 0.0) || !isfinite(m0) || !isfinite(m1) || !(s > 0.0) || !isfinite(s)) {
      atomicOr(&ctl->err, ERR_NUMERIC);
      return;
    }
    double a = (3.0 - s + sqrt((s - 3.0) * (s - 3.0) + 24.0 * s)) / (12.0 * s);
    for (int it = 0; it < 64; ++it) {
      const double step = (log(a) - dev_digamma(a) - s) / (1.0 / a - dev_trigamma(a));
      double an = a - step;
      if (an <= 0.0) an = 0.5 * a;
      const bool done = fabs(an - a) <= 1e-15 * a;
      a = an;
      if (done) break;
    }
    if (!(a > 0.0) || !isfinite(a)) {
      atomicOr(&ctl->err, ERR_NUMERIC);
      return;
    }
    qa = a;
    qb = a / m0;
  } else {
    const double A = exp(m0), B = exp(m1);
    if (!isfinite(m0) || !isfinite(m1) || !(A + B < 1.0)) {
      atomicOr(&ctl->err, ERR_NUMERIC);
      return;
    }
    const double h = 0.5 / (1.0 - A - B);
    double a = 0.5 + A * h, b = 0.5 + B * h;
    bool bad = !(a > 0.0 && b > 0.0 && isfinite(a) && isfinite(b));
    for (int it = 0; it < 128 && !bad; ++it) {
      const double ps = dev_digamma(a + b), ts = dev_trigamma(a + b);
      const double g1 = dev_digamma(a) - ps - m0, g2 = dev_digamma(b) - ps - m1;
      const double h11 = dev_trigamma(a) - ts, h22 = dev_trigamma(b) - ts, h12 = -ts;
      const double det = h11 * h22 - h12 * h12;
      double da = (h22 * g1 - h12 * g2) / det, db = (h11 * g2 - h12 * g1) / det;
      if (!isfinite(da) || !isfinite(db)) {
        bad = true;
        break;
      }
      int halvings = 0;
      while ((a - da <= 0.0 || b - db <= 0.0) && halvings < 64) {
        da *= 0.5;
        db *= 0.5;
        ++halvings;
      }
      if (a - da <= 0.0 || b - db <= 0.0) {
        bad = true;
        break;
      }
      const double rel = fabs(da) / a + fabs(db) / b;
      a -= da;
      b -= db;
      if (rel < 1e-15) break;
    }
    if (bad || !(a > 0.0 && b > 0.0) || !isfinite(a) || !isfinite(b)) {
      atomicOr(&ctl->err, ERR_NUMERIC);
      return;
    }
    qa = a;
    qb = b;
  }
  q[i0] = (float)qa;
  q[i1] = (float)qb;
}

cudaError_t launch_mstep(const LevelView& v, const double* mom, double* m, float* q, double lambda, double sched_p,
                         double var_floor, long long t_host, Ctl* ctl, cudaStream_t s) {
  const long long tot = v.n * v.D;
  if (tot == 0) return cudaSuccess;
  k_mstep<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(v, mom, m, q, lambda, sched_p, var_floor, t_host, ctl);
  return cudaGetLastError();
}

// Mean parameters of proposal parameters (Alg. 1's m_0; App. E's m = (mu, mu^2 + sigma^2)).
__global__ void k_mean_params(LevelView v, const float* __restrict__ q, double* m) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int D = v.D;
  if (i >= v.n * D) return;
  const long long e = i / D;
  const int d = (int)(i % D);
  const long long i0 = (e * 2) * D + d, i1 = (e * 2 + 1) * D + d;
  const double a = q[i0], b = q[i1];
  if (v.qfam == QEM_Q_GAUSS) {
    m[i0] = a;
    m[i1] = a * a + b * b;
  } else if (v.qfam == QEM_Q_GAMMA) {
    m[i0] = a / b;
    m[i1] = dev_digamma(a) - log(b);
  } else {
    m[i0] = dev_digamma(a) - dev_digamma(a + b);
    m[i1] = dev_digamma(b) - dev_digamma(a + b);
  }
}

cudaError_t launch_mean_params(const LevelView& v, const float* q, double* m, cudaStream_t s) {
  const long long tot = v.n * v.D;
  if (tot == 0) return cudaSuccess;
  k_mean_params<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(v, q, m);
  return cudaGetLastError();
}

// Moments of level `lv` rescaled by exp(lp_same - lp_fresh) of their instance
// (the root reached through the parent chain): the self-normalised estimate
// times P_MP(z) / P_MP(z_new), i.e. the moment estimate normalised by a
// second, distinct sample (the remark after Theorem 1).
__global__ void k_moments_rescale(const long long* par1, const long long* par2, const long long* par3, int lv,
                                  long long n, int D, const double* lp_same, const double* lp_fresh, double* mom) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n * 2 * D) return;
  long long e = i / (2 * D);
  if (lv >= 3) e = par3[e];
  if (lv >= 2) e = par2[e];
  if (lv >= 1) e = par1[e];
  mom[i] *= exp(lp_same[e] - lp_fresh[e]);
}

cudaError_t launch_moments_rescale(const LevelView* lvs, int l, const double* lp_same, const double* lp_fresh,
                                   double* mom, cudaStream_t s) {
  const LevelView& v = lvs[l];
  const long long tot = v.n * 2 * v.D;
  if (tot == 0) return cudaSuccess;
  k_moments_rescale<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      l >= 1 ? lvs[1].parent : nullptr, l >= 2 ? lvs[2].parent : nullptr, l >= 3 ? lvs[3].parent : nullptr, l,
      v.n, v.D, lp_same, lp_fresh, mom);
  return cudaGetLastError();
}

// Predictive log-likelihood of held-out observations of each element from
// the last E-step's samples and marginal weights (the paper's diagnostic of
// held-out data):  out[e] = log sum_k w_e[k] prod_n p(y_n | z_e^k, x_n).
// One block per element; FP32 terms with a block-wide max shift.
// ---------------------------------------------------------------------------
// Parent-conditioned proposals (App. A.2, the permutation copy scheme).
// Permutations: per element, the K keys are word (k mod 4) of Philox4x32-10
// with counter (k div 4, e mod 2^32, (e div 2^32) | 2^30, iter) and key seed
// (bit 30 of the third word keeps these counters apart from the noise
// stream's); copies are ordered by (key, k): perm[rank of copy k] = k.  One
// block per element, keys in shared memory, ranks by counting (K^2 / block).
__global__ void k_draw_perm(LevelView v, int K, int* perm, const Ctl* ctl) {
  extern __shared__ uint32_t keys[];
  const long long e = blockIdx.x, ge = e + v.ebase;  // ge: the element's index in the noise streams
  const unsigned long long seed = ctl->seed, iter = ctl->iter;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(k >> 2), (uint32_t)ge, (uint32_t)(ge >> 32) | 0x40000000u,
                                             (uint32_t)iter),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    keys[k] = w[k & 3];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const uint32_t kk = keys[k];
    int rank = 0;
    for (int j = 0; j < K; ++j) {
      const uint32_t kj = keys[j];
      rank += (kj < kk || (kj == kk && j < k)) ? 1 : 0;
    }
    perm[e * K + rank] = k;
  }
}

cudaError_t launch_draw_perm(const LevelView& v, int K, int* perm, const Ctl* ctl, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  if (K > 4096) return cudaErrorInvalidValue;
  k_draw_perm<<<(unsigned)v.n, 256, sizeof(uint32_t) * (size_t)K, s>>>(v, K, perm, ctl);
  return cudaGetLastError();
}

// Residual moments of a qcond level (the Gaussian M-step's statistics of the
// parent-conditioned proposal): with d = z - z_parent[0:D] under the joint
// weights of (parent sample, child sample),
//   E d   = E z - E z_parent,   E d^2 = E z^2 - 2 E[z z_parent] + E z_parent^2,
// E[z z_parent] = sum_k z^k cz^k (cz from the adjoint).  mom holds the level's
// (E z, E z^2) on entry and (E d, E d^2) on exit; FP64 sums.  One block per
// element, one thread per dimension.
__global__ void k_residual_moments(LevelView v, int K, const double* __restrict__ mom_parent, double* mom) {
  const long long e = blockIdx.x;
  const int D = v.D, d = threadIdx.x;
  if (d >= D) return;
  double cross = 0.0;
  for (int k = 0; k < K; ++k) {
    const long long i = (e * K + k) * D + d;
    cross += (double)v.z[i] * (double)v.cz[i];
  }
  const long long p = v.parent[e];
  const double pm1 = mom_parent[(p * 2 + 0) * v.pD + d], pm2 = mom_parent[(p * 2 + 1) * v.pD + d];
  const double m1 = mom[(e * 2 + 0) * D + d], m2 = mom[(e * 2 + 1) * D + d];
  mom[(e * 2 + 0) * D + d] = m1 - pm1;
  mom[(e * 2 + 1) * D + d] = m2 - 2.0 * cross + pm2;
}

cudaError_t launch_residual_moments(const LevelView& v, int K, const double* mom_parent, double* mom, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  const int thr = ((v.D + 31) / 32) * 32;
  k_residual_moments<<<(unsigned)v.n, thr, 0, s>>>(v, K, mom_parent, mom);
  return cudaGetLastError();
}

template <int MAXD>
__global__ void __launch_bounds__(256) k_predictive(LevelView v, int K, const float* __restrict__ xn,
                                                  const float* __restrict__ yn, int nn, double* out) {
  extern __shared__ __align__(16) float psm[];
  __shared__ float red_m[8], red_s[8];
  const long long e = blockIdx.x;
  const int D = v.D;
  float* xs = psm;                 // [nn][D]
  float* ys = xs + nn * D;         // [nn]
  float* cs = ys + nn;             // [nn] per-observation constant
  for (int i = threadIdx.x; i < nn * D; i += blockDim.x) xs[i] = xn ? xn[e * (long long)nn * D + i] : 0.f;
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const float y = yn[e * nn + n];
    ys[n] = y;
    float c = 0.f;
    if (v.lik == QEM_LIK_GAUSS) c = -0.5f * logf(6.283185307179586f * v.lik_var);
    if (v.lik == QEM_LIK_POISSON_LOG || v.lik == QEM_LIK_POISSON_RATE) c = -lgammaf(y + 1.f);
    cs[n] = c;
  }
  __syncthreads();
  float m = -INFINITY, sacc = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float wk = v.w[e * K + k];
    if (!(wk > 0.f)) continue;
    const float* zr = v.z + (e * K + k) * (long long)D;
    float z[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) z[d] = d < D ? zr[d] : 0.f;
    float ll = 0.f;
    for (int n = 0; n < nn; ++n) {
      float sdot = 0.f;
#pragma unroll
      for (int d = 0; d < MAXD; ++d)
        if (d < D) sdot = fmaf(z[d], xs[n * D + d], sdot);
      const float y = ys[n];
      float t = cs[n];
      switch (v.lik) {
        case QEM_LIK_GAUSS: t += -0.5f * (y - sdot) * (y - sdot) / v.lik_var; break;
        case QEM_LIK_BERNOULLI_LOGIT: t += y * sdot - (fmaxf(sdot, 0.f) + log1pf(expf(-fabsf(sdot)))); break;
        case QEM_LIK_POISSON_LOG: t += y * sdot - expf(sdot); break;
        case QEM_LIK_POISSON_RATE: t += y * logf(z[0]) - z[0]; break;
        case QEM_LIK_BERNOULLI_PROB: t += y * logf(z[0]) + (1.f - y) * log1pf(-z[0]); break;
        default: break;
      }
      ll += t;
    }
    const float a = logf(wk) + ll;
    if (a > m) {
      sacc = (m == -INFINITY ? 0.f : sacc * expf(m - a)) + 1.f;
      m = a;
    } else if (a > -INFINITY) {
      sacc += expf(a - m);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int o = 16; o; o >>= 1) {
    const float mo = __shfl_xor_sync(0xffffffffu, m, o), so = __shfl_xor_sync(0xffffffffu, sacc, o);
    const float M = fmaxf(m, mo);
    sacc = (m == -INFINITY ? 0.f : sacc * expf(m - M)) + (mo == -INFINITY ? 0.f : so * expf(mo - M));
    m = M;
  }
  if (lane == 0) {
    red_m[warp] = m;
    red_s[warp] = sacc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float M = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = fmaxf(M, red_m[w]);
    double S = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (red_m[w] > -INFINITY) S += (double)red_s[w] * exp((double)red_m[w] - (double)M);
    out[e] = (double)M + log(S);
  }
}

cudaError_t launch_predictive(const LevelView& v, int K, const float* xn, const float* yn, int nn, double* out,
                              cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  const size_t sm = sizeof(float) * ((size_t)nn * v.D + 2 * (size_t)nn);
  if (sm > 48 * 1024) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)v.n;
  if (v.D <= 4) k_predictive<4><<<g, 256, sm, s>>>(v, K, xn, yn, nn, out);
  else if (v.D <= 8) k_predictive<8><<<g, 256, sm, s>>>(v, K, xn, yn, nn, out);
  else if (v.D <= 20) k_predictive<20><<<g, 256, sm, s>>>(v, K, xn, yn, nn, out);
  else if (v.D <= 40) k_predictive<40><<<g, 256, sm, s>>>(v, K, xn, yn, nn, out);
  else k_predictive<64><<<g, 256, sm, s>>>(v, K, xn, yn, nn, out);
  return cudaGetLastError();
}

}  // namespace qem
