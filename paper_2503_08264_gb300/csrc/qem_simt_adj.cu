// FP32 CUDA-core adjoint of the log-factor contraction: the marginal weights
// (Eq. mmp) on the FP32 path and for the small parent sets of the
// mixed-precision paths.
// Kept in a translation unit of its own so that the library's units compile
// in parallel.
#include <math.h>

#include "qem_internal.cuh"

namespace qem {

constexpr int kRowTile = 128;     // rows per block of the FP32 adjoint
constexpr int kChunk = 32;        // staged parent samples of the FP32 adjoint

// ---------------------------------------------------------------------------
// Loads samples [k0, k0+nk) of element e into shared rows of stride D+1
// (coalesced global reads; conflict-free row reads for odd strides).
__device__ __forceinline__ void stage_samples(const LevelView& v, long long e, int K, int k0, int nk, float* zc) {
  const int D = v.D;
  stage_rows<0>(v.z + (e * K + k0) * (long long)D, nk * D, D, zc);
}

// ---------------------------------------------------------------------------
// K5 (FP32): adjoint of the contraction = marginal weights (Eq. mmp with the
// indicator moment; Sec. 3.2's source-term trick in closed form):
//   w_e[k] = sum_kp w_p[kp] exp( S_e[kp][k] - log sum_k' exp S_e[kp][k'] ),
// over the compacted parent samples.  One thread per child sample k; the kept
// parent samples stream through shared memory with the per-(e, kp) shift
// pc[kp] + ln w_p[kp] - ln K - lt[e][kp] folded in.  Elements whose parent
// keeps more than max_eff samples are left to the tensor-core adjoint
// (max_eff = 0: no limit).  SPLIT: the kept parent rows are pairs
// kp = a K + b of a split parent (as in the forward); cidx, cw and lt hold
// K^2 entries per element.  CROSS (parent-conditioned proposals): also
// cz[e][k] = sum_kp w_p[kp] P(k | kp) z_p^kp[0:D], the child-prior mean of
// each kept parent sample being that sample's first D coordinates.
template <int MAXD, bool SPLIT, bool CROSS>
__global__ void __launch_bounds__(kRowTile) k_adj_compact(LevelView v, LevelView par, int K, int n_rt, int max_eff) {
  constexpr int DP = MAXD / 2;       // dimension pairs
  __shared__ float4 pq[kChunk * DP];  // per kept parent sample and pair: (pm_d, pm_d+1, pp_d, pp_d+1)
  __shared__ float pcs[kChunk];
  const long long e = blockIdx.x / n_rt;
  const int k = (blockIdx.x % n_rt) * blockDim.x + threadIdx.x;
  const int D = v.D;
  const long long p = v.parent[e];
  const long long Kp = SPLIT ? (long long)K * K : K;
  const int n_eff = par.ccnt[p];
  if (max_eff > 0 && n_eff > max_eff) return;  // uniform over the block
  const bool act = k < K;
  extern __shared__ float zc[];  // [blockDim][D+1]
  const int k0 = (int)(blockIdx.x % n_rt) * blockDim.x;
  stage_samples(v, e, K, k0, min((int)blockDim.x, K - k0), zc);
  __syncthreads();
  float zr[MAXD];
#pragma unroll
  for (int d = 0; d < MAXD; ++d) zr[d] = (act && d < D) ? zc[threadIdx.x * (D + 1) + d] : 0.f;
  const float hk = act ? v.htil[e * K + k] : 0.f;
  float acc = 0.f;
  float accp[CROSS ? MAXD : 1];
#pragma unroll
  for (int d = 0; d < (CROSS ? MAXD : 1); ++d) accp[d] = 0.f;
  for (int j0 = 0; j0 < n_eff; j0 += kChunk) {
    const int nj = min(kChunk, n_eff - j0);
    __syncthreads();
    for (int i = threadIdx.x; i < kChunk * DP; i += blockDim.x) {
      const int j = i / DP, d = 2 * (i % DP);
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < nj && d < D) {
        const int kp = par.cidx[p * Kp + j0 + j];
        const int ka = SPLIT ? kp / K : kp, kb = SPLIT ? kp % K : kp;
        const float* pm = par.pm + (p * K + ka) * D;
        const float* pp = par.pp + (p * K + kb) * D;
        t.x = pm[d];
        t.z = pp[d];
        if (d + 1 < D) {
          t.y = pm[d + 1];
          t.w = pp[d + 1];
        }
      }
      pq[i] = t;
    }
    for (int j = threadIdx.x; j < kChunk; j += blockDim.x) {
      float sh = -INFINITY;
      if (j < nj) {
        const int kp = par.cidx[p * Kp + j0 + j];
        const int kb = SPLIT ? kp % K : kp;
        sh = par.pc[p * K + kb] + par.cw[p * Kp + j0 + j] - v.lt[e * Kp + kp];
      }
      pcs[j] = sh;
    }
    __syncthreads();
    if (!act) continue;
#pragma unroll 4
    for (int j = 0; j < kChunk; ++j) {
      const float c = pcs[j];
      if (c == -INFINITY) continue;
      // dimensions in pairs (packed FP32, one 16-byte shared load per pair):
      // a += pp_d (z_d - pm_d)^2
      float a0 = c + hk, a1 = 0.f;
#pragma unroll
      for (int dp = 0; dp < DP; ++dp) {
        const float4 t = pq[j * DP + dp];
        float t0, t1, q0, q1;
        diff2(t0, t1, zr[2 * dp], zr[2 * dp + 1], t.x, t.y);
        mul2(q0, q1, t0, t1, t0, t1);
        fma2(a0, a1, t.z, t.w, q0, q1);
      }
      const float term = expf(a0 + a1);
      acc += term;
      if (CROSS) {
#pragma unroll
        for (int dp = 0; dp < DP; ++dp) {
          const float4 t = pq[j * DP + dp];
          accp[2 * dp] = fmaf(term, t.x, accp[2 * dp]);
          accp[2 * dp + 1] = fmaf(term, t.y, accp[2 * dp + 1]);
        }
      }
    }
  }
  if (act) v.w[e * K + k] = acc;
  if (CROSS && act) {
#pragma unroll
    for (int d = 0; d < (CROSS ? MAXD : 1); ++d)
      if (d < D) v.cz[(e * K + k) * D + d] = accp[d];
  }
}

// Small-set adjoint with its own normaliser (used when the forward ran at a
// different precision): one block per element; for each of the <= kSmallKept
// kept parent samples the log-factor of every child sample is evaluated once
// in FP32 (log2 units, kept in shared memory), its row normaliser
// log sum_k exp S[kp][k] is reduced over the block (maximum, then the sum of
// 2^(a - max)), and the marginal weights follow, so every row of P(k | kp)
// sums to one in the arithmetic that evaluates it.  Elements whose parent
// keeps more samples are left to the tensor-core adjoint.
template <int MAXD>
__global__ void __launch_bounds__(256) k_adj_small(LevelView v, LevelView par, int K) {
  extern __shared__ float dyn[];
  float* zc = dyn;                          // [256][D+1] staged samples
  float* av = zc + 256 * (v.D + 1);         // [kSmallKept][K] log-factors (log2 units)
  __shared__ float pms[kSmallKept * MAXD];
  __shared__ float pps[kSmallKept * MAXD];
  __shared__ float pcs[kSmallKept];
  __shared__ float red[kSmallKept][8];
  __shared__ float colmax[kSmallKept];
  __shared__ float shift[kSmallKept];
  constexpr float kL2e = 1.4426950408889634f;
  const long long e = blockIdx.x;
  const int D = v.D;
  const long long p = v.parent[e];
  const int n_eff = par.ccnt[p];
  if (n_eff > kSmallKept) return;
  for (int i = threadIdx.x; i < kSmallKept * MAXD; i += blockDim.x) {
    const int j = i / MAXD, d = i % MAXD;
    const bool ok = j < n_eff && d < D;
    const int kp = ok ? par.cidx[p * K + j] : 0;
    pms[i] = ok ? par.pm[(p * K + kp) * D + d] : 0.f;
    pps[i] = ok ? kL2e * par.pp[(p * K + kp) * D + d] : 0.f;
  }
  if (threadIdx.x < kSmallKept) {
    const int j = threadIdx.x;
    pcs[j] = j < n_eff ? kL2e * par.pc[p * K + par.cidx[p * K + j]] : 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // pass 1: the log-factors of the kept parent samples (log2 units) from
  // samples staged through shared memory, with each thread's running maximum
  // per parent sample
  float mx[kSmallKept];
#pragma unroll
  for (int j = 0; j < kSmallKept; ++j) mx[j] = -INFINITY;
  for (int k0 = 0; k0 < K; k0 += blockDim.x) {
    const int nk = min((int)blockDim.x, K - k0);
    __syncthreads();
    stage_samples(v, e, K, k0, nk, zc);
    __syncthreads();
    if ((int)threadIdx.x >= nk) continue;
    const int k = k0 + threadIdx.x;
    float zr[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) zr[d] = d < D ? zc[threadIdx.x * (D + 1) + d] : 0.f;
    const float hk = kL2e * v.htil[e * K + k];
#pragma unroll
    for (int j = 0; j < kSmallKept; ++j) {
      if (j < n_eff) {
        float a = pcs[j] + hk;
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
          const float t = zr[d] - pms[j * MAXD + d];
          a = fmaf(pps[j * MAXD + d], t * t, a);
        }
        av[j * K + k] = a;
        mx[j] = fmaxf(mx[j], a);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kSmallKept; ++j) {
    float m = mx[j];
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[j][warp] = m;
  }
  __syncthreads();
  if (threadIdx.x < kSmallKept) {
    float m = -INFINITY;
    for (int w = 0; w < nw; ++w) m = fmaxf(m, red[threadIdx.x][w]);
    colmax[threadIdx.x] = isfinite(m) ? m : 0.f;
  }
  __syncthreads();
  // pass 2: row normalisers sum_k 2^(a - max) of each kept parent sample
  float sm[kSmallKept];
#pragma unroll
  for (int j = 0; j < kSmallKept; ++j) sm[j] = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
#pragma unroll
    for (int j = 0; j < kSmallKept; ++j)
      if (j < n_eff) sm[j] += exp2f(av[j * K + k] - colmax[j]);
  }
#pragma unroll
  for (int j = 0; j < kSmallKept; ++j) {
    float t = sm[j];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[j][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < kSmallKept) {
    const int j = threadIdx.x;
    float S = 0.f;
    for (int w = 0; w < nw; ++w) S += red[j][w];
    // log2 w_p - log2 sum_k 2^a[kp][k]   (cw = ln w_p - ln K)
    shift[j] = j < n_eff ? kL2e * (par.cw[p * K + j] + logf((float)K)) - (colmax[j] + log2f(S)) : -INFINITY;
  }
  __syncthreads();
  // pass 3: the marginal weights
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kSmallKept; ++j)
      if (j < n_eff) acc += exp2f(av[j * K + k] + shift[j]);
    v.w[e * K + k] = acc;
  }
}

cudaError_t launch_adj_small(const LevelView& v, const LevelView& par, int K, cudaStream_t s) {
  if (v.n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)v.n;
  const size_t sm = sizeof(float) * (256 * (size_t)(v.D + 1) + (size_t)kSmallKept * K);
  if (v.D <= 4) k_adj_small<4><<<grid, 256, sm, s>>>(v, par, K);
  else if (v.D <= 8) k_adj_small<8><<<grid, 256, sm, s>>>(v, par, K);
  else if (v.D <= 20) k_adj_small<20><<<grid, 256, sm, s>>>(v, par, K);
  else if (v.D <= 32) k_adj_small<32><<<grid, 256, sm, s>>>(v, par, K);
  else k_adj_small<64><<<grid, 256, sm, s>>>(v, par, K);
  return cudaGetLastError();
}

template <int MAXD>
static cudaError_t adj_small_cfg(size_t sm) {
  return opt_in_smem(k_adj_small<MAXD>, sm);
}

cudaError_t configure_adj_small(int D, int K) {
  const size_t sm = sizeof(float) * (256 * (size_t)(D + 1) + (size_t)kSmallKept * K);
  if (sm <= 48 * 1024) return cudaSuccess;
  if (D <= 4) return adj_small_cfg<4>(sm);
  if (D <= 8) return adj_small_cfg<8>(sm);
  if (D <= 20) return adj_small_cfg<20>(sm);
  if (D <= 32) return adj_small_cfg<32>(sm);
  return adj_small_cfg<64>(sm);
}

template <int MAXD, bool SPLIT, bool CROSS = false>
static cudaError_t adj_compact_dispatch(const LevelView& v, const LevelView& par, int K, int max_eff, cudaStream_t s) {
  const int thr = K >= kRowTile ? kRowTile : ((K + 31) / 32) * 32;
  const int n_rt = (K + thr - 1) / thr;
  k_adj_compact<MAXD, SPLIT, CROSS><<<(unsigned)(v.n * n_rt), thr, sizeof(float) * thr * (size_t)(v.D + 1), s>>>(
      v, par, K, n_rt, max_eff);
  return cudaGetLastError();
}

static cudaError_t adj_compact_cross(const LevelView& v, const LevelView& par, int K, int max_eff, cudaStream_t s) {
  if (v.D <= 4) return adj_compact_dispatch<4, false, true>(v, par, K, max_eff, s);
  if (v.D <= 8) return adj_compact_dispatch<8, false, true>(v, par, K, max_eff, s);
  if (v.D <= 20) return adj_compact_dispatch<20, false, true>(v, par, K, max_eff, s);
  if (v.D <= 32) return adj_compact_dispatch<32, false, true>(v, par, K, max_eff, s);
  return cudaErrorInvalidValue;
}

template <bool SPLIT>
static cudaError_t adj_compact_dims(const LevelView& v, const LevelView& par, int K, int max_eff, cudaStream_t s) {
  if (v.D <= 4) return adj_compact_dispatch<4, SPLIT>(v, par, K, max_eff, s);
  if (v.D <= 8) return adj_compact_dispatch<8, SPLIT>(v, par, K, max_eff, s);
  if (v.D <= 20) return adj_compact_dispatch<20, SPLIT>(v, par, K, max_eff, s);
  if (v.D <= 32) return adj_compact_dispatch<32, SPLIT>(v, par, K, max_eff, s);
  if (SPLIT) return cudaErrorInvalidValue;
  return adj_compact_dispatch<SPLIT ? 32 : 64, SPLIT>(v, par, K, max_eff, s);
}

cudaError_t launch_adj_compact(const LevelView& v, const LevelView& par, int K, int max_eff, cudaStream_t s,
                               bool split) {
  if (v.n == 0) return cudaSuccess;
  if (v.qcond) return split ? cudaErrorInvalidValue : adj_compact_cross(v, par, K, max_eff, s);
  return split ? adj_compact_dims<true>(v, par, K, max_eff, s) : adj_compact_dims<false>(v, par, K, max_eff, s);
}

}  // namespace qem
