// Split root: the E-step of a two-level model whose root (mu, psi) -- the
// global mean and log-variance of App. F's MovieLens model -- is two latents
// with their own sample indices instead of one grouped latent.  A user's
// prior factor N(z_m; mu^a, diag exp(psi^b)) then takes two parent indices,
// so the user's factor after summing out its own index is a K x K table
// L_m[a][b] (the K^(number of parents) tables of the Limitations section);
// Eq. mp_iw over all (a, b, k_1, ..., k_M) factorises as
//   A[a][b]  = f_mu[a] + f_psi[b] + sum_m L_m[a][b],
//   log P_MP = log (1/K^2) sum_{a,b} exp A[a][b],
//   W        = softmax(A),  w_mu[a] = sum_b W[a][b],  w_psi[b] = sum_a W[a][b],
//   w_m[k]   = sum_{a,b} W[a][b] exp(S_m[a][b][k] - L_m[a][b] - log K).
// The user-side kernels (forward, plate sums, compaction, adjoint) are the
// grouped path's FP32 kernels in their K^2-row mode (qem_simt.cu); this file
// holds the root-side kernels.
#include <math.h>

#include "qem_internal.cuh"

namespace qem {

// Root factor of each half of every root sample, in FP64:
//   f_mu[i][k]  = sum_{d < D}  [log N(z_d; 0, v) - log N(z_d; loc_d, scale_d^2)],
//   f_psi[i][k] = the same over d in [D, 2D),
// z the root sample (mu^k, psi^k), v the prior variance, (loc, scale) = q.
__global__ void k_split_unary(LevelView r, int K, const float* __restrict__ q, double* fa, double* fb) {
  __shared__ double s_loc[2 * kMaxDim], s_isd[2 * kMaxDim], s_lsd[2 * kMaxDim];
  const long long i = blockIdx.x;
  const int D2 = r.D, D = D2 / 2;
  const double v = (double)r.prior_a;
  for (int d = threadIdx.x; d < D2; d += blockDim.x) {
    const double sd = (double)q[i * 2 * D2 + D2 + d];
    s_loc[d] = (double)q[i * 2 * D2 + d];
    s_isd[d] = 1.0 / sd;
    s_lsd[d] = log(sd);
  }
  __syncthreads();
  const double half_log_v = 0.5 * log(v), inv_v = 1.0 / v;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const float* z = r.z + (i * K + k) * D2;
    double sa = 0.0, sb = 0.0;
    for (int d = 0; d < D2; ++d) {
      const double zd = (double)z[d];
      const double t = (zd - s_loc[d]) * s_isd[d];
      // the 1/2 log 2 pi of the two densities cancel
      const double f = -0.5 * zd * zd * inv_v - half_log_v + 0.5 * t * t + s_lsd[d];
      if (d < D)
        sa += f;
      else
        sb += f;
    }
    fa[i * K + k] = sa;
    fb[i * K + k] = sb;
  }
}

cudaError_t launch_split_unary(const LevelView& root, int K, const float* q, double* fa, double* fb, cudaStream_t s) {
  if (root.n == 0) return cudaSuccess;
  if (root.D > 2 * kMaxDim) return cudaErrorInvalidValue;
  k_split_unary<<<(unsigned)root.n, 128, 0, s>>>(root, K, q, fa, fb);
  return cudaGetLastError();
}

// Root of each instance over the K^2 pairs (FP64 values, FP64 sums):
//   A[a][b] = f_mu[a] + f_psi[b] + H[a K + b],   log P_MP = LSE A - 2 log K,
//   W = exp(A - LSE A) stored as FP32 for the compaction and the adjoint,
//   w_mu[a] = sum_b W[a][b], w_psi[b] = sum_a W[a][b] (FP64 sums of the stored W).
// wab [n][2][K] receives (w_mu, w_psi); w0 [n][K] (the root level's weights) w_mu.
__global__ void k_split_root(int K, const double* __restrict__ fa, const double* __restrict__ fb,
                             const double* __restrict__ hsum, float* W, float* wab, float* w0, double* log_pmp,
                             double* user_out, Ctl* ctl) {
  const long long i = blockIdx.x;
  const int KK = K * K;
  __shared__ double red[32];
  __shared__ double bc;
  auto a_of = [&](int c) -> double { return fa[i * K + c / K] + fb[i * K + c % K] + hsum[i * KK + c]; };
  double mx = -INFINITY;
  for (int c = threadIdx.x; c < KK; c += blockDim.x) mx = fmax(mx, a_of(c));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = -INFINITY;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) m = fmax(m, red[j]);
    bc = isfinite(m) ? m : 0.0;
  }
  __syncthreads();
  const double m = bc;
  double sacc = 0.0;
  for (int c = threadIdx.x; c < KK; c += blockDim.x) sacc += (double)expf((float)(a_of(c) - m));
  for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += red[j];
    const double lse = m + log(t);
    bc = lse;
    const double lp = lse - 2.0 * log((double)K);
    log_pmp[i] = lp;
    if (user_out) user_out[i] = lp;
    if (!isfinite(lp)) atomicOr(&ctl->err, ERR_NUMERIC);
  }
  __syncthreads();
  const double lse = bc;
  for (int c = threadIdx.x; c < KK; c += blockDim.x) W[i * KK + c] = expf((float)(a_of(c) - lse));
  __syncthreads();  // the block's global writes of W are visible to the block after the barrier
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double sa = 0.0, sb = 0.0;
    for (int j = 0; j < K; ++j) {
      sa += (double)W[i * KK + (long long)k * K + j];
      sb += (double)W[i * KK + (long long)j * K + k];
    }
    wab[(i * 2 + 0) * K + k] = (float)sa;
    wab[(i * 2 + 1) * K + k] = (float)sb;
    w0[i * K + k] = (float)sa;
  }
}

cudaError_t launch_split_root(int n_inst, int K, const double* fa, const double* fb, const double* hsum, float* W,
                              float* wab, float* w0, double* log_pmp, double* user_out, Ctl* ctl, cudaStream_t s) {
  if (n_inst == 0) return cudaSuccess;
  k_split_root<<<(unsigned)n_inst, 256, 0, s>>>(K, fa, fb, hsum, W, wab, w0, log_pmp, user_out, ctl);
  return cudaGetLastError();
}

// Moments of the two root halves (Eq. momone(z)): dimension d < D takes the
// mu weights, d >= D the psi weights; (z, z^2) in FP64.  One thread per dimension.
__global__ void k_split_root_moments(LevelView r, int K, const float* __restrict__ wab, double* mom) {
  const long long i = blockIdx.x;
  const int D2 = r.D, D = D2 / 2;
  const int d = threadIdx.x;
  if (d >= D2) return;
  const float* w = wab + (i * 2 + (d < D ? 0 : 1)) * K;
  double s0 = 0.0, s1 = 0.0;
  for (int k = 0; k < K; ++k) {
    const double z = (double)r.z[(i * K + k) * D2 + d];
    const double wk = (double)w[k];
    s0 += wk * z;
    s1 += wk * z * z;
  }
  mom[(i * 2 + 0) * D2 + d] = s0;
  mom[(i * 2 + 1) * D2 + d] = s1;
}

cudaError_t launch_split_root_moments(const LevelView& root, int K, const float* wab, double* mom, cudaStream_t s) {
  if (root.n == 0) return cudaSuccess;
  const int thr = ((root.D + 31) / 32) * 32;
  if (thr > 1024) return cudaErrorInvalidValue;
  k_split_root_moments<<<(unsigned)root.n, thr, 0, s>>>(root, K, wab, mom);
  return cudaGetLastError();
}

}  // namespace qem
