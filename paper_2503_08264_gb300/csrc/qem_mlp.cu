// Learned warm start: a 37-128-128-36 proposal network for the users of the
// hierarchical logistic model (no counterpart in the paper; the amortised
// start of plain QEM).  For a user with items (x_n, y_n), n = 1..N:
//
//   features  f  = [sum_n x_n y_n (D), sum_n x_n (D), sum_n y_n]      (D = 18)
//   network   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3
//   proposal  q  = N(o[:D], diag exp(o[D:])^2)
//   loss      mean over users of KL(N(m, s^2) || q), m and s the user's QEM
//             proposal, summed over dimensions
//
// Arithmetic: the operands of every product (features / activations and
// weights) are rounded to BF16, products accumulate in FP32; the backward
// pass uses the same rounded operands.  Gradients are accumulated per block
// into the caller's workspace and reduced over blocks in a fixed order, so a
// step is deterministic.  Adam (Kingma & Ba 2015) updates FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "qem.h"

namespace {

constexpr int kD = QEM_MLP_DIM;
constexpr int kIn = 2 * kD + 1;
constexpr int kH = QEM_MLP_HIDDEN;
constexpr int kOut = 2 * kD;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH * kIn;
constexpr int kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH;
constexpr int kOffB3 = kOffW3 + kOut * kH;
constexpr int kP = kOffB3 + kOut;
static_assert(kP == QEM_MLP_PARAMS, "parameter count");
constexpr int kThreads = 256;
constexpr int kRows = 32;   // users per tile

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Weights in shared memory as BF16, transposed (wt[k * outs + j] = W[j][k]) so
// that threads of consecutive outputs read consecutive addresses; the
// backward pass also keeps W2 untransposed (w2[j * kH + k]).
struct Weights {
  __nv_bfloat16 w1t[kIn * kH];
  __nv_bfloat16 w2t[kH * kH];
  __nv_bfloat16 w3t[kH * kOut];
  float b1[kH], b2[kH], b3[kOut];
};

__device__ void load_weights(const float* __restrict__ p, Weights& w, __nv_bfloat16* w2 /* nullable */) {
  for (int i = threadIdx.x; i < kH * kIn; i += blockDim.x) {
    const int j = i / kIn, k = i % kIn;
    w.w1t[k * kH + j] = __float2bfloat16_rn(p[kOffW1 + i]);
  }
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    const int j = i / kH, k = i % kH;
    const __nv_bfloat16 v = __float2bfloat16_rn(p[kOffW2 + i]);
    w.w2t[k * kH + j] = v;
    if (w2) w2[i] = v;
  }
  for (int i = threadIdx.x; i < kOut * kH; i += blockDim.x) {
    const int j = i / kH, k = i % kH;
    w.w3t[k * kOut + j] = __float2bfloat16_rn(p[kOffW3 + i]);
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    w.b1[i] = p[kOffB1 + i];
    w.b2[i] = p[kOffB2 + i];
  }
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) w.b3[i] = p[kOffB3 + i];
}

// z[r][j] = sum_k a[r][k] W[j][k] + b[j] for the tile's R rows; hidden layers
// store the BF16-rounded ReLU (the next layer's operand), the output layer z.
template <int IN, int OUTS, bool HIDDEN>
__device__ void dense(const float* a, const __nv_bfloat16* wt, const float* b, float* out) {
  for (int o = threadIdx.x; o < kRows * OUTS; o += blockDim.x) {
    const int r = o / OUTS, j = o % OUTS;
    const float* ar = a + r * IN;
    float acc = 0.f;
#pragma unroll 8
    for (int k = 0; k < IN; ++k) acc = fmaf(ar[k], __bfloat162float(wt[k * OUTS + j]), acc);
    acc += b[j];
    out[o] = HIDDEN ? bf16r(fmaxf(acc, 0.f)) : acc;
  }
}

__device__ void load_tile(const float* __restrict__ feats, long long row0, int rows, float* x) {
  for (int i = threadIdx.x; i < kRows * kIn; i += blockDim.x) {
    const int r = i / kIn;
    x[i] = r < rows ? bf16r(feats[row0 * kIn + i]) : 0.f;
  }
}

// ---------------------------------------------------------------------------- forward
__global__ void __launch_bounds__(kThreads) k_mlp_forward(const float* __restrict__ params,
                                                          const float* __restrict__ feats, long long n,
                                                          float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Weights& w = *reinterpret_cast<Weights*>(smraw);
  float* x = reinterpret_cast<float*>(smraw + sizeof(Weights));
  float* h1 = x + kRows * kIn;
  float* h2 = h1 + kRows * kH;
  float* o = h2 + kRows * kH;
  load_weights(params, w, nullptr);
  for (long long t = blockIdx.x; t * kRows < n; t += gridDim.x) {
    const long long row0 = t * kRows;
    const int rows = (int)(n - row0 < kRows ? n - row0 : kRows);
    __syncthreads();
    load_tile(feats, row0, rows, x);
    __syncthreads();
    dense<kIn, kH, true>(x, w.w1t, w.b1, h1);
    __syncthreads();
    dense<kH, kH, true>(h1, w.w2t, w.b2, h2);
    __syncthreads();
    dense<kH, kOut, false>(h2, w.w3t, w.b3, o);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * kOut; i += blockDim.x) out[row0 * kOut + i] = o[i];
  }
}

// ---------------------------------------------------------------------------- forward + backward
// Block b accumulates its gradient in part[b][0..kP) and its KL sum in
// part[b][kP] (both zeroed by the block first).
__global__ void __launch_bounds__(kThreads) k_mlp_backward(const float* __restrict__ params,
                                                           const float* __restrict__ feats,
                                                           const float* __restrict__ target, long long n,
                                                           float inv_n, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Weights& w = *reinterpret_cast<Weights*>(smraw);
  __nv_bfloat16* w2 = reinterpret_cast<__nv_bfloat16*>(smraw + sizeof(Weights));
  float* x = reinterpret_cast<float*>(smraw + sizeof(Weights) + sizeof(__nv_bfloat16) * kH * kH);
  float* h1 = x + kRows * kIn;
  float* h2 = h1 + kRows * kH;   // reused for the gradient at h1
  float* go = h2 + kRows * kH;   // network output, then the gradient at it
  float* g2 = go + kRows * kOut;
  __shared__ float red[kThreads / 32];
  float* pg = part + (long long)blockIdx.x * (kP + 1);
  load_weights(params, w, w2);
  for (int i = threadIdx.x; i <= kP; i += blockDim.x) pg[i] = 0.f;
  float lacc = 0.f;
  for (long long t = blockIdx.x; t * kRows < n; t += gridDim.x) {
    const long long row0 = t * kRows;
    const int rows = (int)(n - row0 < kRows ? n - row0 : kRows);
    __syncthreads();
    load_tile(feats, row0, rows, x);
    __syncthreads();
    dense<kIn, kH, true>(x, w.w1t, w.b1, h1);
    __syncthreads();
    dense<kH, kH, true>(h1, w.w2t, w.b2, h2);
    __syncthreads();
    dense<kH, kOut, false>(h2, w.w3t, w.b3, go);
    __syncthreads();
    // loss and its gradient at the output (dimension d owns the pair (mu_d, log sigma_d))
    for (int i = threadIdx.x; i < kRows * kD; i += blockDim.x) {
      const int r = i / kD, d = i % kD;
      float gm = 0.f, gl = 0.f;
      if (r < rows) {
        const float mu = go[r * kOut + d], ls = go[r * kOut + kD + d];
        const float m = target[(row0 + r) * kOut + d], s = target[(row0 + r) * kOut + kD + d];
        const float is2 = expf(-2.f * ls);
        const float q = s * s + (m - mu) * (m - mu);
        lacc += ls - logf(s) + 0.5f * q * is2 - 0.5f;
        gm = (mu - m) * is2 * inv_n;
        gl = (1.f - q * is2) * inv_n;
      }
      go[r * kOut + d] = gm;
      go[r * kOut + kD + d] = gl;
    }
    __syncthreads();
    // layer 3: dW3 += go^T h2, db3 += sum go; g2 = (go W3) * [h2 > 0]
    for (int p = threadIdx.x; p < kOut * kH; p += blockDim.x) {
      const int j = p / kH, k = p % kH;
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc = fmaf(go[r * kOut + j], h2[r * kH + k], acc);
      pg[kOffW3 + p] += acc;
    }
    for (int j = threadIdx.x; j < kOut; j += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc += go[r * kOut + j];
      pg[kOffB3 + j] += acc;
    }
    for (int o = threadIdx.x; o < kRows * kH; o += blockDim.x) {
      const int r = o / kH, k = o % kH;
      float acc = 0.f;
      for (int j = 0; j < kOut; ++j) acc = fmaf(go[r * kOut + j], __bfloat162float(w.w3t[k * kOut + j]), acc);
      g2[o] = h2[o] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // layer 2: dW2 += g2^T h1, db2 += sum g2; g1 = (g2 W2) * [h1 > 0] (into h2's buffer)
    for (int p = threadIdx.x; p < kH * kH; p += blockDim.x) {
      const int j = p / kH, k = p % kH;
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc = fmaf(g2[r * kH + j], h1[r * kH + k], acc);
      pg[kOffW2 + p] += acc;
    }
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc += g2[r * kH + j];
      pg[kOffB2 + j] += acc;
    }
    float* g1 = h2;
    for (int o = threadIdx.x; o < kRows * kH; o += blockDim.x) {
      const int r = o / kH, k = o % kH;
      float acc = 0.f;
      for (int j = 0; j < kH; ++j) acc = fmaf(g2[r * kH + j], __bfloat162float(w2[j * kH + k]), acc);
      g1[o] = h1[o] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // layer 1: dW1 += g1^T x, db1 += sum g1
    for (int p = threadIdx.x; p < kH * kIn; p += blockDim.x) {
      const int j = p / kIn, k = p % kIn;
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc = fmaf(g1[r * kH + j], x[r * kIn + k], acc);
      pg[kOffW1 + p] += acc;
    }
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc += g1[r * kH + j];
      pg[kOffB1 + j] += acc;
    }
  }
  for (int o = 16; o; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    pg[kP] = s;
  }
}

// Sum of the blocks' partial gradients in block order (FP64); the loss sum
// divided by n.
__global__ void k_mlp_reduce(const float* __restrict__ part, int blocks, float inv_n, float* __restrict__ grad,
                             double* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kP) return;
  double acc = 0.0;
  for (int b = 0; b < blocks; ++b) acc += (double)part[(long long)b * (kP + 1) + p];
  if (p < kP)
    grad[p] = (float)acc;
  else if (loss)
    *loss = acc * (double)inv_n;
}

__global__ void k_mlp_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_mlp_features(const float* __restrict__ x, const float* __restrict__ y, long long n, int N,
                               float* __restrict__ f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n * kIn) return;
  const long long u = i / kIn;
  const int c = (int)(i % kIn);
  float acc = 0.f;
  for (int t = 0; t < N; ++t) {
    const float yv = y[u * N + t];
    if (c < kD)
      acc += x[(u * N + t) * kD + c] * yv;
    else if (c < 2 * kD)
      acc += x[(u * N + t) * kD + (c - kD)];
    else
      acc += yv;
  }
  f[i] = acc;
}

// q parameters (loc, scale) of each user from the network output; the log
// scale is clamped to [-12, 6] so a poorly trained network cannot produce a
// degenerate proposal.
__global__ void k_mlp_to_q(const float* __restrict__ out, long long n, float* __restrict__ q) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n * kD) return;
  const long long u = i / kD;
  const int d = (int)(i % kD);
  q[(u * 2) * kD + d] = out[u * kOut + d];
  q[(u * 2 + 1) * kD + d] = expf(fminf(fmaxf(out[u * kOut + kD + d], -12.f), 6.f));
}

constexpr size_t kFwdSmem = sizeof(Weights) + sizeof(float) * kRows * (kIn + 2 * kH + kOut);
constexpr size_t kBwdSmem =
    sizeof(Weights) + sizeof(__nv_bfloat16) * kH * kH + sizeof(float) * kRows * (kIn + 3 * kH + kOut);

int blocks_for(long long n) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms < 1)
    sms = 1;
  const long long tiles = (n + kRows - 1) / kRows;
  return (int)(tiles < sms ? (tiles > 0 ? tiles : 1) : sms);
}

qem_status configured() {
  static bool done = false;
  if (done) return QEM_OK;
  if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem) !=
          cudaSuccess)
    return QEM_ERR_CUDA;
  done = true;
  return QEM_OK;
}

}  // namespace

extern "C" {

qem_status qem_mlp_features(const float* x, const float* y, int64_t n, int n_obs, int dim, float* feats,
                            void* stream) {
  if (n < 0 || n_obs < 0 || (n > 0 && (!x || !y || !feats))) return QEM_ERR_INVALID_ARG;
  if (dim != kD) return QEM_ERR_UNSUPPORTED;
  if (n == 0) return QEM_OK;
  const long long tot = n * kIn;
  k_mlp_features<<<(unsigned)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, y, n, n_obs, feats);
  return cudaGetLastError() == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

qem_status qem_mlp_forward(const float* params, const float* feats, int64_t n, float* out, void* stream) {
  if (!params || n < 0 || (n > 0 && (!feats || !out))) return QEM_ERR_INVALID_ARG;
  if (n == 0) return QEM_OK;
  const qem_status st = configured();
  if (st != QEM_OK) return st;
  k_mlp_forward<<<blocks_for(n) * 2, kThreads, kFwdSmem, (cudaStream_t)stream>>>(params, feats, n, out);
  return cudaGetLastError() == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

qem_status qem_mlp_workspace_size(int64_t n, size_t* bytes) {
  if (n < 0 || !bytes) return QEM_ERR_INVALID_ARG;
  *bytes = sizeof(float) * (size_t)blocks_for(n) * (kP + 1);
  return QEM_OK;
}

qem_status qem_mlp_backward(const float* params, const float* feats, const float* target, int64_t n, float* grad,
                            double* loss, void* workspace, void* stream) {
  if (!params || !grad || !workspace || n < 1 || !feats || !target) return QEM_ERR_INVALID_ARG;
  const qem_status st = configured();
  if (st != QEM_OK) return st;
  const int blocks = blocks_for(n);
  const float inv_n = 1.f / (float)n;
  cudaStream_t s = (cudaStream_t)stream;
  float* part = static_cast<float*>(workspace);
  k_mlp_backward<<<blocks, kThreads, kBwdSmem, s>>>(params, feats, target, n, inv_n, part);
  k_mlp_reduce<<<(kP + 1 + 255) / 256, 256, 0, s>>>(part, blocks, inv_n, grad, loss);
  return cudaGetLastError() == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

qem_status qem_mlp_step(float* params, const float* grad, float* m, float* v, int64_t t, double lr, double beta1,
                        double beta2, double eps, void* stream) {
  if (!params || !grad || !m || !v || t < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return QEM_ERR_INVALID_ARG;
  const float c1 = (float)(1.0 - std::pow(beta1, (double)t)), c2 = (float)(1.0 - std::pow(beta2, (double)t));
  k_mlp_adam<<<(kP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, kP, (float)lr, (float)beta1,
                                                                  (float)beta2, (float)eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

qem_status qem_mlp_to_q(const float* out, int64_t n, float* q_params, void* stream) {
  if (n < 0 || (n > 0 && (!out || !q_params))) return QEM_ERR_INVALID_ARG;
  if (n == 0) return QEM_OK;
  const long long tot = n * kD;
  k_mlp_to_q<<<(unsigned)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(out, n, q_params);
  return cudaGetLastError() == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

}  // extern "C"
