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
// Arithmetic: every product runs on the tensor cores (mma.sync m16n8k16,
// BF16 operands, FP32 accumulation).  Forward: features, activations and
// weights are rounded to BF16.  Backward: the same rounded activations and
// weights; the FP32 gradients at the layer outputs enter as two BF16 terms
// (hi = bf16(g), lo = bf16(g - hi): 16 mantissa bits), so the backward
// products carry errors ~2^-16 relative to the products of the rounded
// operands.  Bias gradients and the loss are summed from FP32 values.
// Gradients are accumulated per block into the caller's workspace, every
// element by one thread in a fixed order, and reduced over blocks in a fixed
// order, so a step is deterministic.  Adam (Kingma & Ba 2015) updates FP32
// master weights.
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
static_assert(kH == 128 && kIn <= 48 && kOut <= 48, "tile shapes below");
constexpr int kThreads = 256;   // 8 warps
constexpr int kRows = 64;       // users per tile (4 MMA row tiles of 16)
constexpr int kInP = 48;        // inputs padded to 3 k-steps of 16
constexpr int kOutP = 48;       // outputs padded to 6 n-tiles of 8
// shared-memory row strides (BF16 elements): multiples of 8 (16-byte rows for
// ldmatrix) whose 16-byte rows fall in distinct banks for 8 consecutive rows
constexpr int kLdIn = 56;       // rows of kInP (X, W1, the output gradient)
constexpr int kLdH = 136;       // rows of kH

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------- warp-level tensor-core products
__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(s_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
               : "=r"(r[0]), "=r"(r[1]) : "r"(s_addr(p)));
}
// c += a b for one 16x8x16 step (row-major A, column-major B, FP32 C)
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// Fragment of the 16x16 block of A at (m0, k0): A row-major [m][k] (AT
// false) or A = S^T with S row-major [k][m] (AT true); ld in elements.
template <bool AT>
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const bf16* base, int ld, int m0, int k0) {
  const int l = threadIdx.x & 31, q = l >> 3, r = l & 7;
  if (AT)
    ldsm_x4_t(a, base + (k0 + r + ((q & 2) ? 8 : 0)) * ld + m0 + ((q & 1) ? 8 : 0));
  else
    ldsm_x4(a, base + (m0 + r + ((q & 1) ? 8 : 0)) * ld + k0 + ((q & 2) ? 8 : 0));
}
// Fragment of the 16x8 block of B at (k0, n0): B given as Bt row-major [n][k]
// (BT false: a weight matrix W[out][in] for x W^T) or B row-major [k][n] (BT true).
template <bool BT>
__device__ __forceinline__ void load_b(uint32_t (&b)[2], const bf16* base, int ld, int k0, int n0) {
  const int l = threadIdx.x & 31, q = (l >> 3) & 1, r = l & 7;
  if (BT)
    ldsm_x2_t(b, base + (k0 + r + q * 8) * ld + n0);
  else
    ldsm_x2(b, base + (n0 + r) * ld + k0 + q * 8);
}
// acc[j] += A[m0..m0+16)[0..K) B[0..K)[n0+8j..+8) for j < NT
template <int NT, bool AT, bool BT>
__device__ __forceinline__ void warp_gemm(float (&acc)[NT][4], const bf16* A, int lda, int m0, const bf16* B, int ldb,
                                          int n0, int K) {
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    load_a<AT>(a, A, lda, m0, k0);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      uint32_t b[2];
      load_b<BT>(b, B, ldb, k0, n0 + 8 * j);
      mma16816(acc[j], a, b);
    }
  }
}
template <int NT>
__device__ __forceinline__ void zero_acc(float (&acc)[NT][4]) {
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
}
__device__ __forceinline__ void st_bf2(bf16* p, float x, float y) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(x, y);
}

// ---------------------------------------------------------------------------- shared-memory tiles
// Weights as BF16 in their natural [out][in] layout (zero padding), biases FP32.
struct Weights {
  bf16 w1[kH * kLdIn];      // [128][56], inputs 37..55 zero
  bf16 w2[kH * kLdH];       // [128][136]
  bf16 w3[kOutP * kLdH];    // [48][136], outputs 36..47 zero
  float b1[kH], b2[kH], b3[kOutP];
};
struct Acts {
  bf16 x[kRows * kLdIn];    // inputs, BF16, columns 37..55 zero
  bf16 h1[kRows * kLdH];    // BF16 ReLU activations
  bf16 h2[kRows * kLdH];
};
struct Grads {
  float go[kRows * kOutP];      // output, then the loss gradient at it (FP32)
  bf16 go_hi[kRows * kLdIn];    // the output gradient as hi + lo (columns 36..55 zero)
  bf16 go_lo[kRows * kLdIn];
  bf16 g2_hi[kRows * kLdH];     // gradient at layer 2's pre-activation
  bf16 g2_lo[kRows * kLdH];
  bf16 g1_hi[kRows * kLdH];     // gradient at layer 1's pre-activation
  bf16 g1_lo[kRows * kLdH];
  float dbp[4][kH];             // per row tile column sums (bias gradients)
};

__device__ void load_weights(const float* __restrict__ p, Weights& w) {
  for (int i = threadIdx.x; i < kH * kLdIn; i += blockDim.x) {
    const int j = i / kLdIn, k = i % kLdIn;
    w.w1[i] = __float2bfloat16_rn(k < kIn ? p[kOffW1 + j * kIn + k] : 0.f);
  }
  for (int i = threadIdx.x; i < kH * kLdH; i += blockDim.x) {
    const int j = i / kLdH, k = i % kLdH;
    w.w2[i] = __float2bfloat16_rn(k < kH ? p[kOffW2 + j * kH + k] : 0.f);
  }
  for (int i = threadIdx.x; i < kOutP * kLdH; i += blockDim.x) {
    const int j = i / kLdH, k = i % kLdH;
    w.w3[i] = __float2bfloat16_rn(j < kOut && k < kH ? p[kOffW3 + j * kH + k] : 0.f);
  }
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    w.b1[i] = p[kOffB1 + i];
    w.b2[i] = p[kOffB2 + i];
  }
  for (int i = threadIdx.x; i < kOutP; i += blockDim.x) w.b3[i] = i < kOut ? p[kOffB3 + i] : 0.f;
}

__device__ void load_tile(const float* __restrict__ feats, long long row0, int rows, bf16* x) {
  for (int i = threadIdx.x; i < kRows * kLdIn; i += blockDim.x) {
    const int r = i / kLdIn, k = i % kLdIn;
    x[i] = __float2bfloat16_rn(r < rows && k < kIn ? feats[(row0 + r) * kIn + k] : 0.f);
  }
}

// Hidden layer: out = bf16(relu(a W^T + b)), a [64][K] row-major (lda), W [128][K]
// (ldw); warp w computes rows 16 (w % 4) .. +16 and columns 64 (w / 4) .. +64.
__device__ __forceinline__ void hidden_layer(const bf16* a, int lda, int K, const bf16* w, int ldw, const float* b,
                                             bf16* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int m0 = 16 * (warp & 3), n0 = 64 * (warp >> 2);
  float acc[8][4];
  zero_acc(acc);
  warp_gemm<8, false, false>(acc, a, lda, m0, w, ldw, n0, K);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = n0 + 8 * j + 2 * t;
    st_bf2(out + (m0 + g) * kLdH + c, fmaxf(acc[j][0] + b[c], 0.f), fmaxf(acc[j][1] + b[c + 1], 0.f));
    st_bf2(out + (m0 + g + 8) * kLdH + c, fmaxf(acc[j][2] + b[c], 0.f), fmaxf(acc[j][3] + b[c + 1], 0.f));
  }
}

// The three layers of one tile; the output layer's FP32 values (bias added)
// go to emit(row, col, value) for col < kOut.
template <class Emit>
__device__ __forceinline__ void forward_tile(const Weights& w, Acts& s, Emit emit) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  hidden_layer(s.x, kLdIn, kInP, w.w1, kLdIn, w.b1, s.h1);
  __syncthreads();
  hidden_layer(s.h1, kLdH, kH, w.w2, kLdH, w.b2, s.h2);
  __syncthreads();
  const int m0 = 16 * (warp & 3), n0 = 24 * (warp >> 2);
  float acc[3][4];
  zero_acc(acc);
  warp_gemm<3, false, false>(acc, s.h2, kLdH, m0, w.w3, kLdH, n0, kH);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int c = n0 + 8 * j + 2 * t;
    if (c < kOut) {
      emit(m0 + g, c, acc[j][0] + w.b3[c]);
      emit(m0 + g, c + 1, acc[j][1] + w.b3[c + 1]);
      emit(m0 + g + 8, c, acc[j][2] + w.b3[c]);
      emit(m0 + g + 8, c + 1, acc[j][3] + w.b3[c + 1]);
    }
  }
}

// ---------------------------------------------------------------------------- forward
__global__ void __launch_bounds__(kThreads) k_mlp_forward(const float* __restrict__ params,
                                                          const float* __restrict__ feats, long long n,
                                                          float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Weights& w = *reinterpret_cast<Weights*>(smraw);
  Acts& s = *reinterpret_cast<Acts*>(smraw + sizeof(Weights));
  load_weights(params, w);
  for (long long tile = blockIdx.x; tile * kRows < n; tile += gridDim.x) {
    const long long row0 = tile * kRows;
    const int rows = (int)(n - row0 < kRows ? n - row0 : kRows);
    __syncthreads();
    load_tile(feats, row0, rows, s.x);
    __syncthreads();
    forward_tile(w, s, [&](int r, int c, float v) {
      if (r < rows) out[(row0 + r) * kOut + c] = v;
    });
  }
}

// Split v into hi + lo BF16 terms at p_hi / p_lo (two adjacent columns).
__device__ __forceinline__ void st_split2(bf16* hi, bf16* lo, float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  *reinterpret_cast<__nv_bfloat162*>(hi) = h;
  *reinterpret_cast<__nv_bfloat162*>(lo) = __floats2bfloat162_rn(x - __low2float(h), y - __high2float(h));
}

// Gradient at a hidden pre-activation from the next layer's: acc = (g_next W)
// masked by the activation (h > 0), stored as hi + lo; per warp and column,
// the sum over its 16 rows into dbp (the bias gradient, from the FP32 values).
// Warp w: rows 16 (w % 4) .. +16, columns 64 (w / 4) .. +64.
__device__ __forceinline__ void hidden_grad(const bf16* g_hi, const bf16* g_lo, int ldg, int K, const bf16* w,
                                            const bf16* h, bf16* out_hi, bf16* out_lo, float (*dbp)[kH]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt = warp & 3, m0 = 16 * mt, n0 = 64 * (warp >> 2);
  float acc[8][4];
  zero_acc(acc);
  warp_gemm<8, false, true>(acc, g_hi, ldg, m0, w, kLdH, n0, K);
  warp_gemm<8, false, true>(acc, g_lo, ldg, m0, w, kLdH, n0, K);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = n0 + 8 * j + 2 * t;
    const int r0 = (m0 + g) * kLdH + c, r1 = (m0 + g + 8) * kLdH + c;
    const float v0 = __bfloat162float(h[r0]) > 0.f ? acc[j][0] : 0.f;
    const float v1 = __bfloat162float(h[r0 + 1]) > 0.f ? acc[j][1] : 0.f;
    const float v2 = __bfloat162float(h[r1]) > 0.f ? acc[j][2] : 0.f;
    const float v3 = __bfloat162float(h[r1 + 1]) > 0.f ? acc[j][3] : 0.f;
    st_split2(out_hi + r0, out_lo + r0, v0, v1);
    st_split2(out_hi + r1, out_lo + r1, v2, v3);
    float s0 = v0 + v2, s1 = v1 + v3;   // rows g and g + 8 of columns c, c + 1
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (g == 0) {
      dbp[mt][c] = s0;
      dbp[mt][c + 1] = s1;
    }
  }
}

// dW[m][n] += sum_r G[r][m] A[r][n] over the tile's 64 rows, G as hi + lo
// ([64][M], ldg), A [64][N] (lda); warp w takes the MT x NT block of 16 x 8
// tiles at m-tile mt0, n-tile nt0; pg rows of length ldp, valid m < Mv, n < Nv.
template <int NT>
__device__ __forceinline__ void weight_grad(const bf16* g_hi, const bf16* g_lo, int ldg, int m0, const bf16* a,
                                            int lda, int n0, float* pg, int ldp, int Mv, int Nv) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[NT][4];
  zero_acc(acc);
  warp_gemm<NT, true, true>(acc, g_hi, ldg, m0, a, lda, n0, kRows);
  warp_gemm<NT, true, true>(acc, g_lo, ldg, m0, a, lda, n0, kRows);
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int c = n0 + 8 * j + 2 * t;
    const int ra = m0 + g, rb = m0 + g + 8;
    if (ra < Mv) {
      if (c < Nv) pg[ra * ldp + c] += acc[j][0];
      if (c + 1 < Nv) pg[ra * ldp + c + 1] += acc[j][1];
    }
    if (rb < Mv) {
      if (c < Nv) pg[rb * ldp + c] += acc[j][2];
      if (c + 1 < Nv) pg[rb * ldp + c + 1] += acc[j][3];
    }
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
  Acts& s = *reinterpret_cast<Acts*>(smraw + sizeof(Weights));
  Grads& gr = *reinterpret_cast<Grads*>(smraw + sizeof(Weights) + sizeof(Acts));
  __shared__ float red[kThreads / 32];
  const int warp = threadIdx.x >> 5;
  float* pg = part + (long long)blockIdx.x * (kP + 1);
  load_weights(params, w);
  for (int i = threadIdx.x; i <= kP; i += blockDim.x) pg[i] = 0.f;
  // the output gradient's padding columns stay zero
  for (int i = threadIdx.x; i < kRows * kLdIn; i += blockDim.x) {
    gr.go_hi[i] = __float2bfloat16_rn(0.f);
    gr.go_lo[i] = __float2bfloat16_rn(0.f);
  }
  float lacc = 0.f;
  for (long long tile = blockIdx.x; tile * kRows < n; tile += gridDim.x) {
    const long long row0 = tile * kRows;
    const int rows = (int)(n - row0 < kRows ? n - row0 : kRows);
    __syncthreads();
    load_tile(feats, row0, rows, s.x);
    __syncthreads();
    forward_tile(w, s, [&](int r, int c, float v) { gr.go[r * kOutP + c] = v; });
    __syncthreads();
    // loss and its gradient at the output (dimension d owns the pair (mu_d, log sigma_d))
    for (int i = threadIdx.x; i < kRows * kD; i += blockDim.x) {
      const int r = i / kD, d = i % kD;
      float gm = 0.f, gl = 0.f;
      if (r < rows) {
        const float mu = gr.go[r * kOutP + d], ls = gr.go[r * kOutP + kD + d];
        const float m = target[(row0 + r) * kOut + d], sd = target[(row0 + r) * kOut + kD + d];
        const float is2 = expf(-2.f * ls);
        const float q = sd * sd + (m - mu) * (m - mu);
        lacc += ls - logf(sd) + 0.5f * q * is2 - 0.5f;
        gm = (mu - m) * is2 * inv_n;
        gl = (1.f - q * is2) * inv_n;
      }
      gr.go[r * kOutP + d] = gm;
      gr.go[r * kOutP + kD + d] = gl;
      const bf16 hm = __float2bfloat16_rn(gm), hl = __float2bfloat16_rn(gl);
      gr.go_hi[r * kLdIn + d] = hm;
      gr.go_lo[r * kLdIn + d] = __float2bfloat16_rn(gm - __bfloat162float(hm));
      gr.go_hi[r * kLdIn + kD + d] = hl;
      gr.go_lo[r * kLdIn + kD + d] = __float2bfloat16_rn(gl - __bfloat162float(hl));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kOut; j += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < kRows; ++r) acc += gr.go[r * kOutP + j];
      pg[kOffB3 + j] += acc;
    }
    // layer 3: dW3 += go^T h2 (warp w: output rows 0..47, hidden columns 16 w .. +16);
    // g2 = (go W3) * [h2 > 0]
    for (int mt = 0; mt < 3; ++mt)
      weight_grad<2>(gr.go_hi, gr.go_lo, kLdIn, 16 * mt, s.h2, kLdH, 16 * warp, pg + kOffW3, kH, kOut, kH);
    hidden_grad(gr.go_hi, gr.go_lo, kLdIn, kOutP, w.w3, s.h2, gr.g2_hi, gr.g2_lo, gr.dbp);
    __syncthreads();
    for (int j = threadIdx.x; j < kH; j += blockDim.x)
      pg[kOffB2 + j] += (gr.dbp[0][j] + gr.dbp[1][j]) + (gr.dbp[2][j] + gr.dbp[3][j]);
    // layer 2: dW2 += g2^T h1 (warp w: rows 16 w .. +16, all 128 columns); g1 = (g2 W2) * [h1 > 0]
    weight_grad<16>(gr.g2_hi, gr.g2_lo, kLdH, 16 * warp, s.h1, kLdH, 0, pg + kOffW2, kH, kH, kH);
    __syncthreads();   // the bias sums above are read before dbp is rewritten
    hidden_grad(gr.g2_hi, gr.g2_lo, kLdH, kH, w.w2, s.h1, gr.g1_hi, gr.g1_lo, gr.dbp);
    __syncthreads();
    for (int j = threadIdx.x; j < kH; j += blockDim.x)
      pg[kOffB1 + j] += (gr.dbp[0][j] + gr.dbp[1][j]) + (gr.dbp[2][j] + gr.dbp[3][j]);
    // layer 1: dW1 += g1^T x (warp w: rows 16 w .. +16, the 48 padded input columns)
    weight_grad<6>(gr.g1_hi, gr.g1_lo, kLdH, 16 * warp, s.x, kLdIn, 0, pg + kOffW1, kIn, kH, kIn);
  }
  for (int o = 16; o; o >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sum += red[i];
    pg[kP] = sum;
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

constexpr size_t kFwdSmem = sizeof(Weights) + sizeof(Acts);
constexpr size_t kBwdSmem = sizeof(Weights) + sizeof(Acts) + sizeof(Grads);
static_assert(kBwdSmem <= 227 * 1024, "shared memory of the backward kernel");

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
