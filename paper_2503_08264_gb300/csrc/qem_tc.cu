// Tensor-core (tcgen05) contraction path of libqem for sm_103a.
//
// The K_parent x K_child log-factor tile of one plate element (Eq. rmp; the
// sum over the child index of Eq. Prmp, organised per Sec. 6) is a
// low-rank bilinear form plus row and column terms:
//   S[kp][k] = rowc[kp] + sum_f A[kp][f] B[k][f] + h[k].
// The bilinear part and the column term run on the 5th-generation tensor
// cores (BF16 operands, FP32 accumulation in TMEM); FP32 rounding is recovered
// with a split-BF16 representation (x = hi + lo, products hi*hi + hi*lo +
// lo*hi) and a three-way split of h.  All values are pre-scaled by log2(e) so
// the epilogue applies ex2 directly.
//   forward : lt[e][kp] = rowc[kp] + ln 2 * log2 sum_k 2^(A B^T + h)[kp][k] - ln K   (online max shift)
//   adjoint : w[e][k]   = sum_kp 2^(B A^T + h + d)[k][kp],  d = log2 e (rowc + ln w_p - lt - ln K)
// The adjoint runs over the parent samples with non-negligible weight only
// (compacted list; the dropped terms are below 2^-40 of the largest weight).
//
// Operand layout: the canonical K-major no-swizzle layout of tcgen05
// (8 x 8 bf16 core matrices of 128 contiguous bytes, core matrices of a row
// group consecutive along K).  Features are written to global memory in that
// layout, so every operand tile is one contiguous bulk copy.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "qem_tc.cuh"
#include "qem_tc_ptx.cuh"

namespace qem {

namespace tc {

// ---------------------------------------------------------------------------- feature builders
// Parent side (A rows of the forward tile, B columns of the adjoint): for each
// parent sample kp, with the children's prior written as
//   log p(z | kp) = pc + sum_d pp_d (z_d - pm_d)^2
// and a per-parent centre c (mean of pm over kp; z' = z - c, pm' = pm - c):
//   mean/log-variance prior: A = log2e [pp_d, -2 pp_d pm'_d],  B = [z'^2, z']
//   fixed-variance prior:    A = log2e [-2 pp pm'_d],          B = [z']      (pp z'^2 joins h)
//   rowc = pc + sum_d pp_d pm'_d^2.
// Row of fk columns: split 3: [Ah | 1 1 1 | Ah | Al | 0..], split 1: [Ah | 1 1 1 | 0..].
__global__ void k_parent_features(LevelView par, int Dc, int mean_logvar, int K, int fk, int nb, int split,
                                  int a_ah2, int a_al, int a_alt, int tail, __nv_bfloat16* afeat, float* rowc,
                                  float* center) {
  const long long p = blockIdx.x;
  __shared__ float cen[kMaxDim];
  __shared__ float red[8][kMaxDim];
  // centre: mean over the parent samples of the children's prior mean
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = 0; d < Dc; ++d) {
      float acc = 0.f;
      for (int kp = threadIdx.x; kp < K; kp += blockDim.x) acc += par.pm[(p * K + kp) * Dc + d];
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) red[warp][d] = acc;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < Dc; d += blockDim.x) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][d];
      cen[d] = t / K;
      center[p * Dc + d] = cen[d];
    }
    __syncthreads();
  }
  for (int kp = blockIdx.y * blockDim.x + threadIdx.x; kp < K; kp += gridDim.y * blockDim.x) {
    const float* pm = par.pm + (p * K + kp) * Dc;
    const float* pp = par.pp + (p * K + kp) * Dc;
    double rc = par.pc[p * K + kp];
    for (int d = 0; d < Dc; ++d) {
      const float dm = pm[d] - cen[d];
      rc += (double)pp[d] * dm * dm;
    }
    if (blockIdx.z == 0) rowc[p * K + kp] = (float)rc;
    __nv_bfloat16* row = afeat + p * (long long)K * fk;
    for (int c0 = 0; c0 < fk; c0 += 8) {
      __align__(16) __nv_bfloat16 g[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + j;
        int f = -1, part = 0;  // part: 0 = hi, 1 = lo
        if (c < nb) f = c;
        else if (c < nb + 3) { g[j] = __float2bfloat16_rn(1.f); continue; }
        else if (split == 3 && c >= a_ah2 && c < a_ah2 + nb) f = c - a_ah2;
        else if (split == 3 && tail > 0 && c >= a_alt && c < a_alt + tail) { f = nb - tail + (c - a_alt); part = 1; }
        else if (split == 3 && c >= a_al && c < a_al + nb - tail) { f = c - a_al; part = 1; }
        if (f >= 0) {
          float a = mean_logvar ? (f < Dc ? pp[f] : -2.f * pp[f - Dc] * (pm[f - Dc] - cen[f - Dc]))
                                : -2.f * pp[f] * (pm[f] - cen[f]);
          a *= kLog2e;
          __nv_bfloat16 hi, lo;
          split2(a, hi, lo);
          g[j] = part == 0 ? hi : lo;
        } else {
          g[j] = __float2bfloat16_rn(0.f);
        }
      }
      *reinterpret_cast<uint4*>(row + canon(kp, c0, fk)) = *reinterpret_cast<const uint4*>(g);
    }
  }
}

// Child side: B row of sample k of element e: split 3: [Bh | h1 h2 h3 | Bl | Bh | 0..],
// split 1: [Bh | h1 h2 h3 | 0..], with h = log2e (htil + [fixed-variance] pp sum z'^2).
// Samples are staged through shared memory (coalesced loads); each thread
// builds the B features of one sample into its own shared row, then writes
// the row as 16-byte granules of the canonical layout.
__global__ void __launch_bounds__(128) k_child_features(LevelView ch, int mean_logvar, float pp_fixed, int K, int fk,
                                                        int nb, int split, int b_bl, int b_bh2, int b_bht, int tail,
                                                        const float* center, __nv_bfloat16* bfeat) {
  extern __shared__ float csm[];
  const long long e = blockIdx.x;
  const int D = ch.D, zst = D + 1, bst = nb + 1;
  const long long p = ch.parent[e];
  float* cen = csm;                      // [D]
  float* zc = cen + D;                   // [128][D+1]
  float* bf = zc + 128 * zst;            // [128][nb+1] B feature values
  float* hs = bf + 128 * bst;            // [128] h (log2 units)
  for (int d = threadIdx.x; d < D; d += blockDim.x) cen[d] = center[p * D + d];
  __nv_bfloat16* out = bfeat + e * (long long)K * fk;
  for (int k0 = 0; k0 < K; k0 += blockDim.x) {
    const int nk = min((int)blockDim.x, K - k0);
    __syncthreads();
    stage_rows<0>(ch.z + (e * K + k0) * (long long)D, nk * D, D, zc);
    __syncthreads();
    if ((int)threadIdx.x < nk) {
      const int r = threadIdx.x;
      float ss = 0.f;
      for (int d = 0; d < D; ++d) {
        const float zp = zc[r * zst + d] - cen[d];
        ss = fmaf(zp, zp, ss);
        if (mean_logvar) {
          bf[r * bst + d] = zp * zp;
          bf[r * bst + D + d] = zp;
        } else {
          bf[r * bst + d] = zp;
        }
      }
      float h = ch.htil[e * K + k0 + r];
      if (!mean_logvar) h = fmaf(pp_fixed, ss, h);
      hs[r] = h * kLog2e;
    }
    __syncthreads();
    // one 16-byte granule (8 features of one sample) per thread and step;
    // consecutive threads take consecutive samples of the same granule column
    const int gran = fk >> 3;
    for (int i = threadIdx.x; i < nk * gran; i += blockDim.x) {
      const int r = i % nk, g = i / nk;
      __align__(16) __nv_bfloat16 q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = g * 8 + j;
        if (c < nb) {
          q[j] = __float2bfloat16_rn(bf[r * bst + c]);
        } else if (c < nb + 3) {
          __nv_bfloat16 h1, h2, h3;
          split3(hs[r], h1, h2, h3);
          q[j] = c == nb ? h1 : (c == nb + 1 ? h2 : h3);
        } else if (split == 3 && c >= b_bl && c < b_bl + nb) {
          const float x = bf[r * bst + c - b_bl];
          q[j] = __float2bfloat16_rn(x - __bfloat162float(__float2bfloat16_rn(x)));
        } else if (split == 3 && b_bh2 >= 0 && c >= b_bh2 && c < b_bh2 + nb) {
          q[j] = __float2bfloat16_rn(bf[r * bst + c - b_bh2]);
        } else if (split == 3 && tail > 0 && c >= b_bht && c < b_bht + tail) {
          q[j] = __float2bfloat16_rn(bf[r * bst + nb - tail + (c - b_bht)]);
        } else {
          q[j] = __float2bfloat16_rn(0.f);
        }
      }
      *reinterpret_cast<uint4*>(out + canon(k0 + r, g * 8, fk)) = *reinterpret_cast<const uint4*>(q);
    }
  }
}

// Compile-time specialisation of the child features for the common widths:
// the sample's features live in registers and every column of the row is
// resolved at compile time (no per-value branches); rows are written as
// 16-byte granules of the canonical layout.
__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <int NB, int SPLIT, bool MLV, int BBL, int BBH2, int FK, int BBT = -1, int TAIL = 0>
__global__ void __launch_bounds__(128) k_child_features_t(LevelView ch, float pp_fixed, int K, const float* center,
                                                          __nv_bfloat16* bfeat) {
  constexpr int D = MLV ? NB / 2 : NB;
  constexpr int ZS = D + 1;
  __shared__ float cen[D];
  __shared__ float zc[128 * ZS];
  const long long e = blockIdx.x;
  const long long p = ch.parent[e];
  for (int d = threadIdx.x; d < D; d += blockDim.x) cen[d] = center[p * D + d];
  __nv_bfloat16* out = bfeat + e * (long long)K * FK;
  for (int k0 = 0; k0 < K; k0 += 128) {
    const int nk = min(128, K - k0);
    __syncthreads();
    stage_rows<D>(ch.z + (e * K + k0) * (long long)D, nk * D, D, zc);
    __syncthreads();
    if ((int)threadIdx.x >= nk) continue;
    const int r = threadIdx.x;
    float b[NB];
    float ss = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float zp = zc[r * ZS + d] - cen[d];
      ss = fmaf(zp, zp, ss);
      if (MLV) {
        b[d] = zp * zp;
        b[D + d] = zp;
      } else {
        b[d] = zp;
      }
    }
    float h = ch.htil[e * K + k0 + r];
    if (!MLV) h = fmaf(pp_fixed, ss, h);
    __nv_bfloat16 h1, h2, h3;
    split3(h * kLog2e, h1, h2, h3);
    __nv_bfloat16 bh[NB], bl[NB];
#pragma unroll
    for (int f = 0; f < NB; ++f) {
      bh[f] = __float2bfloat16_rn(b[f]);
      bl[f] = __float2bfloat16_rn(b[f] - __bfloat162float(bh[f]));
    }
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    uint32_t wv[FK / 2];
#pragma unroll
    for (int c = 0; c < FK; c += 2) {
      __nv_bfloat16 v[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int cc = c + t;
        __nv_bfloat16 x = zero;
        if (cc < NB) x = bh[cc];
        else if (cc == NB) x = h1;
        else if (cc == NB + 1) x = h2;
        else if (cc == NB + 2) x = h3;
        else if (SPLIT == 3 && cc >= BBL && cc < BBL + NB) x = bl[cc - BBL];
        else if (SPLIT == 3 && BBH2 >= 0 && cc >= BBH2 && cc < BBH2 + NB) x = bh[cc - BBH2];
        else if (SPLIT == 3 && TAIL > 0 && cc >= BBT && cc < BBT + TAIL) x = bh[NB - TAIL + (cc - BBT)];
        v[t] = x;
      }
      wv[c / 2] = pack_bf16x2(v[0], v[1]);
    }
    const long long k = k0 + r;
#pragma unroll
    for (int g = 0; g < FK / 8; ++g)
      *reinterpret_cast<uint4*>(out + canon(k, g * 8, FK)) =
          make_uint4(wv[4 * g], wv[4 * g + 1], wv[4 * g + 2], wv[4 * g + 3]);
  }
}

// ---------------------------------------------------------------------------- TF32 operand rows
// TF32 mode: one product per k-step, every operand value an FP32 word rounded
// to TF32 (cvt.rna; the tensor core reads the upper 19 bits), rows of nb + 3
// values padded to a multiple of 8 (one kind::tf32 k-step), in the same
// canonical byte layout (a 16-byte granule holds 4 values; widths and column
// offsets are given in 16-bit units, 2 per value):
//   parent rows  [A (nb) | 1 1 1 | 0..]        child rows  [B (nb) | h1 h2 h3 | 0..]
// with h = h1 + h2 + h3 its three-part TF32 split (33 significant bits).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split3_tf32(float x, float& a, float& b, float& c) {
  if (!(x > kNegBig)) {  // -inf / very negative / NaN-safe, as split3
    a = isnan(x) ? x : kNegBig;
    b = c = 0.f;
    return;
  }
  a = tf32_rna(x);
  const float r1 = x - a;
  b = tf32_rna(r1);
  c = tf32_rna(r1 - b);
}

__global__ void k_parent_features_tf32(LevelView par, int Dc, int mean_logvar, int K, int fk, int nb,
                                       __nv_bfloat16* afeat, float* rowc, float* center) {
  const long long p = blockIdx.x;
  __shared__ float cen[kMaxDim];
  __shared__ float red[8][kMaxDim];
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = 0; d < Dc; ++d) {
      float acc = 0.f;
      for (int kp = threadIdx.x; kp < K; kp += blockDim.x) acc += par.pm[(p * K + kp) * Dc + d];
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) red[warp][d] = acc;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < Dc; d += blockDim.x) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][d];
      cen[d] = t / K;
      center[p * Dc + d] = cen[d];
    }
    __syncthreads();
  }
  for (int kp = blockIdx.y * blockDim.x + threadIdx.x; kp < K; kp += gridDim.y * blockDim.x) {
    const float* pm = par.pm + (p * K + kp) * Dc;
    const float* pp = par.pp + (p * K + kp) * Dc;
    double rc = par.pc[p * K + kp];
    for (int d = 0; d < Dc; ++d) {
      const float dm = pm[d] - cen[d];
      rc += (double)pp[d] * dm * dm;
    }
    if (blockIdx.z == 0) rowc[p * K + kp] = (float)rc;
    __nv_bfloat16* row = afeat + p * (long long)K * fk;
    for (int c0 = 0; c0 < fk / 2; c0 += 4) {
      float g[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int f = c0 + j;
        if (f < nb) {
          const float v = mean_logvar ? (f < Dc ? pp[f] : -2.f * pp[f - Dc] * (pm[f - Dc] - cen[f - Dc]))
                                      : -2.f * pp[f] * (pm[f] - cen[f]);
          g[j] = tf32_rna(v * kLog2e);
        } else {
          g[j] = f < nb + 3 ? 1.f : 0.f;
        }
      }
      *reinterpret_cast<float4*>(row + canon(kp, 2 * c0, fk)) = make_float4(g[0], g[1], g[2], g[3]);
    }
  }
}

__global__ void __launch_bounds__(128) k_child_features_tf32(LevelView ch, int mean_logvar, float pp_fixed, int K,
                                                             int fk, int nb, const float* center,
                                                             __nv_bfloat16* bfeat) {
  extern __shared__ float csm[];
  const long long e = blockIdx.x;
  const int D = ch.D, zst = D + 1, bst = nb + 4;
  const long long p = ch.parent[e];
  float* cen = csm;                      // [D]
  float* zc = cen + D;                   // [128][D+1]
  float* bf = zc + 128 * zst;            // [128][nb+4] row values (features, then h1 h2 h3)
  for (int d = threadIdx.x; d < D; d += blockDim.x) cen[d] = center[p * D + d];
  __nv_bfloat16* out = bfeat + e * (long long)K * fk;
  const int nv = nb + 3, gran = fk >> 3;  // values per row; 16-byte granules per row
  for (int k0 = 0; k0 < K; k0 += blockDim.x) {
    const int nk = min((int)blockDim.x, K - k0);
    __syncthreads();
    stage_rows<0>(ch.z + (e * K + k0) * (long long)D, nk * D, D, zc);
    __syncthreads();
    if ((int)threadIdx.x < nk) {
      const int r = threadIdx.x;
      float ss = 0.f;
      for (int d = 0; d < D; ++d) {
        const float zp = zc[r * zst + d] - cen[d];
        ss = fmaf(zp, zp, ss);
        if (mean_logvar) {
          bf[r * bst + d] = tf32_rna(zp * zp);
          bf[r * bst + D + d] = tf32_rna(zp);
        } else {
          bf[r * bst + d] = tf32_rna(zp);
        }
      }
      float h = ch.htil[e * K + k0 + r];
      if (!mean_logvar) h = fmaf(pp_fixed, ss, h);
      split3_tf32(h * kLog2e, bf[r * bst + nb], bf[r * bst + nb + 1], bf[r * bst + nb + 2]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nk * gran; i += blockDim.x) {
      const int r = i % nk, g = i / nk;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * g + j;
        v[j] = c < nv ? bf[r * bst + c] : 0.f;
      }
      *reinterpret_cast<float4*>(out + canon(k0 + r, g * 8, fk)) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// Adjoint operands of the parents whose compacted weight list is longer than
// `small` (the others are handled on the CUDA cores): the kept rows of the
// parent features, gathered in order (padding rows repeat row 0 and carry a
// -inf shift).
__global__ void k_gather(LevelView par, int K, int fk, int small, const __nv_bfloat16* afeat, __nv_bfloat16* cfeat) {
  const long long p = blockIdx.x;
  const int n_eff = par.ccnt[p];
  if (n_eff <= small) return;
  const int npad = min(K, (n_eff + 15) & ~15);
  const int gran = fk >> 3;
  const uint4* src = reinterpret_cast<const uint4*>(afeat + p * (long long)K * fk);
  uint4* dst = reinterpret_cast<uint4*>(cfeat + p * (long long)K * fk);
  for (int i = threadIdx.x; i < npad * gran; i += blockDim.x) {
    const int j = i / gran, g = i % gran;
    const int kp = par.cidx[p * K + j];
    dst[canon(j, g * 8, fk) >> 3] = src[canon(kp, g * 8, fk) >> 3];
  }
}

// Column shifts of the adjoint tile of element e (log2 units):
//   d_j = log2e (rowc[kp_j] + ln w_p[kp_j] - ln K - lt_e[kp_j]),  -inf on padding.
__global__ void k_dcol(LevelView ch, LevelView par, int K, int small, const float* rowc, float* dcol) {
  const long long e = blockIdx.x;
  const long long p = ch.parent[e];
  const int n_eff = par.ccnt[p];
  if (n_eff <= small) return;
  const int npad = min(K, (n_eff + 15) & ~15);
  for (int j = threadIdx.x; j < npad; j += blockDim.x) {
    float d = -INFINITY;
    if (j < n_eff) {
      const int kp = par.cidx[p * K + j];
      d = (rowc[p * K + kp] + par.cw[p * K + j] - ch.lt[e * K + kp]) * kLog2e;
    }
    dcol[e * K + j] = d;
  }
}


// ---------------------------------------------------------------------------- the contraction kernel
// One work unit = 128 rows of one plate element.  Columns stream in chunks
// of up to 256 (the MMA reaches its full rate only at N = 256: an M = 128,
// K = 16 instruction takes ~128 cycles at N = 128 and at N = 256) through a
// ring of up to 4 bulk copies, one issuing warp per stage; the MMA accumulates
// each chunk in FP32 in TMEM (2 slots of 256 columns, so the MMA of chunk
// g+1 overlaps the epilogue of chunk g); 16 epilogue warps turn TMEM into
// row sums.  The A tile is reloaded only when the unit's row block changes
// (double-buffered when shared memory allows, otherwise single).
constexpr int kNB = 256;          // columns per chunk

struct ContractArgs {
  int K, frow, fcol, ksteps, rt_per_unit, units_per_elt, a_slots, nst;  // nst: column ring depth
  int koff_row[16], koff_col[16];   // per k-step: column offset in the row / column operand
  long long n_units, n_elts;
  const long long* parent;
  const __nv_bfloat16* rows_feat;   // A operand source (forward: parent features, adjoint: child features)
  const __nv_bfloat16* cols_feat;   // B operand source (forward: child features, adjoint: compacted parents)
  const float* rowc;                // forward
  float* lt;                        // forward output [n][K]
  const int* ccnt;                  // adjoint: kept parent samples per parent
  int small;                        //          parents keeping <= small samples are skipped
  const float* dcol;                //          column shifts [n][K] (log2 units)
  float* w_out;                     //          output [n][K]
  Ctl* ctl;
  long long timeout_cycles;
  int expire_test;                  // qem_test_expire_wait
};

struct Smem {
  uint8_t* a0;       // two A blocks (RT row tiles each), a_stride apart
  uint8_t* b0;       // nst B chunks, b_stride apart
  float* d0;         // nst column-shift rows (adjoint), kNB floats apart
  uint32_t a_stride, b_stride;
  uint64_t* a_full;
  uint64_t* a_empty;
  uint64_t* b_full;
  uint64_t* b_empty;
  uint64_t* t_full;
  uint64_t* t_empty;
  uint64_t* d_full;   // adjoint column shifts landed in stage
  uint64_t* d_empty;  // adjoint column shifts of stage consumed by the epilogue
  uint64_t* done;
  uint32_t* tmem_base;
  volatile int* abort_flag;
  volatile int* stop_flag;
  float2* merge;      // [kRows][4] partial (max, sum) of every row
};

__host__ __device__ inline size_t contract_smem_bytes(int frow, int fcol, bool adj, int a_slots, int nst) {
  const size_t a = (size_t)kRows * frow * 2, b = (size_t)kNB * fcol * 2;
  size_t tot = 1024 + a_slots * a + nst * b;
  if (adj) tot += nst * (size_t)kNB * sizeof(float);
  tot += 32 * 8 + 16 + kRows * 4 * sizeof(float2);
  return tot;
}
// Shared-memory budget: a double-buffered row operand first (a new row block
// per unit when parents change from unit to unit), then the deepest column
// ring that fits (a chunk's MMAs are known complete only well after they
// finish, so the ring needs about three chunks of lead).  False when not even
// one row slot and two column stages fit.
__host__ inline bool contract_config(int frow, int fcol, bool adj, int& a_slots, int& nst) {
  static const int opts[][2] = {{2, 4}, {2, 3}, {1, 4}, {1, 3}, {2, 2}, {1, 2}};
  for (const auto& o : opts)
    if (contract_smem_bytes(frow, fcol, adj, o[0], o[1]) <= kSmemLimit) {
      a_slots = o[0];
      nst = o[1];
      return true;
    }
  return false;
}

__device__ __forceinline__ Smem carve(uint8_t* raw, int frow, int fcol, bool adj, int a_slots, int nst) {
  Smem s;
  uint8_t* p = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  const size_t a = (size_t)kRows * frow * 2, b = (size_t)kNB * fcol * 2;
  s.a_stride = (uint32_t)a;
  s.b_stride = (uint32_t)b;
  s.a0 = p;
  p += a_slots * a;
  s.b0 = p;
  p += nst * b;
  if (adj) {
    s.d0 = reinterpret_cast<float*>(p);
    p += nst * kNB * sizeof(float);
  } else {
    s.d0 = nullptr;
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);
  s.a_full = bars + 0;
  s.a_empty = bars + 2;
  s.b_full = bars + 4;
  s.b_empty = bars + 8;
  s.t_full = bars + 12;
  s.t_empty = bars + 14;
  s.d_full = bars + 16;
  s.d_empty = bars + 20;
  s.done = bars + 24;
  p += 32 * 8;
  s.tmem_base = reinterpret_cast<uint32_t*>(p);
  s.abort_flag = reinterpret_cast<volatile int*>(p + 4);
  s.stop_flag = reinterpret_cast<volatile int*>(p + 8);
  p += 16;
  s.merge = reinterpret_cast<float2*>(p);
  return s;
}

// The sequence of work units of a CTA, identical in every role.
// Forward: units u = blockIdx.x + i * gridDim.x, u -> (element u / upe, row
// block u % upe); the parent of the next unit is loaded one unit ahead.
// Adjoint: elements e = blockIdx.x + i * gridDim.x whose parent keeps more
// than `small` weighted samples, each contributing its upe row blocks in
// order; the next element's parent and count are loaded while the current
// element is processed.
struct Unit {
  long long e, p;
  int rb;       // row block
  int ncols;    // columns of the unit
};
template <bool ADJ>
struct Walker {
  const ContractArgs& a;
  long long cur;          // forward: next unit; adjoint: current element
  long long p_next;       // forward: parent of unit `cur`
  long long ep, pp;       // adjoint: element whose units are being yielded and its parent
  int cnt, rb;            //          its kept count and next row block (rb == upe: need a new element)
  long long nxt, p_nx;    //          prefetched element and its parent
  __device__ explicit Walker(const ContractArgs& args) : a(args) {
    if (!ADJ) {
      cur = blockIdx.x;
      p_next = cur < a.n_units ? a.parent[cur / a.units_per_elt] : 0;
    } else {
      rb = a.units_per_elt;
      ep = pp = -1;
      cnt = 0;
      nxt = blockIdx.x;
      p_nx = nxt < a.n_elts ? a.parent[nxt] : 0;
    }
  }
  __device__ bool next(Unit& x) {
    if (!ADJ) {
      if (cur >= a.n_units) return false;
      x.e = cur / a.units_per_elt;
      x.rb = (int)(cur % a.units_per_elt);
      x.p = p_next;
      x.ncols = a.K;
      cur += gridDim.x;
      if (cur < a.n_units) p_next = a.parent[cur / a.units_per_elt];
      return true;
    }
    while (rb >= a.units_per_elt) {  // advance to the next element that has work
      if (nxt >= a.n_elts) return false;
      ep = nxt;
      pp = p_nx;
      cnt = a.ccnt[pp];
      nxt += gridDim.x;
      if (nxt < a.n_elts) p_nx = a.parent[nxt];
      rb = cnt > a.small ? 0 : a.units_per_elt;
    }
    x.e = ep;
    x.p = pp;
    x.rb = rb++;
    x.ncols = min(a.K, max(16, (cnt + 15) & ~15));
    return true;
  }
};

template <bool ADJ, bool TF32>
__global__ void __launch_bounds__(kThreads, 1) k_contract(ContractArgs a) {
  extern __shared__ uint8_t smem_raw[];
  Smem s = carve(smem_raw, a.frow, a.fcol, ADJ, a.a_slots, a.nst);
  const int NA = a.a_slots, NS = a.nst;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = a.K, RT = a.rt_per_unit, frow = a.frow, fcol = a.fcol;
  const uint32_t sbo_a = (uint32_t)(frow >> 3) * 128u, sbo_b = (uint32_t)(fcol >> 3) * 128u;
  const uint32_t tile_bytes = (uint32_t)kRows * frow * 2;
  const long long lim = a.timeout_cycles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.a_full[i], 1);
      mbar_init(&s.a_empty[i], 1);
      mbar_init(&s.t_full[i], 1);
      mbar_init(&s.t_empty[i], kEpiWarps);
    }
    for (int i = 0; i < NS; ++i) {
      mbar_init(&s.b_full[i], 1);
      mbar_init(&s.b_empty[i], 1);
      mbar_init(&s.d_full[i], 1);
      mbar_init(&s.d_empty[i], kEpiWarps);
    }
    mbar_init(s.done, 1);
    *s.abort_flag = 0;
    *s.stop_flag = 0;
    fence_barrier_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(s.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_base;

  if (warp < kProdWarps) {
    // ------------------------------------------------------------ producers
    // Warp 0 loads the row operand (once per row block); warp 1 + i loads the
    // column chunks of ring stage i.  Several issuing warps keep several bulk
    // copies in flight per SM (one thread waiting on every stage in turn
    // serialises them).
    const bool is_a = warp == 0;
    const int my_stage = warp - 1;
    int as = 0;
    uint32_t aph = 0, bph = 0;
    long long g = 0;                // chunk counter of this CTA (all roles count the same chunks)
    uint32_t armed = 0, last = 0;  // bit i: a slot i, bit 2: my b stage, bit 3: my d stage
    long long prev_row = -1;
    bool ok = true;
    Walker<ADJ> wk(a);
    Unit x;
    while (ok && wk.next(x)) {
      const long long row_elt = ADJ ? x.e : x.p;
      const long long row_key = row_elt * a.units_per_elt + x.rb;
      if (row_key != prev_row) {
        if (is_a && lane == 0) {  // new row block: load it into the next A slot
          ok = mbar_wait(&s.a_empty[as], aph ^ 1, lim, s.abort_flag);
          if (ok) {
            const uint32_t bytes = (uint32_t)RT * tile_bytes;
            mbar_expect_tx(&s.a_full[as], bytes);
            bulk_g2s(s.a0 + as * s.a_stride, a.rows_feat + (row_elt * K + (long long)x.rb * RT * kRows) * frow, bytes,
                     &s.a_full[as]);
            armed |= 1u << as;
            last = (last & ~(1u << as)) | (aph << as);
          }
        }
        if (++as == NA) {
          as = 0;
          aph ^= 1;
        }
        prev_row = row_key;
      }
      const long long col_elt = ADJ ? x.p : x.e;
      for (int c0 = 0; c0 < x.ncols && ok; c0 += kNB, ++g) {
        const int bs = (int)(g % NS);
        if (bs == 0 && g > 0) bph ^= 1;
        if (is_a || bs != my_stage || lane != 0) continue;
        const int nc = min(kNB, x.ncols - c0);
        ok = mbar_wait(&s.b_empty[bs], bph ^ 1, lim, s.abort_flag);
        if (ok) {
          const uint32_t bytes = (uint32_t)nc * fcol * 2;
          mbar_expect_tx(&s.b_full[bs], bytes);
          bulk_g2s(s.b0 + bs * s.b_stride, a.cols_feat + (col_elt * K + c0) * fcol, bytes, &s.b_full[bs]);
          armed |= 4u;
          last = (last & ~4u) | (bph << 2);
        }
        // the column shifts live until the epilogue has used them (own barriers)
        if (ADJ && ok) ok = mbar_wait(&s.d_empty[bs], bph ^ 1, lim, s.abort_flag);
        if (ADJ && ok) {
          mbar_expect_tx(&s.d_full[bs], (uint32_t)nc * 4u);
          bulk_g2s(s.d0 + bs * kNB, a.dcol + x.e * K + c0, (uint32_t)nc * 4u, &s.d_full[bs]);
          armed |= 8u;
          last = (last & ~8u) | (bph << 3);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    }
    // no bulk copy of this CTA may still be landing when it exits: wait for
    // the last phase armed on every full barrier this warp armed (bounded,
    // ignores abort)
    if (lane == 0) {
      volatile int never = 0;
      if (is_a) {
        for (int i = 0; i < NA; ++i)
          if (armed & (1u << i)) mbar_wait(&s.a_full[i], (last >> i) & 1u, drain_bound(lim), &never);
      } else {
        if (armed & 4u) mbar_wait(&s.b_full[my_stage], (last >> 2) & 1u, drain_bound(lim), &never);
        if (armed & 8u) mbar_wait(&s.d_full[my_stage], (last >> 3) & 1u, drain_bound(lim), &never);
      }
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer (one elected lane)
    // The whole warp runs the loop (its waits are warp votes, so control flow
    // and descriptors stay warp-uniform); one elected lane issues.
    {
      int as = NA - 1, bs = 0, ts = 0;   // as: slot of the current row block (advanced on each new block)
      uint32_t aph = 1, bph = 0, tph = 0;
      // Descriptors are built once: a k-step at column c of a slot adds c to
      // the start-address field (16-byte units; shared addresses stay below
      // 2^18, so the 14-bit field never carries), so the issue loop is a few
      // integer adds per MMA and keeps the tensor pipe fed.
      uint32_t kro[16], kco[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        kro[i] = (uint32_t)a.koff_row[i];
        kco[i] = (uint32_t)a.koff_col[i];
      }
      const int nks = a.ksteps;
      const uint64_t adesc0 = smem_desc(s.a0, 128, sbo_a), bdesc0 = smem_desc(s.b0, 128, sbo_b);
      const uint32_t a_step = s.a_stride >> 4, b_step = s.b_stride >> 4, t_step = tile_bytes >> 4;
      long long prev_row = -1;
      bool ok = true;
      // test hook (qem_test_expire_wait): a wait on the teardown barrier, which
      // nothing completes before the teardown, runs out and aborts the CTA
      if (a.expire_test) ok = mbar_spin_warp(s.done, 0, lim, s.abort_flag);
      Walker<ADJ> wk(a);
      Unit x;
      while (ok && wk.next(x)) {
        const long long row_key = (ADJ ? x.e : x.p) * a.units_per_elt + x.rb;
        if (row_key != prev_row) {
          if (prev_row >= 0) {  // the previous block's last MMA has been issued
            if (elect_one()) mma_commit(&s.a_empty[as]);
            __syncwarp();
          }
          if (++as == NA) {
            as = 0;
            aph ^= 1;
          }
          ok = mbar_spin_warp(&s.a_full[as], aph, lim, s.abort_flag);
          if (!ok) break;
          prev_row = row_key;
        }
        for (int c0 = 0; c0 < x.ncols; c0 += kNB) {
          const int nc = min(kNB, x.ncols - c0);
          ok = mbar_spin_warp(&s.b_full[bs], bph, lim, s.abort_flag) &&
               mbar_spin_warp(&s.t_empty[ts], tph ^ 1, lim, s.abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t idesc = idesc_fmt(nc, TF32 ? 2u : 1u);
          const uint64_t bd = bdesc0 + (uint64_t)(bs * b_step);
          if (elect_one()) {
            for (int r = 0; r < RT; ++r) {
              const uint32_t d_tmem = tmem + (uint32_t)(ts * 256 + r * kNB);
              const uint64_t ad = adesc0 + (uint64_t)(as * a_step + r * t_step);
#pragma unroll
              for (int ks = 0; ks < 16; ++ks)
                if (ks < nks) mma_kind<TF32>(d_tmem, ad + kro[ks], bd + kco[ks], idesc, ks > 0 ? 1u : 0u);
            }
            mma_commit(&s.b_empty[bs]);
            mma_commit(&s.t_full[ts]);
          }
          __syncwarp();
          if (++bs == NS) {
            bs = 0;
            bph ^= 1;
          }
          ts ^= 1;
          if (ts == 0) tph ^= 1;
        }
      }
      // every issued MMA has completed before the teardown, also after an
      // abort (the wait ignores the abort flag; it is still bounded)
      if (elect_one()) mma_commit(s.done);
      __syncwarp();
      volatile int never = 0;
      mbar_wait(s.done, 0, drain_bound(lim), &never);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (16 warps)
    // Warp w reads TMEM lanes 32 (w % 4) .. +31 (the restriction of
    // tcgen05.ld).  With RT = 2 the four warps of a lane quarter take (row
    // tile, column half); with RT = 1 they take column quarters.  Four warps
    // share each SM sub-partition, so one warp's TMEM-load latency is hidden
    // by the others' exponentials.  Every epilogue warp executes both named
    // barriers of every unit it enters, and the decision to stop is read from
    // a flag written between them, so the warps always agree.
    const int part = (warp - kEpiWarp0) >> 2;
    const int quarter = warp & 3;
    const int r = RT == 2 ? (part >> 1) : 0;
    const int ncp = RT == 2 ? 2 : 4;             // column parts per row tile
    const int cpart = RT == 2 ? (part & 1) : part;
    const int row = quarter * 32 + lane;
    int ts = 0, ds = 0;
    uint32_t tph = 0, dph = 0;
    Walker<ADJ> wk(a);
    Unit x;
    while (wk.next(x)) {
      float m = -INFINITY, sacc = 0.f;
      bool ok = true;
      for (int c0 = 0; c0 < x.ncols && ok; c0 += kNB) {
        const int nc = min(kNB, x.ncols - c0);
        ok = mbar_wait(&s.t_full[ts], tph, lim, s.abort_flag);
        if (ok && ADJ) ok = mbar_wait(&s.d_full[ds], dph, lim, s.abort_flag);
        ok = __all_sync(0xffffffffu, ok);  // the TMEM loads below are warp-collective
        if (!ok) break;
        tc_fence_after();
        const int qw = nc / ncp;  // columns of this warp (multiple of 4)
        const int col0 = cpart * qw;
        const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ts * 256 + r * kNB + col0);
        const float* dsm = ADJ ? s.d0 + ds * kNB + col0 : nullptr;
        int c = 0;
        if (!ADJ) {
          for (; c < qw; c += 32) lse_group32(tbase + c, m, sacc);
        } else {
          for (; c + 32 <= qw; c += 32) {
            float v[32];
            tmem_ld32(tbase + c, v);
            const float4* d4 = reinterpret_cast<const float4*>(dsm + c);
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              const float4 dv = d4[j >> 2];
              add2(v[j], v[j + 1], dv.x, dv.y);
              add2(v[j + 2], v[j + 3], dv.z, dv.w);
              float e0 = ex2f(v[j]), e1 = ex2f(v[j + 1]), e2 = ex2f(v[j + 2]), e3 = ex2f(v[j + 3]);
              add2(p0, p1, e0, e1);
              add2(p2, p3, e2, e3);
            }
            add2(p0, p1, p2, p3);
            sacc += p0 + p1;
          }
          for (; c < qw; c += 4) {
            float v[4];
            tmem_ld4(tbase + c, v);
#pragma unroll
            for (int j = 0; j < 4; ++j) sacc += ex2f(v[j] + dsm[c + j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&s.t_empty[ts]);
          if (ADJ) mbar_arrive(&s.d_empty[ds]);
        }
        ts ^= 1;
        if (ts == 0) tph ^= 1;
        if (++ds == NS) {
          ds = 0;
          dph ^= 1;
        }
      }
      // combine the column parts of each row
      const int mrow = r * kRows + row;
      s.merge[mrow * 4 + cpart] = make_float2(m, sacc);
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
      if (threadIdx.x == 32 * kEpiWarp0) *s.stop_flag = *s.abort_flag;
      if (cpart == 0 && ok) {
        const long long k = (long long)x.rb * RT * kRows + mrow;
        if (ADJ) {
          float S = 0.f;
          for (int i = 0; i < ncp; ++i) S += s.merge[mrow * 4 + i].y;
          a.w_out[x.e * K + k] = S;
        } else {
          float M = -INFINITY;
          for (int i = 0; i < ncp; ++i) M = fmaxf(M, s.merge[mrow * 4 + i].x);
          float S = 0.f;
          for (int i = 0; i < ncp; ++i) {
            const float2 o = s.merge[mrow * 4 + i];
            if (o.x != -INFINITY) S += o.y * ex2f(o.x - M);
          }
          a.lt[x.e * K + k] = a.rowc[x.p * K + k] + (M + log2f(S)) * kLn2 - logf((float)K);
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
      if (*s.stop_flag) break;
    }
  }

  tc_fence_before();
  __syncthreads();
  // after the barrier: every role has stopped, so an abort by any of them is seen
  if (*s.abort_flag && threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_TIMEOUT);
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------- diagnostic GEMM
// out[128][n] = A[128][fk] * B[n][fk]^T through the same descriptors, bulk
// copies, MMA and TMEM loads (validation of the operand layout).
__global__ void __launch_bounds__(128, 1) k_diag_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int fk, int n,
                                                     float* out, Ctl* ctl, long long lim) {
  extern __shared__ uint8_t raw[];
  uint8_t* sa = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sb = sa + (size_t)kRows * fk * 2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sb + (size_t)kMaxN * fk * 2);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(bars + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tbase + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tbase, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  if (threadIdx.x == 0) {
    const uint32_t ab = (uint32_t)kRows * fk * 2, bb = (uint32_t)n * fk * 2;
    mbar_expect_tx(&bars[0], ab + bb);
    bulk_g2s(sa, A, ab, &bars[0]);
    bulk_g2s(sb, B, bb, &bars[0]);
    if (mbar_wait(&bars[0], 0, lim, abort_flag)) {
      tc_fence_after();
      const uint32_t sbo = (uint32_t)(fk >> 3) * 128u;
      for (int ks = 0; ks < fk / 16; ++ks)
        mma_bf16(tmem, smem_desc(sa + ks * 256, 128, sbo), smem_desc(sb + ks * 256, 128, sbo), idesc_bf16(n),
                 ks > 0 ? 1u : 0u);
    }
    mma_commit(&bars[1]);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[1], 0, lim, abort_flag));  // warp-collective loads follow
  tc_fence_after();
  if (ok) {
    const int row = warp * 32 + lane;
    for (int c = 0; c < n; c += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      for (int j = 0; j < 8; ++j) out[(long long)row * n + c + j] = v[j];
    }
  }
  if (threadIdx.x == 0) {
    if (*abort_flag) atomicOr(&ctl->err, ERR_TIMEOUT);
    // neither the bulk copies nor the MMAs may still be in flight at the
    // teardown, also after an abort (bounded waits that ignore the flag)
    volatile int never = 0;
    mbar_wait(&bars[0], 0, drain_bound(lim), &never);
    mbar_wait(&bars[1], 0, drain_bound(lim), &never);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace tc

// ---------------------------------------------------------------------------- host side
using namespace tc;

static int up16(int x) { return (x + 15) & ~15; }
static int up8(int x) { return (x + 7) & ~7; }

// Operand layout of a level with nb bilinear features (see Layout).
// split 0: TF32 rows [X (nb) | 1 1 1 or h1 h2 h3 | 0..], nb + 3 values padded
// to a multiple of 8 (one kind::tf32 k-step of 32 bytes = 16 units).
static Layout make_layout(int nb, int split) {
  Layout L;
  L.nb = nb;
  L.split = split;
  if (split == 0) {
    L.fka = L.fkb = 2 * up8(nb + 3);
    L.nks = L.fka / 16;
    for (int i = 0; i < L.nks; ++i) L.ka[i] = L.kb[i] = 16 * i;
    return L;
  }
  if (split == 1) {
    L.fka = L.fkb = up16(nb + 3);
    L.nks = L.fka / 16;
    for (int i = 0; i < L.nks; ++i) L.ka[i] = L.kb[i] = 16 * i;
    return L;
  }
  const int fk_dup = up16(3 * nb + 3);            // [Bh | h | Bl | Bh]: both rows fk_dup wide
  const int p1 = up8(nb + 3), p2 = up16(p1 + nb);
  const int r = nb % 16, slack = p2 - (p1 + nb);
  const int tail = r <= slack ? r : 0;             // ragged tail of the lo*hi product packed in the padding
  const int q = up16(nb - tail);
  if (p2 < fk_dup && (p2 + q) / 16 <= 16) {        // [Bh | h | Bl | Bh tail], the lo*hi product re-reads Bh
    L.fka = p2 + q;
    L.fkb = p2;
    L.a_ah2 = p1;
    L.a_al = p2;
    L.b_bl = p1;
    L.b_bh2 = -1;
    L.tail = tail;
    L.a_alt = tail ? p1 + nb : -1;
    L.b_bht = tail ? p1 + nb : -1;
    L.nks = 0;
    for (int c = 0; c < p2; c += 16, ++L.nks) L.ka[L.nks] = L.kb[L.nks] = c;
    for (int c = 0; c < q; c += 16, ++L.nks) {
      L.ka[L.nks] = p2 + c;
      L.kb[L.nks] = c;
    }
  } else {
    L.fka = L.fkb = fk_dup;
    L.a_ah2 = nb + 3;
    L.a_al = 2 * nb + 3;
    L.b_bl = nb + 3;
    L.b_bh2 = 2 * nb + 3;
    L.nks = fk_dup / 16;
    for (int i = 0; i < L.nks; ++i) L.ka[i] = L.kb[i] = 16 * i;
  }
  return L;
}

qem_status tc_plan_reserve(qem_plan_t P, const qem_model_desc* desc, char* base, size_t* bytes) {
  *bytes = 0;
  if (P->precision == QEM_PREC_FP32) return QEM_OK;
  const int K = P->K;
  if (K % kRows != 0) return QEM_ERR_UNSUPPORTED;
  const int split = P->precision == QEM_PREC_BF16X3 ? 3 : (P->precision == QEM_PREC_TF32 ? 0 : 1);
  TcBuffers tb;
  tb.split = split;
  tb.tf32 = split == 0;
  size_t off = 0;
  auto take = [&](size_t b) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(b);
    return p;
  };
  for (int l = 1; l < desc->n_levels; ++l) {
    const qem_level_desc& c = desc->levels[l];
    const qem_level_desc& pa = desc->levels[l - 1];
    const int nb = c.prior == QEM_PRIOR_NORMAL_MEAN_LOGVAR ? 2 * c.dim : c.dim;
    const Layout L = make_layout(nb, split);
    if (L.fka > kMaxFK || L.fkb > kMaxFK || L.nks > 16) return QEM_ERR_UNSUPPORTED;
    tb.nb[l] = nb;
    tb.lay[l] = L;
    tb.bfeat[l] = (__nv_bfloat16*)take((size_t)c.n * K * L.fkb * 2);
    tb.afeat[l] = (__nv_bfloat16*)take((size_t)pa.n * K * L.fka * 2);
    tb.cfeat[l] = (__nv_bfloat16*)take((size_t)pa.n * K * L.fka * 2);
    tb.rowc[l] = (float*)take((size_t)pa.n * K * 4);
    tb.center[l] = (float*)take((size_t)pa.n * c.dim * 4);
    tb.dcol[l] = (float*)take((size_t)c.n * K * 4);
  }
  *bytes = off;
  if (base) {
    P->tc = new (std::nothrow) TcBuffers(tb);
    if (!P->tc) return QEM_ERR_OOM;
  }
  return QEM_OK;
}

qem_status tc_plan_init(qem_plan_t P, const qem_model_desc*) {
  if (P->precision == QEM_PREC_FP32) return QEM_OK;
  const bool tf32 = P->tc->tf32;
  for (int l = 1; l < P->L; ++l) {
    const Layout& L = P->tc->lay[l];
    int na, ns;
    if (!contract_config(L.fka, L.fkb, false, na, ns)) return QEM_ERR_UNSUPPORTED;
    if (!contract_config(L.fkb, L.fka, true, na, ns)) return QEM_ERR_UNSUPPORTED;
    const qem_status rs = tc_res_init(L.fka, L.fkb, P->K, tf32);
    if (rs != QEM_OK) return rs;
  }
  cudaError_t e1, e2;
  if (tf32) {
    e1 = opt_in_smem(k_contract<false, true>, 0);
    e2 = opt_in_smem(k_contract<true, true>, 0);
  } else {
    e1 = opt_in_smem(k_contract<false, false>, 0);
    e2 = opt_in_smem(k_contract<true, false>, 0);
  }
  return e1 == cudaSuccess && e2 == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

void tc_plan_release(qem_plan_t P) {
  delete P->tc;
  P->tc = nullptr;
}

static long long timeout_cycles(qem_plan_t P) { return (long long)(P->timeout_s * (double)P->clock_khz * 1e3); }

cudaError_t tc_features(qem_plan_t P, int l) {
  TcBuffers& T = *P->tc;
  const LevelView& ch = P->lv[l];
  const LevelView& pa = P->lv[l - 1];
  const Layout& L = T.lay[l];
  const int K = P->K, nb = T.nb[l];
  const int mlv = ch.prior == QEM_PRIOR_NORMAL_MEAN_LOGVAR ? 1 : 0;
  if (T.tf32) {
    if (pa.n > 0) {
      const dim3 grid((unsigned)pa.n, (unsigned)std::max(1, std::min(16, (int)(2 * P->num_sms / std::max(1LL, pa.n)))));
      k_parent_features_tf32<<<grid, 256, 0, P->stream>>>(pa, ch.D, mlv, K, L.fka, nb, T.afeat[l], T.rowc[l],
                                                          T.center[l]);
    }
    if (ch.n > 0) {
      const size_t sm = sizeof(float) * (size_t)(ch.D + 128 * (ch.D + 1) + 128 * (nb + 4));
      k_child_features_tf32<<<(unsigned)ch.n, 128, sm, P->stream>>>(ch, mlv, -0.5f / ch.prior_a, K, L.fkb, nb,
                                                                    T.center[l], T.bfeat[l]);
    }
    return cudaGetLastError();
  }
  if (pa.n > 0) {
    const dim3 grid((unsigned)pa.n, (unsigned)std::max(1, std::min(16, (int)(2 * P->num_sms / std::max(1LL, pa.n)))));
    k_parent_features<<<grid, 256, 0, P->stream>>>(pa, ch.D, mlv, K, L.fka, nb, T.split, L.a_ah2, L.a_al, L.a_alt,
                                                   L.tail, T.afeat[l], T.rowc[l], T.center[l]);
  }
  if (ch.n > 0) {
    const unsigned g = (unsigned)ch.n;
    const float ppf = -0.5f / ch.prior_a;
    cudaStream_t st = P->stream;
    // compile-time layouts of the common shapes (checked against the plan's layout)
    if (mlv && nb == 36 && T.split == 3 && L.b_bl == 40 && L.b_bh2 < 0 && L.fkb == 80 && L.tail == 4 && L.b_bht == 76)
      k_child_features_t<36, 3, true, 40, -1, 80, 76, 4><<<g, 128, 0, st>>>(ch, ppf, K, T.center[l], T.bfeat[l]);
    else if (mlv && nb == 36 && T.split == 1 && L.fkb == 48)
      k_child_features_t<36, 1, true, -1, -1, 48><<<g, 128, 0, st>>>(ch, ppf, K, T.center[l], T.bfeat[l]);
    else if (!mlv && nb == 8 && T.split == 3 && L.b_bl == 11 && L.b_bh2 == 19 && L.fkb == 32)
      k_child_features_t<8, 3, false, 11, 19, 32><<<g, 128, 0, st>>>(ch, ppf, K, T.center[l], T.bfeat[l]);
    else if (!mlv && nb == 8 && T.split == 1 && L.fkb == 16)
      k_child_features_t<8, 1, false, -1, -1, 16><<<g, 128, 0, st>>>(ch, ppf, K, T.center[l], T.bfeat[l]);
    else {
      const size_t sm = sizeof(float) * (size_t)(ch.D + 128 * (ch.D + 1) + 128 * (nb + 1) + 128);
      k_child_features<<<g, 128, sm, st>>>(ch, mlv, ppf, K, L.fkb, nb, T.split, L.b_bl, L.b_bh2, L.b_bht, L.tail,
                                           T.center[l], T.bfeat[l]);
    }
  }
  return cudaGetLastError();
}

static cudaError_t launch_contract(qem_plan_t P, int l, bool adj) {
  TcBuffers& T = *P->tc;
  const LevelView& ch = P->lv[l];
  const Layout& L = T.lay[l];
  if (ch.n == 0) return cudaSuccess;
  ContractArgs a{};
  a.K = P->K;
  a.ksteps = L.nks;
  a.frow = adj ? L.fkb : L.fka;
  a.fcol = adj ? L.fka : L.fkb;
  for (int i = 0; i < L.nks; ++i) {
    a.koff_row[i] = adj ? L.kb[i] : L.ka[i];
    a.koff_col[i] = adj ? L.ka[i] : L.kb[i];
  }
  a.rt_per_unit = 1;
  a.units_per_elt = P->K / kRows;
  if (!contract_config(a.frow, a.fcol, adj, a.a_slots, a.nst)) return cudaErrorInvalidValue;
  a.n_units = ch.n * a.units_per_elt;
  a.n_elts = ch.n;
  a.parent = ch.parent;
  a.ctl = P->ctl;
  a.timeout_cycles = timeout_cycles(P);
  a.expire_test = P->expire_test;
  if (!adj) {
    a.rows_feat = T.afeat[l];
    a.cols_feat = T.bfeat[l];
    a.rowc = T.rowc[l];
    a.lt = ch.lt;
  } else {
    a.rows_feat = T.bfeat[l];
    a.cols_feat = T.cfeat[l];
    a.ccnt = P->lv[l - 1].ccnt;
    a.small = kSmallKept;
    a.dcol = T.dcol[l];
    a.w_out = ch.w;
  }
  const long long work = adj ? a.n_elts : a.n_units;
  const long long grid = work < P->num_sms ? work : P->num_sms;
  const size_t smem = contract_smem_bytes(a.frow, a.fcol, adj, a.a_slots, a.nst);
  if (T.tf32) {
    if (adj)
      k_contract<true, true><<<(unsigned)grid, kThreads, smem, P->stream>>>(a);
    else
      k_contract<false, true><<<(unsigned)grid, kThreads, smem, P->stream>>>(a);
  } else {
    if (adj)
      k_contract<true, false><<<(unsigned)grid, kThreads, smem, P->stream>>>(a);
    else
      k_contract<false, false><<<(unsigned)grid, kThreads, smem, P->stream>>>(a);
  }
  return cudaGetLastError();
}

// The element-resident schedule when the plan's launch shapes select it (bit
// 0 of tc_sched) and the level's operands fit it, otherwise the streaming one.
cudaError_t tc_forward(qem_plan_t P, int l) {
  const Layout& L = P->tc->lay[l];
  if ((P->tune.tc_sched & 1) && tc_res_fits(L.fka, L.fkb, P->K)) return tc_forward_res(P, l, P->tc->tf32);
  return launch_contract(P, l, false);
}

cudaError_t tc_adjoint_prep(qem_plan_t P, int l) {
  TcBuffers& T = *P->tc;
  const LevelView& pa = P->lv[l - 1];
  const LevelView& ch = P->lv[l];
  if (pa.n > 0)
    k_gather<<<(unsigned)pa.n, 256, 0, P->stream>>>(pa, P->K, T.lay[l].fka, kSmallKept, T.afeat[l], T.cfeat[l]);
  if (ch.n > 0) k_dcol<<<(unsigned)ch.n, 256, 0, P->stream>>>(ch, pa, P->K, kSmallKept, T.rowc[l], T.dcol[l]);
  return cudaGetLastError();
}

cudaError_t tc_adjoint(qem_plan_t P, int l) {
  const Layout& L = P->tc->lay[l];
  if ((P->tune.tc_sched & 2) && tc_adj_res_fits(L.fkb, L.fka, P->K)) return tc_adjoint_res(P, l, P->tc->tf32);
  return launch_contract(P, l, true);
}

}  // namespace qem

extern "C" qem_status qem_diag_tc_gemm(const void* A, const void* B, int fk, int n, float* out, void* stream) {
  using namespace qem;
  using namespace qem::tc;
  if (!A || !B || !out || fk < 16 || fk > kMaxFK || fk % 16 || n < 16 || n > kMaxN || n % 16) return QEM_ERR_INVALID_ARG;
  Ctl* ctl = nullptr;
  if (cudaMalloc(&ctl, sizeof(Ctl)) != cudaSuccess) return QEM_ERR_OOM;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
  const size_t smem = 1024 + (size_t)kRows * fk * 2 + (size_t)kMaxN * fk * 2 + 64;
  cudaFuncSetAttribute(k_diag_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, khz = 2000000;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  k_diag_gemm<<<1, 128, smem, s>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, fk, n, out, ctl,
                                   (long long)khz * 1000 * 2);
  cudaError_t e = cudaGetLastError();
  Ctl h{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(ctl);
  if (e != cudaSuccess) return QEM_ERR_CUDA;
  return (h.err & ERR_TIMEOUT) ? QEM_ERR_TIMEOUT : QEM_OK;
}
