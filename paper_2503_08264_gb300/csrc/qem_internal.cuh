// Internal declarations of libqem: the plan, the per-level device views and
// the device helpers every kernel file uses.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qem.h"

namespace qem {

constexpr int kMaxDim = 64;
// Adjoints: a parent element keeping at most this many weighted samples is
// handled on the CUDA cores, a denser one on the tensor cores.
constexpr int kSmallKept = 4;
constexpr float kLog2Pi = 1.8378770664093453f;
constexpr double kLog2PiD = 1.8378770664093454835606594728112;

// Error bits raised by kernels in the plan's control block.
enum : int { ERR_NUMERIC = 1, ERR_TIMEOUT = 2, ERR_INTERNAL = 4 };

// Device control block: written by tiny kernels so that a captured graph can
// advance the iteration without re-capture.
struct Ctl {
  unsigned long long seed;
  unsigned long long iter;     // noise stream iteration
  long long t;                 // EMA iteration number (>= 1)
  long long trace_row;         // row of the log P_MP trace to write (-1: none)
  int err;                     // ERR_* bits
  int pad;
  long long remaining;         // iterations left in a device-side loop (qem_run)
};

// Device view of one level of the plan (all pointers device).
struct LevelView {
  long long n;        // elements
  int D;              // latent dim
  int prior;          // QEM_PRIOR_*
  float prior_a, prior_b;
  int lik;
  float lik_var;
  int n_obs;
  int qfam;
  int nps;            // noise numbers per sample
  int level;          // index of this level
  int chain;          // days per region of a chain plate (1: plain plate)
  long long ebase;    // index of element 0 in the counter-based noise streams (a shard's offset)
  int qcond;          // parent-conditioned proposal (copies drawn from permuted parent copies)
  const int* perm;    // [n][K] qcond: parent copy of each sample
  const float* pz;    // qcond: the parent level's samples [n_parent][K][pD]
  int pD;             // qcond: the parent's dimension
  float* cz;          // [n][K][D] qcond: joint-weighted parent sample per child sample (adjoint)
  const float* x;     // [n][n_obs][D]
  const float* y;     // [n][n_obs]
  const long long* parent;     // [n] (level > 0)
  const long long* child_off;  // [n+1] offsets of children at level+1 (if any)
  // workspace
  float* z;           // [n][K][D]
  float* loc;         // [n][K]  sample-dependent part of log lik - log q (+ log prior at level 0)
  double* cst;        // [n]     sample-independent part of the same (normalisers, lgamma(y+1), ...)
  float* cshift;      // [n]     maximum taken out of loc by the sampler (joins cst)
  const double* ltab; // [kCountTable] per-count Poisson-log constants (levels with that likelihood)
  float* htil;        // [n][K]  loc + children's sum - off  (relative local factor)
  double* hsum;       // [n][K]  sum over children of their log mean-exp (FP64)
  double* off;        // [n]     constant removed from htil (chain plates: from that day's beta)
  float* lt;          // [n][K]  (level > 0) relative log mean_k exp S_e[kp][k], per parent sample kp
  float* w;           // [n][K]  marginal weights
  float* beta;        // [n][K]  chain plates: relative log mean_k exp S of day d >= 1 per sample of day d-1
  // conditional parameters of this level's children given each of its samples
  float* pm;          // [n][K][Dc] child-prior mean
  float* pp;          // [n][K][Dc] -0.5 * child-prior precision
  float* pc;          // [n][K]     child-prior log normaliser
  int Dc;             // dimension of the children (0: none)
  // weight compaction of this level's samples (levels with children)
  int* cidx;          // [n][K] indices of the kept samples, in order
  int* ccnt;          // [n]    number kept
  float* cw;          // [n][K] ln w - ln K of the kept samples (-inf padding)
  // plate-sum chunks: children of element p are chunks chk_off[p]..chk_off[p+1]
  // of the next level; this level's own chunks (levels > 0) cover
  // elements chk_beg[i]..chk_end[i] with FP64 partial sums [n_chunks][K]
  long long* chk_off;
  long long* chk_beg;
  long long* chk_end;
  long long n_chunks;
  double* partial;
};

struct TcBuffers;  // tensor-core operand buffers (qem_tc.cu)

// Workspace of the split-root E-step (qem_split.cu), allocated on first use.
struct SplitWs {
  void* base = nullptr;
  size_t bytes = 0;
  double* fa = nullptr;        // [n0][K]   root factor of the mu half of each root sample
  double* fb = nullptr;        // [n0][K]   the same for the psi half
  float* lt = nullptr;         // [n1][K^2] user tables L_m[a K + b] (relative, as lt)
  double* partial = nullptr;   // [n1 chunks][K^2] plate-sum partials
  double* hsum = nullptr;      // [n0][K^2] sum over users
  float* W = nullptr;          // [n0][K^2] joint root weights
  int* cidx = nullptr;         // [n0][K^2] kept pairs
  int* ccnt = nullptr;         // [n0]
  float* cw = nullptr;         // [n0][K^2]
  float* wab = nullptr;        // [n0][2][K] (w_mu, w_psi)
};

}  // namespace qem

namespace qem {
// Launch shapes chosen by the autotuner (qem_tune.cu); the defaults are
// what an untuned plan uses.
struct Tune {
  int sample_threads = 128;  // threads per block of the sampler (one block per element)
  int mom_threads = 256;     // threads per block of the moments kernel (one block per element)
  int fwd_rows = 128;        // FP32 contraction: parent samples per block (one per thread)
  int fwd_chunk = 32;        // FP32 contraction: child samples staged per shared-memory round
  int tc_sched = 3;          // tensor-core schedules, bit 0: element-resident forward, bit 1: element-resident
                             // adjoint (each when its operands fit); a clear bit: the streaming schedule
};
}  // namespace qem

struct qem_plan_s {
  int L = 0;
  int K = 0;
  int precision = 0;
  int tile = 0;
  cudaStream_t stream = nullptr;
  double var_floor = 1e-10;
  double timeout_s = 2.0;
  int expire_test = 0;         // qem_test_expire_wait
  int device = 0;
  int num_sms = 0;
  long long clock_khz = 0;
  qem::LevelView lv[QEM_MAX_LEVELS];
  long long q_off[QEM_MAX_LEVELS], eps_off[QEM_MAX_LEVELS], w_off[QEM_MAX_LEVELS], z_off[QEM_MAX_LEVELS];
  long long q_len = 0, eps_len = 0, w_len = 0, z_len = 0;
  double* log_pmp = nullptr;   // [n_inst] of the last E-step
  double* count_tab = nullptr; // [kCountTable] Poisson-log count constants (nullptr: no such level)
  qem::Ctl* ctl = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  qem::TcBuffers* tc = nullptr;
  void* prof = nullptr;        // per-kernel event records (qem_api.cu)
  void* run = nullptr;         // cached device-loop graph of qem_run (qem_api.cu)
  qem::Tune tune;              // launch shapes (defaults, or chosen by qem_tune)
  qem::SplitWs* split = nullptr; // split-root workspace (qem_estep_split_root), allocated on first use
  int* perm_own = nullptr;     // qcond: the plan's drawn permutations [n_1][K]
  const int* perm_user = nullptr; // qcond: caller-supplied permutations (qem_set_perm)
  bool tuned = false;          // qem_tune has run (or a cached choice was applied)
};

namespace qem {

// ---------------------------------------------------------------------------
// Packed FP32 pair arithmetic (one instruction for two lanes of work):
// (a0, a1) <- (a0, a1) + (b0, b1) * (c0, c1), and (d0, d1) = (x0 - y0, x1 - y1).
__device__ __forceinline__ void fma2(float& a0, float& a1, float b0, float b1, float c0, float c1) {
  asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n mov.b64 z, {%0, %1};\n"
      " fma.rn.f32x2 z, x, y, z;\n mov.b64 {%0, %1}, z;\n}\n"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}
__device__ __forceinline__ void diff2(float& d0, float& d1, float x0, float x1, float y0, float y1) {
  asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
      " sub.rn.f32x2 z, x, y;\n mov.b64 {%0, %1}, z;\n}\n"
      : "=f"(d0), "=f"(d1)
      : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}
__device__ __forceinline__ void mul2(float& d0, float& d1, float x0, float x1, float y0, float y1) {
  asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
      " mul.rn.f32x2 z, x, y;\n mov.b64 {%0, %1}, z;\n}\n"
      : "=f"(d0), "=f"(d1)
      : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}

// ---------------------------------------------------------------------------
// Block-wide copy of n consecutive floats (sample rows of width D) from global
// memory into shared rows of stride D + 1: 16-byte loads when the source is
// aligned, four of them in flight per thread before their stores (the copies
// are latency-bound otherwise: one load at a time per thread).
template <int DC>  // DC > 0: the width known at compile time; 0: D at run time
__device__ __forceinline__ void stage_rows(const float* __restrict__ src, int n, int Drt, float* dst) {
  const int D = DC > 0 ? DC : Drt;
  const int ZS = D + 1;
  const int nth = blockDim.x;
  int head = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const int n4 = n >> 2;
    for (int i0 = threadIdx.x; i0 < n4; i0 += 4 * nth) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u * nth < n4) v[u] = s4[i0 + u * nth];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = i0 + u * nth;
        if (idx < n4) {
          const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
          int r = (4 * idx) / D, c = (4 * idx) % D;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            dst[r * ZS + c] = vv[j];
            if (++c == D) {
              c = 0;
              ++r;
            }
          }
        }
      }
    }
    head = n4 << 2;
  }
  for (int i = head + threadIdx.x; i < n; i += nth) dst[(i / D) * ZS + (i % D)] = src[i];
}

// ---------------------------------------------------------------------------
// Counter-based noise: Philox4x32-10 (Salmon et al., SC'11) with the counter
// layout key = seed, ctr = (sample lo, sample hi, level<<24 | idx/4, iter).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// -2 log u for u = (x + 0.5) 2^-32, accurate at both ends of (0, 1).
__device__ __forceinline__ float neg2_log_unit(uint32_t x) {
  if (x < 0x80000000u) return -2.f * logf(((float)x + 0.5f) * 2.3283064365386963e-10f);
  const float one_minus_u = ((float)(0xFFFFFFFFu - x) + 0.5f) * 2.3283064365386963e-10f;
  return -2.f * log1pf(-one_minus_u);
}

__device__ __forceinline__ float unit_of(uint32_t x) { return ((float)x + 0.5f) * 2.3283064365386963e-10f; }

// log(1 + t) for t in [-1/2, 1] without a library call or a branch:
// log(1 + t) = 2 atanh(s), s = t / (2 + t) in [-1/3, 1/3], and the odd series
// of atanh to s^15 (truncation below 1e-8 relative); relative error a few
// units of FP32 rounding, for every t in the range including tiny |t|.
__device__ __forceinline__ float log1p_small(float t) {
  const float s = __fdividef(t, 2.f + t), s2 = s * s;
  float p = 1.f / 15.f;
  p = fmaf(p, s2, 1.f / 13.f);
  p = fmaf(p, s2, 1.f / 11.f);
  p = fmaf(p, s2, 1.f / 9.f);
  p = fmaf(p, s2, 1.f / 7.f);
  p = fmaf(p, s2, 1.f / 5.f);
  p = fmaf(p, s2, 1.f / 3.f);
  p = fmaf(p, s2, 1.f);
  return 2.f * s * p;
}

// -2 log u for the Box-Muller radius: the fast logarithm for u < 1/2 (small
// relative error there), log1p of -(1-u) near u = 1 (1-u carries the low
// bits of the uniform).
__device__ __forceinline__ float neg2_log_unit_fast(uint32_t x) {
  if (x < 0x80000000u) return -2.f * __logf(((float)x + 0.5f) * 2.3283064365386963e-10f);
  const float one_minus_u = ((float)(0xFFFFFFFFu - x) + 0.5f) * 2.3283064365386963e-10f;
  return -2.f * log1p_small(-one_minus_u);
}

// sqrt(r) for r > 0 from the fast reciprocal square root.
__device__ __forceinline__ float sqrt_pos_fast(float r) { return r * rsqrtf(r); }

// Four N(0,1) numbers of block `blk` of one sample (Box-Muller on (u0,u1), (u2,u3)).
// The angle 2 pi u is evaluated as pi + (2 pi u - pi) with the fast sine and
// cosine on (-pi, pi) (absolute error ~2^-21), so the draws agree with an
// exact evaluation of the same uniforms to ~1e-6.
__device__ __forceinline__ float4 normal4(unsigned long long seed, unsigned long long iter, int level,
                                          unsigned long long sample, uint32_t blk) {
  const uint4 r = philox4x32_10(
      make_uint4((uint32_t)sample, (uint32_t)(sample >> 32), ((uint32_t)level << 24) | blk, (uint32_t)iter),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float t0 = fmaf(6.283185307179586f, unit_of(r.y), -3.141592653589793f);
  const float t1 = fmaf(6.283185307179586f, unit_of(r.w), -3.141592653589793f);
  float s0, c0, s1, c1;
  __sincosf(t0, &s0, &c0);
  __sincosf(t1, &s1, &c1);
  const float r0 = sqrt_pos_fast(neg2_log_unit_fast(r.x)), r1 = sqrt_pos_fast(neg2_log_unit_fast(r.z));
  return make_float4(-r0 * c0, -r0 * s0, -r1 * c1, -r1 * s1);
}

// One noise number of index idx (normal or uniform slot, as the family's layout says).
__device__ __forceinline__ float noise_at(unsigned long long seed, unsigned long long iter, int level,
                                          unsigned long long sample, int idx, int qfam) {
  const uint4 r = philox4x32_10(
      make_uint4((uint32_t)sample, (uint32_t)(sample >> 32), ((uint32_t)level << 24) | (uint32_t)(idx >> 2),
                 (uint32_t)iter),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint32_t v[4] = {r.x, r.y, r.z, r.w};
  const int j = idx & 3;
  bool uni = false;
  if (qfam != QEM_Q_GAUSS) {
    const int blk = 2 * QEM_GAMMA_TRIES + 1, rr = idx % blk;
    uni = (rr == blk - 1) || (rr & 1);
  }
  if (uni) return unit_of(v[j]);
  const float rad = sqrtf(neg2_log_unit(v[j & 2]));
  float s, c;
  sincospif(2.f * unit_of(v[(j & 2) + 1]), &s, &c);
  return (j & 1) ? rad * s : rad * c;
}

// Bounded spin on a flag (for device-side waits): returns false on expiry.
__device__ __forceinline__ bool spin_until_ge(const volatile int* flag, int target, long long max_cycles) {
  const long long t0 = clock64();
  while (*flag < target) {
    if (clock64() - t0 > max_cycles) return false;
    __nanosleep(64);
  }
  return true;
}

// ---------------------------------------------------------------------------
// Host-side launchers (qem_simt.cu / qem_tc.cu).
cudaError_t launch_loop_begin(Ctl* ctl, long long iterations, cudaStream_t s);
cudaError_t launch_loop_next(Ctl* ctl, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_set_ctl(Ctl* ctl, unsigned long long seed, unsigned long long iter, long long t,
                           long long trace_row, cudaStream_t s);
cudaError_t launch_advance_ctl(Ctl* ctl, long long n_inst, cudaStream_t s);
// Counts y < kCountTable of a Poisson-log likelihood take their constant
// y s0 - e^s0 - lgamma(y + 1) from a table built once per plan.
// Dynamic shared memory a kernel is opted into (the sm_103a per-block
// maximum).  Kernels are opted into the maximum, not the current plan's
// need: the attribute is per kernel and process-wide, so a plan that set a
// smaller value would make an earlier plan's larger launches fail.
constexpr int kSmemOptIn = 227 * 1024;
// Opt kernel f into all the dynamic shared memory it can have (the maximum
// less its static shared memory); cudaErrorInvalidValue when `need` bytes
// do not fit.
template <class T>
inline cudaError_t opt_in_smem(T* f, size_t need) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  const int avail = kSmemOptIn - (int)fa.sharedSizeBytes;
  if (need > (size_t)avail) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, avail);
}
constexpr int kCountTable = 4096;
cudaError_t launch_count_table(double* tab, cudaStream_t s);
cudaError_t launch_elem_const(const LevelView& v, const float* q, cudaStream_t s);
cudaError_t launch_sample_local(const LevelView& v, int K, int threads, const float* q, const float* eps, const Ctl* ctl,
                                cudaStream_t s);
cudaError_t launch_parent_params(const LevelView& parent, const LevelView& child, int K, cudaStream_t s);
cudaError_t launch_finalize(const LevelView& v, int K, bool has_children, cudaStream_t s);
// split: the parent's rows are the K^2 pairs of its two halves (qem_split.cu).
cudaError_t launch_fwd_simt(const LevelView& v, const LevelView& parent, int K, int rows, int chunk, cudaStream_t s,
                            bool split = false);
cudaError_t launch_plate_sum(const LevelView& parent, const LevelView& child, int K, cudaStream_t s);
cudaError_t launch_root(const LevelView& v, int K, bool has_children, double* log_pmp, double* user_out,
                        double* trace, Ctl* ctl, cudaStream_t s);
// Kc: sample count of the children (0: K).
cudaError_t launch_compact(const LevelView& parent, int K, float rel, cudaStream_t s, int Kc = 0);
// (levels with qcond also write cz, the joint-weighted parent sample per child sample)
cudaError_t launch_adj_compact(const LevelView& v, const LevelView& parent, int K, int max_eff, cudaStream_t s,
                               bool split = false);
cudaError_t launch_adj_small(const LevelView& v, const LevelView& parent, int K, cudaStream_t s);
cudaError_t configure_adj_small(int D, int K);
cudaError_t launch_moments(const LevelView& v, int K, int threads, double* mom, cudaStream_t s);
cudaError_t launch_mstep(const LevelView& v, const double* mom, double* m, float* q, double lambda,
                         double sched_p, double var_floor, long long t_host, Ctl* ctl, cudaStream_t s);
size_t sample_local_smem(const LevelView& v, int K, int threads);
constexpr int kSampleThreadsLimit = 256;   // largest sampler block the tuner tries
cudaError_t configure_sample_local(size_t smem);
cudaError_t launch_mean_params(const LevelView& v, const float* q, double* m, cudaStream_t s);
cudaError_t launch_moments_rescale(const LevelView* lvs, int l, const double* lp_same, const double* lp_fresh,
                                   double* mom, cudaStream_t s);
cudaError_t launch_split_unary(const LevelView& root, int K, const float* q, double* fa, double* fb, cudaStream_t s);
cudaError_t launch_split_root(int n_inst, int K, const double* fa, const double* fb, const double* hsum, float* W,
                              float* wab, float* w0, double* log_pmp, double* user_out, Ctl* ctl, cudaStream_t s);
cudaError_t launch_split_root_moments(const LevelView& root, int K, const float* wab, double* mom, cudaStream_t s);
// Chain plates (qem_chain.cu): the forward over each region's days and the
// root-to-leaf adjoint; one block per region.
cudaError_t launch_chain_forward(const LevelView& v, const LevelView& parent, int K, cudaStream_t s);
cudaError_t launch_chain_adjoint(const LevelView& v, const LevelView& parent, int K, cudaStream_t s);
cudaError_t configure_chain(int D, int K);
// Parent-conditioned proposals (qem_simt.cu): the counter-based permutations
// and the residual moments.
cudaError_t launch_draw_perm(const LevelView& v, int K, int* perm, const Ctl* ctl, cudaStream_t s);
cudaError_t launch_residual_moments(const LevelView& v, int K, const double* mom_parent, double* mom, cudaStream_t s);
cudaError_t launch_predictive(const LevelView& v, int K, const float* xn, const float* yn, int nn, double* out,
                              cudaStream_t s);

}  // namespace qem
