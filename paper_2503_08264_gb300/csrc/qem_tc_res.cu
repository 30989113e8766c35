// Element-resident schedules of the tensor-core contractions (sm_103a): the
// forward (k_fwd_res) and the adjoint (k_adj_res).
//
// Forward tile of plate element e (Eq. Prmp, organised per Sec. 6):
//   S_e[kp][k] = rowc[kp] + sum_f A_p[kp][f] B_e[k][f] + h_e[k]   (log2 units),
//   lt[e][kp]  = rowc[kp] + ln 2 * log2 sum_k 2^(S_e - rowc)[kp][k] - ln K,
// with A_p the parent's operand rows (shared by every child of the parent)
// and B_e the element's own rows.  Adjoint tile (Eq. mmp with the indicator
// moment; Sec. 3.2's source-term weights in closed form) over the parent
// samples the parent keeps (its compacted list of n_eff samples):
//   w[e][k] = sum_j 2^(B_e[k] . A_p[j] + h_e[k] + d_e[j]),
//   d_e[j]  = log2 e (rowc[kp_j] + ln w_p[kp_j] - ln K - lt_e[kp_j]).
//
// The streaming schedule in qem_tc.cu gives each CTA one 128-row block of one
// element and streams the other operand through shared memory chunk by
// chunk, 1.25 B of L2 traffic per pair for the forward's 80-column
// split-BF16 rows.  Here one CTA takes whole elements and keeps one operand
// of the element in shared memory:
//  * forward: B_e (all K rows, 160 KB at K = 1024) stays while the parent's
//    K / 128 row blocks stream through a two-slot ring (0.37 B per pair);
//  * adjoint: the element's rows are taken in passes of four row blocks
//    while the parent's kept rows stream once per pass in chunks of 256
//    (0.55 B per pair at K = 1024).
// Tiles are 128 x 256 (the MMA's full rate; a narrower N is bound by the MMA
// issue rate) in two TMEM slots of 256 columns.  Roles (640 threads, one CTA
// per SM): warp 0 loads the row side, warp 1 the column side (and the
// adjoint's column shifts), warp 2 issues the MMAs (one lane) and owns
// TMEM, warp 3 is idle, warps 4..19 are the epilogue; warp w reads TMEM lanes
// 32 (w % 4) .. +31 (the rule of tcgen05.ld).
// The epilogue is two groups of eight warps that take alternate tiles
// (group g every tile of TMEM slot g), each warp half of a tile's columns in
// two pieces of 64; while one group waits for its tile, loads it or merges,
// the other exponentiates, so the ex2 unit is not left idle between tiles.
// Partial sums meet in shared memory (per row block in the forward, per pass
// of four row blocks in the adjoint), completed by the group that took the
// last tile, without a CTA-wide barrier.  The MMA warp runs converged and one
// elected lane issues.
//
// Every wait is bounded; an expired wait sets the CTA's abort flag, every
// role stops at its next wait, the producers wait (bounded, ignoring the
// flag) for their own copies and the MMA issuer for its MMAs before TMEM is
// freed, and the plan's control block gets ERR_TIMEOUT.
#include "qem_tc.cuh"
#include "qem_tc_ptx.cuh"

namespace qem {
namespace tc {

constexpr int kResMaxChunks = kBStagesMax;  // forward: one producer warp per resident chunk, K <= 1024

__host__ __device__ inline int imin(int x, int y) { return x < y ? x : y; }

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------- forward, columns resident
struct ResArgs {
  int K, R, C;                      // samples, row blocks (K / 128), column chunks (K / 256 rounded up)
  int frow, fcol, ksteps;           // operand row widths (16-bit units) and MMA k-steps
  int koff_row[16], koff_col[16];   // per k-step: 16-bit column offset in the row / column operand
  long long n_elts;
  const long long* parent;
  const __nv_bfloat16* rows_feat;   // A: parent operand rows [n_parent][K][frow]
  const __nv_bfloat16* cols_feat;   // B: element operand rows [n][K][fcol]
  const float* rowc;                // [n_parent][K] row constants (nats)
  float* lt;                        // [n][K] output
  Ctl* ctl;
  long long timeout_cycles;
  int expire_test;                  // qem_test_expire_wait
};

struct ResSmem {
  uint8_t* a0;       // two row blocks, a_stride apart
  uint8_t* b0;       // C column chunks of 256 rows, b_stride apart
  uint32_t a_stride, b_stride;
  uint64_t* a_full;
  uint64_t* a_empty;
  uint64_t* b_full;
  uint64_t* b_empty;
  uint64_t* t_full;   // [2]
  uint64_t* t_empty;  // [2]
  uint64_t* done;
  uint64_t* m_full;  // [2] a row block's partials written (one arrival per producing thread)
  uint64_t* m_free;  // [2] a row block's partials read (one arrival per completing thread)
  uint32_t* tmem_base;
  volatile int* abort_flag;
  float2* merge;     // [2][kRows][4] partial (max, sum) of every row, per (group, half)
};

__host__ __device__ inline size_t res_smem_bytes(int frow, int fcol, int K) {
  const size_t a = (size_t)kRows * frow * 2, b = (size_t)imin(K, kMaxN) * fcol * 2;
  const int C = (K + kMaxN - 1) / kMaxN;
  return 1024 + 2 * a + (size_t)C * b + 32 * 8 + 16 + 2 * kRows * 4 * sizeof(float2);
}

__device__ __forceinline__ ResSmem res_carve(uint8_t* raw, int frow, int fcol, int K) {
  ResSmem s;
  uint8_t* p = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  const int C = (K + kMaxN - 1) / kMaxN;
  s.a_stride = (uint32_t)kRows * frow * 2;
  s.b_stride = (uint32_t)imin(K, kMaxN) * fcol * 2;
  s.a0 = p;
  p += 2 * (size_t)s.a_stride;
  s.b0 = p;
  p += (size_t)C * s.b_stride;
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);
  s.a_full = bars + 0;
  s.a_empty = bars + 2;
  s.b_full = bars + 4;
  s.b_empty = bars + 4 + kResMaxChunks;
  s.t_full = bars + 4 + 2 * kResMaxChunks;
  s.t_empty = s.t_full + 2;
  s.done = s.t_empty + 2;
  s.m_full = s.done + 1;
  s.m_free = s.m_full + 2;
  p += 32 * 8;
  s.tmem_base = reinterpret_cast<uint32_t*>(p);
  s.abort_flag = reinterpret_cast<volatile int*>(p + 4);
  p += 16;
  s.merge = reinterpret_cast<float2*>(p);
  return s;
}

// Roles of the forward: warp 0 loads the parent's row blocks, warp 1 the
// element's column chunks, warp 2 issues the MMAs and owns TMEM, warp 3 is
// idle, warps 4..19 are the epilogue in two groups of 8 (640 threads: up to
// 96 registers per thread, room for a warp to hold 64 values at once).
constexpr int kFwdThreads = 640;
constexpr int kFwdMmaWarp = 2, kFwdEpiWarp0 = 4, kFwdGroupWarps = 8;

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// The 64 values of one row in one warp's piece of a tile, already in
// registers, folded into the row's online log-sum-exp in two passes: the
// exact maximum of the piece and the running one (four chains of
// three-input max), then every value shifted and exponentiated in place,
// then summed.  No exponential waits on another's sum, so all 64 can be in
// flight in the ex2 unit at once, and every term is at most 1 (no overflow).
// The values' registers are overwritten.
__device__ __forceinline__ void lse_regs64(uint32_t (&va)[32], uint32_t (&vb)[32], float& m, float& sacc) {
  const auto F = [](uint32_t x) { return __uint_as_float(x); };
  float c0 = fmaxf(F(va[0]), F(va[1])), c1 = fmaxf(F(va[16]), F(va[17]));
  float c2 = fmaxf(F(vb[0]), F(vb[1])), c3 = fmaxf(F(vb[16]), F(vb[17]));
#pragma unroll
  for (int j = 2; j < 16; j += 2) {
    c0 = max3f(c0, F(va[j]), F(va[j + 1]));
    c1 = max3f(c1, F(va[16 + j]), F(va[17 + j]));
    c2 = max3f(c2, F(vb[j]), F(vb[j + 1]));
    c3 = max3f(c3, F(vb[16 + j]), F(vb[17 + j]));
  }
  const float mn = max3f(max3f(c0, c1, m), c2, c3);
  if (mn != m) sacc *= ex2f(m - mn);  // the running sum moves to the new maximum (0 while m is -inf)
  m = mn;
#pragma unroll
  for (int j = 0; j < 32; j += 2) {
    float x0 = F(va[j]), x1 = F(va[j + 1]), y0 = F(vb[j]), y1 = F(vb[j + 1]);
    sub2(x0, x1, m);
    sub2(y0, y1, m);
    va[j] = __float_as_uint(ex2f(x0));
    va[j + 1] = __float_as_uint(ex2f(x1));
    vb[j] = __float_as_uint(ex2f(y0));
    vb[j + 1] = __float_as_uint(ex2f(y1));
  }
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
  for (int j = 0; j < 32; j += 2) {
    add2(p0, p1, F(va[j]), F(va[j + 1]));
    add2(p2, p3, F(vb[j]), F(vb[j + 1]));
  }
  add2(p0, p1, p2, p3);
  sacc += p0 + p1;
}

template <bool TF32>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd_res(ResArgs a) {
  extern __shared__ uint8_t smem_raw[];
  ResSmem s = res_carve(smem_raw, a.frow, a.fcol, a.K);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = a.K, R = a.R, C = a.C, frow = a.frow, fcol = a.fcol;
  const uint32_t sbo_a = (uint32_t)(frow >> 3) * 128u, sbo_b = (uint32_t)(fcol >> 3) * 128u;
  const uint32_t a_bytes = (uint32_t)kRows * frow * 2;
  const long long lim = a.timeout_cycles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.a_full[i], 1);
      mbar_init(&s.a_empty[i], 1);
      mbar_init(&s.t_full[i], 1);
      mbar_init(&s.t_empty[i], kFwdGroupWarps);
      // a row block's partials come from both groups when it has two tiles or more
      mbar_init(&s.m_full[i], 32 * kFwdGroupWarps * (C >= 2 ? 2 : 1));
      mbar_init(&s.m_free[i], kRows);
    }
    for (int c = 0; c < C; ++c) {
      mbar_init(&s.b_full[c], 1);
      mbar_init(&s.b_empty[c], 1);
    }
    mbar_init(s.done, 1);
    *s.abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kFwdMmaWarp) {
    tmem_alloc(s.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ row blocks of the parent
    if (lane == 0) {
      int as = 0;
      uint32_t aph = 0, armed = 0, last = 0;
      bool ok = true;
      for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x) {
        const long long p = a.parent[e];
        for (int rb = 0; rb < R; ++rb) {
          ok = mbar_wait(&s.a_empty[as], aph ^ 1, lim, s.abort_flag);
          if (!ok) break;
          mbar_expect_tx(&s.a_full[as], a_bytes);
          bulk_g2s(s.a0 + as * s.a_stride, a.rows_feat + (p * K + (long long)rb * kRows) * frow, a_bytes,
                   &s.a_full[as]);
          armed |= 1u << as;
          last = (last & ~(1u << as)) | (aph << as);
          if (++as == 2) {
            as = 0;
            aph ^= 1;
          }
        }
      }
      // no copy of this CTA may still be landing when it exits (bounded, ignores abort)
      volatile int never = 0;
      for (int i = 0; i < 2; ++i)
        if (armed & (1u << i)) mbar_wait(&s.a_full[i], (last >> i) & 1u, drain_bound(lim), &never);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ the element's column chunks
    // Chunk c of the next element is loaded once the last MMAs on chunk c of
    // this one have completed; the releases come in chunk order.
    if (lane == 0) {
      uint32_t armed = 0, last = 0;
      bool ok = true;
      int i = 0;
      for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x, ++i) {
        const uint32_t ph = (uint32_t)i & 1u;
        for (int c = 0; c < C; ++c) {
          const int c0 = c * kMaxN;
          const uint32_t bytes = (uint32_t)imin(kMaxN, K - c0) * fcol * 2;
          ok = mbar_wait(&s.b_empty[c], ph ^ 1u, lim, s.abort_flag);
          if (!ok) break;
          mbar_expect_tx(&s.b_full[c], bytes);
          bulk_g2s(s.b0 + c * s.b_stride, a.cols_feat + (e * K + c0) * fcol, bytes, &s.b_full[c]);
          armed |= 1u << c;
          last = (last & ~(1u << c)) | (ph << c);
        }
        const long long en = e + gridDim.x;  // the CTA's next element: warm L2 while this one is contracted
        if (ok && en < a.n_elts)
          for (int c = 0; c < C; ++c)
            bulk_prefetch_l2(a.cols_feat + (en * K + (long long)c * kMaxN) * fcol,
                             (uint32_t)imin(kMaxN, K - c * kMaxN) * fcol * 2);
      }
      volatile int never = 0;
      for (int c = 0; c < C; ++c)
        if (armed & (1u << c)) mbar_wait(&s.b_full[c], (last >> c) & 1u, drain_bound(lim), &never);
    }
  } else if (warp == kFwdMmaWarp) {
    // ------------------------------------------------------------ MMA issuer (one elected lane)
    {
      const int nks = a.ksteps;
      const uint64_t adesc0 = smem_desc(s.a0, 128, sbo_a), bdesc0 = smem_desc(s.b0, 128, sbo_b);
      const uint32_t a_step = s.a_stride >> 4, b_step = s.b_stride >> 4;
      const uint32_t fmt = TF32 ? 2u : 1u;
      int as = 0, ts = 0, i = 0;
      uint32_t aph = 0, tph = 0;
      bool ok = true;
      // test hook (qem_test_expire_wait): a wait on the teardown barrier, which
      // nothing completes before the teardown, runs out and aborts the CTA
      if (a.expire_test) ok = mbar_spin_warp(s.done, 0, lim, s.abort_flag);
      for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x, ++i) {
        const uint32_t bph = (uint32_t)i & 1u;
        for (int rb = 0; rb < R && ok; ++rb) {
          ok = mbar_spin_warp(&s.a_full[as], aph, lim, s.abort_flag);
          if (!ok) break;
          for (int c = 0; c < C; ++c) {
            const int nc = imin(kMaxN, K - c * kMaxN);
            if (rb == 0) ok = mbar_spin_warp(&s.b_full[c], bph, lim, s.abort_flag);
            if (ok) ok = mbar_spin_warp(&s.t_empty[ts], tph ^ 1u, lim, s.abort_flag);
            if (!ok) break;
            tc_fence_after();
            const uint32_t idesc = idesc_fmt(nc, fmt);
            const uint32_t d_tmem = tmem + (uint32_t)(ts * kMaxN);
            const uint64_t ad = adesc0 + (uint64_t)(as * a_step), bd = bdesc0 + (uint64_t)(c * b_step);
            if (elect_one()) {
#pragma unroll
              for (int ks = 0; ks < 16; ++ks)
                if (ks < nks)  // k-step offsets read from the kernel parameters (constant bank)
                  mma_kind<TF32>(d_tmem, ad + (uint32_t)a.koff_row[ks], bd + (uint32_t)a.koff_col[ks], idesc,
                                 ks > 0 ? 1u : 0u);
              mma_commit(&s.t_full[ts]);
              if (rb == R - 1) mma_commit(&s.b_empty[c]);  // the element's last use of chunk c
            }
            __syncwarp();
            ts ^= 1;
            if (ts == 0) tph ^= 1u;
          }
          if (!ok) break;
          if (elect_one()) mma_commit(&s.a_empty[as]);
          __syncwarp();
          if (++as == 2) {
            as = 0;
            aph ^= 1u;
          }
        }
      }
      // every issued MMA has completed before the teardown (bounded, ignores abort)
      if (elect_one()) mma_commit(s.done);
      __syncwarp();
      volatile int never = 0;
      mbar_wait(s.done, 0, drain_bound(lim), &never);
    }
    __syncwarp();
  } else if (warp >= kFwdEpiWarp0) {
    // ------------------------------------------------------------ epilogue (two groups of 8 warps)
    // The CTA's tiles form one sequence t over its elements, row blocks and
    // column chunks (the MMA issuer's order); tile t is in TMEM slot t % 2
    // and group g takes the tiles of slot g.  Warp (g, half, quarter) reads
    // TMEM lanes 32 quarter .. +31 and columns half * nc / 2 .. +nc / 2 of
    // the tile, 64 at a time, and hands the slot back after its last load.
    // At the end of a row block every producing thread writes its partial
    // (max, sum) to merge buffer n % 2 (n: the CTA's row-block count), and
    // the half-0 warps of the group that took the block's last tile combine
    // the partials into lt.  A group with no tile in the block (one column
    // chunk: the groups alternate row blocks) skips it.
    const int ew = warp - kFwdEpiWarp0;
    const int g = ew >> 3, half = (ew >> 2) & 1, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const float lnK = logf((float)K);
    const int j0 = C >= 2 ? 0 : 2 * g, j1 = C >= 2 ? 4 : 2 * g + 2;  // the producing (group, half) pairs
    uint32_t tph = 0, n = 0;
    int t0 = 0;  // the row block's first tile in the sequence
    bool ok = true;
    for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x) {
      const long long p = a.parent[e];
      for (int rb = 0; rb < R && ok; ++rb, ++n, t0 += C) {
        const int first = t0 + ((g - t0) & 1);
        if (first >= t0 + C) continue;
        const bool fin = half == 0 && ((t0 + C - 1) & 1) == g;
        const long long k = (long long)rb * kRows + row;
        // the row constant, read now so that its latency is spent under the block's tiles
        const float rc = fin ? a.rowc[p * K + k] : 0.f;
        float m = -INFINITY, sacc = 0.f;
        for (int t = first; t < t0 + C; t += 2) {
          const int w = imin(kMaxN, K - (t - t0) * kMaxN) >> 1;  // 128, or 64 in a 128-column last chunk
          ok = mbar_wait(&s.t_full[g], tph, lim, s.abort_flag);
          ok = __all_sync(0xffffffffu, ok);  // the TMEM loads below are warp-collective
          if (!ok) break;
          tc_fence_after();
          uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * kMaxN + half * w);
          uint32_t va[32], vb[32];
          if (w == 128) {
            tmem_ld32_issue(tb, va);
            tmem_ld32_issue(tb + 32u, vb);
            tmem_wait32(va);
            tmem_wait32(vb);
            lse_regs64(va, vb, m, sacc);
            tb += 64u;
          }
          tmem_ld32_issue(tb, va);
          tmem_ld32_issue(tb + 32u, vb);
          tmem_wait32(va);
          tmem_wait32(vb);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&s.t_empty[g]);
          tph ^= 1u;
          lse_regs64(va, vb, m, sacc);
        }
        if (!ok) break;
        const uint32_t bsel = n & 1u, use = n >> 1;
        float2* mb = s.merge + (size_t)bsel * kRows * 4;
        // buffer bsel is free once row block n - 2 has been combined
        if (use > 0) ok = mbar_wait(&s.m_free[bsel], (use - 1) & 1u, lim, s.abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        mb[row * 4 + 2 * g + half] = make_float2(m, sacc);
        mbar_arrive(&s.m_full[bsel]);
        if (fin) {
          ok = mbar_wait(&s.m_full[bsel], use & 1u, lim, s.abort_flag);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          float M = -INFINITY;
          for (int j = j0; j < j1; ++j) M = fmaxf(M, mb[row * 4 + j].x);
          float S = 0.f;
          for (int j = j0; j < j1; ++j) {
            const float2 o = mb[row * 4 + j];
            if (o.x != -INFINITY) S += o.y * ex2f(o.x - M);
          }
          a.lt[e * K + k] = rc + (M + log2f(S)) * kLn2 - lnK;
          mbar_arrive(&s.m_free[bsel]);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // after the barrier: every role has stopped, so an abort by any of them is seen
  if (*s.abort_flag && threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_TIMEOUT);
  if (warp == kFwdMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------- adjoint, rows resident
// The element's K operand rows are taken in passes of up to four 128-row
// blocks (80 KB of split-BF16 rows in shared memory); in each pass the
// parent's kept rows stream once, in chunks of 256 (the MMA's full rate),
// through a two-deep ring with their column shifts, and every chunk meets
// the pass's row blocks in turn (tile = row block x chunk, 128 x 256, two
// TMEM slots).  Each epilogue thread keeps one partial sum per row block of
// the pass; at the pass's end the four column quarters of every row are
// added through shared memory.  Operand traffic: the element's rows once and
// the parent's kept rows once per pass, (2 * 224 + 160) B per kept parent
// sample and child sample pair / K at K = 1024 (0.55 B per pair).
constexpr int kAdjPassRows = 4;   // row blocks per pass

struct AdjResArgs {
  int K, R, frow, fcol, ksteps, nst;  // nst: depth of the chunk ring
  int koff_row[16], koff_col[16];
  long long n_elts;
  const long long* parent;
  const int* ccnt;                    // kept samples per parent
  int small;                          // parents keeping <= small are skipped (CUDA-core adjoint)
  const __nv_bfloat16* rows_feat;     // element operand rows [n][K][frow]
  const __nv_bfloat16* cols_feat;     // compacted parent rows [n_parent][K][fcol]
  const float* dcol;                  // [n][K] column shifts (log2 units)
  float* w_out;                       // [n][K]
  Ctl* ctl;
  long long timeout_cycles;
  int expire_test;                  // qem_test_expire_wait
};

struct AdjSmem {
  uint8_t* a0;       // kAdjPassRows row blocks, a_stride apart
  uint8_t* b0;       // nst column chunks of 256 rows, b_stride apart
  float* d0;         // nst column-shift rows of 256 floats
  float* merge;      // [2][kAdjPassRows][kRows][4] partial row sums of a pass, per (group, half)
  uint32_t a_stride, b_stride;
  uint64_t* a_full;   // [kAdjPassRows]
  uint64_t* a_empty;  // [kAdjPassRows]
  uint64_t* b_full;   // [nst]
  uint64_t* b_empty;  // [nst]
  uint64_t* d_full;   // [nst]
  uint64_t* d_empty;  // [nst]
  uint64_t* t_full;   // [2]
  uint64_t* t_empty;  // [2]
  uint64_t* done;
  uint64_t* m_full;   // [2] a pass's partials written (one arrival per epilogue thread)
  uint64_t* m_free;   // [2] a pass's partials read (one arrival per completing thread)
  uint32_t* tmem_base;
  volatile int* abort_flag;
};

__host__ __device__ inline size_t adj_res_smem_bytes(int frow, int fcol, int nst) {
  return 1024 + (size_t)kAdjPassRows * kRows * frow * 2 + (size_t)nst * kMaxN * fcol * 2 + (size_t)nst * kMaxN * 4 +
         2 * (size_t)kAdjPassRows * kRows * 4 * 4 + 40 * 8 + 16;
}

__device__ __forceinline__ AdjSmem adj_carve(uint8_t* raw, int frow, int fcol, int nst) {
  AdjSmem s;
  uint8_t* p = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  s.a_stride = (uint32_t)kRows * frow * 2;
  s.b_stride = (uint32_t)kMaxN * fcol * 2;
  s.a0 = p;
  p += (size_t)kAdjPassRows * s.a_stride;
  s.b0 = p;
  p += (size_t)nst * s.b_stride;
  s.d0 = reinterpret_cast<float*>(p);
  p += (size_t)nst * kMaxN * 4;
  s.merge = reinterpret_cast<float*>(p);
  p += 2 * (size_t)kAdjPassRows * kRows * 4 * 4;
  uint64_t* bars = reinterpret_cast<uint64_t*>(p);
  s.a_full = bars;
  s.a_empty = bars + kAdjPassRows;
  s.b_full = bars + 2 * kAdjPassRows;
  s.b_empty = s.b_full + 4;
  s.d_full = s.b_empty + 4;
  s.d_empty = s.d_full + 4;
  s.t_full = s.d_empty + 4;
  s.t_empty = s.t_full + 2;
  s.done = s.t_empty + 2;
  s.m_full = s.done + 1;
  s.m_free = s.m_full + 2;
  p += 40 * 8;
  s.tmem_base = reinterpret_cast<uint32_t*>(p);
  s.abort_flag = reinterpret_cast<volatile int*>(p + 4);
  return s;
}

// sum_j 2^(v_j + d_j) over one warp's 64 columns of a tile row, in two
// passes: every value shifted and exponentiated in place, then summed, so
// that no exponential waits on another's sum.
__device__ __forceinline__ float adj_sum64(float (&va)[32], float (&vb)[32], const float* d) {
  const float4* d4 = reinterpret_cast<const float4*>(d);
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 da = d4[j >> 2], db = d4[8 + (j >> 2)];
    add2(va[j], va[j + 1], da.x, da.y);
    add2(va[j + 2], va[j + 3], da.z, da.w);
    add2(vb[j], vb[j + 1], db.x, db.y);
    add2(vb[j + 2], vb[j + 3], db.z, db.w);
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    va[j] = ex2f(va[j]);
    vb[j] = ex2f(vb[j]);
  }
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
  for (int j = 0; j < 32; j += 2) {
    add2(p0, p1, va[j], va[j + 1]);
    add2(p2, p3, vb[j], vb[j + 1]);
  }
  add2(p0, p1, p2, p3);
  return p0 + p1;
}

template <bool TF32>
__global__ void __launch_bounds__(kFwdThreads, 1) k_adj_res(AdjResArgs a) {
  extern __shared__ uint8_t smem_raw[];
  const int NS = a.nst;
  AdjSmem s = adj_carve(smem_raw, a.frow, a.fcol, NS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = a.K, R = a.R, frow = a.frow, fcol = a.fcol;
  const int passes = (R + kAdjPassRows - 1) / kAdjPassRows;
  const uint32_t sbo_a = (uint32_t)(frow >> 3) * 128u, sbo_b = (uint32_t)(fcol >> 3) * 128u;
  const uint32_t a_bytes = (uint32_t)kRows * frow * 2;
  const long long lim = a.timeout_cycles;

  if (threadIdx.x == 0) {
    for (int j = 0; j < kAdjPassRows; ++j) {
      mbar_init(&s.a_full[j], 1);
      mbar_init(&s.a_empty[j], 1);
    }
    for (int i = 0; i < NS; ++i) {
      mbar_init(&s.b_full[i], 1);
      mbar_init(&s.b_empty[i], 1);
      mbar_init(&s.d_full[i], 1);
      mbar_init(&s.d_empty[i], kEpiWarps);  // every epilogue warp, with or without tiles on the chunk
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.t_full[i], 1);
      mbar_init(&s.t_empty[i], kFwdGroupWarps);
      mbar_init(&s.m_full[i], 32 * kEpiWarps);
      mbar_init(&s.m_free[i], kRows);
    }
    mbar_init(s.done, 1);
    *s.abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kFwdMmaWarp) {
    tmem_alloc(s.tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_base;

  // the elements of this CTA whose parent keeps more than `small` samples,
  // the same sequence in every role
  auto kept_of = [&](long long e) { return a.ccnt[a.parent[e]]; };

  if (warp == 0) {
    // ------------------------------------------------------------ row blocks of the element, pass by pass
    if (lane == 0) {
      uint32_t uses = 0, armed = 0, last = 0;  // uses: 4 bits per slot (use count parity in bit 0 of each nibble)
      bool ok = true;
      for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x) {
        if (kept_of(e) <= a.small) continue;
        for (int h = 0; h < passes && ok; ++h) {
          const int nrb = imin(kAdjPassRows, R - h * kAdjPassRows);
          for (int j = 0; j < nrb; ++j) {
            const uint32_t ph = (uses >> j) & 1u;
            ok = mbar_wait(&s.a_empty[j], ph ^ 1u, lim, s.abort_flag);
            if (!ok) break;
            mbar_expect_tx(&s.a_full[j], a_bytes);
            bulk_g2s(s.a0 + j * s.a_stride, a.rows_feat + (e * K + (long long)(h * kAdjPassRows + j) * kRows) * frow,
                     a_bytes, &s.a_full[j]);
            armed |= 1u << j;
            last = (last & ~(1u << j)) | (ph << j);
            uses ^= 1u << j;
          }
        }
      }
      volatile int never = 0;
      for (int j = 0; j < kAdjPassRows; ++j)
        if (armed & (1u << j)) mbar_wait(&s.a_full[j], (last >> j) & 1u, drain_bound(lim), &never);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ parent chunks and column shifts, once per pass
    if (lane == 0) {
      uint32_t armed_b = 0, armed_d = 0, last_b = 0, last_d = 0;
      bool ok = true;
      long long g = 0;
      for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x) {
        const long long p = a.parent[e];
        const int n_eff = a.ccnt[p];
        if (n_eff <= a.small) continue;
        const int npad = imin(K, (n_eff + 15) & ~15);
        for (int h = 0; h < passes && ok; ++h)
          for (int c0 = 0; c0 < npad; c0 += kMaxN, ++g) {
            const int st = (int)(g % NS);
            const uint32_t ph = (uint32_t)((g / NS) & 1);
            const int nc = imin(kMaxN, npad - c0);
            ok = mbar_wait(&s.b_empty[st], ph ^ 1u, lim, s.abort_flag);
            if (!ok) break;
            mbar_expect_tx(&s.b_full[st], (uint32_t)nc * fcol * 2);
            bulk_g2s(s.b0 + st * s.b_stride, a.cols_feat + (p * K + c0) * fcol, (uint32_t)nc * fcol * 2,
                     &s.b_full[st]);
            armed_b |= 1u << st;
            last_b = (last_b & ~(1u << st)) | (ph << st);
            ok = mbar_wait(&s.d_empty[st], ph ^ 1u, lim, s.abort_flag);
            if (!ok) break;
            mbar_expect_tx(&s.d_full[st], (uint32_t)nc * 4u);
            bulk_g2s(s.d0 + st * kMaxN, a.dcol + e * K + c0, (uint32_t)nc * 4u, &s.d_full[st]);
            armed_d |= 1u << st;
            last_d = (last_d & ~(1u << st)) | (ph << st);
          }
      }
      volatile int never = 0;
      for (int st = 0; st < NS; ++st) {
        if (armed_b & (1u << st)) mbar_wait(&s.b_full[st], (last_b >> st) & 1u, drain_bound(lim), &never);
        if (armed_d & (1u << st)) mbar_wait(&s.d_full[st], (last_d >> st) & 1u, drain_bound(lim), &never);
      }
    }
  } else if (warp == kFwdMmaWarp) {
    // ------------------------------------------------------------ MMA issuer (one elected lane)
    {
      const int nks = a.ksteps;
      const uint64_t adesc0 = smem_desc(s.a0, 128, sbo_a), bdesc0 = smem_desc(s.b0, 128, sbo_b);
      const uint32_t a_step = s.a_stride >> 4, b_step = s.b_stride >> 4;
      const uint32_t fmt = TF32 ? 2u : 1u;
      uint32_t uses = 0;  // bit j: use parity of row-block slot j
      int ts = 0;
      uint32_t tph = 0;
      bool ok = true;
      // test hook (qem_test_expire_wait): a wait on the teardown barrier, which
      // nothing completes before the teardown, runs out and aborts the CTA
      if (a.expire_test) ok = mbar_spin_warp(s.done, 0, lim, s.abort_flag);
      long long g = 0;
      for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x) {
        const int n_eff = kept_of(e);
        if (n_eff <= a.small) continue;
        const int npad = imin(K, (n_eff + 15) & ~15);
        for (int h = 0; h < passes && ok; ++h) {
          const int nrb = imin(kAdjPassRows, R - h * kAdjPassRows);
          for (int c0 = 0; c0 < npad && ok; c0 += kMaxN, ++g) {
            const int st = (int)(g % NS);
            const uint32_t bph = (uint32_t)((g / NS) & 1);
            const int nc = imin(kMaxN, npad - c0);
            const bool last_chunk = c0 + kMaxN >= npad;
            ok = mbar_spin_warp(&s.b_full[st], bph, lim, s.abort_flag);
            if (!ok) break;
            const uint32_t idesc = idesc_fmt(nc, fmt);
            const uint64_t bd = bdesc0 + (uint64_t)(st * b_step);
            for (int j = 0; j < nrb; ++j) {
              if (c0 == 0) ok = mbar_spin_warp(&s.a_full[j], (uses >> j) & 1u, lim, s.abort_flag);
              if (ok) ok = mbar_spin_warp(&s.t_empty[ts], tph ^ 1u, lim, s.abort_flag);
              if (!ok) break;
              tc_fence_after();
              const uint32_t d_tmem = tmem + (uint32_t)(ts * kMaxN);
              const uint64_t ad = adesc0 + (uint64_t)(j * a_step);
              if (elect_one()) {
#pragma unroll
                for (int ks = 0; ks < 16; ++ks)
                  if (ks < nks)
                    mma_kind<TF32>(d_tmem, ad + (uint32_t)a.koff_row[ks], bd + (uint32_t)a.koff_col[ks], idesc,
                                   ks > 0 ? 1u : 0u);
                mma_commit(&s.t_full[ts]);
                if (last_chunk) mma_commit(&s.a_empty[j]);
              }
              __syncwarp();
              ts ^= 1;
              if (ts == 0) tph ^= 1u;
              if (last_chunk) uses ^= 1u << j;
            }
            if (ok) {
              if (elect_one()) mma_commit(&s.b_empty[st]);
              __syncwarp();
            }
          }
        }
      }
      if (elect_one()) mma_commit(s.done);
      __syncwarp();
      volatile int never = 0;
      mbar_wait(s.done, 0, drain_bound(lim), &never);
    }
    __syncwarp();
  } else if (warp >= kFwdEpiWarp0) {
    // ------------------------------------------------------------ epilogue (two groups of 8 warps)
    // The CTA's tiles form one sequence T over its elements, passes, chunks
    // and row blocks (the MMA issuer's order); tile T is in TMEM slot T % 2
    // and group g takes the tiles of slot g.  Warp (g, half, quarter) reads
    // TMEM lanes 32 quarter .. +31 and its half of each tile's columns (in
    // 16-column groups, the first half taking the odd one; 128 columns as two
    // pieces of 64 for a full chunk) and keeps one partial sum per row block
    // of the pass.  Every warp waits for every chunk's column shifts and
    // releases them after its tiles of the chunk, also where it has none, so
    // that neither group gets a stage ahead of the other.  At the end of a
    // pass every thread writes its partials to merge buffer np % 2 (np: the
    // CTA's pass count), and the half-0 warps of the group with the pass's
    // last tile add the four partials of every row.
    const int ew = warp - kFwdEpiWarp0;
    const int g = ew >> 3, half = (ew >> 2) & 1, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    uint32_t tph = 0, np = 0;
    int T = 0;
    long long gc = 0;
    bool ok = true;
    for (long long e = blockIdx.x; e < a.n_elts && ok; e += gridDim.x) {
      const int n_eff = kept_of(e);
      if (n_eff <= a.small) continue;
      const int npad = imin(K, (n_eff + 15) & ~15);
      const int nch = (npad + kMaxN - 1) / kMaxN;
      for (int h = 0; h < passes && ok; ++h, ++np) {
        const int nrb = imin(kAdjPassRows, R - h * kAdjPassRows);
        const bool fin = half == 0 && ((T + nch * nrb - 1) & 1) == g;
        float acc[kAdjPassRows] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < npad && ok; c0 += kMaxN, ++gc) {
          const int st = (int)(gc % NS);
          const uint32_t dph = (uint32_t)((gc / NS) & 1);
          const int n16 = imin(kMaxN, npad - c0) >> 4;
          const int cbase = half ? ((n16 + 1) >> 1) << 4 : 0;  // this warp's columns of the chunk
          const int ncw = (half ? n16 >> 1 : (n16 + 1) >> 1) << 4;
          ok = mbar_wait(&s.d_full[st], dph, lim, s.abort_flag);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          const float* dsm = s.d0 + st * kMaxN + cbase;
#pragma unroll
          for (int j = 0; j < kAdjPassRows; ++j) {
            if (j >= nrb) break;
            if (((T + j) & 1) != g) continue;
            ok = mbar_wait(&s.t_full[g], tph, lim, s.abort_flag);
            ok = __all_sync(0xffffffffu, ok);  // the TMEM loads below are warp-collective
            if (!ok) break;
            tc_fence_after();
            const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * kMaxN + cbase);
            float sum = 0.f;
            if (ncw == 128) {
              // each load completes inside its own asm block (this kernel spills a
              // few registers; no spill may fall between a load and its wait)
              float va[32], vb[32];
              tmem_ld32(tb, va);
              tmem_ld32(tb + 32u, vb);
              sum = adj_sum64(va, vb, dsm);
              tmem_ld32(tb + 64u, va);
              tmem_ld32(tb + 96u, vb);
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&s.t_empty[g]);
              sum += adj_sum64(va, vb, dsm + 64);
            } else {
              for (int c = 0; c < ncw; c += 16) {
                float v[16];
                tmem_ld16(tb + (uint32_t)c, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = ex2f(v[q] + dsm[c + q]);
#pragma unroll
                for (int q = 0; q < 16; q += 4) sum += (v[q] + v[q + 1]) + (v[q + 2] + v[q + 3]);
              }
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&s.t_empty[g]);
            }
            acc[j] += sum;
            tph ^= 1u;
          }
          T += nrb;
          __syncwarp();
          if (lane == 0 && ok) mbar_arrive(&s.d_empty[st]);
        }
        if (!ok) break;
        const uint32_t bsel = np & 1u, use = np >> 1;
        float* mb = s.merge + (size_t)bsel * kAdjPassRows * kRows * 4;
        // buffer bsel is free once pass np - 2 has been added up
        if (use > 0) ok = mbar_wait(&s.m_free[bsel], (use - 1) & 1u, lim, s.abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
#pragma unroll
        for (int j = 0; j < kAdjPassRows; ++j) mb[(j * kRows + row) * 4 + 2 * g + half] = acc[j];
        mbar_arrive(&s.m_full[bsel]);
        if (fin) {
          ok = mbar_wait(&s.m_full[bsel], use & 1u, lim, s.abort_flag);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          for (int j = 0; j < nrb; ++j) {
            const float* mr = mb + (j * kRows + row) * 4;
            a.w_out[e * K + (long long)(h * kAdjPassRows + j) * kRows + row] = (mr[0] + mr[1]) + (mr[2] + mr[3]);
          }
          mbar_arrive(&s.m_free[bsel]);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // after the barrier: every role has stopped, so an abort by any of them is seen
  if (*s.abort_flag && threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_TIMEOUT);
  if (warp == kFwdMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace tc

using namespace tc;

bool tc_res_fits(int frow, int fcol, int K) {
  return K % kRows == 0 && K <= kResMaxChunks * kMaxN && res_smem_bytes(frow, fcol, K) <= kSmemLimit;
}

// Deepest chunk ring of the resident adjoint that fits (0: it does not fit).
static int tc_adj_res_stages(int frow, int fcol, int K) {
  if (K % kRows != 0) return 0;
  for (int nst = 4; nst >= 2; --nst)
    if (adj_res_smem_bytes(frow, fcol, nst) <= kSmemLimit) return nst;
  return 0;
}

bool tc_adj_res_fits(int frow, int fcol, int K) { return tc_adj_res_stages(frow, fcol, K) > 0; }

qem_status tc_res_init(int frow, int fcol, int K, bool tf32) {
  cudaError_t e = cudaSuccess;
  if (tc_res_fits(frow, fcol, K)) {
    const size_t bytes = res_smem_bytes(frow, fcol, K);
    e = tf32 ? opt_in_smem(k_fwd_res<true>, bytes) : opt_in_smem(k_fwd_res<false>, bytes);
  }
  // the adjoint's rows are the child operand (fcol wide), its columns the parent's (frow wide)
  const int nst = tc_adj_res_stages(fcol, frow, K);
  if (e == cudaSuccess && nst > 0) {
    const size_t bytes = adj_res_smem_bytes(fcol, frow, nst);
    e = tf32 ? opt_in_smem(k_adj_res<true>, bytes) : opt_in_smem(k_adj_res<false>, bytes);
  }
  return e == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

static long long res_timeout_cycles(qem_plan_t P) { return (long long)(P->timeout_s * (double)P->clock_khz * 1e3); }

cudaError_t tc_forward_res(qem_plan_t P, int l, bool tf32) {
  TcBuffers& T = *P->tc;
  const LevelView& ch = P->lv[l];
  const Layout& L = T.lay[l];
  if (ch.n == 0) return cudaSuccess;
  ResArgs a{};
  a.K = P->K;
  a.R = P->K / kRows;
  a.C = (P->K + kMaxN - 1) / kMaxN;
  a.frow = L.fka;
  a.fcol = L.fkb;
  a.ksteps = L.nks;
  for (int i = 0; i < L.nks; ++i) {
    a.koff_row[i] = L.ka[i];
    a.koff_col[i] = L.kb[i];
  }
  a.n_elts = ch.n;
  a.parent = ch.parent;
  a.rows_feat = T.afeat[l];
  a.cols_feat = T.bfeat[l];
  a.rowc = T.rowc[l];
  a.lt = ch.lt;
  a.ctl = P->ctl;
  a.timeout_cycles = res_timeout_cycles(P);
  a.expire_test = P->expire_test;
  const long long grid = ch.n < P->num_sms ? ch.n : P->num_sms;
  const size_t smem = res_smem_bytes(a.frow, a.fcol, a.K);
  if (tf32)
    k_fwd_res<true><<<(unsigned)grid, kFwdThreads, smem, P->stream>>>(a);
  else
    k_fwd_res<false><<<(unsigned)grid, kFwdThreads, smem, P->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t tc_adjoint_res(qem_plan_t P, int l, bool tf32) {
  TcBuffers& T = *P->tc;
  const LevelView& ch = P->lv[l];
  const Layout& L = T.lay[l];
  if (ch.n == 0) return cudaSuccess;
  AdjResArgs a{};
  a.K = P->K;
  a.R = P->K / kRows;
  a.frow = L.fkb;
  a.fcol = L.fka;
  a.nst = tc_adj_res_stages(a.frow, a.fcol, a.K);
  if (a.nst == 0) return cudaErrorInvalidValue;
  a.ksteps = L.nks;
  for (int i = 0; i < L.nks; ++i) {
    a.koff_row[i] = L.kb[i];
    a.koff_col[i] = L.ka[i];
  }
  a.n_elts = ch.n;
  a.parent = ch.parent;
  a.ccnt = P->lv[l - 1].ccnt;
  a.small = kSmallKept;
  a.rows_feat = T.bfeat[l];
  a.cols_feat = T.cfeat[l];
  a.dcol = T.dcol[l];
  a.w_out = ch.w;
  a.ctl = P->ctl;
  a.timeout_cycles = res_timeout_cycles(P);
  a.expire_test = P->expire_test;
  const long long grid = ch.n < P->num_sms ? ch.n : P->num_sms;
  const size_t smem = adj_res_smem_bytes(a.frow, a.fcol, a.nst);
  if (tf32)
    k_adj_res<true><<<(unsigned)grid, kFwdThreads, smem, P->stream>>>(a);
  else
    k_adj_res<false><<<(unsigned)grid, kFwdThreads, smem, P->stream>>>(a);
  return cudaGetLastError();
}

}  // namespace qem
