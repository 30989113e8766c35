// libqem host side: plan construction (validation, plate CSR, workspace) and
// the C-ABI entry points declared in include/qem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "qem_internal.cuh"
#include "qem_tc.cuh"

using namespace qem;

namespace {

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align256(sizeof(T) * count);
    return count ? p : nullptr;
  }
};

int noise_per_sample(const qem_level_desc& d) {
  if (d.qfam == QEM_Q_GAUSS) return d.dim;
  const int blk = 2 * QEM_GAMMA_TRIES + 1;
  return d.dim * blk * (d.qfam == QEM_Q_GAMMA ? 1 : 2);
}

qem_status validate(const qem_model_desc* desc, const qem_plan_opts* o) {
  if (!desc || !o) return QEM_ERR_INVALID_ARG;
  if (desc->n_levels < 1 || desc->n_levels > QEM_MAX_LEVELS) return QEM_ERR_INVALID_ARG;
  if (o->K < 1 || o->K > 4096) return QEM_ERR_INVALID_ARG;
  if (o->precision < QEM_PREC_FP32 || o->precision > QEM_PREC_TF32) return QEM_ERR_INVALID_ARG;
  if (o->var_floor < 0 || o->timeout_s < 0) return QEM_ERR_INVALID_ARG;
  if (o->tile != 0 && o->tile != QEM_TILE_AUTO) return QEM_ERR_INVALID_ARG;
  const int L = desc->n_levels;
  for (int l = 0; l < L; ++l) {
    const qem_level_desc& d = desc->levels[l];
    if (d.n < 0 || d.dim < 1 || d.n_obs < 0) return QEM_ERR_INVALID_ARG;
    if (d.dim > kMaxDim) return QEM_ERR_UNSUPPORTED;
    if (d.qfam < QEM_Q_GAUSS || d.qfam > QEM_Q_BETA) return QEM_ERR_INVALID_ARG;
    if (d.lik < QEM_LIK_NONE || d.lik > QEM_LIK_BERNOULLI_PROB) return QEM_ERR_INVALID_ARG;
    if (d.lik == QEM_LIK_NONE && d.n_obs != 0) return QEM_ERR_INVALID_ARG;
    if (d.lik != QEM_LIK_NONE && d.n_obs > 0 && d.n > 0 && (!d.x || !d.y)) return QEM_ERR_INVALID_ARG;
    if (d.n_obs > 4096 || (size_t)d.n_obs * d.dim > 8192) return QEM_ERR_UNSUPPORTED;
    if (d.lik == QEM_LIK_GAUSS && !(d.lik_var > 0)) return QEM_ERR_INVALID_ARG;
    if ((d.lik == QEM_LIK_POISSON_RATE && (d.qfam != QEM_Q_GAMMA || d.dim != 1)) ||
        (d.lik == QEM_LIK_BERNOULLI_PROB && (d.qfam != QEM_Q_BETA || d.dim != 1)))
      return QEM_ERR_INVALID_ARG;
    if (L > 1 && d.qfam != QEM_Q_GAUSS) return QEM_ERR_UNSUPPORTED;
    if (d.chain < 0 || d.qcond < 0 || d.qcond > 1) return QEM_ERR_INVALID_ARG;
    if (d.qcond) {
      if (l != 1 || L != 2 || o->precision != QEM_PREC_FP32 || d.dim > 32 || d.qfam != QEM_Q_GAUSS || d.chain > 1)
        return QEM_ERR_UNSUPPORTED;
    }
    if (d.chain > 1) {
      if (l != 1 || L != 2 || o->precision != QEM_PREC_FP32 || d.dim > 8 || d.qfam != QEM_Q_GAUSS || o->K > 1024)
        return QEM_ERR_UNSUPPORTED;
      if (d.n % d.chain != 0 || !(d.prior_b > 0)) return QEM_ERR_INVALID_ARG;
      if (d.n > 0 && d.parent)
        for (int64_t e = 0; e < d.n; ++e)
          if (d.parent[e] != d.parent[e - e % d.chain]) return QEM_ERR_INVALID_ARG;
    }
    if (l == 0) {
      if (d.parent) return QEM_ERR_INVALID_ARG;
      if (d.prior == QEM_PRIOR_STD_NORMAL) {
        if (!(d.prior_a > 0) || d.qfam != QEM_Q_GAUSS) return QEM_ERR_INVALID_ARG;
      } else if (d.prior == QEM_PRIOR_GAMMA) {
        if (!(d.prior_a > 0 && d.prior_b > 0) || d.qfam != QEM_Q_GAMMA) return QEM_ERR_INVALID_ARG;
      } else if (d.prior == QEM_PRIOR_BETA) {
        if (!(d.prior_a > 0 && d.prior_b > 0) || d.qfam != QEM_Q_BETA) return QEM_ERR_INVALID_ARG;
      } else {
        return QEM_ERR_INVALID_ARG;
      }
    } else {
      const qem_level_desc& p = desc->levels[l - 1];
      if (d.prior == QEM_PRIOR_NORMAL_FIXED_VAR) {
        if (p.dim != d.dim || !(d.prior_a > 0)) return QEM_ERR_INVALID_ARG;
      } else if (d.prior == QEM_PRIOR_NORMAL_MEAN_LOGVAR) {
        if (p.dim != 2 * d.dim) return QEM_ERR_INVALID_ARG;
      } else {
        return QEM_ERR_INVALID_ARG;
      }
      if (d.n > 0) {
        if (!d.parent) return QEM_ERR_INVALID_ARG;
        int64_t prev = 0;
        for (int64_t e = 0; e < d.n; ++e) {
          const int64_t pe = d.parent[e];
          if (pe < 0 || pe >= p.n || pe < prev) return QEM_ERR_INVALID_ARG;
          prev = pe;
        }
      }
    }
  }
  return QEM_OK;
}

#define QEM_TRY(expr)                          \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) return QEM_ERR_CUDA; \
  } while (0)

// Per-kernel CUDA-event records of a plan (qem_profile_*).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  cudaEvent_t get() {
    if (next == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[next++];
  }
  ~Prof() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

inline Prof* prof_of(qem_plan_t P) { return static_cast<Prof*>(P->prof); }

// qem_run's graph: one conditional (while) node whose body is one iteration
// (E-step, EMA + M-step, loop control), instantiated once per argument set.
struct RunGraph {
  const void* key[4] = {};
  double lambda = -1.0, sched_p = -1.0;
  cudaGraph_t g = nullptr;
  cudaGraph_t body = nullptr;   // the while node's body (owned by g)
  cudaGraphExec_t ge = nullptr;
  ~RunGraph() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
  }
};
inline RunGraph* run_of(qem_plan_t P) { return static_cast<RunGraph*>(P->run); }

// Launch `expr` (a cudaError_t expression), bracketed by events when profiling.
#define QEM_LAUNCH(P, kind, expr)                                          \
  do {                                                                     \
    Prof* _pf = prof_of(P);                                                \
    cudaEvent_t _a = nullptr, _b = nullptr;                                \
    if (_pf && _pf->on) {                                                  \
      _a = _pf->get();                                                     \
      _b = _pf->get();                                                     \
      if (_a) cudaEventRecord(_a, (P)->stream);                            \
    }                                                                      \
    QEM_TRY(expr);                                                         \
    if (_a && _b) {                                                        \
      cudaEventRecord(_b, (P)->stream);                                    \
      _pf->recs.push_back({kind, _a, _b});                                 \
    }                                                                      \
  } while (0)

// The E-step from sampling through the plate sums into the root (Eq. Prmp
// over the plate tree, leaves first), enqueued on the plan's stream.
qem_status estep_tree(qem_plan_t P, const float* q, const float* eps) {
  cudaStream_t s = P->stream;
  const int L = P->L, K = P->K;
  for (int l = 0; l < L; ++l) {
    if (P->lv[l].qcond && !P->perm_user) QEM_LAUNCH(P, QEM_K_SAMPLE, launch_draw_perm(P->lv[l], K, P->perm_own, P->ctl, s));
    QEM_LAUNCH(P, QEM_K_SAMPLE,
               launch_sample_local(P->lv[l], K, P->tune.sample_threads, q + P->q_off[l],
                                   eps ? eps + P->eps_off[l] : nullptr, P->ctl, s));
    QEM_LAUNCH(P, QEM_K_SAMPLE, launch_elem_const(P->lv[l], q + P->q_off[l], s));
  }
  for (int l = 0; l + 1 < L; ++l) QEM_LAUNCH(P, QEM_K_PARENT, launch_parent_params(P->lv[l], P->lv[l + 1], K, s));
  for (int l = L - 1; l >= 1; --l) {
    const bool has_children = l + 1 < L;
    if (has_children) QEM_LAUNCH(P, QEM_K_FINALIZE, launch_finalize(P->lv[l], K, has_children, s));
    if (P->lv[l].chain > 1) {
      QEM_LAUNCH(P, QEM_K_FORWARD, launch_chain_forward(P->lv[l], P->lv[l - 1], K, s));
    } else if (P->precision == QEM_PREC_FP32) {
      QEM_LAUNCH(P, QEM_K_FORWARD, launch_fwd_simt(P->lv[l], P->lv[l - 1], K, P->tune.fwd_rows, P->tune.fwd_chunk, s));
    } else {
      QEM_LAUNCH(P, QEM_K_OPERANDS, tc_features(P, l));
      QEM_LAUNCH(P, QEM_K_FORWARD, tc_forward(P, l));
    }
    QEM_LAUNCH(P, QEM_K_PLATE_SUM, launch_plate_sum(P->lv[l - 1], P->lv[l], K, s));
  }
  return QEM_OK;
}

// Forward half of the E-step (sampling through log P_MP and the root
// weights: Eq. Prmp over the plate tree), enqueued on the plan's stream.
qem_status estep_forward(qem_plan_t P, const float* q, const float* eps, double* user_lp, double* trace) {
  const qem_status st = estep_tree(P, q, eps);
  if (st != QEM_OK) return st;
  QEM_LAUNCH(P, QEM_K_ROOT, launch_root(P->lv[0], P->K, P->L > 1, P->log_pmp, user_lp, trace, P->ctl, P->stream));
  return QEM_OK;
}

// Second half of the E-step: the adjoint (marginal weights, Eq. mmp) root to
// leaves and the moments, after the root step.
qem_status estep_adjoint(qem_plan_t P, double* moments) {
  cudaStream_t s = P->stream;
  const int L = P->L, K = P->K;
  for (int l = 1; l < L; ++l) {
    if (P->lv[l].chain > 1) {
      QEM_LAUNCH(P, QEM_K_ADJOINT, launch_chain_adjoint(P->lv[l], P->lv[l - 1], K, s));
      continue;
    }
    // parent samples below rel * the largest weight are dropped from the
    // adjoint: 2^-40 on the FP32 path, 2^-24 on the mixed-precision paths
    const float rel = P->precision == QEM_PREC_FP32 ? 9.094947017729282e-13f : 5.9604644775390625e-08f;
    QEM_LAUNCH(P, QEM_K_OPERANDS, launch_compact(P->lv[l - 1], K, rel, s));
    if (P->precision == QEM_PREC_FP32) {
      QEM_LAUNCH(P, QEM_K_ADJOINT, launch_adj_compact(P->lv[l], P->lv[l - 1], K, 0, s));
    } else {
      QEM_LAUNCH(P, QEM_K_ADJ_SMALL, launch_adj_small(P->lv[l], P->lv[l - 1], K, s));
      QEM_LAUNCH(P, QEM_K_OPERANDS, tc_adjoint_prep(P, l));
      QEM_LAUNCH(P, QEM_K_ADJOINT, tc_adjoint(P, l));
    }
  }
  for (int l = 0; l < L; ++l) {
    QEM_LAUNCH(P, QEM_K_MOMENTS, launch_moments(P->lv[l], K, P->tune.mom_threads, moments + P->q_off[l], s));
    if (P->lv[l].qcond)
      QEM_LAUNCH(P, QEM_K_MOMENTS,
                 launch_residual_moments(P->lv[l], K, moments + P->q_off[l - 1], moments + P->q_off[l], s));
  }
  return QEM_OK;
}

// The E-step body (Eq. mp_iw over the plate tree): the forward half, then the
// adjoint and the moments.
qem_status estep_body(qem_plan_t P, const float* q, const float* eps, double* moments, double* user_lp,
                      double* trace) {
  const qem_status st = estep_forward(P, q, eps, user_lp, trace);
  if (st != QEM_OK) return st;
  return estep_adjoint(P, moments);
}

qem_status mstep_body(qem_plan_t P, const double* moments, double* m, float* q, double lambda, double sched_p,
                      long long t_host) {
  for (int l = 0; l < P->L; ++l)
    QEM_LAUNCH(P, QEM_K_MSTEP,
               launch_mstep(P->lv[l], moments ? moments + P->q_off[l] : nullptr, m + P->q_off[l], q + P->q_off[l],
                            lambda, sched_p, P->var_floor, t_host, P->ctl, P->stream));
  return QEM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the launch shapes (Tune): a coordinate search over each knob's
// candidates, timing whole E-steps with CUDA events on the plan's stream and
// keeping a candidate only when it is at least 3% faster.  The choice is
// cached per shape signature (precision, K, SM count; per level: element
// count to a power of two, dimension, observations, likelihood, proposal
// family) for the process and, when the environment variable QEM_TUNE_CACHE
// names a file, across processes (one "signature|values" line per entry).
std::mutex g_tune_mu;
std::map<std::string, Tune> g_tune_cache;
bool g_tune_file_read = false;

const int kSampleCand[] = {64, 128, 256};
const int kMomCand[] = {128, 256, 512};
const int kRowsCand[] = {64, 128, 256};
const int kChunkCand[] = {16, 32, 64};
const int kSchedCand[] = {3, 1, 0, 2};

template <size_t N>
bool one_of(int v, const int (&c)[N]) {
  for (int x : c)
    if (x == v) return true;
  return false;
}
bool tune_valid(const Tune& t) {
  return one_of(t.sample_threads, kSampleCand) && one_of(t.mom_threads, kMomCand) && one_of(t.fwd_rows, kRowsCand) &&
         one_of(t.fwd_chunk, kChunkCand) && one_of(t.tc_sched, kSchedCand);
}

std::string tune_signature(const qem_plan_s* P) {
  char buf[160];
  std::snprintf(buf, sizeof buf, "p%d K%d sm%d", P->precision, P->K, P->num_sms);
  std::string sig = buf;
  for (int l = 0; l < P->L; ++l) {
    const LevelView& v = P->lv[l];
    int b = 0;
    while (b < 62 && (1LL << b) < v.n) ++b;
    std::snprintf(buf, sizeof buf, " L%d:n2^%d,D%d,o%d,lik%d,q%d", l, b, v.D, v.n_obs, v.lik, v.qfam);
    sig += buf;
  }
  return sig;
}

const char* tune_file() {
  const char* f = std::getenv("QEM_TUNE_CACHE");
  return f && *f ? f : nullptr;
}

void tune_read_file_locked() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = tune_file();
  FILE* f = path ? std::fopen(path, "r") : nullptr;
  if (!f) return;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    char* bar = std::strchr(line, '|');
    if (!bar) continue;
    *bar = 0;
    Tune t;
    if (std::sscanf(bar + 1, "%d %d %d %d %d", &t.sample_threads, &t.mom_threads, &t.fwd_rows, &t.fwd_chunk,
                    &t.tc_sched) == 5 &&
        tune_valid(t))
      g_tune_cache[line] = t;
  }
  std::fclose(f);
}

void tune_store_locked(const std::string& sig, const Tune& t) {
  g_tune_cache[sig] = t;
  const char* path = tune_file();
  FILE* f = path ? std::fopen(path, "a") : nullptr;
  if (!f) return;
  std::fprintf(f, "%s|%d %d %d %d %d\n", sig.c_str(), t.sample_threads, t.mom_threads, t.fwd_rows, t.fwd_chunk,
               t.tc_sched);
  std::fclose(f);
}

// Mean time of `reps` E-steps after one warm-up (profiling is off meanwhile).
qem_status time_esteps(qem_plan_t P, const float* q, double* mom, int reps, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  qem_status st = QEM_OK;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) st = QEM_ERR_CUDA;
  if (st == QEM_OK) st = estep_body(P, q, nullptr, mom, nullptr, nullptr);
  if (st == QEM_OK && cudaEventRecord(a, P->stream) != cudaSuccess) st = QEM_ERR_CUDA;
  for (int r = 0; r < reps && st == QEM_OK; ++r) st = estep_body(P, q, nullptr, mom, nullptr, nullptr);
  if (st == QEM_OK && (cudaEventRecord(b, P->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                       cudaEventElapsedTime(ms, a, b) != cudaSuccess))
    st = QEM_ERR_CUDA;
  if (st == QEM_OK) *ms /= (float)reps;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return st;
}

}  // namespace

extern "C" qem_status qem_tune(qem_plan_t P, const float* q_params, int flags) {
  if (!P || !q_params || (flags & ~QEM_TUNE_FORCE)) return QEM_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(P->stream, &cs) != cudaSuccess) return QEM_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return QEM_ERR_INVALID_ARG;  // timing cannot run inside a capture
  const std::string sig = tune_signature(P);
  if (!(flags & QEM_TUNE_FORCE)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_read_file_locked();
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      P->tune = it->second;
      P->tuned = true;
      return QEM_OK;
    }
  }
  Prof* pf = prof_of(P);
  const bool prof_was_on = pf && pf->on;
  if (pf) pf->on = false;
  double* mom = nullptr;
  qem_status st = cudaMalloc(&mom, sizeof(double) * (size_t)(P->q_len > 0 ? P->q_len : 1)) == cudaSuccess
                      ? QEM_OK
                      : QEM_ERR_OOM;
  if (st == QEM_OK && launch_set_ctl(P->ctl, 0x5eedULL, 1, 1, -1, P->stream) != cudaSuccess) st = QEM_ERR_CUDA;
  Tune best = P->tune;
  float best_ms = 0.f;
  if (st == QEM_OK) st = time_esteps(P, q_params, mom, 2, &best_ms);
  auto try_knob = [&](int Tune::*field, const int* cand, int nc) {
    for (int i = 0; i < nc && st == QEM_OK; ++i) {
      if (cand[i] == best.*field) continue;
      Tune t = best;
      t.*field = cand[i];
      P->tune = t;
      float ms = 0.f;
      st = time_esteps(P, q_params, mom, 2, &ms);
      if (st == QEM_OK && ms < 0.97f * best_ms) {
        best = t;
        best_ms = ms;
      }
    }
    P->tune = best;
  };
  try_knob(&Tune::sample_threads, kSampleCand, 3);
  try_knob(&Tune::mom_threads, kMomCand, 3);
  if (P->precision == QEM_PREC_FP32 && P->L > 1) {
    try_knob(&Tune::fwd_rows, kRowsCand, 3);
    try_knob(&Tune::fwd_chunk, kChunkCand, 3);
  }
  if (P->precision != QEM_PREC_FP32 && P->L > 1) try_knob(&Tune::tc_sched, kSchedCand, 4);
  P->tune = best;
  delete static_cast<RunGraph*>(P->run);  // a loop graph built before holds the old launch shapes
  P->run = nullptr;
  if (mom) {
    if (cudaStreamSynchronize(P->stream) != cudaSuccess && st == QEM_OK) st = QEM_ERR_CUDA;
    cudaFree(mom);
  }
  if (st == QEM_OK) {
    P->tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_read_file_locked();
    tune_store_locked(sig, best);
  }
  if (pf) pf->on = prof_was_on;
  return st;
}

extern "C" qem_status qem_tune_set(qem_plan_t P, const int* params) {
  if (!P || !params) return QEM_ERR_INVALID_ARG;
  Tune t;
  t.sample_threads = params[0];
  t.mom_threads = params[1];
  t.fwd_rows = params[2];
  t.fwd_chunk = params[3];
  t.tc_sched = params[4];
  if (!tune_valid(t)) return QEM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
  P->tune = t;
  P->tuned = true;
  delete static_cast<RunGraph*>(P->run);  // the loop graph holds the old launch shapes
  P->run = nullptr;
  return QEM_OK;
}

extern "C" qem_status qem_tune_get(qem_plan_t P, int* params) {
  if (!P || !params) return QEM_ERR_INVALID_ARG;
  params[0] = P->tune.sample_threads;
  params[1] = P->tune.mom_threads;
  params[2] = P->tune.fwd_rows;
  params[3] = P->tune.fwd_chunk;
  params[4] = P->tune.tc_sched;
  return QEM_OK;
}

namespace {

// qem_estep / qem_run with QEM_TILE_AUTO: tune on first use outside a capture.
qem_status maybe_autotune(qem_plan_t P, const float* q) {
  if (P->tile != QEM_TILE_AUTO || P->tuned) return QEM_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(P->stream, &cs) != cudaSuccess) return QEM_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return QEM_OK;  // defaults until a call outside a capture
  return qem_tune(P, q, 0);
}

// Split-root workspace (qem_estep_split_root): carved from one allocation.
qem_status split_alloc(qem_plan_t P) {
  if (P->split) return QEM_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(P->stream, &cs) != cudaSuccess) return QEM_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return QEM_ERR_UNSUPPORTED;
  SplitWs* W = new (std::nothrow) SplitWs();
  if (!W) return QEM_ERR_OOM;
  const size_t K = (size_t)P->K, KK = K * K, n0 = (size_t)P->lv[0].n, n1 = (size_t)P->lv[1].n;
  const size_t nch = (size_t)P->lv[1].n_chunks;
  for (int pass = 0; pass < 2; ++pass) {
    Carver cv;
    if (pass == 1) {
      if (cudaMalloc(&W->base, W->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete W;
        return QEM_ERR_OOM;
      }
      cv.base = (char*)W->base;
    }
    W->fa = cv.take<double>(n0 * K);
    W->fb = cv.take<double>(n0 * K);
    W->lt = cv.take<float>(n1 * KK);
    W->partial = cv.take<double>(nch * KK);
    W->hsum = cv.take<double>(n0 * KK);
    W->W = cv.take<float>(n0 * KK);
    W->cidx = cv.take<int>(n0 * KK);
    W->ccnt = cv.take<int>(n0);
    W->cw = cv.take<float>(n0 * KK);
    W->wab = cv.take<float>(n0 * 2 * K);
    if (pass == 0) W->bytes = std::max<size_t>(cv.off, 256);
  }
  P->split = W;
  return QEM_OK;
}

void split_free(qem_plan_t P) {
  if (!P->split) return;
  if (P->split->base) cudaFree(P->split->base);
  delete P->split;
  P->split = nullptr;
}

}  // namespace

extern "C" {

const char* qem_status_string(qem_status s) {
  switch (s) {
    case QEM_OK: return "QEM_OK";
    case QEM_ERR_INVALID_ARG: return "QEM_ERR_INVALID_ARG: invalid size, pointer or descriptor field";
    case QEM_ERR_UNSUPPORTED: return "QEM_ERR_UNSUPPORTED: valid request that is not implemented";
    case QEM_ERR_OOM: return "QEM_ERR_OOM: workspace allocation failed";
    case QEM_ERR_CUDA: return "QEM_ERR_CUDA: a CUDA call or kernel failed";
    case QEM_ERR_NUMERIC: return "QEM_ERR_NUMERIC: non-finite log P_MP or weights";
    case QEM_ERR_TIMEOUT: return "QEM_ERR_TIMEOUT: a bounded device wait expired";
  }
  return "QEM_ERR_UNKNOWN";
}

qem_status qem_plan(const qem_model_desc* desc, const qem_plan_opts* opts, qem_plan_t* out) {
  if (!out) return QEM_ERR_INVALID_ARG;
  *out = nullptr;
  qem_status st = validate(desc, opts);
  if (st != QEM_OK) return st;
  qem_plan_s* P = new (std::nothrow) qem_plan_s();
  if (!P) return QEM_ERR_OOM;
  P->L = desc->n_levels;
  P->K = opts->K;
  P->precision = opts->precision;
  P->tile = opts->tile;
  P->stream = (cudaStream_t)opts->stream;
  P->var_floor = opts->var_floor > 0 ? opts->var_floor : 1e-10;
  P->timeout_s = opts->timeout_s > 0 ? opts->timeout_s : 2.0;
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    delete P;
    return QEM_ERR_CUDA;
  }
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, P->device);
  P->num_sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrClockRate, P->device);
  P->clock_khz = v > 0 ? v : 2000000;

  const int L = P->L, K = P->K;
  // offsets of the flat user buffers
  long long qo = 0, eo = 0, wo = 0, zo = 0;
  for (int l = 0; l < L; ++l) {
    const qem_level_desc& d = desc->levels[l];
    P->q_off[l] = qo;
    P->eps_off[l] = eo;
    P->w_off[l] = wo;
    P->z_off[l] = zo;
    qo += d.n * 2 * d.dim;
    eo += d.n * (long long)K * noise_per_sample(d);
    wo += d.n * (long long)K;
    zo += d.n * (long long)K * d.dim;
  }
  P->q_len = qo;
  P->eps_len = eo;
  P->w_len = wo;
  P->z_len = zo;

  // children CSR offsets of every level that has a next level
  std::vector<std::vector<long long>> child_off(L);
  for (int l = 0; l + 1 < L; ++l) {
    const qem_level_desc& c = desc->levels[l + 1];
    std::vector<long long>& co = child_off[l];
    co.assign((size_t)desc->levels[l].n + 1, 0);
    for (int64_t e = 0; e < c.n; ++e) co[(size_t)c.parent[e] + 1] += 1;
    for (size_t i = 1; i < co.size(); ++i) co[i] += co[i - 1];
  }

  // plate-sum chunks: the children of each element, at most kChunkChildren per chunk
  struct Chunks {
    std::vector<long long> beg, end, par_off;
  };
  const long long kChunkChildren = 32;
  std::vector<Chunks> chunks(L);
  for (int l = 1; l < L; ++l) {
    Chunks& ck = chunks[l];
    const std::vector<long long>& co = child_off[l - 1];
    ck.par_off.assign(co.size(), 0);
    for (size_t p = 0; p + 1 < co.size(); ++p) {
      ck.par_off[p] = (long long)ck.beg.size();
      for (long long c = co[p]; c < co[p + 1]; c += kChunkChildren) {
        ck.beg.push_back(c);
        ck.end.push_back(std::min(co[p + 1], c + kChunkChildren));
      }
    }
    ck.par_off.back() = (long long)ck.beg.size();
  }

  // two passes: size, then carve
  for (int pass = 0; pass < 2; ++pass) {
    Carver cv;
    if (pass == 1) {
      if (cudaMalloc(&P->ws, P->ws_bytes) != cudaSuccess) {
        delete P;
        return QEM_ERR_OOM;
      }
      cv.base = (char*)P->ws;
    }
    P->ctl = cv.take<Ctl>(1);
    P->log_pmp = cv.take<double>((size_t)desc->levels[0].n);
    bool counts = false;
    for (int l = 0; l < L; ++l) counts = counts || desc->levels[l].lik == QEM_LIK_POISSON_LOG;
    P->count_tab = counts ? cv.take<double>((size_t)kCountTable) : nullptr;
    for (int l = 0; l < L; ++l) {
      const qem_level_desc& d = desc->levels[l];
      LevelView& lv = P->lv[l];
      const size_t nK = (size_t)d.n * K;
      const bool has_children = l + 1 < L;
      lv.n = d.n;
      lv.D = d.dim;
      lv.prior = d.prior;
      lv.prior_a = (float)d.prior_a;
      lv.prior_b = (float)d.prior_b;
      lv.lik = d.lik;
      lv.lik_var = (float)d.lik_var;
      lv.n_obs = d.lik == QEM_LIK_NONE ? 0 : d.n_obs;
      lv.qfam = d.qfam;
      lv.nps = noise_per_sample(d);
      lv.level = l;
      lv.chain = d.chain > 1 ? d.chain : 1;
      lv.ebase = 0;
      lv.qcond = d.qcond;
      lv.pD = l > 0 ? desc->levels[l - 1].dim : 0;
      lv.x = d.x;
      lv.y = d.y;
      lv.Dc = has_children ? desc->levels[l + 1].dim : 0;
      lv.parent = l > 0 ? cv.take<long long>((size_t)d.n) : nullptr;
      lv.child_off = has_children ? cv.take<long long>((size_t)d.n + 1) : nullptr;
      lv.z = cv.take<float>(nK * d.dim);
      lv.loc = cv.take<float>(nK);
      lv.cst = cv.take<double>((size_t)d.n);
      lv.cshift = cv.take<float>((size_t)d.n);
      lv.ltab = d.lik == QEM_LIK_POISSON_LOG ? P->count_tab : nullptr;
      lv.htil = has_children ? cv.take<float>(nK) : lv.loc;
      lv.hsum = has_children ? cv.take<double>(nK) : nullptr;
      lv.off = (has_children || d.chain > 1) ? cv.take<double>((size_t)d.n) : nullptr;
      lv.lt = l > 0 ? cv.take<float>(nK) : nullptr;
      lv.w = cv.take<float>(nK);
      lv.beta = d.chain > 1 ? cv.take<float>(nK) : nullptr;
      lv.cz = d.qcond ? cv.take<float>(nK * d.dim) : nullptr;
      if (d.qcond) {
        P->perm_own = cv.take<int>(nK);
        lv.perm = P->perm_own;
        lv.pz = P->lv[l - 1].z;
      }
      lv.pm = has_children ? cv.take<float>(nK * lv.Dc) : nullptr;
      lv.pp = has_children ? cv.take<float>(nK * lv.Dc) : nullptr;
      lv.pc = has_children ? cv.take<float>(nK) : nullptr;
      lv.cidx = has_children ? cv.take<int>(nK) : nullptr;
      lv.ccnt = has_children ? cv.take<int>((size_t)d.n) : nullptr;
      lv.cw = has_children ? cv.take<float>(nK) : nullptr;
      lv.chk_off = has_children ? cv.take<long long>((size_t)d.n + 1) : nullptr;
      lv.n_chunks = l > 0 ? (long long)chunks[l].beg.size() : 0;
      lv.chk_beg = l > 0 ? cv.take<long long>((size_t)lv.n_chunks) : nullptr;
      lv.chk_end = l > 0 ? cv.take<long long>((size_t)lv.n_chunks) : nullptr;
      lv.partial = l > 0 ? cv.take<double>((size_t)lv.n_chunks * K) : nullptr;
    }
    size_t tc_bytes = 0;
    st = tc_plan_reserve(P, desc, pass == 1 ? cv.base + cv.off : nullptr, &tc_bytes);
    if (st != QEM_OK) {
      if (P->ws) cudaFree(P->ws);
      delete P;
      return st;
    }
    cv.off += align256(tc_bytes);
    if (pass == 0) P->ws_bytes = std::max<size_t>(cv.off, 256);
  }
  // upload the plate structure
  cudaError_t ce = cudaMemsetAsync(P->ctl, 0, sizeof(Ctl), P->stream);
  for (int l = 0; l < L && ce == cudaSuccess; ++l) {
    const qem_level_desc& d = desc->levels[l];
    if (l > 0 && d.n > 0)
      ce = cudaMemcpyAsync((void*)P->lv[l].parent, d.parent, sizeof(long long) * (size_t)d.n, cudaMemcpyHostToDevice,
                           P->stream);
    if (ce == cudaSuccess && l + 1 < L)
      ce = cudaMemcpyAsync((void*)P->lv[l].child_off, child_off[l].data(), sizeof(long long) * child_off[l].size(),
                           cudaMemcpyHostToDevice, P->stream);
    if (ce == cudaSuccess && P->lv[l].hsum)
      ce = cudaMemsetAsync(P->lv[l].hsum, 0, sizeof(double) * (size_t)d.n * K, P->stream);
    if (ce == cudaSuccess && l + 1 < L)
      ce = cudaMemcpyAsync(P->lv[l].chk_off, chunks[l + 1].par_off.data(), sizeof(long long) * chunks[l + 1].par_off.size(),
                           cudaMemcpyHostToDevice, P->stream);
    if (ce == cudaSuccess && l > 0 && P->lv[l].n_chunks > 0) {
      ce = cudaMemcpyAsync(P->lv[l].chk_beg, chunks[l].beg.data(), sizeof(long long) * chunks[l].beg.size(),
                           cudaMemcpyHostToDevice, P->stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(P->lv[l].chk_end, chunks[l].end.data(), sizeof(long long) * chunks[l].end.size(),
                             cudaMemcpyHostToDevice, P->stream);
    }
  }
  if (ce == cudaSuccess && P->count_tab) ce = launch_count_table(P->count_tab, P->stream);
  size_t smem = 0;
  for (int l = 0; l < L; ++l) smem = std::max(smem, sample_local_smem(P->lv[l], K, kSampleThreadsLimit));
  if (ce == cudaSuccess) ce = configure_sample_local(smem);
  for (int l = 1; l < L && ce == cudaSuccess; ++l) ce = configure_adj_small(P->lv[l].D, K);
  for (int l = 1; l < L && ce == cudaSuccess; ++l)
    if (P->lv[l].chain > 1) ce = configure_chain(P->lv[l].D, K);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(P->stream);
  if (ce == cudaSuccess) {
    st = tc_plan_init(P, desc);
    if (st != QEM_OK) {
      cudaFree(P->ws);
      delete P;
      return st;
    }
  }
  if (ce != cudaSuccess) {
    cudaFree(P->ws);
    delete P;
    return QEM_ERR_CUDA;
  }
  *out = P;
  return QEM_OK;
}

qem_status qem_plan_destroy(qem_plan_t P) {
  if (!P) return QEM_OK;
  cudaError_t e = cudaStreamSynchronize(P->stream);
  tc_plan_release(P);
  split_free(P);
  delete prof_of(P);
  delete run_of(P);
  if (P->ws) cudaFree(P->ws);
  delete P;
  return e == cudaSuccess ? QEM_OK : QEM_ERR_CUDA;
}

qem_status qem_workspace_size(const qem_plan_t P, size_t* bytes) {
  if (!P || !bytes) return QEM_ERR_INVALID_ARG;
  *bytes = P->ws_bytes;
  return QEM_OK;
}

qem_status qem_layout(const qem_plan_t P, int level, int64_t* q_off, int64_t* eps_off, int64_t* w_off) {
  if (!P || level < 0 || level >= P->L) return QEM_ERR_INVALID_ARG;
  if (q_off) *q_off = P->q_off[level];
  if (eps_off) *eps_off = P->eps_off[level];
  if (w_off) *w_off = P->w_off[level];
  return QEM_OK;
}

qem_status qem_sizes(const qem_plan_t P, int64_t* q_len, int64_t* eps_len, int64_t* w_len, int64_t* n_inst) {
  if (!P) return QEM_ERR_INVALID_ARG;
  if (q_len) *q_len = P->q_len;
  if (eps_len) *eps_len = P->eps_len;
  if (w_len) *w_len = P->w_len;
  if (n_inst) *n_inst = P->lv[0].n;
  return QEM_OK;
}

qem_status qem_estep(qem_plan_t P, const float* q_params, const float* eps, uint64_t seed, uint64_t iter,
                     double* moments, double* log_pmp) {
  if (!P || !q_params || !moments) return QEM_ERR_INVALID_ARG;
  const qem_status ts = maybe_autotune(P, q_params);
  if (ts != QEM_OK) return ts;
  QEM_TRY(launch_set_ctl(P->ctl, seed, iter, 1, -1, P->stream));
  return estep_body(P, q_params, eps, moments, log_pmp, nullptr);
}

qem_status qem_log_pmp_fresh(qem_plan_t P, const float* q_params, uint64_t seed, uint64_t iter, double* log_pmp) {
  if (!P || !q_params) return QEM_ERR_INVALID_ARG;
  const qem_status ts = maybe_autotune(P, q_params);
  if (ts != QEM_OK) return ts;
  QEM_TRY(launch_set_ctl(P->ctl, seed, iter, 1, -1, P->stream));
  return estep_forward(P, q_params, nullptr, log_pmp, nullptr);
}

qem_status qem_set_perm(qem_plan_t P, const int32_t* perm) {
  if (!P) return QEM_ERR_INVALID_ARG;
  int lq = -1;
  for (int l = 0; l < P->L; ++l)
    if (P->lv[l].qcond) lq = l;
  if (lq < 0) return QEM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
  P->perm_user = perm;
  P->lv[lq].perm = perm ? perm : P->perm_own;
  delete run_of(P);  // the loop graph holds the old pointer
  P->run = nullptr;
  return QEM_OK;
}

qem_status qem_test_expire_wait(qem_plan_t P, int on) {
  if (!P) return QEM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
  P->expire_test = on ? 1 : 0;
  delete run_of(P);  // the loop graph holds the old kernel arguments
  P->run = nullptr;
  return QEM_OK;
}

qem_status qem_set_elem_base(qem_plan_t P, const int64_t* base) {
  if (!P || !base) return QEM_ERR_INVALID_ARG;
  for (int l = 0; l < P->L; ++l)
    if (base[l] < 0) return QEM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
  for (int l = 0; l < P->L; ++l) P->lv[l].ebase = (long long)base[l];
  delete run_of(P);  // the loop graph holds the old level views
  P->run = nullptr;
  return QEM_OK;
}

qem_status qem_estep_shard_forward(qem_plan_t P, const float* q_params, const float* eps, uint64_t seed,
                                   uint64_t iter, double* root_G) {
  if (!P || !q_params || !root_G) return QEM_ERR_INVALID_ARG;
  if (P->L < 2) return QEM_ERR_UNSUPPORTED;
  const qem_status ts = maybe_autotune(P, q_params);
  if (ts != QEM_OK) return ts;
  QEM_TRY(launch_set_ctl(P->ctl, seed, iter, 1, -1, P->stream));
  const qem_status st = estep_tree(P, q_params, eps);
  if (st != QEM_OK) return st;
  QEM_TRY(cudaMemcpyAsync(root_G, P->lv[0].hsum, sizeof(double) * (size_t)P->lv[0].n * P->K,
                          cudaMemcpyDeviceToDevice, P->stream));
  return QEM_OK;
}

qem_status qem_estep_shard_finish(qem_plan_t P, const double* root_G, double* moments, double* log_pmp) {
  if (!P || !root_G || !moments) return QEM_ERR_INVALID_ARG;
  if (P->L < 2) return QEM_ERR_UNSUPPORTED;
  QEM_TRY(cudaMemcpyAsync(P->lv[0].hsum, root_G, sizeof(double) * (size_t)P->lv[0].n * P->K,
                          cudaMemcpyDeviceToDevice, P->stream));
  QEM_LAUNCH(P, QEM_K_ROOT, launch_root(P->lv[0], P->K, true, P->log_pmp, log_pmp, nullptr, P->ctl, P->stream));
  return estep_adjoint(P, moments);
}

qem_status qem_estep_split_root(qem_plan_t P, const float* q_params, const float* eps, uint64_t seed, uint64_t iter,
                                double* moments, double* log_pmp, float* root_weights) {
  if (!P || !q_params || !moments) return QEM_ERR_INVALID_ARG;
  if (P->L != 2) return QEM_ERR_UNSUPPORTED;
  const LevelView& r = P->lv[0];
  const LevelView& u = P->lv[1];
  if (r.prior != QEM_PRIOR_STD_NORMAL || r.qfam != QEM_Q_GAUSS || r.lik != QEM_LIK_NONE ||
      u.prior != QEM_PRIOR_NORMAL_MEAN_LOGVAR || r.D != 2 * u.D || u.D > 32 || u.chain > 1 || u.qcond ||
      P->K > 1024)
    return QEM_ERR_UNSUPPORTED;
  qem_status st = split_alloc(P);
  if (st != QEM_OK) return st;
  SplitWs& W = *P->split;
  cudaStream_t s = P->stream;
  const int K = P->K, KK = K * K;
  QEM_TRY(launch_set_ctl(P->ctl, seed, iter, 1, -1, s));
  for (int l = 0; l < 2; ++l) {
    QEM_LAUNCH(P, QEM_K_SAMPLE,
               launch_sample_local(P->lv[l], K, P->tune.sample_threads, q_params + P->q_off[l],
                                   eps ? eps + P->eps_off[l] : nullptr, P->ctl, s));
    QEM_LAUNCH(P, QEM_K_SAMPLE, launch_elem_const(P->lv[l], q_params + P->q_off[l], s));
  }
  QEM_LAUNCH(P, QEM_K_PARENT, launch_parent_params(r, u, K, s));
  QEM_LAUNCH(P, QEM_K_ROOT, launch_split_unary(r, K, q_params + P->q_off[0], W.fa, W.fb, s));
  // users: K^2-row tables, their plate sums, the root over the pairs
  LevelView uk = u;
  uk.lt = W.lt;
  uk.partial = W.partial;
  LevelView rk = r;
  rk.hsum = W.hsum;
  rk.w = W.W;
  rk.cidx = W.cidx;
  rk.ccnt = W.ccnt;
  rk.cw = W.cw;
  QEM_LAUNCH(P, QEM_K_FORWARD, launch_fwd_simt(uk, r, K, P->tune.fwd_rows, P->tune.fwd_chunk, s, true));
  QEM_LAUNCH(P, QEM_K_PLATE_SUM, launch_plate_sum(rk, uk, KK, s));
  QEM_LAUNCH(P, QEM_K_ROOT,
             launch_split_root((int)r.n, K, W.fa, W.fb, W.hsum, W.W, root_weights ? root_weights : W.wab, r.w,
                               P->log_pmp, log_pmp, P->ctl, s));
  // adjoint over the kept pairs (2^-40 of the largest joint weight: FP32 path)
  QEM_LAUNCH(P, QEM_K_OPERANDS, launch_compact(rk, KK, 9.094947017729282e-13f, s, K));
  QEM_LAUNCH(P, QEM_K_ADJOINT, launch_adj_compact(uk, rk, K, 0, s, true));
  QEM_LAUNCH(P, QEM_K_MOMENTS, launch_moments(u, K, P->tune.mom_threads, moments + P->q_off[1], s));
  QEM_LAUNCH(P, QEM_K_MOMENTS,
             launch_split_root_moments(r, K, root_weights ? root_weights : W.wab, moments + P->q_off[0], s));
  return QEM_OK;
}

qem_status qem_predictive(qem_plan_t P, int level, const float* x_new, const float* y_new, int n_obs_new,
                          double* out) {
  if (!P || level < 0 || level >= P->L || n_obs_new < 1 || !y_new || !out) return QEM_ERR_INVALID_ARG;
  const LevelView& v = P->lv[level];
  if (v.lik == QEM_LIK_NONE) return QEM_ERR_INVALID_ARG;
  if (!x_new && v.lik != QEM_LIK_POISSON_RATE && v.lik != QEM_LIK_BERNOULLI_PROB) return QEM_ERR_INVALID_ARG;
  if (sizeof(float) * ((size_t)n_obs_new * v.D + 2 * (size_t)n_obs_new) > 48 * 1024) return QEM_ERR_UNSUPPORTED;
  QEM_TRY(launch_predictive(v, P->K, x_new, y_new, n_obs_new, out, P->stream));
  return QEM_OK;
}

qem_status qem_moments_rescale(qem_plan_t P, const double* log_pmp_same, const double* log_pmp_fresh,
                               double* moments) {
  if (!P || !log_pmp_same || !log_pmp_fresh || !moments) return QEM_ERR_INVALID_ARG;
  for (int l = 0; l < P->L; ++l)
    QEM_TRY(launch_moments_rescale(P->lv, l, log_pmp_same, log_pmp_fresh, moments + P->q_off[l], P->stream));
  return QEM_OK;
}

qem_status qem_mstep(qem_plan_t P, const double* moments, double* mean_params, float* q_params, double lambda,
                     double sched_p, int64_t t) {
  if (!P || !mean_params || !q_params) return QEM_ERR_INVALID_ARG;
  if (!(lambda >= 0.0 && lambda <= 1.0) || !(sched_p >= 0.0 && sched_p < 1.0) || t < 1) return QEM_ERR_INVALID_ARG;
  return mstep_body(P, moments, mean_params, q_params, lambda, sched_p, t);
}

qem_status qem_mean_params(qem_plan_t P, const float* q_params, double* mean_params) {
  if (!P || !q_params || !mean_params) return QEM_ERR_INVALID_ARG;
  for (int l = 0; l < P->L; ++l)
    QEM_TRY(launch_mean_params(P->lv[l], q_params + P->q_off[l], mean_params + P->q_off[l], P->stream));
  return QEM_OK;
}

qem_status qem_log_pmp(qem_plan_t P, double* host_out) {
  if (!P || !host_out) return QEM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
  Ctl c;
  if (cudaMemcpy(&c, P->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return QEM_ERR_CUDA;
  if (P->lv[0].n > 0 &&
      cudaMemcpy(host_out, P->log_pmp, sizeof(double) * (size_t)P->lv[0].n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return QEM_ERR_CUDA;
  if (c.err & ERR_TIMEOUT) return QEM_ERR_TIMEOUT;
  for (long long i = 0; i < P->lv[0].n; ++i)
    if (!std::isfinite(host_out[i])) return QEM_ERR_NUMERIC;
  if (c.err & ERR_NUMERIC) return QEM_ERR_NUMERIC;
  return QEM_OK;
}

qem_status qem_weights(qem_plan_t P, float* weights) {
  if (!P || !weights) return QEM_ERR_INVALID_ARG;
  for (int l = 0; l < P->L; ++l) {
    const size_t nK = (size_t)P->lv[l].n * P->K;
    if (nK)
      QEM_TRY(cudaMemcpyAsync(weights + P->w_off[l], P->lv[l].w, sizeof(float) * nK, cudaMemcpyDeviceToDevice,
                              P->stream));
  }
  return QEM_OK;
}

qem_status qem_samples(qem_plan_t P, float* z) {
  if (!P || !z) return QEM_ERR_INVALID_ARG;
  for (int l = 0; l < P->L; ++l) {
    const size_t cnt = (size_t)P->lv[l].n * P->K * P->lv[l].D;
    if (cnt)
      QEM_TRY(cudaMemcpyAsync(z + P->z_off[l], P->lv[l].z, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, P->stream));
  }
  return QEM_OK;
}

qem_status qem_run(qem_plan_t P, int64_t T, int64_t t0, double lambda, double sched_p, uint64_t seed,
                   double* mean_params, float* q_params, double* moments, double* log_pmp_trace) {
  if (!P || T < 0 || t0 < 1 || !mean_params || !q_params || !moments) return QEM_ERR_INVALID_ARG;
  if (!(lambda >= 0.0 && lambda <= 1.0) || !(sched_p >= 0.0 && sched_p < 1.0)) return QEM_ERR_INVALID_ARG;
  cudaStream_t own = nullptr;
  Prof* pf = prof_of(P);
  const bool prof_was_on = pf && pf->on;
  if (pf) pf->on = false;  // event records cannot sit inside a conditional body
  if (P->stream == nullptr) {  // the legacy stream cannot be captured: a private stream, finished synchronously
    if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) return QEM_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) {
      cudaStreamDestroy(own);
      return QEM_ERR_CUDA;
    }
    P->stream = own;
  }
  qem_status st = QEM_OK;
  do {
    st = mstep_body(P, nullptr, mean_params, q_params, lambda, sched_p, 1);  // Q_1 = set(m_0)
    if (st == QEM_OK && T > 0) st = maybe_autotune(P, q_params);
    if (st != QEM_OK) break;
    // iteration t0 first: the noise stream (seed, t) and the schedule's t continue a saved run
    if (launch_set_ctl(P->ctl, seed, (unsigned long long)t0, t0, log_pmp_trace ? 0 : -1, P->stream) != cudaSuccess) {
      st = QEM_ERR_CUDA;
      break;
    }
    if (T == 0) break;
    RunGraph* R = run_of(P);
    const void* key[4] = {mean_params, q_params, moments, log_pmp_trace};
    const bool same = R && std::memcmp(R->key, key, sizeof(key)) == 0 && R->lambda == lambda && R->sched_p == sched_p;
    if (!same) {
      delete R;
      R = new (std::nothrow) RunGraph();
      P->run = R;
      if (!R) { st = QEM_ERR_OOM; break; }
      std::memcpy(R->key, key, sizeof(key));
      R->lambda = lambda;
      R->sched_p = sched_p;
      cudaGraphConditionalHandle h;
      cudaGraphNodeParams np = {};
      cudaGraphNode_t node;
      if (cudaGraphCreate(&R->g, 0) != cudaSuccess ||
          cudaGraphConditionalHandleCreate(&h, R->g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        st = QEM_ERR_CUDA;
        break;
      }
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      if (cudaGraphAddNode(&node, R->g, nullptr, nullptr, 0, &np) != cudaSuccess) { st = QEM_ERR_CUDA; break; }
      cudaGraph_t body = np.conditional.phGraph_out[0];
      R->body = body;
      if (cudaStreamBeginCaptureToGraph(P->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
          cudaSuccess) {
        st = QEM_ERR_CUDA;
        break;
      }
      qem_status sb = estep_body(P, q_params, nullptr, moments, nullptr, log_pmp_trace);
      if (sb == QEM_OK) sb = mstep_body(P, moments, mean_params, q_params, lambda, sched_p, 0);
      if (sb == QEM_OK && launch_loop_next(P->ctl, h, P->stream) != cudaSuccess) sb = QEM_ERR_CUDA;
      cudaGraph_t captured = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(P->stream, &captured);
      if (sb != QEM_OK || ec != cudaSuccess) { st = sb != QEM_OK ? sb : QEM_ERR_CUDA; break; }
      if (cudaGraphInstantiate(&R->ge, R->g, 0) != cudaSuccess) { st = QEM_ERR_CUDA; break; }
    }
    if (launch_loop_begin(P->ctl, T, P->stream) != cudaSuccess || cudaGraphLaunch(R->ge, P->stream) != cudaSuccess)
      st = QEM_ERR_CUDA;
  } while (0);
  if (st != QEM_OK && run_of(P) && !run_of(P)->ge) {  // a half-built graph is not kept
    delete run_of(P);
    P->run = nullptr;
  }
  if (own) {
    if (cudaStreamSynchronize(own) != cudaSuccess && st == QEM_OK) st = QEM_ERR_CUDA;
    cudaStreamDestroy(own);
    P->stream = nullptr;
  }
  if (pf) pf->on = prof_was_on;
  return st;
}

qem_status qem_adjoint_pairs(qem_plan_t P, double* kept_tc, double* kept_all) {
  if (!P) return QEM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
  double tc = 0.0, all = 0.0;
  for (int l = 1; l < P->L; ++l) {
    const LevelView& pa = P->lv[l - 1];
    if (pa.n == 0 || P->lv[l].chain > 1) continue;
    std::vector<int> cnt((size_t)pa.n);
    std::vector<long long> co((size_t)pa.n + 1);
    if (cudaMemcpy(cnt.data(), pa.ccnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(co.data(), pa.child_off, sizeof(long long) * co.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return QEM_ERR_CUDA;
    for (long long p = 0; p < pa.n; ++p) {
      const double pairs = (double)cnt[(size_t)p] * (double)(co[(size_t)p + 1] - co[(size_t)p]) * P->K;
      all += pairs;
      if (P->precision != QEM_PREC_FP32 && cnt[(size_t)p] > kSmallKept) tc += pairs;
    }
  }
  if (kept_tc) *kept_tc = tc;
  if (kept_all) *kept_all = all;
  return QEM_OK;
}

qem_status qem_run_kernels(qem_plan_t P, int64_t* per_iteration, int64_t* per_call) {
  if (!P || !per_iteration || !per_call) return QEM_ERR_INVALID_ARG;
  RunGraph* R = run_of(P);
  if (!R || !R->body) return QEM_ERR_INVALID_ARG;
  size_t n = 0;
  if (cudaGraphGetNodes(R->body, nullptr, &n) != cudaSuccess) return QEM_ERR_CUDA;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(R->body, nodes.data(), &n) != cudaSuccess) return QEM_ERR_CUDA;
  int64_t k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) return QEM_ERR_CUDA;
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *per_iteration = k;
  *per_call = P->L + 2;  // the initial M-step (one kernel per level), the control set-up, the loop set-up
  return QEM_OK;
}

static const char* kKindNames[QEM_K_COUNT] = {"sample_local", "parent_params", "finalize", "forward",
                                              "plate_sum",    "root",          "adjoint",  "moments",
                                              "mstep",        "operands",      "adjoint_small"};

const char* qem_profile_name(int kind) { return kind >= 0 && kind < QEM_K_COUNT ? kKindNames[kind] : nullptr; }

qem_status qem_profile_enable(qem_plan_t P, int on) {
  if (!P) return QEM_ERR_INVALID_ARG;
  Prof* pf = prof_of(P);
  if (!pf) {
    pf = new (std::nothrow) Prof();
    if (!pf) return QEM_ERR_OOM;
    P->prof = pf;
  }
  if (on) {
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
    pf->recs.clear();
    pf->next = 0;
  }
  pf->on = on != 0;
  return QEM_OK;
}

qem_status qem_profile_read(qem_plan_t P, int kind, double* ms, int64_t* launches) {
  if (!P || kind < 0 || kind >= QEM_K_COUNT) return QEM_ERR_INVALID_ARG;
  Prof* pf = prof_of(P);
  double tot = 0.0;
  int64_t cnt = 0;
  if (pf) {
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return QEM_ERR_CUDA;
    for (const Prof::Rec& r : pf->recs) {
      if (r.kind != kind) continue;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return QEM_ERR_CUDA;
      tot += t;
      ++cnt;
    }
  }
  if (ms) *ms = tot;
  if (launches) *launches = cnt;
  return QEM_OK;
}

}  // extern "C"
