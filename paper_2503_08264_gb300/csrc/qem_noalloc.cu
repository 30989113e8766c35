// Allocation-free E-step for single-level models (one latent per instance).
//
// Some callers cannot call cudaMalloc at the point where they need an
// E-step: memory-pool-managed runtimes that forbid allocations outside their
// pool, or real-time loops where an allocation's latency and implicit
// synchronisation are not acceptable.  For them this entry point keeps its
// scratch (samples, local factors, weights, per-instance constants and the
// control block) in one file-scope device array instead of a plan workspace,
// and allocates nothing on the device or the host.
//
// The array holds at most kNoAllocScratchBytes bytes (32 MiB); every GPU that
// loads the library keeps it until the process exits.  All calls share it:
// calls whose GPU work overlaps (different streams, or different host
// threads) race on it.  Its contents persist between calls; everything a
// call reads is written by that call first, and the control block is
// cleared at the start of every call.
#include <cuda_runtime.h>

#include "qem_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device with that
// device current (host code must not use the symbol itself as an address).
// A cudaDeviceReset releases the module that holds the array, so a kept
// address is not valid after one (documented in the header).
void* g_scratch_addr[kMaxDevices] = {};

inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" qem_status qem_estep_single_noalloc(const qem_level_desc* level, int K, const float* q_params,
                                               const float* eps, uint64_t seed, uint64_t iter, double* moments,
                                               double* log_pmp, void* stream) {
  using namespace qem;
  if (!level || !q_params || !moments || K < 1 || K > 4096) return QEM_ERR_INVALID_ARG;
  const qem_level_desc& d = *level;
  if (d.parent || d.n < 0 || d.dim < 1 || d.n_obs < 0 || d.chain < 0) return QEM_ERR_INVALID_ARG;
  if (d.chain > 1 || d.qcond) return QEM_ERR_UNSUPPORTED;
  if (d.dim > kMaxDim || d.n_obs > 4096 || (size_t)d.n_obs * d.dim > 8192) return QEM_ERR_UNSUPPORTED;
  if (d.qfam < QEM_Q_GAUSS || d.qfam > QEM_Q_BETA || d.lik < QEM_LIK_NONE || d.lik > QEM_LIK_BERNOULLI_PROB)
    return QEM_ERR_INVALID_ARG;
  if (d.lik == QEM_LIK_NONE && d.n_obs != 0) return QEM_ERR_INVALID_ARG;
  if (d.lik != QEM_LIK_NONE && d.n_obs > 0 && d.n > 0 && (!d.x || !d.y)) return QEM_ERR_INVALID_ARG;
  if (d.lik == QEM_LIK_GAUSS && !(d.lik_var > 0)) return QEM_ERR_INVALID_ARG;
  if ((d.lik == QEM_LIK_POISSON_RATE && (d.qfam != QEM_Q_GAMMA || d.dim != 1)) ||
      (d.lik == QEM_LIK_BERNOULLI_PROB && (d.qfam != QEM_Q_BETA || d.dim != 1)))
    return QEM_ERR_INVALID_ARG;
  if (!((d.prior == QEM_PRIOR_STD_NORMAL && d.qfam == QEM_Q_GAUSS && d.prior_a > 0) ||
        (d.prior == QEM_PRIOR_GAMMA && d.qfam == QEM_Q_GAMMA && d.prior_a > 0 && d.prior_b > 0) ||
        (d.prior == QEM_PRIOR_BETA && d.qfam == QEM_Q_BETA && d.prior_a > 0 && d.prior_b > 0)))
    return QEM_ERR_INVALID_ARG;
  if (d.n == 0) return QEM_OK;

  // scratch layout: control block, log P_MP, per-instance constants and
  // shifts, the count table (Poisson-log only), local factors, weights,
  // samples
  const size_t nK = (size_t)d.n * K;
  const bool counts = d.lik == QEM_LIK_POISSON_LOG;
  const size_t need = up256(sizeof(Ctl)) + up256(sizeof(double) * (size_t)d.n) * 2 + up256(sizeof(float) * (size_t)d.n) +
                      (counts ? up256(sizeof(double) * kCountTable) : 0) + up256(sizeof(float) * nK) * 2 +
                      up256(sizeof(float) * nK * d.dim);
  if (need > kNoAllocScratchBytes) return QEM_ERR_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QEM_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return QEM_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += up256(bytes);
    return p;
  };
  Ctl* ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  double* lp_internal = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d.n));
  LevelView v{};
  v.n = d.n;
  v.D = d.dim;
  v.prior = d.prior;
  v.prior_a = (float)d.prior_a;
  v.prior_b = (float)d.prior_b;
  v.lik = d.lik;
  v.lik_var = (float)d.lik_var;
  v.n_obs = d.lik == QEM_LIK_NONE ? 0 : d.n_obs;
  v.qfam = d.qfam;
  v.nps = d.qfam == QEM_Q_GAUSS ? d.dim : d.dim * (2 * QEM_GAMMA_TRIES + 1) * (d.qfam == QEM_Q_GAMMA ? 1 : 2);
  v.level = 0;
  v.chain = 1;
  v.beta = nullptr;
  v.qcond = 0;
  v.perm = nullptr;
  v.pz = nullptr;
  v.pD = 0;
  v.cz = nullptr;
  v.x = d.x;
  v.y = d.y;
  v.cst = reinterpret_cast<double*>(take(sizeof(double) * (size_t)d.n));
  v.cshift = reinterpret_cast<float*>(take(sizeof(float) * (size_t)d.n));
  double* tab = counts ? reinterpret_cast<double*>(take(sizeof(double) * kCountTable)) : nullptr;
  v.ltab = tab;
  v.loc = reinterpret_cast<float*>(take(sizeof(float) * nK));
  v.htil = v.loc;
  v.w = reinterpret_cast<float*>(take(sizeof(float) * nK));
  v.z = reinterpret_cast<float*>(take(sizeof(float) * nK * d.dim));

  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess) return QEM_ERR_CUDA;
  if (launch_set_ctl(ctl, seed, iter, 1, -1, s) != cudaSuccess) return QEM_ERR_CUDA;
  const Tune dflt;
  if (configure_sample_local(sample_local_smem(v, K, dflt.sample_threads)) != cudaSuccess) return QEM_ERR_CUDA;
  if (tab && launch_count_table(tab, s) != cudaSuccess) return QEM_ERR_CUDA;
  if (launch_sample_local(v, K, dflt.sample_threads, q_params, eps, ctl, s) != cudaSuccess) return QEM_ERR_CUDA;
  if (launch_elem_const(v, q_params, s) != cudaSuccess) return QEM_ERR_CUDA;
  if (launch_root(v, K, false, lp_internal, log_pmp, nullptr, ctl, s) != cudaSuccess) return QEM_ERR_CUDA;
  if (launch_moments(v, K, dflt.mom_threads, moments, s) != cudaSuccess) return QEM_ERR_CUDA;
  return QEM_OK;
}
