// FP32 CUDA-core forward contraction (Eq. Prmp) for latent dimensions 33..64
// (grouped mode), in a unit of its own: its unrolled code dominates the
// library's compile time.
#include "qem_simt_fwd.cuh"

namespace qem {

cudaError_t fwd_simt_d64(const LevelView& v, const LevelView& par, int K, int rows, int chunk, cudaStream_t s) {
  return fwd_simt_dispatch<64, false>(v, par, K, rows, chunk, s);
}

}  // namespace qem
