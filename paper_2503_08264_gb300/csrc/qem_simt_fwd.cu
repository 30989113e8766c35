// FP32 CUDA-core forward contraction (Eq. Prmp): latent dimensions up to 32,
// both modes, and the entry point.
#include "qem_simt_fwd.cuh"

namespace qem {

template <bool SPLIT>
static cudaError_t fwd_simt_dims(const LevelView& v, const LevelView& par, int K, int rows, int chunk,
                                 cudaStream_t s) {
  if (v.D <= 4) return fwd_simt_dispatch<4, SPLIT>(v, par, K, rows, chunk, s);
  if (v.D <= 8) return fwd_simt_dispatch<8, SPLIT>(v, par, K, rows, chunk, s);
  if (v.D <= 20) return fwd_simt_dispatch<20, SPLIT>(v, par, K, rows, chunk, s);
  if (v.D <= 32) return fwd_simt_dispatch<32, SPLIT>(v, par, K, rows, chunk, s);
  if (SPLIT) return cudaErrorInvalidValue;
  return fwd_simt_d64(v, par, K, rows, chunk, s);
}

// rows: parent samples per block (a multiple of 32, at most 256); chunk: child
// samples staged per round (16, 32, or 64 for D <= 20; others take 32).
cudaError_t launch_fwd_simt(const LevelView& v, const LevelView& par, int K, int rows, int chunk, cudaStream_t s,
                            bool split) {
  if (v.n == 0) return cudaSuccess;
  if (rows < 32 || rows > kFwdRowsMax || rows % 32) return cudaErrorInvalidValue;
  return split ? fwd_simt_dims<true>(v, par, K, rows, chunk, s) : fwd_simt_dims<false>(v, par, K, rows, chunk, s);
}

}  // namespace qem
