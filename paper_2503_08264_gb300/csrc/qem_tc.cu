// Tensor-core contraction path (placeholder until the tcgen05 kernels land).
#include "qem_tc.cuh"

namespace qem {

qem_status tc_plan_reserve(qem_plan_t P, const qem_model_desc*, char*, size_t* bytes) {
  *bytes = 0;
  return P->precision == QEM_PREC_FP32 ? QEM_OK : QEM_ERR_UNSUPPORTED;
}
qem_status tc_plan_init(qem_plan_t, const qem_model_desc*) { return QEM_OK; }
void tc_plan_release(qem_plan_t) {}
cudaError_t tc_forward(qem_plan_t, int) { return cudaErrorNotSupported; }
cudaError_t tc_adjoint(qem_plan_t, int) { return cudaErrorNotSupported; }

}  // namespace qem
