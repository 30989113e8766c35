// Tensor-core (tcgen05) contraction path of libqem: plan-time reservation of
// the operand buffers and the forward / adjoint launches for one level.
#pragma once

#include "qem_internal.cuh"

namespace qem {

// Bytes of workspace the tensor-core path needs (base == nullptr: size only;
// otherwise carve the buffers from base).
qem_status tc_plan_reserve(qem_plan_t P, const qem_model_desc* desc, char* base, size_t* bytes);
// One-time set-up after the workspace exists (kernel attributes, constant operands).
qem_status tc_plan_init(qem_plan_t P, const qem_model_desc* desc);
void tc_plan_release(qem_plan_t P);
// Operand features of level l (l >= 1) and its parent level, after the
// level's relative local factors are final.
cudaError_t tc_features(qem_plan_t P, int l);
// Forward contraction of level l into lv[l].lt.
cudaError_t tc_forward(qem_plan_t P, int l);
// Adjoint of level l into lv[l].w for the elements whose parent keeps more
// than kSmallKept weighted samples (the rest run on the CUDA cores):
// operand gathering and column shifts, then the contraction.
cudaError_t tc_adjoint_prep(qem_plan_t P, int l);
cudaError_t tc_adjoint(qem_plan_t P, int l);

}  // namespace qem
