// Tensor-core (tcgen05) contraction path of libqem: plan-time reservation of
// the operand buffers and the forward / adjoint launches for one level.
#pragma once

#include "qem_internal.cuh"

#include <cuda_bf16.h>

namespace qem {

// Column layout of the operand rows of one level (16-bit columns, canonical
// K-major core-matrix layout; a TF32 value takes two columns).  Parent rows (A of the forward):
//   [Ah | 1 1 1 | .. | Ah at a_ah2 | .. | Al at a_al | 0..]   (split 3)
// child rows (B of the forward):
//   [Bh | h1 h2 h3 | .. | Bl at b_bl | (Bh at b_bh2) | 0..]
// and a table of MMA k-steps pairing parent columns ka[i]..+16 with child
// columns kb[i]..+16.  When it saves child bytes, the lo*hi product re-reads
// the first Bh block instead of storing Bh twice (b_bh2 = -1), with the
// ragged tail of that product packed into the padding (tail, a_alt, b_bht).
struct Layout {
  int nb = 0, split = 1;
  int fka = 0, fkb = 0;
  int a_ah2 = -1, a_al = -1, b_bl = -1, b_bh2 = -1;
  // compact form: the last `tail` features of the lo*hi product sit in the
  // padding after the Ah/Bl block (parent Al at a_alt, child Bh copy at
  // b_bht); the Al block at a_al then holds only the first nb - tail.
  int tail = 0, a_alt = -1, b_bht = -1;
  int nks = 0;
  int ka[16] = {}, kb[16] = {};
};

struct TcBuffers {
  Layout lay[QEM_MAX_LEVELS];
  int nb[QEM_MAX_LEVELS] = {};   // bilinear features of child level l
  int split = 3;                 // 3: split BF16, 1: BF16, 0: TF32 rows
  bool tf32 = false;
  __nv_bfloat16* bfeat[QEM_MAX_LEVELS] = {};   // child level l:   [n_l][K rows][fkb] canonical
  __nv_bfloat16* afeat[QEM_MAX_LEVELS] = {};   // parent of l:     [n_{l-1}][K rows][fka]
  __nv_bfloat16* cfeat[QEM_MAX_LEVELS] = {};   // compacted parent rows, same layout
  float* rowc[QEM_MAX_LEVELS] = {};            // [n_{l-1}][K] row constants (nats)
  float* center[QEM_MAX_LEVELS] = {};          // [n_{l-1}][D_l]
  float* dcol[QEM_MAX_LEVELS] = {};            // [n_l][K] adjoint column shifts (log2 units)
};

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
// Element-resident schedule of the forward (qem_tc_res.cu): whether operand
// rows of these widths (16-bit units) and K samples fit it, its one-time
// kernel set-up, and the launch for level l.
bool tc_res_fits(int frow, int fcol, int K);
qem_status tc_res_init(int frow, int fcol, int K, bool tf32);
cudaError_t tc_forward_res(qem_plan_t P, int l, bool tf32);
// Element-resident schedule of the adjoint (rows: the child's operand, frow
// wide; columns: the parent's, fcol wide): whether it fits, and the launch.
bool tc_adj_res_fits(int frow, int fcol, int K);
cudaError_t tc_adjoint_res(qem_plan_t P, int l, bool tf32);

}  // namespace qem
