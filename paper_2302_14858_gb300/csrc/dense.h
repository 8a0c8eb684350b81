// Dense per-block operator D = A^-1 B on the tensor cores (see dense_tc.cu).
#pragma once
#include "cfd_internal.h"

namespace cfd {

// One stage of the dense path over a group of same-size blocks: a GEMM of
// 128-pencil tiles against the digit images of up to two operators per pass.
struct DenseParams {
  const void *in;            // field buffer (dtype) or FP64 scratch
  void *out;                 // final output buffer (dtype)
  void *scratch_out;         // FP64 scratch for intermediate results
  const int *blocks;         // [nblk] global block ids
  const long long *extpre, *intpre;
  int nblk, nf, nops, N, g;
  int in_field;              // 1: in is the field buffer
  unsigned long long in_box, out_box;  // scratch box sizes (elements)
  int axis, t1, t2;          // box axes (0 z, 1 y, 2 x); t2 fastest
  int in_dims[3], out_dims[3], in_start[3], out_start[3];
  int n1, n2;                // transverse pencil counts
  int int_lo1, int_hi1, int_lo2, int_hi2;  // transverse range that writes final outputs
  int passes, rows;          // MMA passes per tile, output rows per pass (multiple of 16, <= 48)
  int nseg[2];               // operators (segments of N rows) per pass
  const uint16_t *seg_img[2][2];
  const int *seg_exp[2][2];
  int seg_mode[2][2];        // -1 skip, 0 final store, 2 FP64 scratch
  int seg_op[2][2];          // op index in the output for final stores
  int *status;
};

cfd_status dense_bind(cfd_blocks_s *B);
cfd_status dense_workspace(cfd_blocks_s *B, int nf, unsigned mask, cfd_precision prec, int n_iter, size_t *bytes);
cfd_status dense_apply(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, cfd_precision prec, int n_iter,
                       void *out, void *work, size_t work_bytes, cudaStream_t st);
}  // namespace cfd
