// Dense per-block operator D = A^-1 B on the tensor cores (see dense_tc.cu).
#pragma once
#include "cfd_internal.h"

namespace cfd {
cfd_status dense_bind(cfd_blocks_s *B);
cfd_status dense_workspace(cfd_blocks_s *B, int nf, unsigned mask, cfd_precision prec, int n_iter, size_t *bytes);
cfd_status dense_apply(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, cfd_precision prec, int n_iter,
                       void *out, void *work, size_t work_bytes, cudaStream_t st);
}  // namespace cfd
