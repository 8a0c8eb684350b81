// Dense per-block operator path on the tensor cores (placeholder until the
// tcgen05 kernels land): every request is reported as unsupported.
#include "dense.h"

namespace cfd {
cfd_status dense_bind(cfd_blocks_s *) { return CFD_OK; }
cfd_status dense_workspace(cfd_blocks_s *, int, unsigned, cfd_precision, int, size_t *) {
  set_error("tensor-core precisions are not built yet");
  return CFD_ERR_UNSUPPORTED;
}
cfd_status dense_apply(cfd_blocks_s *, const void *, int, unsigned, cfd_precision, int, void *, void *, size_t,
                       cudaStream_t) {
  set_error("tensor-core precisions are not built yet");
  return CFD_ERR_UNSUPPORTED;
}
}  // namespace cfd
