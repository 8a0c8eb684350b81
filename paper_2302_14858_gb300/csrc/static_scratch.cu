// Allocation-free variant of the FP64 banded apply (closures only).
//
// Who needs it: code that embeds these operators where device allocation is
// not available at the call site -- a host simulation that hands all device
// memory to its own pool at start-up and forbids later cudaMalloc/cudaFree,
// a solver step running under a fixed memory budget, or any caller that must
// not synchronise the device (cudaFree does) in the middle of its time loop.
// Such callers can still bind the blocks once at start-up; this entry point
// then needs no workspace argument and allocates nothing per call.
//
// The scratch it needs (the D_j intermediate of the mixed derivatives, on rows
// extended along i) lives in one file-scope device array of fixed size.  Every
// GPU that loads this library holds that array until the process exits.  Host
// code cannot use the array's name as a device address, so the address is
// looked up with cudaGetSymbolAddress once per device (on the first call made
// on that device, with that device current) and handed to the kernels.
#include <mutex>

#include "cfd_internal.h"

namespace cfd {
size_t banded_closed_scratch_bytes(const cfd_blocks_s *B, int nf, unsigned mask);
cfd_status apply_banded_closed(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, void *out,
                               double *scratch, cudaStream_t st);
}  // namespace cfd

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of g_static_scratch, per device ordinal

}  // namespace

using namespace cfd;

extern "C" cfd_status cfd_apply_static(cfd_blocks_t B, const void *fields, int nfields, unsigned op_mask, void *out,
                                       void *stream) {
  if (!B || !fields || !out || nfields < 1 || !op_mask || (op_mask & ~CFD_OP_ALL)) {
    set_error("cfd_apply_static: bad argument");
    return CFD_ERR_ARG;
  }
  for (auto &grp : B->groups)
    if ((long long)grp.size() * nfields > 65535) {
      set_error("cfd_apply_static: blocks of one size x nfields exceeds 65535");
      return CFD_ERR_UNSUPPORTED;
    }
  const size_t need = banded_closed_scratch_bytes(B, nfields, op_mask);
  if (need > kStaticScratchBytes) {
    set_error("cfd_apply_static: this request needs " + std::to_string(need) +
              " bytes of scratch but the static array holds " + std::to_string(kStaticScratchBytes) +
              "; split the fields or blocks over several calls");
    return CFD_ERR_ARG;
  }
  int dev = -1;
  cfd_status s = cuda_fail(cudaGetDevice(&dev), "cfd_apply_static: cudaGetDevice");
  if (s != CFD_OK) return s;
  if (dev != B->device) {
    set_error("cfd_apply_static: the current device is not the one the blocks were bound on");
    return CFD_ERR_ARG;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("cfd_apply_static: device ordinal out of range");
    return CFD_ERR_UNSUPPORTED;
  }
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      s = cuda_fail(cudaGetSymbolAddress(&p, g_static_scratch), "cfd_apply_static: cudaGetSymbolAddress");
      if (s != CFD_OK) return s;
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  // Nothing in the scratch has to start at zero: every intermediate value is
  // written by the first stage before the second stage reads it.
  return apply_banded_closed(B, fields, nfields, op_mask, out, static_cast<double *>(scratch),
                             (cudaStream_t)stream);
}
