// Ghost regions exchanged between processes (each owning a subset of the MeshBlocks): the
// remote part of the communication matrix G of Eq. example_G.  A plan lists (block,
// direction) items; pack copies, for every item, the owner block's interior slab that fills a
// ghost region in that direction of its neighbour into a contiguous buffer; unpack writes a
// buffer into the ghost regions of the receiving blocks.  Items, per item nfields slabs in
// (z, y, x) order, in the order of the plan: a pack plan on the owner and an unpack plan on the
// receiver that list the same regions in the same order move the same values.
#include <algorithm>
#include <new>
#include <vector>

#include "cfd_internal.h"

struct cfd_halo_plan_s {
  cfd_blocks_s *B = nullptr;
  int n = 0, maxslab = 0;
  long long total = 0;              // slab elements of one field over all items
  int *d_items = nullptr;           // [n][4]: block, dz, dy, dx
  long long *d_off = nullptr;       // [n]: element offset of item i (one field)
  std::vector<long long> off;
};

namespace cfd {
namespace {

__device__ __forceinline__ int extent(int d, int N, int g) { return d == 0 ? N : g; }

// One thread per slab element of one (item, field).  dir > 0: pack (read the owner's interior
// at ghost - d N), dir < 0: unpack (write the receiver's ghost region).
template <typename T>
__global__ void k_halo(T *fields, T *buf, const int *__restrict__ items, const long long *__restrict__ off,
                       const long long *__restrict__ extpre, const int *__restrict__ nvec, int nf, int g,
                       long long total, int pack) {
  const int it = blockIdx.y, q = blockIdx.z;
  const int b = items[4 * it + 0], dz = items[4 * it + 1], dy = items[4 * it + 2], dx = items[4 * it + 3];
  const int N = nvec[b], E = N + 2 * g;
  const int rz = extent(dz, N, g), ry = extent(dy, N, g), rx = extent(dx, N, g);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rz * ry * rx) return;
  const int zi = e / (ry * rx), rem = e - zi * ry * rx, yi = rem / rx, xi = rem - yi * rx;
  // ghost-region coordinates of the receiving block (interior k = 0..N-1)
  const int z = dz < 0 ? zi - g : (dz > 0 ? N + zi : zi);
  const int y = dy < 0 ? yi - g : (dy > 0 ? N + yi : yi);
  const int x = dx < 0 ? xi - g : (dx > 0 ? N + xi : xi);
  T *blk = fields + (long long)nf * extpre[b] + (long long)q * E * E * E;
  T *slot = buf + (long long)q * total + off[it] + e;
  if (pack) {
    const int zs = z - dz * N, ys = y - dy * N, xs = x - dx * N;   // the owner's interior
    *slot = blk[((long long)(zs + g) * E + (ys + g)) * E + (xs + g)];
  } else {
    blk[((long long)(z + g) * E + (y + g)) * E + (x + g)] = *slot;
  }
}

cfd_status run_halo(cfd_halo_plan_s *P, void *fields, int nf, void *buf, bool pack, cudaStream_t st) {
  if (!P || !fields || !buf || nf < 1) { set_error("cfd_halo: bad argument"); return CFD_ERR_ARG; }
  if (P->n == 0) return CFD_OK;
  if (P->n > 65535 || nf > 65535) { set_error("cfd_halo: too many items or fields"); return CFD_ERR_UNSUPPORTED; }
  cfd_blocks_s *B = P->B;
  dim3 grid((unsigned)((P->maxslab + 255) / 256), (unsigned)P->n, (unsigned)nf);
  launch_begin(KF_EXCHANGE, st);
  if (B->dtype == CFD_F32)
    k_halo<float><<<grid, 256, 0, st>>>(static_cast<float *>(fields), static_cast<float *>(buf), P->d_items,
                                        P->d_off, B->d_extpre, B->d_nvec, nf, B->ng, P->total, pack ? 1 : 0);
  else
    k_halo<double><<<grid, 256, 0, st>>>(static_cast<double *>(fields), static_cast<double *>(buf), P->d_items,
                                         P->d_off, B->d_extpre, B->d_nvec, nf, B->ng, P->total, pack ? 1 : 0);
  launch_end(KF_EXCHANGE, st);
  return cuda_fail(cudaGetLastError(), "k_halo launch");
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_halo_plan_create(cfd_blocks_t B, const int *items, int n, cfd_halo_plan_t *out) {
  if (!B || !out || n < 0 || (n > 0 && !items)) { set_error("cfd_halo_plan_create: bad argument"); return CFD_ERR_ARG; }
  cfd_halo_plan_s *P = new (std::nothrow) cfd_halo_plan_s();
  if (!P) { set_error("out of host memory"); return CFD_ERR_ALLOC; }
  P->B = B;
  P->n = n;
  std::vector<int> it4((size_t)n * 4);
  P->off.resize(n);
  long long off = 0;
  for (int i = 0; i < n; ++i) {
    const int b = items[2 * i], r = items[2 * i + 1];
    if (b < 0 || b >= B->nblocks || r < 0 || r >= CFD_NDIRS) {
      delete P;
      set_error("cfd_halo_plan_create: block or direction out of range");
      return CFD_ERR_ARG;
    }
    const int rr = r >= 13 ? r + 1 : r;          // skip the centre of the 3x3x3 enumeration
    const int dz = rr / 9 - 1, dy = (rr / 3) % 3 - 1, dx = rr % 3 - 1;
    const int N = B->n[b], g = B->ng;
    const int rz = dz == 0 ? N : g, ry = dy == 0 ? N : g, rx = dx == 0 ? N : g;
    it4[4 * i] = b;
    it4[4 * i + 1] = dz;
    it4[4 * i + 2] = dy;
    it4[4 * i + 3] = dx;
    P->off[i] = off;
    off += (long long)rz * ry * rx;
    P->maxslab = std::max(P->maxslab, rz * ry * rx);
  }
  P->total = off;
  cfd_status s = CFD_OK;
  if (n > 0) {
    s = cuda_fail(cudaMalloc((void **)&P->d_items, it4.size() * sizeof(int)), "cudaMalloc");
    if (s == CFD_OK) s = cuda_fail(cudaMemcpy(P->d_items, it4.data(), it4.size() * sizeof(int), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (s == CFD_OK) s = cuda_fail(cudaMalloc((void **)&P->d_off, P->off.size() * sizeof(long long)), "cudaMalloc");
    if (s == CFD_OK)
      s = cuda_fail(cudaMemcpy(P->d_off, P->off.data(), P->off.size() * sizeof(long long), cudaMemcpyHostToDevice),
                    "cudaMemcpy");
  }
  if (s != CFD_OK) {
    cfd_halo_plan_destroy(P);
    return s;
  }
  *out = P;
  return CFD_OK;
}

cfd_status cfd_halo_plan_bytes(cfd_halo_plan_t P, int nfields, size_t *bytes) {
  if (!P || nfields < 1 || !bytes) { set_error("cfd_halo_plan_bytes: bad argument"); return CFD_ERR_ARG; }
  *bytes = (size_t)P->total * nfields * (P->B->dtype == CFD_F32 ? 4 : 8);
  return CFD_OK;
}

cfd_status cfd_halo_pack(cfd_halo_plan_t P, const void *fields, int nfields, void *buf, void *stream) {
  return run_halo(P, const_cast<void *>(fields), nfields, buf, true, (cudaStream_t)stream);
}

cfd_status cfd_halo_unpack(cfd_halo_plan_t P, void *fields, int nfields, const void *buf, void *stream) {
  return run_halo(P, fields, nfields, const_cast<void *>(buf), false, (cudaStream_t)stream);
}

void cfd_halo_plan_destroy(cfd_halo_plan_t P) {
  if (!P) return;
  if (P->d_items) cudaFree(P->d_items);
  if (P->d_off) cudaFree(P->d_off);
  delete P;
}

}  // extern "C"
