// Classical RK4 (ERK4) driver for the linear wave system
//   d/dt Phi = K,  d/dt K = sum_i D2_i Phi   (Eq. toyShiftWaveEqnSys, zero shift)
// on MeshBlocks.  Each stage: ghost exchange of the stage Phi, the three
// second derivatives through cfd_apply, then one elementwise combine kernel.
// The combine uses separate multiply and add (no contraction) in the order
//   acc = k1; acc = acc + 2 k2; acc = acc + 2 k3; acc = acc + k4;
//   Phi <- Phi + (dt/6) acc.
#include "cfd_internal.h"

namespace cfd {
namespace {

struct StageArgs {
  double *phi;          // field layout (ghosts) : the state Phi
  double *K;            // field layout          : the state K
  double *phis;         // field layout          : stage Phi (input of the next Laplacian)
  double *Ks;           // interior              : stage K
  const double *lap;    // interior, 3 ops       : d_xx, d_yy, d_zz of the stage Phi
  double *accP, *accK;  // interior
  const long long *extpre, *intpre;
  const int *blocks;
  int N, g, stage;
  double c;             // 0.5 dt, 0.5 dt, dt, dt/6
};

// NC: the block size as a compile-time constant (0: taken from A.N at run time).
template <int NC>
__global__ void k_rk_combine(const StageArgs A) {
  const int N = NC ? NC : A.N, E = N + 2 * A.g;
  const int n3 = N * N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int b = A.blocks[blockIdx.y];
  const int x = i % N, y = (i / N) % N, z = i / (N * N);
  const long long e = A.extpre[b] + ((z + A.g) * E + (y + A.g)) * E + (x + A.g);
  const long long in = A.intpre[b] + i;
  const double *L = A.lap + 3 * A.intpre[b];
  const double lap = __dadd_rn(__dadd_rn(L[i], L[n3 + i]), L[2 * n3 + i]);
  // k_P of this stage is the stage K (stage 1: the state K)
  const double kp = (A.stage == 1) ? A.K[e] : A.Ks[in];
  const double kk = lap;
  double ap, ak;
  if (A.stage == 1) {
    ap = kp;
    ak = kk;
  } else if (A.stage == 4) {
    ap = __dadd_rn(A.accP[in], kp);
    ak = __dadd_rn(A.accK[in], kk);
  } else {
    ap = __dadd_rn(A.accP[in], __dmul_rn(2.0, kp));
    ak = __dadd_rn(A.accK[in], __dmul_rn(2.0, kk));
  }
  if (A.stage < 4) {
    A.accP[in] = ap;
    A.accK[in] = ak;
    A.phis[e] = __dadd_rn(A.phi[e], __dmul_rn(A.c, kp));
    A.Ks[in] = __dadd_rn(A.K[e], __dmul_rn(A.c, kk));
  } else {
    A.phi[e] = __dadd_rn(A.phi[e], __dmul_rn(A.c, ap));
    A.K[e] = __dadd_rn(A.K[e], __dmul_rn(A.c, ak));
  }
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct WaveLayout {
  size_t ext = 0, in = 0, apply = 0;
  size_t total() const { return al(ext * 8) + al(in * 8) * 3 + al(3 * in * 8) + apply + 256; }
};

cfd_status wave_layout(cfd_blocks_s *B, cfd_precision prec, int n_iter, WaveLayout &L) {
  for (int b = 0; b < B->nblocks; ++b) {
    const size_t N = B->n[b], E = N + 2 * B->ng;
    L.ext += E * E * E;
    L.in += N * N * N;
  }
  return cfd_apply_workspace(B, 1, CFD_OP_DXX | CFD_OP_DYY | CFD_OP_DZZ, prec, n_iter, &L.apply);
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" cfd_status cfd_wave_workspace(cfd_blocks_t B, cfd_precision prec, int n_iter, size_t *bytes) {
  if (!B || !bytes) { set_error("cfd_wave_workspace: bad argument"); return CFD_ERR_ARG; }
  WaveLayout L;
  cfd_status s = wave_layout(B, prec, n_iter, L);
  if (s != CFD_OK) return s;
  *bytes = L.total();
  return CFD_OK;
}

extern "C" cfd_status cfd_wave_rk_step(cfd_blocks_t B, void *phi, void *K, double dt, cfd_precision prec, int n_iter,
                                       void *work, size_t work_bytes, void *stream) {
  if (!B || !phi || !K || !work) { set_error("cfd_wave_rk_step: bad argument"); return CFD_ERR_ARG; }
  if (B->dtype != CFD_F64) { set_error("cfd_wave_rk_step: FP64 fields only"); return CFD_ERR_UNSUPPORTED; }
  if (!B->s[1].present) { set_error("cfd_wave_rk_step: needs the second-degree scheme"); return CFD_ERR_ARG; }
  for (int v : B->nbr)
    if (v < 0) { set_error("cfd_wave_rk_step: every ghost region needs a neighbour"); return CFD_ERR_UNSUPPORTED; }
  WaveLayout L;
  cfd_status s = wave_layout(B, prec, n_iter, L);
  if (s != CFD_OK) return s;
  if (work_bytes < L.total()) { set_error("cfd_wave_rk_step: workspace too small"); return CFD_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  char *base = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double *phis = (double *)base;  base += al(L.ext * 8);
  double *Ks = (double *)base;    base += al(L.in * 8);
  double *accP = (double *)base;  base += al(L.in * 8);
  double *accK = (double *)base;  base += al(L.in * 8);
  double *lap = (double *)base;   base += al(3 * L.in * 8);
  void *aw = base;
  const unsigned ops = CFD_OP_DXX | CFD_OP_DYY | CFD_OP_DZZ;
  const double cs[5] = {0, 0.5 * dt, 0.5 * dt, dt, dt / 6.0};
  for (int stage = 1; stage <= 4; ++stage) {
    double *src = stage == 1 ? (double *)phi : phis;
    if ((s = cfd_exchange_ghosts(B, src, 1, stream)) != CFD_OK) return s;
    if ((s = cfd_apply(B, src, 1, ops, prec, n_iter, lap, aw, L.apply, stream)) != CFD_OK) return s;
    for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
      StageArgs A;
      A.phi = (double *)phi;
      A.K = (double *)K;
      A.phis = phis;
      A.Ks = Ks;
      A.lap = lap;
      A.accP = accP;
      A.accK = accK;
      A.extpre = B->d_extpre;
      A.intpre = B->d_intpre;
      A.blocks = B->d_groups[gi];
      A.N = B->sizes[gi];
      A.g = B->ng;
      A.stage = stage;
      A.c = cs[stage];
      const long long n3 = (long long)A.N * A.N * A.N;
      dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)B->groups[gi].size());
      launch_begin(KF_RK, st);
      if (A.N == 32) k_rk_combine<32><<<grid, 256, 0, st>>>(A);
      else if (A.N == 16) k_rk_combine<16><<<grid, 256, 0, st>>>(A);
      else if (A.N == 8) k_rk_combine<8><<<grid, 256, 0, st>>>(A);
      else k_rk_combine<0><<<grid, 256, 0, st>>>(A);
      launch_end(KF_RK, st);
      if ((s = cuda_fail(cudaGetLastError(), "k_rk_combine launch")) != CFD_OK) return s;
    }
  }
  return CFD_OK;
}
