// Classical RK4 (ERK4) driver for the linear wave system
//   d/dt Phi = K,  d/dt K = sum_i D2_i Phi   (Eq. toyShiftWaveEqnSys, zero shift)
// on MeshBlocks.  Each stage: ghost exchange of the stage Phi, the three
// second derivatives through cfd_apply, then one elementwise combine kernel.
// The combine uses separate multiply and add (no contraction) in the order
//   acc = k1; acc = acc + 2 k2; acc = acc + 2 k3; acc = acc + k4;
//   Phi <- Phi + (dt/6) acc.
#include <string.h>

#include <type_traits>

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

// ---------------------------------------------------------------- 2S low-storage RK + KO dissipation

struct RhsArgs {
  const double *phi, *K;     // field layout, ghosts exchanged (K's only when ko_on)
  double *lap;               // interior, 3 ops: d_xx, d_yy, d_zz in; F_K, F_Phi out (slots 0, 1)
  const long long *extpre, *intpre;
  const int *blocks;
  const double *scale;       // [b][degree][axis x, y, z] = 1/dx^d
  int N, g, r, ko_on;
  double ko;                 // -((-1)^r / 2^{2r}) sigma
  int c[13];                 // (D_+)^r (D_-)^r stencil (2r)E_r, m = -r..r
};

// Right-hand side of the wave system with Kreiss-Oliger terms (Eq. dissdef) at every
// interior point: F_K = (d_xx + d_yy) + d_zz + sum_i Q_i[K], F_Phi = K + sum_i Q_i[Phi].
// TK is the precision of the dissipation stencil sums.
template <int NC, typename TK>
__global__ void k_wave_rhs(const RhsArgs A) {
  const int N = NC ? NC : A.N, g = A.g, E = N + 2 * g;
  const int n3 = N * N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int b = A.blocks[blockIdx.y];
  const int x = i % N, y = (i / N) % N, z = i / (N * N);
  const long long e = A.extpre[b] + ((z + g) * E + (y + g)) * E + (x + g);
  double *L = A.lap + 3 * A.intpre[b];
  double fk = __dadd_rn(__dadd_rn(L[i], L[n3 + i]), L[2 * n3 + i]);
  double fp = A.K[e];
  if (A.ko_on) {
    const long long stride[3] = {1, E, (long long)E * E};   // x, y, z
    for (int a = 0; a < 3; ++a) {
      const double w = __dmul_rn(A.ko, A.scale[(b * 2 + 0) * 3 + a]);
      TK sp = 0, sk = 0;
      for (int m = -A.r; m <= A.r; ++m) {
        const long long o = e + m * stride[a];
        sp += (TK)A.c[m + A.r] * (TK)A.phi[o];
        sk += (TK)A.c[m + A.r] * (TK)A.K[o];
      }
      fp = __dadd_rn(fp, __dmul_rn(w, (double)sp));
      fk = __dadd_rn(fk, __dmul_rn(w, (double)sk));
    }
  }
  L[i] = fk;
  L[n3 + i] = fp;
}

struct UpdArgs {
  double *phi, *K;           // field layout: S1, updated in place (interior)
  double *s2p, *s2k;         // interior: S2
  const double *lap;         // F_K, F_Phi (slots 0, 1)
  const long long *extpre, *intpre;
  const int *blocks;
  int N, g, first;
  double gamma1, gamma2, bdt, delta;
};

// S2 <- S2 + delta S1;  S1 <- (gamma1 S1 + gamma2 S2) + (beta dt) F, per field.
template <int NC>
__global__ void k_lsrk_update(const UpdArgs A) {
  const int N = NC ? NC : A.N, g = A.g, E = N + 2 * g;
  const int n3 = N * N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int b = A.blocks[blockIdx.y];
  const int x = i % N, y = (i / N) % N, z = i / (N * N);
  const long long e = A.extpre[b] + ((z + g) * E + (y + g)) * E + (x + g);
  const long long in = A.intpre[b] + i;
  const double *L = A.lap + 3 * A.intpre[b];
  const double p = A.phi[e], k = A.K[e];
  const double sp = A.first ? __dmul_rn(A.delta, p) : __dadd_rn(A.s2p[in], __dmul_rn(A.delta, p));
  const double sk = A.first ? __dmul_rn(A.delta, k) : __dadd_rn(A.s2k[in], __dmul_rn(A.delta, k));
  A.s2p[in] = sp;
  A.s2k[in] = sk;
  A.phi[e] = __dadd_rn(__dadd_rn(__dmul_rn(A.gamma1, p), __dmul_rn(A.gamma2, sp)), __dmul_rn(A.bdt, L[n3 + i]));
  A.K[e] = __dadd_rn(__dadd_rn(__dmul_rn(A.gamma1, k), __dmul_rn(A.gamma2, sk)), __dmul_rn(A.bdt, L[i]));
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

extern "C" cfd_status cfd_wave_lsrk_workspace(cfd_blocks_t B, cfd_precision prec, int n_iter, size_t *bytes) {
  if (!B || !bytes) { set_error("cfd_wave_lsrk_workspace: bad argument"); return CFD_ERR_ARG; }
  WaveLayout L;
  cfd_status s = wave_layout(B, prec, n_iter, L);
  if (s != CFD_OK) return s;
  *bytes = al(L.in * 8) * 2 + al(3 * L.in * 8) + L.apply + 256;
  return CFD_OK;
}

extern "C" cfd_status cfd_wave_lsrk_step(cfd_blocks_t B, void *phi, void *K, double dt, const cfd_lsrk_desc *rk,
                                         double sigma, int ko_r, cfd_precision prec, int n_iter, void *work,
                                         size_t work_bytes, void *stream) {
  if (!B || !phi || !K || !work || !rk) { set_error("cfd_wave_lsrk_step: bad argument"); return CFD_ERR_ARG; }
  if (rk->stages < 1 || rk->stages > 8 || !rk->gamma1 || !rk->gamma2 || !rk->beta || !rk->delta) {
    set_error("cfd_wave_lsrk_step: 1..8 stages with all four coefficient arrays");
    return CFD_ERR_ARG;
  }
  if (!(sigma >= 0) || (sigma > 0 && (ko_r < 1 || ko_r > B->ng || ko_r > 6))) {
    set_error("cfd_wave_lsrk_step: sigma >= 0 and 1 <= ko_r <= min(ng, 6)");
    return CFD_ERR_ARG;
  }
  if (B->dtype != CFD_F64) { set_error("cfd_wave_lsrk_step: FP64 fields only"); return CFD_ERR_UNSUPPORTED; }
  if (!B->s[1].present) { set_error("cfd_wave_lsrk_step: needs the second-degree scheme"); return CFD_ERR_ARG; }
  for (int v : B->nbr)
    if (v < 0) { set_error("cfd_wave_lsrk_step: every ghost region needs a neighbour"); return CFD_ERR_UNSUPPORTED; }
  WaveLayout L;
  cfd_status s = wave_layout(B, prec, n_iter, L);
  if (s != CFD_OK) return s;
  const size_t need = al(L.in * 8) * 2 + al(3 * L.in * 8) + L.apply + 256;
  if (work_bytes < need) { set_error("cfd_wave_lsrk_step: workspace too small"); return CFD_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  char *base = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double *s2p = (double *)base;  base += al(L.in * 8);
  double *s2k = (double *)base;  base += al(L.in * 8);
  double *lap = (double *)base;  base += al(3 * L.in * 8);
  void *aw = base;
  const unsigned ops = CFD_OP_DXX | CFD_OP_DYY | CFD_OP_DZZ;
  const bool ko_on = sigma > 0;
  RhsArgs R;
  memset(&R, 0, sizeof(R));
  R.phi = (const double *)phi;
  R.K = (const double *)K;
  R.lap = lap;
  R.extpre = B->d_extpre;
  R.intpre = B->d_intpre;
  R.scale = B->d_scale;
  R.g = B->ng;
  R.ko_on = ko_on ? 1 : 0;
  if (ko_on) {
    // (D_+)^r (D_-)^r: (-1)^(r+m) C(2r, r+m); prefactor -((-1)^r / 2^{2r}) sigma
    const int r = ko_r;
    R.r = r;
    long long binom = 1;
    for (int j = 0; j <= 2 * r; ++j) {
      R.c[j] = (int)((j % 2 == 0 ? 1 : -1) * binom);  // m = j - r: (-1)^(r+m) C(2r, r+m) = (-1)^j C(2r, j)
      binom = binom * (2 * r - j) / (j + 1);
    }
    R.ko = -((r % 2 == 0) ? 1.0 : -1.0) / (double)(1ll << (2 * r)) * sigma;
  }
  auto launch1 = [&](auto nc, const RhsArgs &A, dim3 grid) {
    if (prec == CFD_FP64_BANDED) k_wave_rhs<decltype(nc)::value, double><<<grid, 256, 0, st>>>(A);
    else k_wave_rhs<decltype(nc)::value, float><<<grid, 256, 0, st>>>(A);
  };
  for (int stage = 0; stage < rk->stages; ++stage) {
    if ((s = cfd_exchange_ghosts(B, phi, 1, stream)) != CFD_OK) return s;
    if (ko_on && (s = cfd_exchange_ghosts(B, K, 1, stream)) != CFD_OK) return s;
    if ((s = cfd_apply(B, phi, 1, ops, prec, n_iter, lap, aw, L.apply, stream)) != CFD_OK) return s;
    for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
      const int N = B->sizes[gi];
      const long long n3 = (long long)N * N * N;
      dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)B->groups[gi].size());
      RhsArgs A = R;
      A.blocks = B->d_groups[gi];
      A.N = N;
      launch_begin(KF_RK, st);
      if (N == 32) launch1(std::integral_constant<int, 32>(), A, grid);
      else if (N == 16) launch1(std::integral_constant<int, 16>(), A, grid);
      else launch1(std::integral_constant<int, 0>(), A, grid);
      launch_end(KF_RK, st);
      if ((s = cuda_fail(cudaGetLastError(), "k_wave_rhs launch")) != CFD_OK) return s;
      UpdArgs U;
      U.phi = (double *)phi;
      U.K = (double *)K;
      U.s2p = s2p;
      U.s2k = s2k;
      U.lap = lap;
      U.extpre = B->d_extpre;
      U.intpre = B->d_intpre;
      U.blocks = B->d_groups[gi];
      U.N = N;
      U.g = B->ng;
      U.first = stage == 0;
      U.gamma1 = rk->gamma1[stage];
      U.gamma2 = rk->gamma2[stage];
      U.bdt = rk->beta[stage] * dt;
      U.delta = rk->delta[stage];
      launch_begin(KF_RK, st);
      if (N == 32) k_lsrk_update<32><<<grid, 256, 0, st>>>(U);
      else if (N == 16) k_lsrk_update<16><<<grid, 256, 0, st>>>(U);
      else k_lsrk_update<0><<<grid, 256, 0, st>>>(U);
      launch_end(KF_RK, st);
      if ((s = cuda_fail(cudaGetLastError(), "k_lsrk_update launch")) != CFD_OK) return s;
    }
  }
  return CFD_OK;
}
