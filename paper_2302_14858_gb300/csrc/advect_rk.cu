// Time stepping of the advection equation u_t = beta^i d_i u (Sec. "Two dimensional advection",
// Eq. tr2pde with c = -beta; the shift-advection term of Sec. "Z4c: system description") with
// the upwinded biased operators, Kreiss-Oliger dissipation (Eq. dissdef) and the two-register
// (2S) low-storage Runge-Kutta recurrence.
#include <string.h>

#include <type_traits>

#include "cfd_internal.h"

namespace cfd {
namespace {

struct KoArgs {
  const double *u;         // field layout, ghosts exchanged
  double *F;               // interior [block][field][N^3]
  const long long *extpre, *intpre;
  const int *blocks;
  const double *scale;     // [b][degree][axis x, y, z] = 1/dx^d
  int N, g, nf, r, ko_on;
  double ko;               // -((-1)^r / 2^{2r}) sigma
  int c[13];               // (D_+)^r (D_-)^r stencil, m = -r..r
};

// F = sum_i Q_i[u] (0 without dissipation), axes x, y, z, taps m = -r..r in FP64.  RC: the
// stencil order r as a compile-time constant (0: taken from A.r).
template <int NC, int RC>
__global__ void k_ko_fields(const KoArgs A) {
  const int N = NC ? NC : A.N, g = A.g, E = N + 2 * g;
  const int r = RC ? RC : A.r;
  const int n3 = N * N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int job = blockIdx.y;
  const int lb = job / A.nf, q = job - lb * A.nf;
  const int b = A.blocks[lb];
  const int x = i % N, y = (i / N) % N, z = i / (N * N);
  const long long E3 = (long long)E * E * E;
  const long long e = (long long)A.nf * A.extpre[b] + q * E3 + ((long long)(z + g) * E + (y + g)) * E + (x + g);
  double f = 0.0;
  if (A.ko_on) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long st = a == 0 ? 1ll : (a == 1 ? (long long)E : (long long)E * E);   // x, y, z
      const double w = A.ko * A.scale[(b * 2 + 0) * 3 + a];
      double s = 0.0;
#pragma unroll
      for (int m = -r; m <= r; ++m) s = fma((double)A.c[m + r], __ldg(A.u + e + m * st), s);
      f = fma(w, s, f);
    }
  }
  A.F[(long long)A.nf * A.intpre[b] + (long long)q * n3 + i] = f;
}

struct UpdFArgs {
  double *u;               // field layout: S1, updated in place (interior)
  double *s2;              // interior: S2
  const double *F;
  const long long *extpre, *intpre;
  const int *blocks;
  int N, g, nf, first;
  double gamma1, gamma2, bdt, delta;
};

// S2 <- S2 + delta S1;  S1 <- (gamma1 S1 + gamma2 S2) + (beta dt) F.
template <int NC>
__global__ void k_lsrk_fields(const UpdFArgs A) {
  const int N = NC ? NC : A.N, g = A.g, E = N + 2 * g;
  const int n3 = N * N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int job = blockIdx.y;
  const int lb = job / A.nf, q = job - lb * A.nf;
  const int b = A.blocks[lb];
  const int x = i % N, y = (i / N) % N, z = i / (N * N);
  const long long E3 = (long long)E * E * E;
  const long long e = (long long)A.nf * A.extpre[b] + q * E3 + ((long long)(z + g) * E + (y + g)) * E + (x + g);
  const long long in = (long long)A.nf * A.intpre[b] + (long long)q * n3 + i;
  const double u = A.u[e];
  const double s = A.first ? __dmul_rn(A.delta, u) : __dadd_rn(A.s2[in], __dmul_rn(A.delta, u));
  A.s2[in] = s;
  A.u[e] = __dadd_rn(__dadd_rn(__dmul_rn(A.gamma1, u), __dmul_rn(A.gamma2, s)), __dmul_rn(A.bdt, A.F[in]));
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t interior_elems(const cfd_blocks_s *B) {
  size_t n = 0;
  for (int b = 0; b < B->nblocks; ++b) n += (size_t)B->n[b] * B->n[b] * B->n[b];
  return n;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" cfd_status cfd_advect_lsrk_workspace(cfd_blocks_t B, int nfields, cfd_precision prec, int n_iter,
                                                size_t *bytes) {
  if (!B || nfields < 1 || !bytes) { set_error("cfd_advect_lsrk_workspace: bad argument"); return CFD_ERR_ARG; }
  size_t bws = 0;
  cfd_status s = cfd_biased_workspace(B, nfields, prec, n_iter, &bws);
  if (s != CFD_OK) return s;
  *bytes = 2 * al256(interior_elems(B) * nfields * 8) + bws + 256;
  return CFD_OK;
}

extern "C" cfd_status cfd_advect_lsrk_step(cfd_blocks_t B, void *u, int nfields, const void *beta, double dt,
                                           const cfd_lsrk_desc *rk, double sigma, int ko_r, cfd_precision prec,
                                           int n_iter, void *work, size_t work_bytes, void *stream) {
  if (!B || !u || !beta || !work || !rk || nfields < 1) {
    set_error("cfd_advect_lsrk_step: bad argument");
    return CFD_ERR_ARG;
  }
  if (rk->stages < 1 || rk->stages > 8 || !rk->gamma1 || !rk->gamma2 || !rk->beta || !rk->delta) {
    set_error("cfd_advect_lsrk_step: 1..8 stages with all four coefficient arrays");
    return CFD_ERR_ARG;
  }
  if (!(sigma >= 0) || (sigma > 0 && (ko_r < 1 || ko_r > B->ng || ko_r > 6))) {
    set_error("cfd_advect_lsrk_step: sigma >= 0 and 1 <= ko_r <= min(ng, 6)");
    return CFD_ERR_ARG;
  }
  if (B->dtype != CFD_F64) { set_error("cfd_advect_lsrk_step: FP64 fields only"); return CFD_ERR_UNSUPPORTED; }
  for (auto &grp : B->groups)
    if ((long long)grp.size() * nfields > 65535) {
      set_error("cfd_advect_lsrk_step: blocks of one size x nfields exceeds 65535");
      return CFD_ERR_UNSUPPORTED;
    }
  for (int v : B->nbr)
    if (v < 0) { set_error("cfd_advect_lsrk_step: every ghost region needs a neighbour"); return CFD_ERR_UNSUPPORTED; }
  size_t need = 0;
  cfd_status s = cfd_advect_lsrk_workspace(B, nfields, prec, n_iter, &need);
  if (s != CFD_OK) return s;
  if (work_bytes < need) { set_error("cfd_advect_lsrk_step: workspace too small"); return CFD_ERR_ARG; }
  size_t bws = 0;
  if ((s = cfd_biased_workspace(B, nfields, prec, n_iter, &bws)) != CFD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t in_bytes = al256(interior_elems(B) * nfields * 8);
  char *base = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double *F = (double *)base;   base += in_bytes;
  double *S2 = (double *)base;  base += in_bytes;
  void *bw = bws ? (void *)base : nullptr;
  KoArgs K;
  memset(&K, 0, sizeof(K));
  K.u = (const double *)u;
  K.F = F;
  K.extpre = B->d_extpre;
  K.intpre = B->d_intpre;
  K.scale = B->d_scale;
  K.g = B->ng;
  K.nf = nfields;
  K.ko_on = sigma > 0;
  if (K.ko_on) {
    const int r = ko_r;
    K.r = r;
    long long binom = 1;
    for (int j = 0; j <= 2 * r; ++j) {
      K.c[j] = (int)((j % 2 == 0 ? 1 : -1) * binom);  // (-1)^j C(2r, j) at m = j - r
      binom = binom * (2 * r - j) / (j + 1);
    }
    K.ko = -((r % 2 == 0) ? 1.0 : -1.0) / (double)(1ll << (2 * r)) * sigma;
  }
  for (int stage = 0; stage < rk->stages; ++stage) {
    if ((s = cfd_exchange_ghosts(B, u, nfields, stream)) != CFD_OK) return s;
    for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
      const int N = B->sizes[gi];
      dim3 grid((unsigned)((N * N * N + 255) / 256), (unsigned)(B->groups[gi].size() * nfields));
      KoArgs A = K;
      A.blocks = B->d_groups[gi];
      A.N = N;
      launch_begin(KF_RK, st);
      const bool r4 = K.ko_on && K.r == 4;
      if (N == 32) { if (r4) k_ko_fields<32, 4><<<grid, 256, 0, st>>>(A); else k_ko_fields<32, 0><<<grid, 256, 0, st>>>(A); }
      else if (N == 16) { if (r4) k_ko_fields<16, 4><<<grid, 256, 0, st>>>(A); else k_ko_fields<16, 0><<<grid, 256, 0, st>>>(A); }
      else k_ko_fields<0, 0><<<grid, 256, 0, st>>>(A);
      launch_end(KF_RK, st);
      if ((s = cuda_fail(cudaGetLastError(), "k_ko_fields launch")) != CFD_OK) return s;
    }
    if ((s = advect_accumulate(B, u, nfields, beta, F, 1, 0, prec, n_iter, bw, bws, st)) != CFD_OK) return s;
    for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
      const int N = B->sizes[gi];
      dim3 grid((unsigned)((N * N * N + 255) / 256), (unsigned)(B->groups[gi].size() * nfields));
      UpdFArgs U;
      U.u = (double *)u;
      U.s2 = S2;
      U.F = F;
      U.extpre = B->d_extpre;
      U.intpre = B->d_intpre;
      U.blocks = B->d_groups[gi];
      U.N = N;
      U.g = B->ng;
      U.nf = nfields;
      U.first = stage == 0;
      U.gamma1 = rk->gamma1[stage];
      U.gamma2 = rk->gamma2[stage];
      U.bdt = rk->beta[stage] * dt;
      U.delta = rk->delta[stage];
      launch_begin(KF_RK, st);
      if (N == 32) k_lsrk_fields<32><<<grid, 256, 0, st>>>(U);
      else if (N == 16) k_lsrk_fields<16><<<grid, 256, 0, st>>>(U);
      else k_lsrk_fields<0><<<grid, 256, 0, st>>>(U);
      launch_end(KF_RK, st);
      if ((s = cuda_fail(cudaGetLastError(), "k_lsrk_fields launch")) != CFD_OK) return s;
    }
  }
  return CFD_OK;
}
