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

// The same right-hand side for N in {16, 32} and r = RR, tiled: a CTA of N x TY threads owns
// TY rows of one block and marches along z.  The x and y stencil taps come from the current z
// plane staged in shared memory (with an RR-wide halo), the z taps from a queue of 2RR+1 values
// per thread in registers, so every field value is read from global memory about once per
// plane instead of 2r+1 times per direction, and converted to the stencil precision TK once (a
// double-to-float conversion runs on the FP64 pipe).  In FP64 the arithmetic and its order are
// those of k_wave_rhs (taps m = -r..r summed per axis, axes x, y, z added in that order); in
// FP32 the weighted directions are also summed in FP32 before the one FP64 add per field.
template <int N, typename TK, int RR>
__global__ void __launch_bounds__(256) k_wave_rhs_tiled(const RhsArgs A) {
  constexpr int TY = 256 / N, W = N + 2 * RR, H = TY + 2 * RR, Q = 2 * RR + 1;
  __shared__ TK sp_[H][W], sk_[H][W];
  const int g = A.g, E = N + 2 * g;
  const long long E2 = (long long)E * E;
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * N + tx;
  const int y0 = blockIdx.x * TY;
  const int b = A.blocks[blockIdx.y];
  const int n3 = N * N * N;
  const double *phi = A.phi + A.extpre[b], *K = A.K + A.extpre[b];
  double *L = A.lap + 3 * A.intpre[b];
  const double wx = __dmul_rn(A.ko, A.scale[(b * 2 + 0) * 3 + 0]);
  const double wy = __dmul_rn(A.ko, A.scale[(b * 2 + 0) * 3 + 1]);
  const double wz = __dmul_rn(A.ko, A.scale[(b * 2 + 0) * 3 + 2]);
  TK c[Q];
#pragma unroll
  for (int m = 0; m < Q; ++m) c[m] = (TK)A.c[m];
  // this thread's column (x, y) in the ghost-extended block
  const long long col = (long long)(y0 + ty + g) * E + (tx + g);
  TK qp[Q], qk[Q];
#pragma unroll
  for (int m = 0; m < Q - 1; ++m) {  // z = -RR .. RR-1 (ghost planes exist: RR <= g)
    qp[m + 1] = (TK)phi[(long long)(g + m - RR) * E2 + col];
    qk[m + 1] = (TK)K[(long long)(g + m - RR) * E2 + col];
  }
  for (int z = 0; z < N; ++z) {
    // shift the z queue and load plane z + RR
#pragma unroll
    for (int m = 0; m < Q - 1; ++m) { qp[m] = qp[m + 1]; qk[m] = qk[m + 1]; }
    qp[Q - 1] = (TK)phi[(long long)(g + z + RR) * E2 + col];
    qk[Q - 1] = (TK)K[(long long)(g + z + RR) * E2 + col];
    __syncthreads();  // the previous plane's taps are read
    const long long plane = (long long)(g + z) * E2;
    for (int i = t; i < H * W; i += 256) {
      const int r = i / W, xx = i - r * W;
      const long long o = plane + (long long)(y0 + r - RR + g) * E + (xx - RR + g);
      sp_[r][xx] = (TK)phi[o];
      sk_[r][xx] = (TK)K[o];
    }
    __syncthreads();
    const int i = (z * N + (y0 + ty)) * N + tx;
    double fk = __dadd_rn(__dadd_rn(L[i], L[n3 + i]), L[2 * n3 + i]);
    double fp = K[plane + col];
    TK px = 0, kx = 0, py = 0, ky = 0, pz = 0, kz = 0;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      px += c[m] * sp_[ty + RR][tx + m];
      kx += c[m] * sk_[ty + RR][tx + m];
      py += c[m] * sp_[ty + m][tx + RR];
      ky += c[m] * sk_[ty + m][tx + RR];
      pz += c[m] * qp[m];
      kz += c[m] * qk[m];
    }
    if constexpr (sizeof(TK) == 8) {
      fp = __dadd_rn(fp, __dmul_rn(wx, px));
      fk = __dadd_rn(fk, __dmul_rn(wx, kx));
      fp = __dadd_rn(fp, __dmul_rn(wy, py));
      fk = __dadd_rn(fk, __dmul_rn(wy, ky));
      fp = __dadd_rn(fp, __dmul_rn(wz, pz));
      fk = __dadd_rn(fk, __dmul_rn(wz, kz));
    } else {
      // FP32 stencil precision: the three directions are combined in FP32 too, so that one
      // conversion and one FP64 add per field remain on the FP64 pipe
      fp = __dadd_rn(fp, (double)((TK)wx * px + (TK)wy * py + (TK)wz * pz));
      fk = __dadd_rn(fk, (double)((TK)wx * kx + (TK)wy * ky + (TK)wz * kz));
    }
    L[i] = fk;
    L[n3 + i] = fp;
  }
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
  *bytes = al(L.in * 8) * 2 + al(3 * L.in * 8) + al(L.apply) + 256;
  return CFD_OK;
}

namespace cfd {
namespace {

// One 2S step of the wave system with Kreiss-Oliger terms; with `beta` the shifted system of
// Eq. toyShiftWaveEqnSys (flat gamma): the upwinded advective terms beta^i d_i Phi and
// beta^i d_i K are added to F_Phi and F_K.
cfd_status lsrk_impl(const char *who, cfd_blocks_s *B, void *phi, void *K, const void *beta, double dt,
                     const cfd_lsrk_desc *rk, double sigma, int ko_r, cfd_precision prec, int n_iter, void *work,
                     size_t work_bytes, cudaStream_t st) {
  auto fail = [&](cfd_status code, const char *msg) {
    set_error(std::string(who) + ": " + msg);
    return code;
  };
  if (!B || !phi || !K || !work || !rk) return fail(CFD_ERR_ARG, "bad argument");
  if (rk->stages < 1 || rk->stages > 8 || !rk->gamma1 || !rk->gamma2 || !rk->beta || !rk->delta)
    return fail(CFD_ERR_ARG, "1..8 stages with all four coefficient arrays");
  if (!(sigma >= 0) || (sigma > 0 && (ko_r < 1 || ko_r > B->ng || ko_r > 6)))
    return fail(CFD_ERR_ARG, "sigma >= 0 and 1 <= ko_r <= min(ng, 6)");
  if (B->dtype != CFD_F64) return fail(CFD_ERR_UNSUPPORTED, "FP64 fields only");
  if (!B->s[1].present) return fail(CFD_ERR_ARG, "needs the second-degree scheme");
  if (beta && !B->biased.present) return fail(CFD_ERR_ARG, "the shift terms need a biased scheme (cfd_scheme_set_biased)");
  for (int v : B->nbr)
    if (v < 0) return fail(CFD_ERR_UNSUPPORTED, "every ghost region needs a neighbour");
  WaveLayout L;
  cfd_status s = wave_layout(B, prec, n_iter, L);
  if (s != CFD_OK) return s;
  size_t bws = 0;
  if (beta && (s = cfd_biased_workspace(B, 1, prec, n_iter, &bws)) != CFD_OK) return s;
  const size_t need = al(L.in * 8) * 2 + al(3 * L.in * 8) + al(L.apply) + bws + 256;
  if (work_bytes < need) return fail(CFD_ERR_ARG, "workspace too small");
  char *base = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double *s2p = (double *)base;  base += al(L.in * 8);
  double *s2k = (double *)base;  base += al(L.in * 8);
  double *lap = (double *)base;  base += al(3 * L.in * 8);
  void *aw = base;               base += al(L.apply);
  void *bw = bws ? (void *)base : nullptr;
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
    if ((s = cfd_exchange_ghosts(B, phi, 1, st)) != CFD_OK) return s;
    if ((ko_on || beta) && (s = cfd_exchange_ghosts(B, K, 1, st)) != CFD_OK) return s;
    if ((s = cfd_apply(B, phi, 1, ops, prec, n_iter, lap, aw, L.apply, st)) != CFD_OK) return s;
    for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
      const int N = B->sizes[gi];
      const long long n3 = (long long)N * N * N;
      dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)B->groups[gi].size());
      RhsArgs A = R;
      A.blocks = B->d_groups[gi];
      A.N = N;
      launch_begin(KF_RK, st);
      if (ko_on && ko_r == 4 && (N == 32 || N == 16)) {
        const dim3 tg((unsigned)(N / (256 / N)), (unsigned)B->groups[gi].size());
        const dim3 tb((unsigned)N, (unsigned)(256 / N));
        if (N == 32) {
          if (prec == CFD_FP64_BANDED) k_wave_rhs_tiled<32, double, 4><<<tg, tb, 0, st>>>(A);
          else k_wave_rhs_tiled<32, float, 4><<<tg, tb, 0, st>>>(A);
        } else {
          if (prec == CFD_FP64_BANDED) k_wave_rhs_tiled<16, double, 4><<<tg, tb, 0, st>>>(A);
          else k_wave_rhs_tiled<16, float, 4><<<tg, tb, 0, st>>>(A);
        }
      } else if (N == 32) launch1(std::integral_constant<int, 32>(), A, grid);
      else if (N == 16) launch1(std::integral_constant<int, 16>(), A, grid);
      else launch1(std::integral_constant<int, 0>(), A, grid);
      launch_end(KF_RK, st);
      if ((s = cuda_fail(cudaGetLastError(), "k_wave_rhs launch")) != CFD_OK) return s;
    }
    if (beta) {
      // F_Phi (slot 1) += beta . grad Phi, F_K (slot 0) += beta . grad K, upwinded
      if ((s = advect_accumulate(B, phi, 1, beta, lap, 3, 1, prec, n_iter, bw, bws, st)) != CFD_OK) return s;
      if ((s = advect_accumulate(B, K, 1, beta, lap, 3, 0, prec, n_iter, bw, bws, st)) != CFD_OK) return s;
    }
    for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
      const int N = B->sizes[gi];
      const long long n3 = (long long)N * N * N;
      dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)B->groups[gi].size());
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

}  // namespace
}  // namespace cfd

extern "C" cfd_status cfd_wave_lsrk_step(cfd_blocks_t B, void *phi, void *K, double dt, const cfd_lsrk_desc *rk,
                                         double sigma, int ko_r, cfd_precision prec, int n_iter, void *work,
                                         size_t work_bytes, void *stream) {
  return lsrk_impl("cfd_wave_lsrk_step", B, phi, K, nullptr, dt, rk, sigma, ko_r, prec, n_iter, work, work_bytes,
                   (cudaStream_t)stream);
}

extern "C" cfd_status cfd_shifted_wave_workspace(cfd_blocks_t B, cfd_precision prec, int n_iter, size_t *bytes) {
  if (!B || !bytes) { set_error("cfd_shifted_wave_workspace: bad argument"); return CFD_ERR_ARG; }
  WaveLayout L;
  cfd_status s = wave_layout(B, prec, n_iter, L);
  if (s != CFD_OK) return s;
  size_t bws = 0;
  if ((s = cfd_biased_workspace(B, 1, prec, n_iter, &bws)) != CFD_OK) return s;
  *bytes = al(L.in * 8) * 2 + al(3 * L.in * 8) + al(L.apply) + bws + 256;
  return CFD_OK;
}

extern "C" cfd_status cfd_shifted_wave_lsrk_step(cfd_blocks_t B, void *phi, void *K, const void *beta, double dt,
                                                 const cfd_lsrk_desc *rk, double sigma, int ko_r, cfd_precision prec,
                                                 int n_iter, void *work, size_t work_bytes, void *stream) {
  if (!beta) { set_error("cfd_shifted_wave_lsrk_step: beta is null (use cfd_wave_lsrk_step)"); return CFD_ERR_ARG; }
  return lsrk_impl("cfd_shifted_wave_lsrk_step", B, phi, K, beta, dt, rk, sigma, ko_r, prec, n_iter, work,
                   work_bytes, (cudaStream_t)stream);
}
