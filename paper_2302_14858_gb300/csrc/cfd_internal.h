// Internal structures of the CFD library (host API <-> CUDA kernels).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cfd.h"

namespace cfd {

constexpr int kMaxN = 32;        // largest block interior size
constexpr int kMaxM = 5;         // largest interior half-width
constexpr int kMaxH = 6;         // largest closure half-width
constexpr int kMaxIter = kMaxN + 4;

// Coefficients of one centred tridiagonal scheme (host copy).
struct SchemeCoef {
  bool present = false;
  int d = 0, order = 0, M = 0, h = 0;
  double a = 0.0;
  double rhs[2 * kMaxM + 1] = {};
  double clo[2 * kMaxH + 1] = {};
};

// Biased first-degree scheme (left-biased form) as given to cfd_scheme_set_biased.
constexpr int kBOff = 6;                 // coefficient of offset m stored at m + kBOff
constexpr int kBTaps = 2 * kBOff + 1;    // offsets -6..6
struct BiasedCoef {
  bool present = false;
  int order = 0, lo = 0, hi = 0, clo = 0, chi = 0, kc = 1;  // offset ranges (inclusive)
  double a = 0.0, csup = 0.0;
  double rhs[kBTaps] = {}, cl[kBTaps] = {};
};

// Per block size: what one biased pencil solve needs (passed by value).
struct BiasedTables {
  int N, kc;
  double a, csup;
  double inv01;            // 1 / (1 - csup a): the 2x2 coupling of the closure row
  double cyc_inv;          // 1 / (1 - (-a)^N): cyclic (single-block periodic) axis
  double rhs[kBTaps], clo[kBTaps];
  double pw[kMaxN + 1];    // (-a)^j
  // Halo-only passes: row N-kc of the left-biased and row kc-1 of the right-biased block
  // operator ([side][0 closed, 1 iterated][ghost-extended index]) and, for the iterated
  // operator, the coefficient of the fixed value at k^c.
  double hrow[2][2][kMaxN + 16];
  double hc[2];
};

// One biased axis pass over a group of same-size blocks.
struct BiasedParams {
  const void *in;          // field buffer (dtype)
  const void *beta;        // shift fields (advect mode)
  void *out;
  const int *blocks;
  const long long *extpre, *intpre;
  const int *nbr;
  const double *scale;     // [nblocks][2][3]; the degree-1 entries are used
  const double *halo_in;   // [nblocks][nf][N^2][2]: (d+ at N-kc, d- at kc-1) of the previous iterate
  double *halo_out;
  int nblk, nf, nops, opidx;
  int axis, t1, t2;        // box axes (0 z, 1 y, 2 x)
  int mode;                // 0 d[S+], 1 d[S-], 2 advect (beta_+ d[S+] + beta_- d[S-])
  int accum;               // 1: add into out
  int pass, last;
};

void build_biased_tables(const BiasedCoef &c, int N, int g, BiasedTables &T);
// dense form of a biased block system (kind 0 closed, 1 iterated, 2 cyclic), unscaled
void biased_operator(const BiasedCoef &c, int N, int g, int side, int kind, std::vector<long double> &W,
                     std::vector<long double> &coup);

// Everything one pencil solve needs for one (block size N, degree d).
// Passed to kernels by value.
struct LineTables {
  int N, M, h, d;
  double a;
  double rhs[2 * kMaxM + 1];
  double clo[2 * kMaxH + 1];
  // Closed system of Eq. sch_cent_om, rows k = 0..N-1 (Thomas factors):
  //   forward  y_k = (r_k - lo_k y_{k-1}) * inv_k,  back  x_k = y_k - c_k x_{k+1}.
  double lo[kMaxN], c[kMaxN], inv[kMaxN];
  // Iterated system of Eq. iter_center_P, rows k = -2..N+1 stored at k + 2.
  double ilo[kMaxIter], ic[kMaxIter], iinv[kMaxIter];
  // Cyclic (undecomposed periodic) system by Sherman-Morrison: Thomas factors
  // of the corner-modified tridiagonal T, the solution z of T z = u and
  // 1/(1 + v.z); x = y - (y_0 - a y_{N-1}) * vfac * z.
  double ylo[kMaxN], yc[kMaxN], yinv[kMaxN], z[kMaxN];
  double vfac;
};

// One axis-solve stage over a group of same-size blocks.
struct LineParams {
  const void *in;          // field buffer or scratch (double)
  void *out;               // output buffer, scratch or nothing (halo-only pass)
  const int *blocks;       // [nblk] global block ids of this group
  const long long *extpre; // [nblocks] sum over previous blocks of E^3
  const long long *intpre; // [nblocks] sum over previous blocks of N^3
  const int *nbr;          // [nblocks][26]
  const double *scale;     // [nblocks][2][3] 1/dx^d per degree, axis (x, y, z)
  const double *halo_in;   // [nblocks][nf][P][2] values exported by neighbours
  double *halo_out;
  int nblk, nf, nops, opidx;
  int g;
  int in_field;            // 1: in is the field buffer (dtype), 0: double scratch
  int out_mode;            // 0 store final, 1 average into final, 2 store scratch, 3 halo only
  int axis;                // 0 z, 1 y, 2 x (box axis order)
  int t1, t2;              // transverse box axes (t2 fastest)
  int in_dims[3], out_dims[3];
  int in_start[3], out_start[3];
  int n1, n2;              // transverse counts
  int pass;                // 0 closed solve, >0 iterated
  int last;                // 1 if this pass writes the output
  int deg;                 // 1 or 2
  unsigned long long in_box, out_box;  // scratch box sizes (elements)
  int *status;
};

struct OpSet {           // device copies per distinct block size
  int N;
  LineTables tab[2];     // degree 1, 2
};

}  // namespace cfd

struct cfd_scheme_s {
  cfd::SchemeCoef s[2];
  cfd::BiasedCoef biased;
};

struct cfd_blocks_s {
  cfd::SchemeCoef s[2];
  int device = 0, num_sms = 0;
  int nblocks = 0, ng = 0;
  cfd_dtype dtype = CFD_F64;
  std::vector<int> n;                  // per block
  std::vector<int> nbr;                // [nblocks * 26]
  std::vector<double> dx;              // [nblocks * 3]
  std::vector<long long> extpre, intpre;
  std::vector<int> sizes;              // distinct N, increasing
  std::vector<std::vector<int>> groups;  // block ids per distinct N
  std::vector<cfd::OpSet> ops;         // per distinct N
  cfd::BiasedCoef biased;
  std::vector<cfd::BiasedTables> btab; // per distinct N (when biased.present)
  bool iter_ok = true;                 // same-size face neighbours everywhere
  bool mixed_one_order = false;        // FP64 banded path: d_ij as D_i D_j only (cfd_blocks_set_mixed_order)
  // device copies
  int *d_nbr = nullptr;
  long long *d_extpre = nullptr, *d_intpre = nullptr;
  // ghost exchange: per block its 26 neighbours' field offsets (extpre of the neighbour, -1 for
  // none) and its own (entry 26), so a copy needs one table load
  long long *d_exch = nullptr;
  std::vector<int> group_b0;           // per group: first block id if the group's ids are consecutive, else -1
  double *d_scale = nullptr;
  int *d_nvec = nullptr;
  std::vector<int *> d_groups;
  int *d_status = nullptr;
  // dense operators for the tensor-core path (per distinct N), see dense_tc.cu:
  // host-side state, its deleter, and the device allocations it refers to
  void *dense_state = nullptr;
  void (*dense_free)(void *) = nullptr;
  std::vector<void *> d_dense_ptrs;
};

namespace cfd {

void set_error(const std::string &msg);
cfd_status cuda_fail(cudaError_t e, const char *what);

// launch accounting (profile.cpp)
enum KernelFamily { KF_EXCHANGE = 0, KF_LINE = 1, KF_RK = 2, KF_DENSE = 3, KF_HALO = 4, KF_BIASED = 5, KF_COUNT = 6 };
void launch_begin(int family, cudaStream_t st);
void launch_end(int family, cudaStream_t st);

// biased.cu: out[block][field][slot out_opidx of out_nops] += sum_i beta^i_+ D_i[S-] f + beta^i_- D_i[S+] f
// for nf fields (`work` as cfd_biased_workspace(B, nf, prec, n_iter))
cfd_status advect_accumulate(cfd_blocks_s *B, const void *fields, int nf, const void *beta, void *out, int out_nops,
                             int out_opidx, cfd_precision prec, int n_iter, void *work, size_t work_bytes,
                             cudaStream_t st);
// biased.cu: out slot = (accum_all ? out : 0) + sum_{i=x,y,z} beta^i (beta^i > 0 ? T[2i+1] : T[2i]),
// T = [block][field][6][N^3] (both biased derivatives of every axis)
cfd_status advect_combine(cfd_blocks_s *B, const void *tmp6, const void *beta, int nf, void *out, int out_nops,
                          int out_opidx, bool accum_all, cudaStream_t st);
// dense_tc.cu: the biased operators on the tensor cores
size_t dense_biased_workspace(const cfd_blocks_s *B, int nf, int n_iter, bool advect);
cfd_status dense_biased(cfd_blocks_s *B, const void *fields, int nf, const void *beta, const int *axes, int naxes,
                        int mode, cfd_precision prec, int n_iter, void *out, int out_nops, int out_opidx,
                        bool accum_all, void *work, size_t work_bytes, cudaStream_t st);

// kernels (banded.cu)
cfd_status launch_exchange(cfd_blocks_s *B, void *fields, int nfields, cudaStream_t st);
cfd_status launch_line(const LineParams &P, const LineTables &T, cudaStream_t st, cfd_dtype dt);

}  // namespace cfd
