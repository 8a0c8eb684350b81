// FP64 biased (upwind) path: per-pencil bidiagonal solves of the left-biased
// block system (Eq. closure_left_X), its mirror closed at k*_+, their iteration
// (Eq. iter_left_X) and the upwinded shift-advection term (Eq. biasderapproxadv).
//
// One thread owns one pencil of one block and field.  The ghost-extended pencil
// is held in registers; each row's right-hand side is an FMA chain over the
// (compile-time) stencil window, scaled by 1/dx.  The solves are first-order
// recurrences: left-biased rows run k = 0..N-1 (a 2x2 solve couples the closure
// row k*_- with row 1), right-biased rows run k = N-1..0.  In advect mode the
// right-biased derivative is kept in registers and combined with the left-biased
// one as it is produced, so one pass over the pencil yields the upwinded right-hand-side term
// beta d f = beta_+ D[S-] f + beta_- D[S+] f for that axis (transport velocity -beta: the
// right-biased scheme where beta > 0, the left-biased one where beta < 0).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "cfd_internal.h"

namespace cfd {

// Biased block operator in dense form: the block system (closed: N rows,
// Eq. closure_left_X or its mirror; iterated: N + kc rows with the value at k^c fixed,
// Eq. iter_left_X; cyclic: the undecomposed periodic system) solved for every right-hand-side
// column (f at ghost-extended index j, and the fixed value) in long double, without dx scaling.
// W: N x E row-major (the N interior rows), coup: the N coefficients of the fixed value.
void biased_operator(const BiasedCoef &c, int N, int g, int side, int kind, std::vector<long double> &W,
                     std::vector<long double> &coup) {
  const int E = N + 2 * g, kc = c.kc;
  const bool iter = kind == 1, cyc = kind == 2;
  const int n = iter ? N + kc : N;
  const int k0 = (iter && side > 0) ? -kc : 0;   // local index of unknown 0
  std::vector<long double> A((size_t)n * n, 0), X((size_t)n * (E + 1), 0);
  for (int u = 0; u < n; ++u) {
    const int k = k0 + u;
    A[(size_t)u * n + u] = 1;
    if (iter && ((side > 0 && u == 0) || (side < 0 && u == n - 1))) {
      X[(size_t)u * (E + 1) + E] = 1;               // fixed node
      continue;
    }
    const bool clo = !iter && !cyc && ((side > 0 && k == 0) || (side < 0 && k == N - 1));
    int off = side > 0 ? (clo ? 1 : -1) : (clo ? -1 : 1);
    int col = u + off;
    if (cyc) col = (col + n) % n;
    A[(size_t)u * n + col] += clo ? c.csup : c.a;
    const double *co = clo ? c.cl : c.rhs;
    for (int m = -kBOff; m <= kBOff; ++m) {
      const double v = co[m + kBOff];
      if (v == 0) continue;
      int j = side > 0 ? k + m : k - m;             // mirror: -alpha_m at offset -m
      if (cyc) j = ((j % N) + N) % N;               // periodic line: the interior point itself
      X[(size_t)u * (E + 1) + j + g] += side > 0 ? v : -v;
    }
  }
  // Gauss-Jordan elimination with partial pivoting
  for (int col = 0; col < n; ++col) {
    int pr = col;
    for (int r = col + 1; r < n; ++r)
      if (fabsl(A[(size_t)r * n + col]) > fabsl(A[(size_t)pr * n + col])) pr = r;
    if (pr != col) {
      for (int q = 0; q < n; ++q) std::swap(A[(size_t)pr * n + q], A[(size_t)col * n + q]);
      for (int q = 0; q <= E; ++q) std::swap(X[(size_t)pr * (E + 1) + q], X[(size_t)col * (E + 1) + q]);
    }
    const long double d = A[(size_t)col * n + col];
    for (int q = 0; q < n; ++q) A[(size_t)col * n + q] /= d;
    for (int q = 0; q <= E; ++q) X[(size_t)col * (E + 1) + q] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const long double f = A[(size_t)r * n + col];
      if (f == 0) continue;
      for (int q = 0; q < n; ++q) A[(size_t)r * n + q] -= f * A[(size_t)col * n + q];
      for (int q = 0; q <= E; ++q) X[(size_t)r * (E + 1) + q] -= f * X[(size_t)col * (E + 1) + q];
    }
  }
  W.assign((size_t)N * E, 0);
  coup.assign(N, 0);
  for (int k = 0; k < N; ++k) {
    const int u = k - k0;
    for (int j = 0; j < E; ++j) W[(size_t)k * E + j] = X[(size_t)u * (E + 1) + j];
    coup[k] = X[(size_t)u * (E + 1) + E];
  }
}

void build_biased_tables(const BiasedCoef &c, int N, int g, BiasedTables &T) {
  memset(&T, 0, sizeof(T));
  T.N = N;
  T.kc = c.kc;
  T.a = c.a;
  T.csup = c.csup;
  T.inv01 = 1.0 / (1.0 - c.csup * c.a);
  double p = 1.0;
  for (int j = 0; j <= N; ++j) {
    T.pw[j] = p;   // (-a)^j
    p *= -c.a;
  }
  T.cyc_inv = 1.0 / (1.0 - T.pw[N]);
  for (int i = 0; i < kBTaps; ++i) {
    T.rhs[i] = c.rhs[i];
    T.clo[i] = c.cl[i];
  }
  const int E = N + 2 * g;
  if (E > kMaxN + 16 || c.kc > N) return;   // refused later by the request checks
  std::vector<long double> W, coup;
  for (int side = 0; side < 2; ++side)
    for (int it = 0; it < 2; ++it) {
      const int sg = side == 0 ? 1 : -1;
      const int k = sg > 0 ? N - c.kc : c.kc - 1;
      biased_operator(c, N, g, sg, it, W, coup);
      for (int j = 0; j < E; ++j) T.hrow[side][it][j] = (double)W[(size_t)k * E + j];
      if (it == 1) T.hc[side] = (double)coup[k];
    }
}

namespace {

__device__ __forceinline__ int dir_index(int dz, int dy, int dx) {
  int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
  return r > 13 ? r - 1 : r;
}

// 1 if v > 0, 2 if v < 0, 0 if v is a zero (integer tests on the bits)
__device__ __forceinline__ int sign_bits(double v) {
  const long long u = __double_as_longlong(v);
  return (u << 1) == 0 ? 0 : (u < 0 ? 2 : 1);
}
__device__ __forceinline__ int sign_bits(float v) {
  const int u = __float_as_int(v);
  return (u << 1) == 0 ? 0 : (u < 0 ? 2 : 1);
}

// Stencil windows compiled in: interior offsets ILO..IHI and closure offsets
// CLO..CHI of the left-biased scheme (the mirror uses the negated offsets).
// A tap that falls outside the ghost-extended pencil is dropped at compile time;
// the host checks that every such tap has a zero coefficient for the rows used.
template <int NT, int G, int ILO, int IHI, int CLO, int CHI, typename T>
__global__ void __launch_bounds__(128) k_biased(const BiasedParams P, const BiasedTables Tb) {
  constexpr int E = NT + 2 * G;
  constexpr int np = NT * NT;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int job = blockIdx.y;
  const int lb = job / P.nf, q = job - lb * P.nf;
  const int b = P.blocks[lb];
  const int t1 = p / NT, t2 = p - t1 * NT;
  const int ax = P.axis;
  const int ez = ax == 0, ey = ax == 1, ex = ax == 2;
  const int nlo = P.nbr[b * 26 + dir_index(-ez, -ey, -ex)];
  const int nhi = P.nbr[b * 26 + dir_index(ez, ey, ex)];
  const bool cyclic = (nlo == b && nhi == b);
  if (cyclic && P.pass > 0) return;  // finished in pass 0
  const bool last = cyclic || P.last;

  // strides of the (E, E, E) box along box axis i (0 z, 1 y, 2 x); selects, not an indexed array
  auto estr = [](int i) { return i == 0 ? (long long)E * E : (i == 1 ? (long long)E : 1ll); };
  constexpr long long box = (long long)E * E * E;
  const long long sa = estr(ax);
  const long long tr = (long long)(t1 + G) * estr(P.t1) + (long long)(t2 + G) * estr(P.t2);
  const T *fin = static_cast<const T *>(P.in) + (long long)P.nf * P.extpre[b] + (long long)q * box + tr;

  double fv[E];
#pragma unroll
  for (int j = 0; j < E; ++j) fv[j] = static_cast<double>(__ldg(fin + j * sa));

  const double scale = P.scale[(b * 2 + 0) * 3 + (2 - ax)];
  const double a = Tb.a;

  // unscaled sums; k is a compile-time constant after unrolling
  auto left_int = [&](int k) {
    double acc = 0.0;
#pragma unroll
    for (int m = ILO; m <= IHI; ++m) {
      const int j = k + m + G;
      if (j >= 0 && j < E) acc = fma(Tb.rhs[m + kBOff], fv[j], acc);
    }
    return acc;
  };
  auto left_clo = [&](int k) {
    double acc = 0.0;
#pragma unroll
    for (int m = CLO; m <= CHI; ++m) {
      const int j = k + m + G;
      if (j >= 0 && j < E) acc = fma(Tb.clo[m + kBOff], fv[j], acc);
    }
    return acc;
  };
  // mirror: alpha^{(0)}_m -> -alpha^{(0)}_{-m}; the sign is applied by the caller
  auto right_int = [&](int k) {
    double acc = 0.0;
#pragma unroll
    for (int m = ILO; m <= IHI; ++m) {
      const int j = k - m + G;
      if (j >= 0 && j < E) acc = fma(Tb.rhs[m + kBOff], fv[j], acc);
    }
    return acc;
  };
  auto right_clo = [&](int k) {
    double acc = 0.0;
#pragma unroll
    for (int m = CLO; m <= CHI; ++m) {
      const int j = k - m + G;
      if (j >= 0 && j < E) acc = fma(Tb.clo[m + kBOff], fv[j], acc);
    }
    return acc;
  };

  const bool do_p = P.mode != 1, do_m = P.mode != 0;
  const long long hp = (long long)np * 2;

  if (!last) {
    // halo-only pass: the two values the neighbours read next pass (d+ at N-kc, d- at kc-1),
    // each one row of the dense block operator (closed for pass 0, iterated after that)
    const int it = P.pass > 0 ? 1 : 0;
    double *h = P.halo_out + ((long long)b * P.nf + q) * hp + 2 * p;
    if (do_p) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < E; ++j) acc = fma(Tb.hrow[0][it][j], fv[j], acc);
      double v = acc * scale;
      if (it) v = fma(Tb.hc[0], P.halo_in[((long long)nlo * P.nf + q) * hp + 2 * p + 0], v);
      h[0] = v;
    }
    if (do_m) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < E; ++j) acc = fma(Tb.hrow[1][it][j], fv[j], acc);
      double v = acc * scale;
      if (it) v = fma(Tb.hc[1], P.halo_in[((long long)nhi * P.nf + q) * hp + 2 * p + 1], v);
      h[1] = v;
    }
    return;
  }

  // advect: a side whose shift sign does not occur on this pencil is not needed
  const T *bet = P.mode == 2 ? static_cast<const T *>(P.beta) + 3ll * P.extpre[b] + (long long)(2 - ax) * box + tr +
                                   (long long)G * sa
                             : nullptr;
  bool need_p = do_p, need_m = do_m;
  if (P.mode == 2) {
    int any = 0;
#pragma unroll
    for (int k = 0; k < NT; ++k) any |= sign_bits(__ldg(bet + k * sa));
    need_p = (any & 2) != 0;   // beta < 0 somewhere: left-biased
    need_m = (any & 1) != 0;   // beta > 0 somewhere: right-biased
  }

  // ---- right-biased derivative (S-), rows k = N-1 .. 0, kept in registers
  double dm[NT];
  if (need_m) {
    const double ms = -scale;
    if (cyclic) {
      // y_{N-1} = r_{N-1}, y_k = r_k - a y_{k+1};  d_k = y_k + (-a)^{N-k} d_0, d_0 = y_0 / (1 - (-a)^N)
#pragma unroll
      for (int k = NT - 1; k >= 0; --k) {
        const double r = right_int(k) * ms;
        dm[k] = (k == NT - 1) ? r : fma(-a, dm[k + 1], r);
      }
      const double d0 = dm[0] * Tb.cyc_inv;
#pragma unroll
      for (int k = 1; k < NT; ++k) dm[k] = fma(Tb.pw[NT - k], d0, dm[k]);
      dm[0] = d0;
    } else if (P.pass == 0) {
      // closure row N-1 (csup d_{N-2} + d_{N-1}) coupled with interior row N-2
      const double rc = right_clo(NT - 1) * ms;
      const double r2 = right_int(NT - 2) * ms;
      dm[NT - 1] = fma(-Tb.csup, r2, rc) * Tb.inv01;
      dm[NT - 2] = fma(-a, dm[NT - 1], r2);
#pragma unroll
      for (int k = NT - 3; k >= 0; --k) dm[k] = fma(-a, dm[k + 1], right_int(k) * ms);
    } else {
      // iterated: d at k^c_+ = N-1+kc is the right neighbour's previous iterate
      double h = P.halo_in[((long long)nhi * P.nf + q) * hp + 2 * p + 1];
      if (Tb.kc >= 3) h = fma(-a, h, right_int(NT + 1) * ms);
      if (Tb.kc >= 2) h = fma(-a, h, right_int(NT) * ms);
#pragma unroll
      for (int k = NT - 1; k >= 0; --k) {
        h = fma(-a, h, right_int(k) * ms);
        dm[k] = h;
      }
    }
  }

  // ---- outputs
  constexpr long long n3 = (long long)NT * NT * NT;
  auto ostr = [](int i) { return i == 0 ? (long long)NT * NT : (i == 1 ? (long long)NT : 1ll); };
  const long long oa = ostr(ax);
  T *o = static_cast<T *>(P.out) + (long long)P.nf * P.nops * P.intpre[b] + ((long long)q * P.nops + P.opidx) * n3 +
         (long long)t1 * ostr(P.t1) + (long long)t2 * ostr(P.t2);
  auto emit = [&](int k, double dp) {
    double v;
    if (P.mode == 0) {
      v = dp;
    } else if (P.mode == 1) {
      v = dm[k];
    } else {
      // beta_+ dm + beta_- dp: beta dm where beta > 0, beta dp where beta < 0, 0 where beta = 0
      const T braw = __ldg(bet + k * sa);
      const int sg = sign_bits(braw);
      const double bb = static_cast<double>(braw);
      v = sg == 1 ? bb * dm[k] : (sg == 2 ? bb * dp : 0.0);
    }
    if (P.accum) v = static_cast<double>(o[k * oa]) + v;
    o[k * oa] = static_cast<T>(v);
  };

  // ---- left-biased derivative (S+), rows k = 0 .. N-1, emitted as produced
  if (need_p) {
    if (cyclic) {
      // y_0 = r_0, y_k = r_k - a y_{k-1};  d_k = y_k + (-a)^{k+1} d_{N-1}, d_{N-1} = y_{N-1} / (1 - (-a)^N)
      double y = 0.0;
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        const double r = left_int(k) * scale;
        y = (k == 0) ? r : fma(-a, y, r);
      }
      const double dl = y * Tb.cyc_inv;
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        const double r = left_int(k) * scale;
        y = (k == 0) ? r : fma(-a, y, r);
        emit(k, fma(Tb.pw[k + 1], dl, y));
      }
    } else {
      double d;
      int k0;
      if (P.pass == 0) {
        // closure row 0 (d_0 + csup d_1) coupled with interior row 1
        const double r0 = left_clo(0) * scale;
        const double r1 = left_int(1) * scale;
        d = fma(-Tb.csup, r1, r0) * Tb.inv01;
        emit(0, d);
        d = fma(-a, d, r1);
        emit(1, d);
        k0 = 2;
      } else {
        // iterated: d at k^c_- = -kc is the left neighbour's previous iterate
        d = P.halo_in[((long long)nlo * P.nf + q) * hp + 2 * p + 0];
        if (Tb.kc >= 3) d = fma(-a, d, left_int(-2) * scale);
        if (Tb.kc >= 2) d = fma(-a, d, left_int(-1) * scale);
        k0 = 0;
      }
#pragma unroll
      for (int k = 0; k < NT; ++k) {
        if (k < k0) continue;
        d = fma(-a, d, left_int(k) * scale);
        emit(k, d);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NT; ++k) emit(k, 0.0);
  }
}

template <int G, int ILO, int IHI, int CLO, int CHI>
cfd_status launch_window(const BiasedParams &P, const BiasedTables &T, cudaStream_t st, cfd_dtype dt) {
  const int np = T.N * T.N;
  dim3 grid((np + 127) / 128, P.nblk * P.nf);
  auto go = [&](auto nt) {
    constexpr int NT = decltype(nt)::value;
    if (dt == CFD_F32) k_biased<NT, G, ILO, IHI, CLO, CHI, float><<<grid, 128, 0, st>>>(P, T);
    else k_biased<NT, G, ILO, IHI, CLO, CHI, double><<<grid, 128, 0, st>>>(P, T);
  };
  switch (T.N) {
    case 8: go(std::integral_constant<int, 8>()); break;
    case 16: go(std::integral_constant<int, 16>()); break;
    case 32: go(std::integral_constant<int, 32>()); break;
    default: set_error("biased path: block size must be 8, 16 or 32"); return CFD_ERR_UNSUPPORTED;
  }
  return cuda_fail(cudaGetLastError(), "k_biased launch");
}

// The compiled (ng, window) combinations; the first that contains the scheme's
// offset ranges is used.
struct Window { int g, ilo, ihi, clo, chi; };
constexpr Window kWindows[] = {{4, -3, 4, -4, 4}, {4, -4, 4, -4, 5}, {6, -5, 5, -5, 6}};

int pick_window(const BiasedCoef &c, int g) {
  for (int i = 0; i < (int)(sizeof(kWindows) / sizeof(kWindows[0])); ++i) {
    const Window &w = kWindows[i];
    if (w.g == g && c.lo >= w.ilo && c.hi <= w.ihi && c.clo >= w.clo && c.chi <= w.chi) return i;
  }
  return -1;
}

cfd_status launch_biased(int win, const BiasedParams &P, const BiasedTables &T, cudaStream_t st, cfd_dtype dt) {
  launch_begin(KF_BIASED, st);
  cfd_status s;
  switch (win) {
    case 0: s = launch_window<4, -3, 4, -4, 4>(P, T, st, dt); break;
    case 1: s = launch_window<4, -4, 4, -4, 5>(P, T, st, dt); break;
    case 2: s = launch_window<6, -5, 5, -5, 6>(P, T, st, dt); break;
    default: set_error("biased path: no compiled stencil window"); s = CFD_ERR_UNSUPPORTED;
  }
  launch_end(KF_BIASED, st);
  return s;
}

size_t halo_elems(const cfd_blocks_s *B, int nf, int n_iter) {
  if (n_iter <= 0) return 0;
  int nmax = 0;
  for (int N : B->sizes) nmax = std::max(nmax, N);
  return (size_t)B->nblocks * nf * nmax * nmax * 2;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Checks shared by cfd_apply_biased and cfd_advect.
cfd_status check_request(cfd_blocks_s *B, int nf, cfd_precision prec, int n_iter, int *win) {
  if (!B->biased.present) {
    set_error("no biased scheme bound (cfd_scheme_set_biased before cfd_blocks_bind)");
    return CFD_ERR_ARG;
  }
  if (prec != CFD_FP64_BANDED && prec != CFD_TC_BF16_EXACT && prec != CFD_TC_BF16X3) {
    set_error("biased path: CFD_FP64_BANDED, CFD_TC_BF16_EXACT or CFD_TC_BF16X3");
    return CFD_ERR_UNSUPPORTED;
  }
  if (n_iter < 0 || n_iter > 64) { set_error("biased path: n_iter out of range"); return CFD_ERR_ARG; }
  const BiasedCoef &c = B->biased;
  const int g = B->ng;
  *win = pick_window(c, g);
  if (*win < 0) {
    set_error("biased path: stencil offsets and ng outside the compiled windows");
    return CFD_ERR_UNSUPPORTED;
  }
  // taps the rows in use reach: closure row k = 0, interior rows from 1 (closed),
  // 0 (cyclic) or 1 - kc (iterated) to N - 1; mirrored for S-
  const int kfirst = n_iter > 0 ? 1 - c.kc : 0;
  if (c.clo < -g || c.lo + kfirst < -g || c.hi > g) {
    set_error("biased path: stencil reaches beyond the ghost layers");
    return CFD_ERR_UNSUPPORTED;
  }
  for (int N : B->sizes)
    if (N < 2 || c.chi > N - 1 + g || c.kc > N) {
      set_error("biased path: block too small for the closure or kc");
      return CFD_ERR_UNSUPPORTED;
    }
  if (n_iter > 0 && !B->iter_ok) {
    set_error("biased path: iteration needs same-size face neighbours on every decomposed axis");
    return CFD_ERR_UNSUPPORTED;
  }
  for (auto &grp : B->groups)
    if ((long long)grp.size() * nf > 65535) {
      set_error("biased path: blocks of one size x nfields exceeds 65535");
      return CFD_ERR_UNSUPPORTED;
    }
  return CFD_OK;
}

// axes: box axes in output order; mode 0/1 derivative (one op per axis), 2 advect (one op, summed)
cfd_status run_biased(cfd_blocks_s *B, const void *fields, int nf, const void *beta, const int *axes, int naxes,
                      int mode, int n_iter, int win, void *out, void *work, cudaStream_t st, int out_nops = 0,
                      int out_opidx = 0, bool accum_all = false) {
  double *halo[2] = {nullptr, nullptr};
  const size_t he = halo_elems(B, nf, n_iter);
  if (he) {
    char *base = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
    halo[0] = (double *)base;
    halo[1] = (double *)(base + align256(he * 8));
  }
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const BiasedTables &T = B->btab[gi];
    BiasedParams P;
    memset(&P, 0, sizeof(P));
    P.in = fields;
    P.beta = beta;
    P.out = out;
    P.blocks = B->d_groups[gi];
    P.extpre = B->d_extpre;
    P.intpre = B->d_intpre;
    P.nbr = B->d_nbr;
    P.scale = B->d_scale;
    P.nblk = (int)B->groups[gi].size();
    P.nf = nf;
    P.nops = out_nops > 0 ? out_nops : (mode == 2 ? 1 : naxes);
    P.mode = mode;
    for (int i = 0; i < naxes; ++i) {
      const int a = axes[i];
      P.axis = a;
      P.t1 = a == 0 ? 1 : 0;
      P.t2 = a == 2 ? 1 : 2;
      P.opidx = mode == 2 ? out_opidx : i;
      P.accum = (mode == 2 && (i > 0 || accum_all)) ? 1 : 0;
      for (int pass = 0; pass <= n_iter; ++pass) {
        P.pass = pass;
        P.last = pass == n_iter;
        P.halo_in = pass > 0 ? halo[(pass - 1) & 1] : nullptr;
        P.halo_out = halo[pass & 1];
        cfd_status s = launch_biased(win, P, T, st, B->dtype);
        if (s != CFD_OK) return s;
      }
    }
  }
  return CFD_OK;
}

cfd_status check_work(cfd_blocks_s *B, int nf, cfd_precision prec, int n_iter, void *work, size_t work_bytes) {
  size_t need = 0;
  cfd_status s = cfd_biased_workspace(B, nf, prec, n_iter, &need);
  if (s != CFD_OK) return s;
  if (need > 0 && (!work || work_bytes < need)) {
    set_error("biased path: workspace too small (see cfd_biased_workspace)");
    return CFD_ERR_ARG;
  }
  return CFD_OK;
}

// Upwind blend of the two biased derivatives of every axis (tensor-core path): one thread per
// interior point of one block, looping over the fields (the shift is read once per point);
// axes added in the order x, y, z, in the field precision (FP32 fields in FP32: GB300's FP64
// pipe, not memory, bounded this kernel when FP32 values were widened to FP64).
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_advect_combine(const T *__restrict__ tmp, const T *__restrict__ beta, T *out,
                                 const int *__restrict__ blocks, const long long *__restrict__ extpre,
                                 const long long *__restrict__ intpre, int N_, int g, int nf, int out_nops,
                                 int out_opidx, int accum_all) {
  const int N = NC ? NC : N_;
  const int n3 = N * N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int b = blocks[blockIdx.y];
  const int x = i % N, y = (i / N) % N, z = i / (N * N);
  const int E = N + 2 * g;
  const long long E3 = (long long)E * E * E;
  const T *bt = beta + 3 * extpre[b] + ((long long)(z + g) * E + (y + g)) * E + (x + g);
  // the shift and, per axis, which biased derivative it takes: beta > 0 the right-biased one
  // (slot 2c+1), beta < 0 the left-biased one (slot 2c), beta = 0 none
  T bv[3];
  int slot[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bv[c] = __ldg(bt + c * E3);
    const int sg = sign_bits(bv[c]);
    slot[c] = 2 * c + (sg == 1 ? 1 : 0);
    if (sg == 0) bv[c] = T(0);  // a zero shift adds nothing (+0 times a finite derivative)
  }
  const T *tp = tmp + (long long)nf * 6 * intpre[b] + i;
  T *o = out + (long long)nf * out_nops * intpre[b] + (long long)out_opidx * n3 + i;
  // fields in groups of QB, every load of a group issued before its first store
  constexpr int QB = 4;
  for (int q0 = 0; q0 < nf; q0 += QB) {
    T dv[QB][3], prev[QB];
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      prev[u] = T(0);
      if (q0 + u < nf) {
        const T *tq = tp + (long long)(q0 + u) * 6 * n3;
#pragma unroll
        for (int c = 0; c < 3; ++c) dv[u][c] = __ldg(tq + (long long)slot[c] * n3);
        if (accum_all) prev[u] = o[(long long)(q0 + u) * out_nops * n3];
      }
    }
    // x, y, z as one FMA chain (three FP64-pipe operations per point and field for FP64 fields)
#pragma unroll
    for (int u = 0; u < QB; ++u) {
      if (q0 + u >= nf) break;
      T acc = accum_all ? fma(bv[0], dv[u][0], prev[u]) : bv[0] * dv[u][0];
      acc = fma(bv[1], dv[u][1], acc);
      acc = fma(bv[2], dv[u][2], acc);
      o[(long long)(q0 + u) * out_nops * n3] = acc;
    }
  }
}

}  // namespace

cfd_status advect_combine(cfd_blocks_s *B, const void *tmp6, const void *beta, int nf, void *out, int out_nops,
                          int out_opidx, bool accum_all, cudaStream_t st) {
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const int N = B->sizes[gi];
    const int n3 = N * N * N;
    dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)B->groups[gi].size());
    launch_begin(KF_BIASED, st);
    auto go = [&](auto tag, auto nc) {
      using T = decltype(tag);
      k_advect_combine<T, decltype(nc)::value><<<grid, 256, 0, st>>>(
          static_cast<const T *>(tmp6), static_cast<const T *>(beta), static_cast<T *>(out), B->d_groups[gi],
          B->d_extpre, B->d_intpre, N, B->ng, nf, out_nops, out_opidx, accum_all);
    };
    auto by_n = [&](auto tag) {
      if (N == 32) go(tag, std::integral_constant<int, 32>());
      else if (N == 16) go(tag, std::integral_constant<int, 16>());
      else go(tag, std::integral_constant<int, 0>());
    };
    if (B->dtype == CFD_F32) by_n(float());
    else by_n(double());
    launch_end(KF_BIASED, st);
    cfd_status s = cuda_fail(cudaGetLastError(), "k_advect_combine launch");
    if (s != CFD_OK) return s;
  }
  return CFD_OK;
}

cfd_status advect_accumulate(cfd_blocks_s *B, const void *fields, int nf, const void *beta, void *out, int out_nops,
                             int out_opidx, cfd_precision prec, int n_iter, void *work, size_t work_bytes,
                             cudaStream_t st) {
  int win;
  cfd_status s = check_request(B, nf, prec, n_iter, &win);
  if (s != CFD_OK) return s;
  if ((s = check_work(B, nf, prec, n_iter, work, work_bytes)) != CFD_OK) return s;
  const int axes[3] = {2, 1, 0};
  if (prec != CFD_FP64_BANDED)
    return dense_biased(B, fields, nf, beta, axes, 3, 2, prec, n_iter, out, out_nops, out_opidx, true, work,
                        work_bytes, st);
  return run_biased(B, fields, nf, beta, axes, 3, 2, n_iter, win, out, work, st, out_nops, out_opidx, true);
}

}  // namespace cfd

using namespace cfd;

extern "C" {

cfd_status cfd_scheme_set_biased(cfd_scheme_t scheme, const cfd_biased_desc *d) {
  if (!scheme || !d || !d->rhs || !d->closure) { set_error("cfd_scheme_set_biased: null argument"); return CFD_ERR_ARG; }
  if (d->rhs_n < 1 || d->closure_n < 1 || d->rhs_lo < -kBOff || d->rhs_lo + d->rhs_n - 1 > kBOff ||
      d->closure_lo < -kBOff || d->closure_lo + d->closure_n - 1 > kBOff) {
    set_error("cfd_scheme_set_biased: stencil offsets outside -6..6");
    return CFD_ERR_ARG;
  }
  if (d->kc < 1 || d->kc > 3 || d->order < 1) { set_error("cfd_scheme_set_biased: kc must be 1..3, order >= 1"); return CFD_ERR_ARG; }
  if (!(std::fabs(d->a) < 1.0) || !(std::fabs(d->a * d->closure_sup) < 1.0)) {
    set_error("cfd_scheme_set_biased: need |a| < 1 and |a closure_sup| < 1");
    return CFD_ERR_ARG;
  }
  BiasedCoef c;
  c.present = true;
  c.order = d->order;
  c.kc = d->kc;
  c.a = d->a;
  c.csup = d->closure_sup;
  c.lo = d->rhs_lo;
  c.hi = d->rhs_lo + d->rhs_n - 1;
  c.clo = d->closure_lo;
  c.chi = d->closure_lo + d->closure_n - 1;
  for (int i = 0; i < d->rhs_n; ++i) {
    if (!std::isfinite(d->rhs[i])) { set_error("cfd_scheme_set_biased: non-finite coefficient"); return CFD_ERR_ARG; }
    c.rhs[d->rhs_lo + i + kBOff] = d->rhs[i];
  }
  for (int i = 0; i < d->closure_n; ++i) {
    if (!std::isfinite(d->closure[i])) { set_error("cfd_scheme_set_biased: non-finite coefficient"); return CFD_ERR_ARG; }
    c.cl[d->closure_lo + i + kBOff] = d->closure[i];
  }
  scheme->biased = c;
  return CFD_OK;
}

cfd_status cfd_biased_workspace(cfd_blocks_t B, int nfields, cfd_precision prec, int n_iter, size_t *bytes) {
  if (!B || nfields < 1 || n_iter < 0 || !bytes) { set_error("cfd_biased_workspace: bad argument"); return CFD_ERR_ARG; }
  if (prec == CFD_TC_BF16_EXACT || prec == CFD_TC_BF16X3) {
    *bytes = dense_biased_workspace(B, nfields, n_iter, true);
    return CFD_OK;
  }
  const size_t he = halo_elems(B, nfields, n_iter);
  *bytes = he ? 2 * align256(he * 8) + 256 : 0;
  return CFD_OK;
}

cfd_status cfd_apply_biased(cfd_blocks_t B, const void *fields, int nfields, unsigned axis_mask, int side,
                            cfd_precision prec, int n_iter, void *out, void *work, size_t work_bytes,
                            void *stream) {
  if (!B || !fields || !out || nfields < 1 || !axis_mask || (axis_mask & ~(CFD_OP_DX | CFD_OP_DY | CFD_OP_DZ)) ||
      (side != 1 && side != -1)) {
    set_error("cfd_apply_biased: bad argument");
    return CFD_ERR_ARG;
  }
  int win;
  cfd_status s = check_request(B, nfields, prec, n_iter, &win);
  if (s != CFD_OK) return s;
  if ((s = check_work(B, nfields, prec, n_iter, work, work_bytes)) != CFD_OK) return s;
  int axes[3], n = 0;
  if (axis_mask & CFD_OP_DX) axes[n++] = 2;
  if (axis_mask & CFD_OP_DY) axes[n++] = 1;
  if (axis_mask & CFD_OP_DZ) axes[n++] = 0;
  if (prec != CFD_FP64_BANDED)
    return dense_biased(B, fields, nfields, nullptr, axes, n, side > 0 ? 0 : 1, prec, n_iter, out, 0, 0, false,
                        work, work_bytes, (cudaStream_t)stream);
  return run_biased(B, fields, nfields, nullptr, axes, n, side > 0 ? 0 : 1, n_iter, win, out, work,
                    (cudaStream_t)stream);
}

cfd_status cfd_advect(cfd_blocks_t B, const void *fields, int nfields, const void *beta, cfd_precision prec,
                      int n_iter, void *out, void *work, size_t work_bytes, void *stream) {
  if (!B || !fields || !beta || !out || nfields < 1) { set_error("cfd_advect: bad argument"); return CFD_ERR_ARG; }
  int win;
  cfd_status s = check_request(B, nfields, prec, n_iter, &win);
  if (s != CFD_OK) return s;
  if ((s = check_work(B, nfields, prec, n_iter, work, work_bytes)) != CFD_OK) return s;
  const int axes[3] = {2, 1, 0};  // x, y, z
  if (prec != CFD_FP64_BANDED)
    return dense_biased(B, fields, nfields, beta, axes, 3, 2, prec, n_iter, out, 1, 0, false, work, work_bytes,
                        (cudaStream_t)stream);
  return run_biased(B, fields, nfields, beta, axes, 3, 2, n_iter, win, out, work, (cudaStream_t)stream);
}

}  // extern "C"
