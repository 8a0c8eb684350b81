// FP64 banded path: ghost exchange (matrix G, Eq. example_G) and the per-pencil
// closed / iterated / cyclic tridiagonal solves (Eqs. sch_cent_om, iter_center_P).
//
// One thread owns one pencil.  The right-hand side of row k is the FMA chain
// sum_m c_m f_{k+m} over m = -M..M (or the closure's -h..h) in increasing m,
// then scaled by dx^{-d}; the solve uses the precomputed Thomas factors of the
// block system (identical for every pencil of a block size).
#include <type_traits>

#include "cfd_internal.h"

namespace cfd {

namespace {

__device__ __forceinline__ int dir_index(int dz, int dy, int dx) {
  int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
  return r > 13 ? r - 1 : r;
}

template <typename T>
__device__ __forceinline__ double ldg_d(const T *p) { return static_cast<double>(__ldg(p)); }

// ---------------------------------------------------------------- ghost exchange

template <typename T, int V> struct VecOf { using type = T; };
template <> struct VecOf<double, 2> { using type = double2; };
template <> struct VecOf<float, 4> { using type = float4; };

// One thread per kVPT groups of V consecutive ghost cells along x (V values = 16 bytes where
// the ghost width, N and the rows keep 16-byte alignment; V = 1 otherwise), enumerated without
// idle threads: part A covers the rows (fixed z, y) that lie in the ghost shell along y or z
// (all of x), part B the x ghosts of the N^2 interior rows.  Consecutive threads take
// consecutive x, so destination rows and source segments are contiguous.  The field offsets
// of the block and its 26 neighbours come from one table (one load each, independent of the
// data), and each thread issues its kVPT copies together, so the copies, not a chain of
// dependent table loads, set the pace.  The common (N, g) pairs are compiled with constant
// sizes (divisions become multiply-shifts); NC = 0 takes them at run time.
constexpr int kVPT = 4;

template <typename T, int NC, int GC, int V>
__global__ void __launch_bounds__(256) k_exchange(T *f, int nf, const int *__restrict__ blocks, int b0, int N_,
                                                  int g_, const long long *__restrict__ tab) {
  using VT = typename VecOf<T, V>::type;
  const int N = NC ? NC : N_, g = NC ? GC : g_;
  const int E = N + 2 * g, Ev = E / V, gv = g / V, Nv = N / V, G2v = 2 * gv;
  const int nA = (E * E - N * N) * Ev, nB = N * N * G2v;
  const int job = blockIdx.y;
  const int lb = job / nf, q = job - lb * nf;
  const int b = b0 >= 0 ? b0 + lb : blocks[lb];
  const long long *tb = tab + (long long)b * 27;
  const long long cells = (long long)E * E * E;
  T *base = f + nf * tb[26] + q * cells;
  int dst[kVPT], src[kVPT];
  long long nbo[kVPT];
#pragma unroll
  for (int u = 0; u < kVPT; ++u) {
    const int idx = (blockIdx.x * kVPT + u) * blockDim.x + threadIdx.x;
    nbo[u] = -1;
    dst[u] = src[u] = 0;
    if (idx >= nA + nB) continue;
    int x, y, z;
    if (idx < nA) {
      const int r = idx / Ev;
      x = (idx - r * Ev) * V;
      const int G2 = 2 * g;
      if (r < G2 * E) {              // z in the ghost shell: whole planes
        const int zz = r / E;
        y = r - zz * E;
        z = zz < g ? zz : zz + N;
      } else {                       // z interior, y in the ghost shell
        const int r2 = r - G2 * E, zz = r2 / G2, yy = r2 - zz * G2;
        z = g + zz;
        y = yy < g ? yy : yy + N;
      }
    } else {                         // interior row, x ghosts
      const int r = idx - nA, row = r / G2v, xx = r - row * G2v, zz = row / N;
      x = (xx < gv ? xx : xx + Nv) * V;
      y = g + row - zz * N;
      z = g + zz;
    }
    const int dx = x < g ? -1 : (x >= N + g ? 1 : 0);
    const int dy = y < g ? -1 : (y >= N + g ? 1 : 0);
    const int dz = z < g ? -1 : (z >= N + g ? 1 : 0);
    nbo[u] = __ldg(tb + dir_index(dz, dy, dx));
    dst[u] = (z * E + y) * E + x;
    src[u] = dst[u] - ((dz * E + dy) * E + dx) * N;
  }
  VT v[kVPT];
#pragma unroll
  for (int u = 0; u < kVPT; ++u)
    if (nbo[u] >= 0) v[u] = *reinterpret_cast<const VT *>(f + nf * nbo[u] + q * cells + src[u]);
#pragma unroll
  for (int u = 0; u < kVPT; ++u)
    if (nbo[u] >= 0) *reinterpret_cast<VT *>(base + dst[u]) = v[u];
}

// ---------------------------------------------------------------- pencil solves

// Window of the pencil kept in registers: ghost-extended indices g-W .. g+N+W-1.
template <int NT, int MT, int HT>
struct Shape {
  static constexpr int W = (HT > MT + 1 ? HT : MT + 1);
  static constexpr int L = NT + 2 * W;
};

template <int NT, int MT, int HT, typename TI, typename TO>
__global__ void __launch_bounds__(128) k_line(const LineParams P, const LineTables T) {
  constexpr int W = Shape<NT, MT, HT>::W;
  constexpr int L = Shape<NT, MT, HT>::L;
  const int np = P.n1 * P.n2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int job = blockIdx.y;
  const int lb = job / P.nf, q = job - lb * P.nf;
  const int b = P.blocks[lb];
  const int t1 = p / P.n2, t2 = p - t1 * P.n2;
  const int g = P.g;

  // axis <-> neighbour directions (box axis 0 = z, 1 = y, 2 = x)
  const int ez = P.axis == 0, ey = P.axis == 1, ex = P.axis == 2;
  const int nlo = P.nbr[b * 26 + dir_index(-ez, -ey, -ex)];
  const int nhi = P.nbr[b * 26 + dir_index(ez, ey, ex)];
  const bool cyclic = (nlo == b && nhi == b);
  if (cyclic && P.pass > 0) return;  // finished in pass 0
  const bool last = cyclic ? true : P.last;

  // ---- input pencil
  const long long is0 = (long long)P.in_dims[1] * P.in_dims[2], is1 = P.in_dims[2];
  const long long istr[3] = {is0, is1, 1};
  long long ib;
  if (P.in_field) {
    const long long E = NT + 2 * g;
    ib = (long long)P.nf * P.extpre[b] + (long long)q * E * E * E;
  } else {
    ib = ((long long)lb * P.nf + q) * (long long)P.in_box;
  }
  ib += (long long)(P.in_start[P.t1] + t1) * istr[P.t1] + (long long)(P.in_start[P.t2] + t2) * istr[P.t2];
  const long long sa = istr[P.axis];
  const TI *fin = static_cast<const TI *>(P.in) + ib + (long long)(g - W) * sa;

  double fv[L];
#pragma unroll
  for (int j = 0; j < L; ++j) fv[j] = ldg_d(fin + (long long)j * sa);

  const double scale = P.scale[(b * 2 + (P.deg - 1)) * 3 + (2 - P.axis)];

  double x[NT + 4];  // x[k] holds interior k after the solve
  if (cyclic) {
    // all rows interior (periodic), Sherman-Morrison on the corner-modified T
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      double acc = T.rhs[0] * fv[k - MT + W];
#pragma unroll
      for (int i = 1; i <= 2 * MT; ++i) acc = fma(T.rhs[i], fv[k + i - MT + W], acc);
      const double r = acc * scale;
      x[k] = (k == 0) ? r * T.yinv[0] : fma(-T.ylo[k], x[k - 1], r) * T.yinv[k];
    }
#pragma unroll
    for (int k = NT - 2; k >= 0; --k) x[k] = fma(-T.yc[k], x[k + 1], x[k]);
    const double s = fma(-T.a, x[NT - 1], x[0]) * T.vfac;
#pragma unroll
    for (int k = 0; k < NT; ++k) x[k] = fma(-s, T.z[k], x[k]);
  } else if (P.pass == 0) {
    // closed system: closure rows 0 and N-1, interior rows between
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      double acc;
      if (k == 0 || k == NT - 1) {
        acc = T.clo[0] * fv[k - HT + W];
#pragma unroll
        for (int i = 1; i <= 2 * HT; ++i) acc = fma(T.clo[i], fv[k + i - HT + W], acc);
      } else {
        acc = T.rhs[0] * fv[k - MT + W];
#pragma unroll
        for (int i = 1; i <= 2 * MT; ++i) acc = fma(T.rhs[i], fv[k + i - MT + W], acc);
      }
      const double r = acc * scale;
      x[k] = (k == 0) ? r * T.inv[0] : fma(-T.lo[k], x[k - 1], r) * T.inv[k];
    }
#pragma unroll
    for (int k = NT - 2; k >= 0; --k) x[k] = fma(-T.c[k], x[k + 1], x[k]);
  } else {
    // iterated system: rows k = -2 .. N+1 at index k + 2; ends fixed by neighbours
    const long long hp = (long long)np * 2;
    const double dlo = P.halo_in[((long long)nlo * P.nf + q) * hp + 2 * p + 1];
    const double dhi = P.halo_in[((long long)nhi * P.nf + q) * hp + 2 * p + 0];
    x[0] = dlo;
#pragma unroll
    for (int i = 1; i <= NT + 2; ++i) {
      const int k = i - 2;
      double acc = T.rhs[0] * fv[k - MT + W];
#pragma unroll
      for (int m = 1; m <= 2 * MT; ++m) acc = fma(T.rhs[m], fv[k + m - MT + W], acc);
      const double r = acc * scale;
      x[i] = fma(-T.ilo[i], x[i - 1], r) * T.iinv[i];
    }
    x[NT + 3] = fma(-T.ilo[NT + 3], x[NT + 2], dhi) * T.iinv[NT + 3];
#pragma unroll
    for (int i = NT + 2; i >= 2; --i) x[i] = fma(-T.ic[i], x[i + 1], x[i]);
    // keep the interior rows k = 0..N-1 (stored at k + 2)
#pragma unroll
    for (int k = 0; k < NT; ++k) x[k] = x[k + 2];
  }

  if (!last) {
    const long long hp = (long long)np * 2;
    double *h = P.halo_out + ((long long)b * P.nf + q) * hp + 2 * p;
    h[0] = x[1];
    h[1] = x[NT - 2];
    return;
  }

  // ---- output
  const long long os0 = (long long)P.out_dims[1] * P.out_dims[2], os1 = P.out_dims[2];
  const long long ostr[3] = {os0, os1, 1};
  long long ob;
  if (P.out_mode <= 1) {
    const long long n3 = (long long)NT * NT * NT;
    ob = (long long)P.nf * P.nops * P.intpre[b] + ((long long)q * P.nops + P.opidx) * n3;
  } else {
    ob = ((long long)lb * P.nf + q) * (long long)P.out_box;
  }
  ob += (long long)(P.out_start[P.t1] + t1) * ostr[P.t1] + (long long)(P.out_start[P.t2] + t2) * ostr[P.t2];
  const long long oa = ostr[P.axis];
  if (P.out_mode == 0) {
    TO *o = static_cast<TO *>(P.out) + ob + (long long)P.out_start[P.axis] * oa;
#pragma unroll
    for (int k = 0; k < NT; ++k) o[(long long)k * oa] = static_cast<TO>(x[k]);
  } else if (P.out_mode == 1) {
    TO *o = static_cast<TO *>(P.out) + ob + (long long)P.out_start[P.axis] * oa;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const long long ix = (long long)k * oa;
      o[ix] = static_cast<TO>((static_cast<double>(o[ix]) + x[k]) * 0.5);
    }
  } else {
    double *o = static_cast<double *>(P.out) + ob + (long long)P.out_start[P.axis] * oa;
#pragma unroll
    for (int k = 0; k < NT; ++k) o[(long long)k * oa] = x[k];
  }
}

template <int NT, int MT, int HT>
cfd_status dispatch_types(const LineParams &P, const LineTables &T, cudaStream_t st, cfd_dtype dt) {
  const int np = P.n1 * P.n2;
  dim3 grid((np + 127) / 128, P.nblk * P.nf);
  const bool in_f32 = P.in_field && dt == CFD_F32;
  const bool out_f32 = P.out_mode <= 1 && dt == CFD_F32;
  launch_begin(KF_LINE, st);
  if (in_f32 && out_f32) k_line<NT, MT, HT, float, float><<<grid, 128, 0, st>>>(P, T);
  else if (in_f32) k_line<NT, MT, HT, float, double><<<grid, 128, 0, st>>>(P, T);
  else if (out_f32) k_line<NT, MT, HT, double, float><<<grid, 128, 0, st>>>(P, T);
  else k_line<NT, MT, HT, double, double><<<grid, 128, 0, st>>>(P, T);
  launch_end(KF_LINE, st);
  return cuda_fail(cudaGetLastError(), "k_line launch");
}

template <int NT>
cfd_status dispatch_widths(const LineParams &P, const LineTables &T, cudaStream_t st, cfd_dtype dt) {
  if (T.M == 3 && T.h == 4) return dispatch_types<NT, 3, 4>(P, T, st, dt);
  if (T.M == 2 && T.h == 4) return dispatch_types<NT, 2, 4>(P, T, st, dt);
  if (T.M == 1 && T.h == 3) return dispatch_types<NT, 1, 3>(P, T, st, dt);
  if (T.M == 3 && T.h == 5) return dispatch_types<NT, 3, 5>(P, T, st, dt);
  set_error("banded path: unsupported stencil widths (M, closure half-width)");
  return CFD_ERR_UNSUPPORTED;
}

}  // namespace

cfd_status launch_line(const LineParams &P, const LineTables &T, cudaStream_t st, cfd_dtype dt) {
  if (P.g < (T.h > T.M + 1 ? T.h : T.M + 1)) {
    set_error("ghost width too small for the stencil");
    return CFD_ERR_ARG;
  }
  switch (T.N) {
    case 8: return dispatch_widths<8>(P, T, st, dt);
    case 16: return dispatch_widths<16>(P, T, st, dt);
    case 32: return dispatch_widths<32>(P, T, st, dt);
    default:
      set_error("banded path: block size must be 8, 16 or 32");
      return CFD_ERR_UNSUPPORTED;
  }
}

cfd_status launch_exchange(cfd_blocks_s *B, void *fields, int nf, cudaStream_t st) {
  for (auto &grp : B->groups)
    if ((long long)grp.size() * nf > 65535) {  // (block, field) pairs of one size go in gridDim.y
      set_error("ghost exchange: blocks of one size x nfields exceeds 65535");
      return CFD_ERR_UNSUPPORTED;
    }
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const int N = B->sizes[gi];
    const int nblk = (int)B->groups[gi].size();
    const long long E = N + 2 * B->ng;
    const long long ghosts = E * E * E - (long long)N * N * N;
    const int g = B->ng;
    launch_begin(KF_EXCHANGE, st);
    auto go = [&](auto tag, auto nc, auto gc, auto vc) {
      using T = decltype(tag);
      constexpr int V = decltype(vc)::value;
      dim3 grid((unsigned)((ghosts / V + 256 * kVPT - 1) / (256 * kVPT)), nblk * nf);
      k_exchange<T, decltype(nc)::value, decltype(gc)::value, V><<<grid, 256, 0, st>>>(
          static_cast<T *>(fields), nf, B->d_groups[gi], B->group_b0[gi], N, g, B->d_exch);
    };
    auto by_size = [&](auto tag, auto vc) {
      using I = std::integral_constant<int, 0>;
      if (g == 4 && N == 16) go(tag, std::integral_constant<int, 16>(), std::integral_constant<int, 4>(), vc);
      else if (g == 4 && N == 32) go(tag, std::integral_constant<int, 32>(), std::integral_constant<int, 4>(), vc);
      else if (g == 4 && N == 8) go(tag, std::integral_constant<int, 8>(), std::integral_constant<int, 4>(), vc);
      else go(tag, I(), I(), vc);
    };
    // 16-byte copies need g, N (hence E) multiples of the vector width and an aligned buffer
    const bool al16 = ((uintptr_t)fields & 15) == 0;
    if (B->dtype == CFD_F64) {
      if (al16 && g % 2 == 0) by_size(double(), std::integral_constant<int, 2>());
      else by_size(double(), std::integral_constant<int, 1>());
    } else {
      if (al16 && g % 4 == 0 && N % 4 == 0) by_size(float(), std::integral_constant<int, 4>());
      else by_size(float(), std::integral_constant<int, 1>());
    }
    launch_end(KF_EXCHANGE, st);
    cfd_status s = cuda_fail(cudaGetLastError(), "k_exchange launch");
    if (s != CFD_OK) return s;
  }
  return CFD_OK;
}

}  // namespace cfd
