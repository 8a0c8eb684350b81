// Host side of the C ABI: scheme construction (closure by C_0 matching),
// MeshBlock binding (operator tables per block size) and launch planning.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "cfd_internal.h"
#include "dense.h"

namespace cfd {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

cfd_status cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return CFD_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return CFD_ERR_CUDA;
}

namespace {

typedef long double ld;

ld fact(int n) {
  ld r = 1;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// Power series helpers in u = eta^2 (centred schemes have even expansions).
std::vector<ld> series_div(const std::vector<ld> &a, const std::vector<ld> &b) {
  std::vector<ld> q(a.size(), 0);
  for (size_t k = 0; k < a.size(); ++k) {
    ld s = a[k];
    for (size_t i = 0; i < k; ++i) s -= q[i] * b[k - i];
    q[k] = s / b[0];
  }
  return q;
}

// Leading error constant C_0 of eps(eta) = eta~^d / eta^d - 1 ~ C_0 eta^order
// for a centred tridiagonal scheme (Eq. fdpwerrdef, Eq. errrelmodwavcent).
//   d = 1:  eta~ / eta = 2 sum_{m>0} a_m sin(m eta) / eta  /  (1 + 2 a cos eta)
//   d = 2:  eta~^2 / eta^2 = -(a_0 + 2 sum_{m>0} a_m cos(m eta)) / eta^2  /  (1 + 2 a cos eta)
ld interior_C0(const SchemeCoef &s) {
  const int K = s.order / 2 + 3;
  std::vector<ld> den(K, 0), num(K + 1, 0);
  for (int k = 0; k < K; ++k) den[k] = ((k % 2) ? -1 : 1) * 2.0L * (ld)s.a / fact(2 * k);
  den[0] += 1;
  const int M = s.M;
  if (s.d == 1) {
    for (int k = 0; k < K; ++k) {
      ld acc = 0;
      for (int m = 1; m <= M; ++m) acc += (ld)s.rhs[M + m] * powl((ld)m, 2 * k + 1);
      num[k] = ((k % 2) ? -1 : 1) * 2.0L * acc / fact(2 * k + 1);
    }
    num.resize(K);
  } else {
    for (int k = 0; k <= K; ++k) {
      ld acc = (k == 0) ? (ld)s.rhs[M] : 0;
      for (int m = 1; m <= M; ++m) acc += 2.0L * (ld)s.rhs[M + m] * powl((ld)m, 2 * k);
      num[k] = -((k % 2) ? -1 : 1) * acc / (k == 0 ? 1 : fact(2 * k));
    }
    // drop the eta^0 term (consistency makes it vanish) and divide by eta^2
    num.erase(num.begin());
  }
  std::vector<ld> r = series_div(num, den);
  return r[s.order / 2];  // coefficient of u^{order/2} = eta^{order}; eps = r - 1
}

bool solve_dense(std::vector<ld> A, std::vector<ld> b, int n, std::vector<ld> &x) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
    if (A[p * n + c] == 0) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[p * n + k], A[c * n + k]);
      std::swap(b[p], b[c]);
    }
    for (int r = c + 1; r < n; ++r) {
      const ld f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  x.assign(n, 0);
  for (int r = n - 1; r >= 0; --r) {
    ld s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
    x[r] = s / A[r * n + r];
  }
  return true;
}

// Explicit centred closure of half-width h = order/2 + 1 (Sec. domdec_drp):
// formal order `order` plus the eta^order error constant equal to the
// interior's C_0.  Unknowns use the (anti)symmetry of centred stencils.
bool build_closure(SchemeCoef &s) {
  const ld C0 = interior_C0(s);
  const int h = s.order / 2 + 1;
  if (h > kMaxH) return false;
  std::vector<ld> A, b, x;
  if (s.d == 1) {
    // unknowns b_1..b_h; alpha-bar_{+-m} = +-b_m
    const int n = h;
    A.assign(n * n, 0);
    b.assign(n, 0);
    int row = 0;
    for (int q = 1; q < s.order; q += 2, ++row) {
      for (int m = 1; m <= h; ++m) A[row * n + (m - 1)] = 2.0L * powl((ld)m, q) / fact(q);
      b[row] = (q == 1) ? 1 : 0;
    }
    const int sg = ((s.order / 2) % 2) ? -1 : 1;
    for (int m = 1; m <= h; ++m) A[row * n + (m - 1)] = sg * 2.0L * powl((ld)m, s.order + 1) / fact(s.order + 1);
    b[row] = C0;
    if (!solve_dense(A, b, n, x)) return false;
    for (int i = 0; i < 2 * kMaxH + 1; ++i) s.clo[i] = 0;
    s.clo[h] = 0.0;
    for (int m = 1; m <= h; ++m) {
      s.clo[h + m] = (double)x[m - 1];
      s.clo[h - m] = -(double)x[m - 1];
    }
  } else {
    // unknowns b_0..b_h; alpha-bar_0 = b_0, alpha-bar_{+-m} = b_m
    const int n = h + 1;
    A.assign(n * n, 0);
    b.assign(n, 0);
    A[0] = 1;
    for (int m = 1; m <= h; ++m) A[m] = 2;
    int row = 1;
    for (int k = 1; k <= s.order / 2 + 1; ++k, ++row) {
      const int sg = (k % 2) ? -1 : 1;
      for (int m = 1; m <= h; ++m) A[row * n + m] = sg * 2.0L * powl((ld)m, 2 * k) / fact(2 * k);
      b[row] = (k == 1) ? -1.0L : (k == s.order / 2 + 1 ? -C0 : 0);
    }
    if (!solve_dense(A, b, n, x)) return false;
    for (int i = 0; i < 2 * kMaxH + 1; ++i) s.clo[i] = 0;
    s.clo[h] = (double)x[0];
    for (int m = 1; m <= h; ++m) s.clo[h + m] = s.clo[h - m] = (double)x[m];
  }
  s.h = h;
  return true;
}

cfd_status copy_desc(const cfd_scheme_desc *d, int deg, SchemeCoef &s) {
  if (!d) return CFD_OK;
  if (d->deriv != deg) { set_error("scheme degree does not match its slot"); return CFD_ERR_ARG; }
  if (d->M < 1 || d->M > kMaxM || !d->rhs) { set_error("interior half-width M out of range"); return CFD_ERR_ARG; }
  if (d->order < 2 || d->order % 2 || d->order > 10) { set_error("order must be even, 2..10"); return CFD_ERR_ARG; }
  if (!(fabs(d->lhs_offdiag) * 2 < 1)) { set_error("system not diagonally dominant (2|a| >= 1)"); return CFD_ERR_ARG; }
  s.present = true;
  s.d = deg;
  s.order = d->order;
  s.M = d->M;
  s.a = d->lhs_offdiag;
  double mx = 0;
  for (int i = 0; i < 2 * d->M + 1; ++i) {
    s.rhs[i] = d->rhs[i];
    mx = std::max(mx, fabs(d->rhs[i]));
  }
  for (int m = 1; m <= d->M; ++m) {
    const double lo = d->rhs[d->M - m], hi = d->rhs[d->M + m];
    const double bad = deg == 1 ? fabs(lo + hi) : fabs(lo - hi);
    if (bad > 1e-14 * mx) { set_error("interior stencil is not centred ((anti)symmetric)"); return CFD_ERR_ARG; }
  }
  if (d->closure) {
    if (d->closure_halfwidth < 1 || d->closure_halfwidth > kMaxH) {
      set_error("closure half-width out of range");
      return CFD_ERR_ARG;
    }
    s.h = d->closure_halfwidth;
    for (int i = 0; i < 2 * s.h + 1; ++i) s.clo[i] = d->closure[i];
  } else if (!build_closure(s)) {
    set_error("closure construction failed");
    return CFD_ERR_ARG;
  }
  return CFD_OK;
}

// Thomas factors of a tridiagonal system with rows (lo_k, 1, up_k), computed
// in FP64 in the textbook order: den_k = 1 - lo_k c_{k-1}, c_k = up_k / den_k.
void thomas_factors(int n, const double *lo, const double *up, double *c, double *inv) {
  double cprev = 0;
  for (int k = 0; k < n; ++k) {
    const double den = 1.0 - lo[k] * cprev;
    c[k] = (k < n - 1) ? up[k] / den : 0.0;
    inv[k] = 1.0 / den;
    cprev = c[k];
  }
}

void build_tables(const SchemeCoef &s, int N, LineTables &T) {
  memset(&T, 0, sizeof(T));
  T.N = N;
  T.M = s.M;
  T.h = s.h;
  T.d = s.d;
  T.a = s.a;
  for (int i = 0; i < 2 * s.M + 1; ++i) T.rhs[i] = s.rhs[i];
  for (int i = 0; i < 2 * s.h + 1; ++i) T.clo[i] = s.clo[i];
  // closed system: unit rows at k = 0 and N-1
  double up[kMaxIter];
  for (int k = 0; k < N; ++k) {
    const bool unit = (k == 0 || k == N - 1);
    T.lo[k] = unit ? 0.0 : s.a;
    up[k] = unit ? 0.0 : s.a;
  }
  thomas_factors(N, T.lo, up, T.c, T.inv);
  // iterated system: rows k = -2..N+1 at k + 2; unit rows at both ends
  const int n = N + 4;
  for (int i = 0; i < n; ++i) {
    const bool unit = (i == 0 || i == n - 1);
    T.ilo[i] = unit ? 0.0 : s.a;
    up[i] = unit ? 0.0 : s.a;
  }
  thomas_factors(n, T.ilo, up, T.ic, T.iinv);
  // cyclic: A = T + u v^T, gamma = -1, u = (gamma, 0.., a), v = (1, 0.., -a)
  //   T_00 = 1 - gamma = 2, T_{N-1,N-1} = 1 + a^2 (rows of T scaled to unit
  //   diagonal for the Thomas factors below).
  {
    double dl[kMaxN], dd[kMaxN], du[kMaxN];
    for (int k = 0; k < N; ++k) {
      dl[k] = (k == 0) ? 0.0 : s.a;
      du[k] = (k == N - 1) ? 0.0 : s.a;
      dd[k] = 1.0;
    }
    dd[0] = 2.0;
    dd[N - 1] = 1.0 + s.a * s.a;
    // general Thomas with diagonal: den_k = dd_k - dl_k c_{k-1}
    double cprev = 0;
    for (int k = 0; k < N; ++k) {
      const double den = dd[k] - dl[k] * cprev;
      T.yc[k] = (k < N - 1) ? du[k] / den : 0.0;
      T.yinv[k] = 1.0 / den;
      T.ylo[k] = dl[k];
      cprev = T.yc[k];
    }
    // z = T^-1 u
    double u[kMaxN] = {};
    u[0] = -1.0;
    u[N - 1] = s.a;
    double y[kMaxN];
    for (int k = 0; k < N; ++k) y[k] = (u[k] - (k ? T.ylo[k] * y[k - 1] : 0.0)) * T.yinv[k];
    for (int k = N - 2; k >= 0; --k) y[k] -= T.yc[k] * y[k + 1];
    for (int k = 0; k < N; ++k) T.z[k] = y[k];
    T.vfac = 1.0 / (1.0 + (T.z[0] - s.a * T.z[N - 1]));
  }
}

int dir_index(int dz, int dy, int dx) {
  int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
  return r > 13 ? r - 1 : r;
}

template <typename T>
cfd_status upload(T **dst, const T *src, size_t n) {
  cfd_status s = cuda_fail(cudaMalloc((void **)dst, n * sizeof(T) + 16), "cudaMalloc");
  if (s != CFD_OK) return s;
  return cuda_fail(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice), "cudaMemcpy");
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct OpList {
  int n = 0;
  int bit[9];
};

OpList ops_of(unsigned mask) {
  OpList o;
  for (int i = 0; i < 9; ++i)
    if (mask & (1u << i)) o.bit[o.n++] = i;
  return o;
}

// box axis index of a letter: x -> 2, y -> 1, z -> 0
const int kAxisOfOp1[3] = {2, 1, 0};                 // dx, dy, dz
const int kMixed[3][2] = {{2, 1}, {2, 0}, {1, 0}};   // (i, j): dxy, dxz, dyz

struct Workspace {
  double *scratch = nullptr;
  double *halo[2] = {nullptr, nullptr};
  size_t scratch_elems = 0, halo_elems = 0;
};

void banded_workspace_sizes(const cfd_blocks_s *B, int nf, unsigned mask, int n_iter, size_t *scratch,
                            size_t *halo) {
  size_t sc = 0, hp = 0;
  const bool mixed = (mask & (CFD_OP_DXY | CFD_OP_DXZ | CFD_OP_DYZ)) != 0;
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const size_t N = B->sizes[gi], E = N + 2 * B->ng;
    if (mixed) sc = std::max(sc, B->groups[gi].size() * nf * E * N * N);
    hp = std::max(hp, E * N);
  }
  *scratch = sc;
  *halo = n_iter > 0 ? (size_t)B->nblocks * nf * hp * 2 : 0;
}

cfd_status run_stage(cfd_blocks_s *B, LineParams P, const LineTables &T, int n_iter, Workspace &ws,
                     cudaStream_t st) {
  for (int pass = 0; pass <= n_iter; ++pass) {
    P.pass = pass;
    P.last = pass == n_iter;
    P.halo_in = pass > 0 ? ws.halo[(pass - 1) & 1] : nullptr;
    P.halo_out = ws.halo[pass & 1];
    cfd_status s = launch_line(P, T, st, B->dtype);
    if (s != CFD_OK) return s;
  }
  return CFD_OK;
}

cfd_status apply_banded(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, int n_iter, void *out,
                        Workspace &ws, cudaStream_t st) {
  const OpList ol = ops_of(mask);
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const int N = B->sizes[gi], g = B->ng, E = N + 2 * g;
    LineParams P;
    memset(&P, 0, sizeof(P));
    P.blocks = B->d_groups[gi];
    P.extpre = B->d_extpre;
    P.intpre = B->d_intpre;
    P.nbr = B->d_nbr;
    P.scale = B->d_scale;
    P.nblk = (int)B->groups[gi].size();
    P.nf = nf;
    P.nops = ol.n;
    P.g = g;
    P.status = B->d_status;
    for (int oi = 0; oi < ol.n; ++oi) {
      const int bit = ol.bit[oi];
      P.opidx = oi;
      if (bit < 6) {
        const int a = kAxisOfOp1[bit % 3];
        const int deg = bit < 3 ? 1 : 2;
        const OpSet &os = B->ops[gi];
        if (!B->s[deg - 1].present) { set_error("op needs a scheme that was not given"); return CFD_ERR_ARG; }
        LineParams Q = P;
        Q.in = fields;
        Q.in_field = 1;
        Q.out = out;
        Q.out_mode = 0;
        Q.axis = a;
        Q.t1 = a == 0 ? 1 : 0;
        Q.t2 = a == 2 ? 1 : 2;
        for (int t = 0; t < 3; ++t) {
          Q.in_dims[t] = E;
          Q.out_dims[t] = N;
          Q.in_start[t] = (t == a) ? 0 : g;
          Q.out_start[t] = 0;
        }
        Q.n1 = N;
        Q.n2 = N;
        Q.deg = deg;
        cfd_status s = run_stage(B, Q, os.tab[deg - 1], n_iter, ws, st);
        if (s != CFD_OK) return s;
      } else {
        if (!B->s[0].present) { set_error("mixed ops need the first-degree scheme"); return CFD_ERR_ARG; }
        const int mi = bit - 6;
        const int norders = B->mixed_one_order ? 1 : 2;  // one order: written directly (out_mode 0)
        for (int order = 0; order < norders; ++order) {
          const int ai = order == 0 ? kMixed[mi][0] : kMixed[mi][1];  // outer (applied last)
          const int aj = order == 0 ? kMixed[mi][1] : kMixed[mi][0];  // inner
          const int ak = 3 - ai - aj;
          // stage 1: D_j on rows extended along i
          LineParams S1 = P;
          S1.in = fields;
          S1.in_field = 1;
          S1.out = ws.scratch;
          S1.out_mode = 2;
          S1.axis = aj;
          S1.t1 = std::min(ai, ak);
          S1.t2 = std::max(ai, ak);
          for (int t = 0; t < 3; ++t) {
            S1.in_dims[t] = E;
            S1.in_start[t] = (t == ak) ? g : 0;
            S1.out_dims[t] = (t == ai) ? E : N;
            S1.out_start[t] = 0;
          }
          S1.n1 = (S1.t1 == ai) ? E : N;
          S1.n2 = (S1.t2 == ai) ? E : N;
          S1.out_box = (unsigned long long)E * N * N;
          S1.deg = 1;
          cfd_status s = run_stage(B, S1, B->ops[gi].tab[0], n_iter, ws, st);
          if (s != CFD_OK) return s;
          // stage 2: D_i on the intermediate
          LineParams S2 = P;
          S2.in = ws.scratch;
          S2.in_field = 0;
          S2.in_box = (unsigned long long)E * N * N;
          S2.out = out;
          S2.out_mode = order == 0 ? 0 : 1;
          S2.axis = ai;
          S2.t1 = std::min(aj, ak);
          S2.t2 = std::max(aj, ak);
          for (int t = 0; t < 3; ++t) {
            S2.in_dims[t] = S1.out_dims[t];
            S2.in_start[t] = 0;
            S2.out_dims[t] = N;
            S2.out_start[t] = 0;
          }
          S2.n1 = N;
          S2.n2 = N;
          S2.deg = 1;
          s = run_stage(B, S2, B->ops[gi].tab[0], n_iter, ws, st);
          if (s != CFD_OK) return s;
        }
      }
    }
  }
  return CFD_OK;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

const char *cfd_last_error(void) { return g_err.c_str(); }

cfd_status cfd_scheme_create(const cfd_scheme_desc *first, const cfd_scheme_desc *second, cfd_scheme_t *out) {
  if (!out || (!first && !second)) { set_error("cfd_scheme_create: null argument"); return CFD_ERR_ARG; }
  cfd_scheme_s *s = new (std::nothrow) cfd_scheme_s();
  if (!s) { set_error("out of host memory"); return CFD_ERR_ALLOC; }
  cfd_status st = copy_desc(first, 1, s->s[0]);
  if (st == CFD_OK) st = copy_desc(second, 2, s->s[1]);
  if (st != CFD_OK) { delete s; return st; }
  *out = s;
  return CFD_OK;
}

cfd_status cfd_scheme_closure(cfd_scheme_t scheme, int deriv, double *closure, int *halfwidth) {
  if (!scheme || (deriv != 1 && deriv != 2) || !closure || !halfwidth) {
    set_error("cfd_scheme_closure: bad argument");
    return CFD_ERR_ARG;
  }
  const SchemeCoef &s = scheme->s[deriv - 1];
  if (!s.present) { set_error("cfd_scheme_closure: degree not present"); return CFD_ERR_ARG; }
  *halfwidth = s.h;
  for (int i = 0; i < 2 * s.h + 1; ++i) closure[i] = s.clo[i];
  return CFD_OK;
}

void cfd_scheme_destroy(cfd_scheme_t scheme) { delete scheme; }

void cfd_blocks_destroy(cfd_blocks_t B) {
  if (!B) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(B->device);
  cudaFree(B->d_nbr);
  cudaFree(B->d_extpre);
  cudaFree(B->d_exch);
  cudaFree(B->d_intpre);
  cudaFree(B->d_scale);
  cudaFree(B->d_nvec);
  cudaFree(B->d_status);
  for (int *p : B->d_groups) cudaFree(p);
  for (void *p : B->d_dense_ptrs) cudaFree(p);
  if (B->dense_state && B->dense_free) B->dense_free(B->dense_state);
  cudaSetDevice(prev);
  delete B;
}

cfd_status cfd_blocks_bind(cfd_scheme_t scheme, int nblocks, const int *block_n, const double *dx,
                           const int *neighbors, int ng, cfd_dtype dtype, cfd_blocks_t *out) {
  if (!scheme || nblocks < 1 || !block_n || !dx || !neighbors || !out) {
    set_error("cfd_blocks_bind: null or empty argument");
    return CFD_ERR_ARG;
  }
  if (dtype != CFD_F64 && dtype != CFD_F32) { set_error("cfd_blocks_bind: dtype"); return CFD_ERR_ARG; }
  int need = 0;
  for (int d = 0; d < 2; ++d) {
    const SchemeCoef &s = scheme->s[d];
    if (s.present) need = std::max(need, std::max(s.h, s.M + 1));
  }
  if (ng < need || ng > 8) { set_error("cfd_blocks_bind: ghost width too small for the stencils (or > 8)"); return CFD_ERR_ARG; }
  cfd_blocks_s *B = new (std::nothrow) cfd_blocks_s();
  if (!B) { set_error("out of host memory"); return CFD_ERR_ALLOC; }
  B->s[0] = scheme->s[0];
  B->s[1] = scheme->s[1];
  B->biased = scheme->biased;
  cudaGetDevice(&B->device);
  if (cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess) B->num_sms = 0;
  B->nblocks = nblocks;
  B->ng = ng;
  B->dtype = dtype;
  B->n.assign(block_n, block_n + nblocks);
  B->nbr.assign(neighbors, neighbors + (size_t)nblocks * 26);
  B->dx.assign(dx, dx + (size_t)nblocks * 3);
  auto fail = [&](cfd_status s, const char *msg) {
    if (msg) set_error(msg);
    cfd_blocks_destroy(B);
    return s;
  };
  for (int b = 0; b < nblocks; ++b) {
    const int N = B->n[b];
    if (N != 8 && N != 16 && N != 32) return fail(CFD_ERR_UNSUPPORTED, "cfd_blocks_bind: block size must be 8, 16 or 32");
    if (N < ng) return fail(CFD_ERR_ARG, "cfd_blocks_bind: N < ng");
    for (int a = 0; a < 3; ++a)
      if (!(B->dx[b * 3 + a] > 0)) return fail(CFD_ERR_ARG, "cfd_blocks_bind: dx must be positive");
    for (int r = 0; r < 26; ++r) {
      const int nb = B->nbr[b * 26 + r];
      if (nb < -1 || nb >= nblocks) return fail(CFD_ERR_ARG, "cfd_blocks_bind: neighbour index out of range");
      if (nb >= 0 && B->n[nb] != N) return fail(CFD_ERR_ARG, "cfd_blocks_bind: neighbour of another size (pass -1)");
    }
    // iteration needs face neighbours along every axis that is not cyclic
    for (int a = 0; a < 3; ++a) {
      const int dz = a == 0, dy = a == 1, dxx = a == 2;
      const int lo = B->nbr[b * 26 + dir_index(-dz, -dy, -dxx)], hi = B->nbr[b * 26 + dir_index(dz, dy, dxx)];
      if (lo == b && hi == b) continue;
      if (lo < 0 || hi < 0 || lo == b || hi == b) B->iter_ok = false;
    }
  }
  // prefix offsets
  B->extpre.resize(nblocks);
  B->intpre.resize(nblocks);
  long long e = 0, i = 0;
  for (int b = 0; b < nblocks; ++b) {
    B->extpre[b] = e;
    B->intpre[b] = i;
    const long long N = B->n[b], E = N + 2 * ng;
    e += E * E * E;
    i += N * N * N;
  }
  // groups by size
  std::map<int, std::vector<int>> gm;
  for (int b = 0; b < nblocks; ++b) gm[B->n[b]].push_back(b);
  for (auto &kv : gm) {
    B->sizes.push_back(kv.first);
    B->groups.push_back(kv.second);
    OpSet os;
    memset(&os, 0, sizeof(os));
    os.N = kv.first;
    for (int d = 0; d < 2; ++d)
      if (B->s[d].present) build_tables(B->s[d], kv.first, os.tab[d]);
    B->ops.push_back(os);
    if (B->biased.present) {
      BiasedTables bt;
      build_biased_tables(B->biased, kv.first, ng, bt);
      B->btab.push_back(bt);
    }
  }
  // per-block scale 1/dx^d, [b][deg][axis x,y,z]
  std::vector<double> scale((size_t)nblocks * 6);
  for (int b = 0; b < nblocks; ++b)
    for (int a = 0; a < 3; ++a) {
      const double h = B->dx[b * 3 + a];
      scale[(b * 2 + 0) * 3 + a] = 1.0 / h;
      scale[(b * 2 + 1) * 3 + a] = 1.0 / (h * h);
    }
  cfd_status s;
  if ((s = upload(&B->d_nbr, B->nbr.data(), B->nbr.size())) != CFD_OK) return fail(s, nullptr);
  if ((s = upload(&B->d_extpre, B->extpre.data(), B->extpre.size())) != CFD_OK) return fail(s, nullptr);
  if ((s = upload(&B->d_intpre, B->intpre.data(), B->intpre.size())) != CFD_OK) return fail(s, nullptr);
  if ((s = upload(&B->d_scale, scale.data(), scale.size())) != CFD_OK) return fail(s, nullptr);
  if ((s = upload(&B->d_nvec, B->n.data(), B->n.size())) != CFD_OK) return fail(s, nullptr);
  for (auto &grp : B->groups) {
    int *p = nullptr;
    if ((s = upload(&p, grp.data(), grp.size())) != CFD_OK) return fail(s, nullptr);
    B->d_groups.push_back(p);
    bool consecutive = true;
    for (size_t k = 0; k < grp.size(); ++k)
      if (grp[k] != grp[0] + (int)k) consecutive = false;
    B->group_b0.push_back(consecutive ? grp[0] : -1);
  }
  {
    std::vector<long long> exch((size_t)nblocks * 27);
    for (int b = 0; b < nblocks; ++b) {
      for (int d = 0; d < 26; ++d) {
        const int nb = B->nbr[(size_t)b * 26 + d];
        exch[(size_t)b * 27 + d] = nb >= 0 ? B->extpre[nb] : -1;
      }
      exch[(size_t)b * 27 + 26] = B->extpre[b];
    }
    if ((s = upload(&B->d_exch, exch.data(), exch.size())) != CFD_OK) return fail(s, nullptr);
  }
  if ((s = cuda_fail(cudaMalloc((void **)&B->d_status, sizeof(int)), "cudaMalloc")) != CFD_OK) return fail(s, nullptr);
  if ((s = cuda_fail(cudaMemset(B->d_status, 0, sizeof(int)), "cudaMemset")) != CFD_OK) return fail(s, nullptr);
  if ((s = dense_bind(B)) != CFD_OK) return fail(s, nullptr);
  *out = B;
  return CFD_OK;
}

cfd_status cfd_exchange_ghosts(cfd_blocks_t B, void *fields, int nfields, void *stream) {
  if (!B || !fields || nfields < 1) { set_error("cfd_exchange_ghosts: bad argument"); return CFD_ERR_ARG; }
  return launch_exchange(B, fields, nfields, (cudaStream_t)stream);
}

cfd_status cfd_apply_workspace(cfd_blocks_t B, int nfields, unsigned op_mask, cfd_precision prec, int n_iter,
                               size_t *bytes) {
  if (!B || nfields < 1 || !bytes || (op_mask & ~CFD_OP_ALL) || !op_mask || n_iter < 0) {
    set_error("cfd_apply_workspace: bad argument");
    return CFD_ERR_ARG;
  }
  if (prec == CFD_FP64_BANDED) {
    size_t sc, ha;
    banded_workspace_sizes(B, nfields, op_mask, n_iter, &sc, &ha);
    *bytes = align256(sc * 8) + 2 * align256(ha * 8) + 256;
    return CFD_OK;
  }
  return dense_workspace(B, nfields, op_mask, prec, n_iter, bytes);
}

cfd_status cfd_apply(cfd_blocks_t B, const void *fields, int nfields, unsigned op_mask, cfd_precision prec,
                     int n_iter, void *out, void *work, size_t work_bytes, void *stream) {
  if (!B || !fields || !out || nfields < 1 || !op_mask || (op_mask & ~CFD_OP_ALL) || n_iter < 0 || n_iter > 64) {
    set_error("cfd_apply: bad argument");
    return CFD_ERR_ARG;
  }
  if (n_iter > 0 && !B->iter_ok) {
    set_error("cfd_apply: hybrid iteration needs same-size face neighbours on every decomposed axis");
    return CFD_ERR_UNSUPPORTED;
  }
  for (auto &grp : B->groups)
    if ((long long)grp.size() * nfields > 65535) {
      set_error("cfd_apply: blocks of one size x nfields exceeds 65535");
      return CFD_ERR_UNSUPPORTED;
    }
  size_t need = 0;
  cfd_status s = cfd_apply_workspace(B, nfields, op_mask, prec, n_iter, &need);
  if (s != CFD_OK) return s;
  if (need > 256 && (!work || work_bytes < need)) {
    set_error("cfd_apply: workspace too small (see cfd_apply_workspace)");
    return CFD_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CFD_FP64_BANDED) {
    size_t sc, ha;
    banded_workspace_sizes(B, nfields, op_mask, n_iter, &sc, &ha);
    Workspace ws;
    char *base = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
    ws.scratch = sc ? (double *)base : nullptr;
    base += align256(sc * 8);
    ws.halo[0] = ha ? (double *)base : nullptr;
    base += align256(ha * 8);
    ws.halo[1] = ha ? (double *)base : nullptr;
    return apply_banded(B, fields, nfields, op_mask, n_iter, out, ws, st);
  }
  return dense_apply(B, fields, nfields, op_mask, prec, n_iter, out, work, work_bytes, st);
}

cfd_status cfd_autotune(cfd_blocks_t B, const void *fields, int nfields, unsigned op_mask, cfd_precision prec,
                        int n_iter, void *out, void *work, size_t work_bytes, void *stream) {
  if (!B || prec == CFD_FP64_BANDED) {
    set_error("cfd_autotune: a blocks handle and a tensor-core precision are needed");
    return CFD_ERR_ARG;
  }
  dense_set_tuning(B, true);
  const cfd_status s = cfd_apply(B, fields, nfields, op_mask, prec, n_iter, out, work, work_bytes, stream);
  dense_set_tuning(B, false);
  return s;
}

cfd_status cfd_autotune_report(cfd_blocks_t B, char *buf, size_t len, size_t *needed) {
  if (!B || (!buf && len) || !needed) { set_error("cfd_autotune_report: bad argument"); return CFD_ERR_ARG; }
  const std::string r = dense_tuning_report(B);
  *needed = r.size() + 1;
  if (buf && len) {
    const size_t n = std::min(len - 1, r.size());
    memcpy(buf, r.data(), n);
    buf[n] = 0;
  }
  return CFD_OK;
}

cfd_status cfd_blocks_set_mixed_order(cfd_blocks_t B, int one_order) {
  if (!B || (one_order != 0 && one_order != 1)) {
    set_error("cfd_blocks_set_mixed_order: bad argument");
    return CFD_ERR_ARG;
  }
  if (one_order && !B->iter_ok) {
    set_error("cfd_blocks_set_mixed_order: one order needs same-size face neighbours on every decomposed axis");
    return CFD_ERR_UNSUPPORTED;
  }
  B->mixed_one_order = one_order != 0;
  return CFD_OK;
}

cfd_status cfd_sync_status(cfd_blocks_t B, void *stream) {
  if (!B) { set_error("cfd_sync_status: null handle"); return CFD_ERR_ARG; }
  cfd_status s = cuda_fail(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  if (s != CFD_OK) return s;
  int v = 0;
  s = cuda_fail(cudaMemcpy(&v, B->d_status, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy status");
  if (s != CFD_OK) return s;
  if (v == 0) return CFD_OK;
  cudaMemset(B->d_status, 0, sizeof(int));
  set_error(v == CFD_ERR_TIMEOUT ? "device: bounded wait ran out" : "device: self-check failed");
  return v == CFD_ERR_TIMEOUT ? CFD_ERR_TIMEOUT : CFD_ERR_DEVICE_ASSERT;
}

}  // extern "C"

// Internal hooks for the allocation-free entry point (static_scratch.cu):
// the FP64 banded apply with closures only, running on a caller-provided
// scratch region instead of the workspace argument.
namespace cfd {

size_t banded_closed_scratch_bytes(const cfd_blocks_s *B, int nf, unsigned mask) {
  size_t sc = 0, ha = 0;
  banded_workspace_sizes(B, nf, mask, 0, &sc, &ha);
  return sc * sizeof(double);
}

cfd_status apply_banded_closed(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, void *out,
                               double *scratch, cudaStream_t st) {
  Workspace ws;
  ws.scratch = scratch;
  return apply_banded(B, fields, nf, mask, 0, out, ws, st);
}

}  // namespace cfd
