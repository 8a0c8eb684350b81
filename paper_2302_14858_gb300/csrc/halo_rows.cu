// Halo passes of the hybrid iteration on the CUDA cores, in compensated FP32.
//
// The hybrid iteration (Eq. iter_center_P for the centred schemes, Eq. iter_left_X for the
// biased ones) needs, before each final pass along a decomposed axis, the values every block's
// neighbours read at their k^c nodes: four rows of a block operator (rows 1 and N-2 of [0]D per
// degree, or of the iterated operator with the previous iterate's halo columns) applied to each
// pencil.  That is four dot products of length N + 2g (+ 4) per pencil: not a GEMM, and on
// GB300 the FP64 pipe (1/58 of the FP32 rate) makes plain FP64 dot products as slow as a
// tensor-core pass over the whole pencil.  This kernel computes them in FP32 with error-free
// transformations instead:
//   - the pencil is scaled by a power of two 2^-U (U the largest exponent of its values) and
//     each value is split, with integer instructions only, into an FP32 pair f = f_h + f_l
//     (47 significant bits; values below 2^-100 of the scale, and subnormals, are zero);
//   - each coefficient is an FP32 pair c = c_h + c_l, prepared on the host;
//   - per row, c_h f_h is formed exactly (product and FMA residual) and added with TwoSum into
//     a (sum, error) pair; c_h f_l + c_l f_h and the residuals go into the error word.
// The result carries ~2^-46 relative to sum_j |c_j f_j|, more than the tensor-core digits keep
// (2^-39 of the pencil scale), so the final pass sees the same halo values to its own
// accuracy.  A NaN or an infinity in a pencil makes its four values NaN, as on the tensor-core
// path.  The pencil addressing is the tensor-core stage's own.
#include <cuda_runtime.h>

#include "dense.h"

namespace cfd {

void halo_rows_from(const std::vector<long double> &M, int cols, HaloRows &R) {
  for (int r = 0; r < 4; ++r)
    for (int j = 0; j < 48; ++j) {
      const long double c = j < cols ? M[(size_t)r * cols + j] : 0.0L;
      const float h = (float)c;
      R.h[j][r] = h;
      R.l[j][r] = (float)(c - (long double)h);
    }
}

namespace {

__device__ __forceinline__ long long hr_stride(int axis, long long s0, long long s1) {
  return axis == 0 ? s0 : (axis == 1 ? s1 : 1);
}
__device__ __forceinline__ int hr_dir(int dz, int dy, int dx) {
  const int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
  return r > 13 ? r - 1 : r;
}

// Unbiased exponent of a finite nonzero normal value; kZeroExp for zeros and subnormals,
// kBadExp for NaN and infinities.
constexpr int kZeroExp = -100000, kBadExp = 100000;
__device__ __forceinline__ int hr_exp(double v) {
  const int e = (__double2hiint(v) >> 20) & 0x7FF;
  return e == 0 ? kZeroExp : (e == 0x7FF ? kBadExp : e - 1023);
}
__device__ __forceinline__ int hr_exp(float v) {
  const int e = (__float_as_int(v) >> 23) & 0xFF;
  return e == 0 ? kZeroExp : (e == 0xFF ? kBadExp : e - 127);
}

// v * 2^-U as an FP32 pair (h + l equals it to 2^-47 relative, by truncation), for U at least
// the exponent of v.  h holds the sign, exponent and leading 23 fraction bits; l the next 23
// fraction bits, made a float by placing them under the exponent of 2^(es - 23) and
// subtracting that power of two (exact).
__device__ __forceinline__ void hr_split(double v, int U, float &h, float &l) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int es = e - 1023 - U;  // <= 0
  if (e == 0 || es < -100) { h = 0.f; l = 0.f; return; }
  const unsigned sg = hi & 0x80000000u;
  h = __uint_as_float(sg | ((unsigned)(es + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
  const unsigned eb = (unsigned)(es + 104) << 23;
  const float t = __fsub_rn(__uint_as_float(eb | ((lo >> 6) & 0x7FFFFFu)), __uint_as_float(eb));
  l = __uint_as_float(__float_as_uint(t) | sg);
}
__device__ __forceinline__ void hr_split(float v, int U, float &h, float &l) {
  const unsigned u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xFFu);
  const int es = e - 127 - U;
  l = 0.f;
  if (e == 0 || es < -100) { h = 0.f; return; }
  h = __uint_as_float((u & 0x807FFFFFu) | ((unsigned)(es + 127) << 23));
}

// (sh, sl) += (ch + cl)(fh + fl), dropping cl fl (2^-48 relative).  The rounded intrinsics
// keep the compiler from contracting the TwoSum steps into FMAs.
template <bool LOW>
__device__ __forceinline__ void hr_acc(float &sh, float &sl, float ch, float cl, float fh, float fl) {
  const float p = __fmul_rn(ch, fh);
  const float pe = __fmaf_rn(ch, fh, -p);  // ch fh = p + pe exactly
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // sh + p = s + er
  sh = s;
  const float cross = LOW ? __fmaf_rn(ch, fl, __fmul_rn(cl, fh)) : __fmul_rn(cl, fh);
  sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(er, pe), cross));
}

// An FP32 value as a double, exactly, with integer instructions (zeros and the negligible
// subnormal error words give zero).
__device__ __forceinline__ double hr_f2d(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu)), (int)(u << 29));
}

// (sh + sl) * 2^U: one FP64 add, the scale as an exponent-field add (ldexp where the result
// would leave the normal range).
__device__ __forceinline__ double hr_result(float sh, float sl, int U) {
  const double d = hr_f2d(sh) + hr_f2d(sl);
  const int hi = __double2hiint(d), lo = __double2loint(d);
  const int e = (hi >> 20) & 0x7FF;
  if (e == 0) return d;
  if (e + U >= 1 && e + U <= 2046) return __hiloint2double(hi + (U << 20), lo);
  return ldexp(d, U);
}

// The rows applied to one pencil: element j of the pencil is load(j), j < E, then the four halo
// columns hv; coefficients (h, l) per column from shared memory.  NR = 4: both degrees; NR = 2:
// the degree-1 rows only (rows 2 and 3 are written as zero).
template <typename TI, int NR, typename Load>
__device__ __forceinline__ void hr_rows(Load load, int E, const double (&hv)[4], bool with_halo,
                                        const float4 *ch4, const float4 *cl4, double *o) {
  int U = kZeroExp;
#pragma unroll 4
  for (int j = 0; j < E; ++j) U = max(U, hr_exp(load(j)));
#pragma unroll
  for (int m = 0; m < 4; ++m) U = max(U, hr_exp(hv[m]));
  if (U == kBadExp || U == kZeroExp) {
    const double v = U == kBadExp ? __longlong_as_double(0x7FF8000000000000ll) : 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) o[r] = r < NR ? v : 0.0;
    return;
  }
  float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
  constexpr bool LOW = sizeof(TI) == 8;
#pragma unroll 4
  for (int j = 0; j < E; ++j) {
    float fh, fl;
    hr_split(load(j), U, fh, fl);
    const float4 ch = ch4[j], cl = cl4[j];
    hr_acc<LOW>(sh[0], sl[0], ch.x, cl.x, fh, fl);
    hr_acc<LOW>(sh[1], sl[1], ch.y, cl.y, fh, fl);
    if constexpr (NR == 4) {
      hr_acc<LOW>(sh[2], sl[2], ch.z, cl.z, fh, fl);
      hr_acc<LOW>(sh[3], sl[3], ch.w, cl.w, fh, fl);
    }
  }
  if (with_halo) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float fh, fl;
      hr_split(hv[m], U, fh, fl);
      const float4 ch = ch4[E + m], cl = cl4[E + m];
      hr_acc<true>(sh[0], sl[0], ch.x, cl.x, fh, fl);
      hr_acc<true>(sh[1], sl[1], ch.y, cl.y, fh, fl);
      if constexpr (NR == 4) {
        hr_acc<true>(sh[2], sl[2], ch.z, cl.z, fh, fl);
        hr_acc<true>(sh[3], sl[3], ch.w, cl.w, fh, fl);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) o[r] = r < NR ? hr_result(sh[r], sl[r], U) : 0.0;
}

// One thread per pencil, 128 threads per CTA.  Each warp first stages its 32 pencils in
// shared memory with loads that do not depend on each other (many in flight per thread):
// along y and z a warp's pencils are consecutive x positions, so every element load is
// coalesced as it is; along x every pencil is a contiguous row, and consecutive lanes take
// consecutive elements of the warp's rows.  Then each lane works on its row from there.
constexpr int kHaloThreads = 128;

template <typename TI, int NR>
__global__ void __launch_bounds__(kHaloThreads) k_halo_rows(const __grid_constant__ DenseParams P,
                                                            const __grid_constant__ HaloRows R) {
  extern __shared__ __align__(16) unsigned char hr_smem[];
  __shared__ float4 s_ch[48], s_cl[48];
  for (int i = threadIdx.x; i < 48; i += blockDim.x) {
    s_ch[i] = make_float4(R.h[i][0], R.h[i][1], R.h[i][2], R.h[i][3]);
    s_cl[i] = make_float4(R.l[i][0], R.l[i][1], R.l[i][2], R.l[i][3]);
  }
  const long long np = (long long)P.n1 * P.n2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < np * P.nblk * P.nf;
  const long long job = valid ? t / np : 0;
  const int p = valid ? (int)(t - job * np) : 0;
  const int lb = (int)(job / P.nf), q = (int)(job - (long long)lb * P.nf);
  const int b = P.contig ? P.b0 + lb : P.blocks[lb];
  const int t1 = p / P.n2, t2 = p - t1 * P.n2;
  const int E = P.N + 2 * P.g;
  const long long E3 = (long long)E * E * E;
  const long long is0 = (long long)P.in_dims[1] * P.in_dims[2], is1 = P.in_dims[2];
  const long long s_t1 = hr_stride(P.t1, is0, is1), s_t2 = hr_stride(P.t2, is0, is1),
                  s_ax = hr_stride(P.axis, is0, is1);
  long long ib = !P.in_field ? job * (long long)P.in_box
                 : P.contig  ? (long long)P.nf * P.ext0 + job * E3
                             : (long long)P.nf * P.extpre[b] + (long long)q * E3;
  ib += (long long)(P.in_start[P.t1] + t1) * s_t1 + (long long)(P.in_start[P.t2] + t2) * s_t2;
  const TI *src = static_cast<const TI *>(P.in) + ib;
  TI *tile = reinterpret_cast<TI *>(hr_smem) + (size_t)(threadIdx.x >> 5) * 32 * (E + 1);
  const int lane = threadIdx.x & 31;
  if (P.axis == 2) {
    // element k of the warp's 32 rows: row k / E (exact in FP32: k < 32 E <= 1536), column k % E
    const float invE = 1.0f / (float)E;
#pragma unroll 8
    for (int it = 0; it < E; ++it) {
      const int k = it * 32 + lane;
      const int r = __float2int_rz(((float)k + 0.5f) * invE), c = k - r * E;
      const TI *rs = reinterpret_cast<const TI *>(__shfl_sync(0xffffffffu, (long long)src, r));
      const bool rv = __shfl_sync(0xffffffffu, valid, r);
      if (rv) tile[r * (E + 1) + c] = __ldg(rs + c);
    }
  } else if (valid) {
#pragma unroll 8
    for (int j = 0; j < E; ++j) tile[lane * (E + 1) + j] = __ldg(src + j * s_ax);
  }
  __syncthreads();  // the coefficients (and each warp's rows)
  if (!valid) return;

  // the neighbours' previous iterate (columns E .. E+3: lower neighbour's row N-2, upper
  // neighbour's row 1, per degree)
  double hv[4] = {0.0, 0.0, 0.0, 0.0};
  if (P.halo_in) {
    const int ez = P.axis == 0, ey = P.axis == 1, ex = P.axis == 2;
#pragma unroll
    for (int jq = 0; jq < 2; ++jq) {
      const int nb = P.nbr[b * 26 + hr_dir(jq ? ez : -ez, jq ? ey : -ey, jq ? ex : -ex)];
      const long long hp = ((long long)nb * P.nf + q) * np + p;
#pragma unroll
      for (int d = 0; d < 2; ++d)
        hv[2 * d + jq] = ((P.halo_deg_mask >> d) & 1) ? P.halo_in[hp * 4 + 2 * d + (jq ? 0 : 1)] : 0.0;
    }
  }
  double *o = P.halo_out + (((long long)b * P.nf + q) * np + p) * 4;
  const TI *row = tile + lane * (E + 1);
  hr_rows<TI, NR>([&](int j) { return row[j]; }, E, hv, P.halo_in != nullptr, s_ch, s_cl, o);
}

}  // namespace

cfd_status halo_rows_launch(const DenseParams &P, const HaloRows &R, bool f32_in, cudaStream_t st) {
  const int E = P.N + 2 * P.g;
  if (E + (P.halo_in ? 4 : 0) > 48) {
    set_error("halo rows: more than 48 columns");
    return CFD_ERR_UNSUPPORTED;
  }
  const long long total = (long long)P.n1 * P.n2 * P.nblk * P.nf;
  if (total <= 0) return CFD_OK;
  const unsigned grid = (unsigned)((total + kHaloThreads - 1) / kHaloThreads);
  // pencils staged in shared memory: 4 warps x 32 pencils x (E + 1) values (<= 46 KB)
  const size_t smem = (size_t)(kHaloThreads / 32) * 32 * (E + 1) * (f32_in ? 4 : 8);
  launch_begin(KF_HALO, st);
  // a stage whose final pass reads only the degree-1 halo values (halo_deg_mask 1: the T stages
  // of the mixed derivatives) needs rows 0 and 1 only
  const bool deg1 = P.halo_deg_mask == 1;
  if (f32_in) {
    if (deg1) k_halo_rows<float, 2><<<grid, kHaloThreads, smem, st>>>(P, R);
    else k_halo_rows<float, 4><<<grid, kHaloThreads, smem, st>>>(P, R);
  } else {
    if (deg1) k_halo_rows<double, 2><<<grid, kHaloThreads, smem, st>>>(P, R);
    else k_halo_rows<double, 4><<<grid, kHaloThreads, smem, st>>>(P, R);
  }
  launch_end(KF_HALO, st);
  return cuda_fail(cudaGetLastError(), "k_halo_rows launch");
}

}  // namespace cfd
