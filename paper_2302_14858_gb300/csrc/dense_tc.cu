// Dense per-block operator on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// For every block size N and axis, the closed block system of Eq. sch_cent_om
// is inverted once at bind time: D = A^-1 B dx^-d, an N x (N + 2g) matrix
// ([0]D of Eq. iter_scheme restricted to the interior rows).  Applying it to
// all pencils of a block is a dense contraction
//     out[p, i] = sum_j f[p, j] D[i, j]      (p: pencil, j: ghost-extended index)
// run as a GEMM with M = 128 pencils per tile, N = output rows, K = N + 2g.
//
// Precision ("exact integer slices").  D row i is scaled by a power of two
// sigma_i >= max_j |D_ij| and written as 5 signed 8-bit digits
//     D_ij / sigma_i = sum_t b_t 2^{-7-8t},  |b_t| <= 128,
// each exact in BF16; every pencil p gets a power-of-two scale tau_p and the
// same 5-digit split a_s of its values (done in the kernel from the IEEE bits).
// A BF16 x BF16 product of digits is an integer below 2^14, a K <= 48 sum is
// below 2^20, and the pairs (s, t) of one level k = s + t (at most 5 of them)
// are accumulated in the same FP32 TMEM columns, staying below 2^22: every
// accumulator is an exact integer.  Levels k <= L are kept; the epilogue forms
// Y = sum_k acc_k 2^{8(L-k)} as a 64-bit integer and writes
//     out = Y * 2^{e(sigma_i) + e(tau_p) - 14 - 8L}
// by assembling the IEEE bits with integer instructions (no FP64 arithmetic).
// (S, L) = (5, 4) keeps 15 slice pairs: the error is below ~2^-37 of
// sum_j |D_ij f_j|, i.e. FP64-level for these operators.  (S, L) = (2, 1) is
// the 3-product hi/lo split.
//
// Kernel structure: a persistent, warp-specialised CTA per SM (producers stage
// and split the pencils of a tile, one thread issues tcgen05.mma, epilogue warps
// read TMEM and rebuild the outputs), described at k_dense below.  The halo
// passes of the hybrid iteration run on the CUDA cores (halo_rows.cu).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "dense.h"

namespace cfd {

namespace {

constexpr int kS = 5;              // digit slices kept for exact mode
constexpr int kTile = 128;         // pencils per tile (MMA M)
constexpr int kTmemCols = 512;
constexpr long long kWaitLimit = 4000000000LL;  // clock cycles (~2 s) before giving up

// ------------------------------------------------------------------ host: wait limit of the main loop

long long g_wait_limit = kWaitLimit;
long long dense_wait_limit() { return g_wait_limit; }

// ------------------------------------------------------------------ host: operator digits

typedef long double ld;

// Solve the closed system A x = B for all columns; A tridiagonal with unit
// rows 0 and N-1.  Row-major D (N x E), long double.
void closed_operator(const SchemeCoef &s, int N, int g, ld scale, std::vector<ld> &D) {
  const int E = N + 2 * g;
  std::vector<ld> A(N * N, 0), Bm(N * E, 0);
  for (int k = 0; k < N; ++k) {
    A[k * N + k] = 1;
    const bool clo = (k == 0 || k == N - 1);
    if (!clo) {
      A[k * N + k - 1] = s.a;
      A[k * N + k + 1] = s.a;
      for (int m = -s.M; m <= s.M; ++m) Bm[k * E + k + m + g] = s.rhs[m + s.M];
    } else {
      for (int m = -s.h; m <= s.h; ++m) Bm[k * E + k + m + g] = s.clo[m + s.h];
    }
  }
  // Gaussian elimination (diagonally dominant: no pivoting needed)
  for (int c = 0; c < N; ++c) {
    for (int r = c + 1; r < N; ++r) {
      const ld f = A[r * N + c] / A[c * N + c];
      if (f == 0) continue;
      for (int k = c; k < N; ++k) A[r * N + k] -= f * A[c * N + k];
      for (int k = 0; k < E; ++k) Bm[r * E + k] -= f * Bm[c * E + k];
    }
  }
  D.assign(N * E, 0);
  for (int r = N - 1; r >= 0; --r)
    for (int k = 0; k < E; ++k) {
      ld v = Bm[r * E + k];
      for (int q = r + 1; q < N; ++q) v -= A[r * N + q] * D[q * E + k];
      D[r * E + k] = v / A[r * N + r];
    }
  for (auto &v : D) v *= scale;
}

// Periodic (undecomposed) operator of one whole line: circulant A_c^-1 B_c,
// written on the ghost-extended index with zeros in the ghost columns.
void cyclic_operator(const SchemeCoef &s, int N, int g, ld scale, std::vector<ld> &D) {
  const int E = N + 2 * g;
  std::vector<ld> A(N * N, 0), Bm(N * N, 0);
  for (int k = 0; k < N; ++k) {
    A[k * N + k] += 1;
    A[k * N + (k + N - 1) % N] += s.a;
    A[k * N + (k + 1) % N] += s.a;
    for (int m = -s.M; m <= s.M; ++m) Bm[k * N + ((k + m) % N + N) % N] += s.rhs[m + s.M];
  }
  // Gauss-Jordan with partial pivoting
  std::vector<int> piv(N);
  for (int c = 0; c < N; ++c) {
    int p = c;
    for (int r = c + 1; r < N; ++r)
      if (fabsl(A[r * N + c]) > fabsl(A[p * N + c])) p = r;
    if (p != c) {
      for (int k = 0; k < N; ++k) std::swap(A[p * N + k], A[c * N + k]);
      for (int k = 0; k < N; ++k) std::swap(Bm[p * N + k], Bm[c * N + k]);
    }
    const ld d = A[c * N + c];
    for (int k = 0; k < N; ++k) { A[c * N + k] /= d; Bm[c * N + k] /= d; }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const ld f = A[r * N + c];
      if (f == 0) continue;
      for (int k = 0; k < N; ++k) { A[r * N + k] -= f * A[c * N + k]; Bm[r * N + k] -= f * Bm[c * N + k]; }
    }
  }
  D.assign(N * E, 0);
  for (int r = 0; r < N; ++r)
    for (int k = 0; k < N; ++k) D[r * E + k + g] = Bm[r * N + k] * scale;
}

uint16_t bf16_of_small_int(int a) {
  float f = (float)a;
  uint32_t u;
  memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

// Digit image of one operator: kS slices x rows x Kp columns (row-major D of
// `cols` columns, cols <= Kp, rows a multiple of 8), canonical K-major smem
// layout per slice: [row/8][k/8][row%8][k%8] bf16.  Row i is scaled by
// 2^rowexp[i] >= max_j |D_ij|.
void digit_image(const std::vector<ld> &D, int rows, int cols, int Kp, std::vector<uint16_t> &img,
                 std::vector<int> &rowexp) {
  img.assign((size_t)kS * rows * Kp, 0);
  rowexp.assign(rows, 0);
  for (int i = 0; i < rows; ++i) {
    ld mx = 0;
    for (int j = 0; j < cols; ++j) mx = std::max(mx, fabsl(D[(size_t)i * cols + j]));
    int e = 0;
    if (mx > 0) frexpl(mx, &e);  // mx < 2^e
    rowexp[i] = e;
    for (int j = 0; j < cols; ++j) {
      long long F = llrintl(ldexpl(D[(size_t)i * cols + j], 39 - e));  // |F| <= 2^39
      int dig[kS];
      for (int t = kS - 1; t >= 1; --t) {
        long long r = F & 0xFF;
        if (r >= 128) r -= 256;
        dig[t] = (int)r;
        F = (F - r) >> 8;
      }
      dig[0] = (int)F;
      for (int t = 0; t < kS; ++t) {
        const size_t off = (size_t)t * rows * Kp + ((size_t)(i / 8) * (Kp / 8) + j / 8) * 64 + (i % 8) * 8 + (j % 8);
        img[off] = bf16_of_small_int(dig[t]);
      }
    }
  }
}

// TF32 image of one operator (the one-product TF32 form): D_ij / 2^rowexp[i] rounded to TF32
// (nearest, ties to even), canonical K-major smem layout of 32-bit elements:
// [row/8][k/4][row%8][k%4].  Same row exponents as the digit image.
void tf32_image(const std::vector<ld> &D, int rows, int cols, int Kp, std::vector<uint32_t> &img) {
  img.assign((size_t)rows * Kp, 0);
  for (int i = 0; i < rows; ++i) {
    ld mx = 0;
    for (int j = 0; j < cols; ++j) mx = std::max(mx, fabsl(D[(size_t)i * cols + j]));
    int e = 0;
    if (mx > 0) frexpl(mx, &e);
    for (int j = 0; j < cols; ++j) {
      const float f = (float)ldexpl(D[(size_t)i * cols + j], -e);
      uint32_t u;
      memcpy(&u, &f, 4);
      u = (u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu;
      img[((size_t)(i / 8) * (Kp / 4) + j / 4) * 32 + (i % 8) * 4 + (j % 4)] = u;
    }
  }
}

// Iterated block system of Eq. iter_center_P in dense form (no dx scaling):
// unknowns k = -1..N with the derivative fixed at k = -2 (d_lo) and k = N+1
// (d_hi);  d[k] = sum_j D1[k][j] f_j + cm[k] d_lo + cp[k] d_hi for k = 0..N-1.
void iterated_operator(const SchemeCoef &s, int N, int g, std::vector<ld> &D1, std::vector<ld> &cm,
                       std::vector<ld> &cp) {
  const int E = N + 2 * g, n = N + 2;
  std::vector<ld> A(n * n, 0), Bm(n * E, 0), Ic(n * 2, 0);
  for (int r = 0; r < n; ++r) {
    const int k = r - 1;
    A[r * n + r] = 1;
    if (r > 0) A[r * n + r - 1] = s.a;
    if (r < n - 1) A[r * n + r + 1] = s.a;
    for (int m = -s.M; m <= s.M; ++m) Bm[r * E + k + m + g] = s.rhs[m + s.M];
  }
  Ic[0 * 2 + 0] = -s.a;          // row k = -1 carries -a d_lo
  Ic[(n - 1) * 2 + 1] = -s.a;    // row k = N carries -a d_hi
  for (int c = 0; c < n; ++c)
    for (int r = c + 1; r < n; ++r) {
      const ld f = A[r * n + c] / A[c * n + c];
      if (f == 0) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < E; ++k) Bm[r * E + k] -= f * Bm[c * E + k];
      for (int k = 0; k < 2; ++k) Ic[r * 2 + k] -= f * Ic[c * 2 + k];
    }
  std::vector<ld> X(n * E), Y(n * 2);
  for (int r = n - 1; r >= 0; --r) {
    for (int k = 0; k < E; ++k) {
      ld v = Bm[r * E + k];
      for (int q = r + 1; q < n; ++q) v -= A[r * n + q] * X[q * E + k];
      X[r * E + k] = v / A[r * n + r];
    }
    for (int k = 0; k < 2; ++k) {
      ld v = Ic[r * 2 + k];
      for (int q = r + 1; q < n; ++q) v -= A[r * n + q] * Y[q * 2 + k];
      Y[r * 2 + k] = v / A[r * n + r];
    }
  }
  D1.assign(N * E, 0);
  cm.assign(N, 0);
  cp.assign(N, 0);
  for (int k = 0; k < N; ++k) {
    for (int j = 0; j < E; ++j) D1[k * E + j] = X[(k + 1) * E + j];
    cm[k] = Y[(k + 1) * 2 + 0];
    cp[k] = Y[(k + 1) * 2 + 1];
  }
}

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// BF16 bit pattern (high half of a float) of a small integer, exact for |a| < 2^22.
__device__ __forceinline__ uint32_t small_int_f32bits(int a) {
  return __float_as_uint(__int_as_float(0x4B400000 + a) - 12582912.0f);
}

// Every TMEM accumulator starts at kAccBias = 1.5 * 2^23 (one extra MMA per pass) and the
// digit sums added to it stay below 2^22 in magnitude, so the FP32 value stays in
// [2^23, 2^24), where the bit pattern is kAccBiasBits + (the integer sum): reading an
// accumulator as an integer is one subtraction, which the epilogue folds into its
// multiply-adds.
constexpr uint32_t kAccBiasBits = 0x4B400000u;
constexpr float kAccBias = 12582912.0f;
constexpr int kBadTau = 1 << 20;  // pencil scale of a pencil holding a NaN or an infinity

// Y * 2^E as an IEEE double (|Y| < 2^55).  The 64-bit conversion runs on the FP64 pipe,
// which nothing else in this kernel uses; the power-of-two scale is an add to the exponent
// field.  `checked`: results below the normal range flush to a signed zero, results above
// it become infinities, and `bad` gives a NaN; without it the caller has established that
// the exponent stays in range for every Y.
template <bool checked>
__device__ __forceinline__ double scaled_double(double d, int E, bool bad) {
  const int hi = __double2hiint(d), lo = __double2loint(d);
  if (!checked) return d == 0.0 ? 0.0 : __hiloint2double(hi + (E << 20), lo);
  const int fe = (hi >> 20) & 0x7FF;  // 0 only for d = 0 here (d is an integer or an FP32 value)
  if (bad) return __longlong_as_double(0x7FF8000000000000ll);
  if (fe == 0 || fe + E <= 0) return __hiloint2double(hi & (int)0x80000000, 0);
  if (fe + E >= 2047) return __hiloint2double((hi & (int)0x80000000) | 0x7FF00000, 0);
  return __hiloint2double(hi + (E << 20), lo);
}
template <bool checked>
__device__ __forceinline__ double scaled_int_to_double(long long Y, int E, bool bad) {
  return scaled_double<checked>(__ll2double_rn(Y), E, bad);
}

// v / tau as TF32 (rounded to nearest, ties away from zero), tau = 2^(emax - bias + 1) the
// pencil's power-of-two scale: an add to the exponent field keeps every element a normal number
// (elements more than 2^-60 below the pencil maximum, and subnormals, are zero), then one
// rounding to FP32 and one to TF32.
__device__ __forceinline__ uint32_t cvt_rna_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint32_t tf32_of(double v, int emax) {
  const int hi = __double2hiint(v), lo = __double2loint(v);
  const int e = (hi >> 20) & 0x7FF;
  if (e == 0 || e + 60 < emax) return 0u;
  return cvt_rna_tf32(__double2float_rn(__hiloint2double(hi - ((emax - 1022) << 20), lo)));
}
__device__ __forceinline__ uint32_t tf32_of(float v, int emax) {
  const uint32_t u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xFF);
  if (e == 0 || e + 60 < emax) return 0u;
  return cvt_rna_tf32(__uint_as_float(u - ((uint32_t)(emax - 126) << 23)));
}

// y * 2^E in FP32 for |E| <= 300: two exact power-of-two factors (each a normal float),
// so the only rounding is that of the final product (under- and overflow as IEEE).
__device__ __forceinline__ float scale_pow2(float y, int E) {
  E = max(-300, min(300, E));
  const int e1 = E / 2, e2 = E - e1;
  return y * __int_as_float((e1 + 127) << 23) * __int_as_float((e2 + 127) << 23);
}

// Signed fixed-point value F = round(v / tau * 2^39), |F| <= 2^39, of one input element;
// tau = 2^(emax - bias + 1) is the pencil's power-of-two scale (emax the largest biased
// exponent of the pencil, below that of infinities).  Integer instructions only: the 53-bit
// significand m (implicit bit included) is shifted right by emax + 14 - e with one extra bit
// kept for rounding (half away from zero).  Elements below 2^-40 tau round to zero; subnormal
// elements are taken as zero.
__device__ __forceinline__ long long fixed_of(double v, int emax) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  const long long F = (long long)(((m >> min(emax + 13 - e, 63)) + 1ull) >> 1);
  return e == 0 ? 0ll : ((int)hi < 0 ? -F : F);
}

__device__ __forceinline__ long long fixed_of(float v, int emax) {
  const uint32_t u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xFF);
  const unsigned long long m = (u & 0x7FFFFFu) | 0x800000u;
  const int sh = e - emax + 15;  // <= 15
  long long U;
  if (e == 0) U = 0;
  else if (sh >= 0) U = (long long)(m << sh);
  else U = (-sh) > 40 ? 0ll : (long long)(((m >> (-sh - 1)) + 1ull) >> 1);
  return (u >> 31) ? -U : U;
}

// Balanced base-256 digits d_0..d_4 (d_1..d_4 in [-128, 127], |d_0| <= 128, d_0 most
// significant) of a two's-complement F with |F| <= 2^39; returns the leading S as FP32
// bit patterns.  Adding 128 to each of the four low digit positions absorbs the carries:
// the low word of V = F + 0x80808080 holds the bytes d_t + 128 and V >> 32 is d_0.  A
// byte is turned into a float by placing it under the exponent of 2^23 (1 PRMT) and
// subtracting 2^23 + 128 (exact).
template <int S>
__device__ __forceinline__ void digits_of(long long F, uint32_t (&out)[S]) {
  const long long V = F + 0x80808080ll;
  const uint32_t lo = (uint32_t)V;
  out[0] = small_int_f32bits((int)(V >> 32));
#pragma unroll
  for (int t = 1; t < S; ++t) {
    const uint32_t sel = 0x5440u | (uint32_t)(4 - t);  // byte 4-t of lo, then 0x00 0x00 0x4B
    out[t] = __float_as_uint(__uint_as_float(__byte_perm(lo, 0x4B00u, sel)) - 8388736.0f);
  }
}

__device__ __forceinline__ int biased_exp(double v) {
  return (int)((((unsigned long long)__double_as_longlong(v)) >> 52) & 0x7FF);
}
__device__ __forceinline__ int biased_exp(float v) { return (int)((__float_as_uint(v) >> 23) & 0xFF); }
__device__ __forceinline__ int tau_exp(int emax, double) { return emax - 1022; }
__device__ __forceinline__ int tau_exp(int emax, float) { return emax - 126; }
__device__ __forceinline__ int nonfinite_exp(double) { return 0x7FF; }
__device__ __forceinline__ int nonfinite_exp(float) { return 0xFF; }

// Wait for the phase `parity` of an mbarrier for at most `limit` clock cycles.  The main loop
// uses the launch's limit (DenseParams::wait_limit); the exit path, which drains the CTA's own
// copies and MMAs before it frees TMEM, always uses kWaitLimit.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar_addr, uint32_t parity, long long limit = kWaitLimit) {
  const long long t0 = clock64();
  uint32_t done = 0;
  while (!done) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar_addr), "r"(parity));
    if (!done && clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ long long stride_of(int axis, long long s0, long long s1) {
  return axis == 0 ? s0 : (axis == 1 ? s1 : 1ll);
}

// ------------------------------------------------------------------ the kernel
//
// Persistent, one CTA of 16 warps per SM, warp-specialised:
//   warps 0-7   producers: stage the next tile's pencils (TMA boxes, or
//               cp.async), split the current one into 5 digit rows of A[buf]
//               (two A buffers), publish the pencil scales (meta_full); then
//               thread 0 issues tcgen05.mma for every pass of the tile into
//               one of three TMEM pass buffers (t_full on commit) and frees
//               A[buf] with a last commit (a_empty);
//   warps 8-15  epilogue: wait t_full, read their TMEM lanes, free the pass
//               buffer (t_empty), rebuild the outputs and store them.
// Every wait is bounded; a timeout latches CFD_ERR_TIMEOUT and ends the CTA.

#ifndef CFD_DENSE_PRODUCER_WARPS
#define CFD_DENSE_PRODUCER_WARPS 8
#endif
constexpr int kProdWarps = CFD_DENSE_PRODUCER_WARPS;  // multiple of 4
constexpr int kProducers = kProdWarps * 32;          // warps 0 .. kProdWarps-1
constexpr int kParts = kProducers / 128;             // threads per pencil
constexpr int kEpilogue = 256;                       // the next 8 warps: two per TMEM lane quadrant
constexpr int kThreads = kProducers + kEpilogue;
constexpr int kPassCols = 160;    // TMEM columns per pass buffer ((L + 1) * R <= 160)
constexpr int kPassBufs = 3;
constexpr int kBiasRows = 160;    // rows of the bias MMA's B operand (>= (L + 1) * R)
constexpr int kBiasBytes = (kTile + kBiasRows) * 16 * 2;

// One group of RH rows of a pass: read the LEV level accumulators of this thread's pencil
// (TMEM lane) from the pass buffer, release it (the last group), rebuild every output as
// Y * 2^(rowexp + ebase) and store it.  `checked` selects the conversion that handles
// non-finite pencils and exponents outside the normal range (see scaled_int_to_double).
template <int RH, int LEV, typename TO, bool checked, int TFM>
__device__ __forceinline__ void epilogue_rows(uint32_t taddr, uint32_t lev_stride, int ebase, bool bad,
                                              const int *rowexp, TO *fin_base, long long fin_stride, double *sc_base,
                                              long long sc_stride, bool write_fin, bool write_sc, int i0,
                                              uint32_t t_empty_addr, bool vec, double *sc_x,
                                              double *sc_y) {
  uint32_t acc[LEV][RH];
#pragma unroll
  for (int k = 0; k < LEV; ++k) {
    const uint32_t addr = taddr + (uint32_t)k * lev_stride;
    if constexpr (RH == 16) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(acc[k][0]), "=r"(acc[k][1]), "=r"(acc[k][2]), "=r"(acc[k][3]), "=r"(acc[k][4]), "=r"(acc[k][5]),
            "=r"(acc[k][6]), "=r"(acc[k][7]), "=r"(acc[k][8]), "=r"(acc[k][9]), "=r"(acc[k][10]),
            "=r"(acc[k][11]), "=r"(acc[k][12]), "=r"(acc[k][13]), "=r"(acc[k][14]), "=r"(acc[k][15])
          : "r"(addr));
    } else {
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(acc[k][0]), "=r"(acc[k][1]), "=r"(acc[k][2]), "=r"(acc[k][3]), "=r"(acc[k][4]),
                     "=r"(acc[k][5]), "=r"(acc[k][6]), "=r"(acc[k][7])
                   : "r"(addr));
    }
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;");
  // the pass buffer can be reused as soon as every epilogue thread has its values
  if (t_empty_addr) {  // last row group of the pass: the buffer can be reused
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(t_empty_addr));
  }
  if (!write_fin && !write_sc) return;  // a pencil outside the outputs of this pass
  // 16-byte vector stores where the output axis is contiguous (x): pencil rows are
  // 16-byte aligned (N and the output offsets are multiples of 16 elements)
  constexpr int V = 16 / sizeof(TO);
#pragma unroll
  for (int c0 = 0; c0 < RH; c0 += V) {
    TO o[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int c = c0 + u;
      const int ex = rowexp[c] + ebase;
      // Y = sum_k a_k 2^(8 (LEV-1-k)), a_k = acc_k - kAccBiasBits (exact integers; the
      // 32-bit partial sums are exact modulo 2^32 and their true values fit)
      auto exact_y = [&]() -> long long {
        if constexpr (LEV == 5) {
          const int t1 = (int)(acc[0][c] * 256u + acc[1][c] - 257u * kAccBiasBits);
          const int t2 = (int)(acc[2][c] * 256u + acc[3][c] - 257u * kAccBiasBits);
          return (long long)t1 * 16777216ll + (long long)t2 * 256ll + (long long)(int)(acc[4][c] - kAccBiasBits);
        } else {
          long long Y = 0;
#pragma unroll
          for (int k = 0; k < LEV; ++k) Y = Y * 256ll + (long long)(int)(acc[k][c] - kAccBiasBits);
          return Y;
        }
      };
      TO val;
      double dv = 0.0;  // the FP64 value the intermediates keep
      if constexpr (TFM) {
        // TF32 form: one FP32 accumulator per output, scaled by 2^(rowexp + etau)
        const float a = __uint_as_float(acc[0][c]);
        if constexpr (sizeof(TO) == 8) {
          val = dv = scaled_double<checked>((double)a, ex, bad);
        } else {
          if constexpr (checked) val = bad ? __int_as_float(0x7FC00000) : scale_pow2(a, ex);
          else val = a * __int_as_float((ex + 127) << 23);
          if (write_sc) dv = scaled_double<true>((double)a, ex, bad);
        }
      } else if constexpr (sizeof(TO) == 8) {
        val = dv = scaled_int_to_double<checked>(exact_y(), ex, bad);
      } else {
        // FP32 outputs: the levels as exact floats, Horner in FP32 (each rounding is relative to
        // a partial sum no larger than a few times the result), one power-of-two scale
        float y = __uint_as_float(acc[0][c]) - kAccBias;
#pragma unroll
        for (int k = 1; k < LEV; ++k) y = fmaf(y, 256.0f, __uint_as_float(acc[k][c]) - kAccBias);
        if constexpr (checked) val = bad ? __int_as_float(0x7FC00000) : scale_pow2(y, ex);
        else val = y * __int_as_float((ex + 127) << 23);
        if (write_sc) dv = scaled_int_to_double<true>(exact_y(), ex, bad);
      }
      o[u] = val;
      const long long i = i0 + c;
      if (write_sc) {
        sc_base[i * sc_stride] = dv;
        if (sc_x) sc_x[i * sc_stride] = dv;  // the face neighbour's ghost column
        if (sc_y) sc_y[i * sc_stride] = dv;
      }
      if (write_fin && !vec) fin_base[i * fin_stride] = val;
    }
    if (write_fin && vec) {
      if constexpr (sizeof(TO) == 8)
        *reinterpret_cast<double2 *>(fin_base + i0 + c0) = make_double2(o[0], o[1]);
      else
        *reinterpret_cast<float4 *>(fin_base + i0 + c0) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
}

// The common cases of the epilogue, without the per-output branches of epilogue_rows: 8 rows
// from the exact levels, every output in the normal range, final outputs (FP64 or FP32) and,
// with SC, the FP64 intermediate (and the face neighbours' ghost copies where sc_x / sc_y are
// set).  VEC: 16-byte stores along a contiguous output axis.
template <int LEV, typename TO, bool VEC, bool SC, int TFM>
__device__ __forceinline__ void epilogue_fast8(uint32_t taddr, uint32_t lev_stride, int ebase, const int *rowexp,
                                               TO *fin_base, long long fin_stride, double *sc_base,
                                               long long sc_stride, double *sc_x, double *sc_y, int i0,
                                               uint32_t t_empty_addr) {
  uint32_t acc[LEV][8];
#pragma unroll
  for (int k = 0; k < LEV; ++k)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(acc[k][0]), "=r"(acc[k][1]), "=r"(acc[k][2]), "=r"(acc[k][3]), "=r"(acc[k][4]),
                   "=r"(acc[k][5]), "=r"(acc[k][6]), "=r"(acc[k][7])
                 : "r"(taddr + (uint32_t)k * lev_stride));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
  if (t_empty_addr) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(t_empty_addr));
  }
  const int4 ra = *reinterpret_cast<const int4 *>(rowexp), rb = *reinterpret_cast<const int4 *>(rowexp + 4);
  const int rx[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
  TO o[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ex = rx[c] + ebase;
    double dv = 0.0;
    if constexpr (TFM) {
      // TF32 form: one FP32 accumulator a per output; a * 2^ex as FP64 from its bits (zero gives
      // zero; an FP32 subnormal, which the exact products cannot produce above 2^-126 of the
      // scale, takes the library conversion)
      const uint32_t u = acc[0][c];
      const float a = __uint_as_float(u);
      const int ef = (int)((u >> 23) & 0xFFu);
      if (sizeof(TO) == 8 || SC) {
        if (ef)
          dv = __hiloint2double((int)((u & 0x80000000u) | ((uint32_t)(ef + 896 + ex) << 20) | ((u >> 3) & 0xFFFFFu)),
                                (int)(u << 29));
        else
          dv = (u & 0x7FFFFFFFu) ? ldexp((double)a, ex) : __hiloint2double((int)(u & 0x80000000u), 0);
      }
      if constexpr (sizeof(TO) == 8) o[c] = dv;
      else o[c] = a * __int_as_float((ex + 127) << 23);
    } else if (sizeof(TO) == 8 || SC) {
      // Y = sum_k a_k 2^(8 (LEV-1-k)) as a 64-bit integer, one conversion, the scale as an
      // exponent-field add (Y = 0 gives 0)
      long long Y;
      if constexpr (LEV == 5) {
        const int t1 = (int)(acc[0][c] * 256u + acc[1][c] - 257u * kAccBiasBits);
        const int t2 = (int)(acc[2][c] * 256u + acc[3][c] - 257u * kAccBiasBits);
        Y = (long long)t1 * 16777216ll + (long long)t2 * 256ll + (long long)(int)(acc[4][c] - kAccBiasBits);
      } else {
        Y = 0;
#pragma unroll
        for (int k = 0; k < LEV; ++k) Y = Y * 256ll + (long long)(int)(acc[k][c] - kAccBiasBits);
      }
      const double d = __ll2double_rn(Y);
      const int hi = __double2hiint(d), lo = __double2loint(d);
      dv = __hiloint2double(hi ? hi + (ex << 20) : 0, lo);
    }
    if constexpr (TFM) {
    } else if constexpr (sizeof(TO) == 8) {
      o[c] = dv;
    } else {
      // FP32 outputs: the levels as exact floats, Horner in FP32, one power-of-two scale
      float y = __uint_as_float(acc[0][c]) - kAccBias;
#pragma unroll
      for (int k = 1; k < LEV; ++k) y = fmaf(y, 256.0f, __uint_as_float(acc[k][c]) - kAccBias);
      o[c] = y * __int_as_float((ex + 127) << 23);
    }
    if constexpr (SC) {
      const long long i = i0 + c;
      sc_base[i * sc_stride] = dv;
      if (sc_x) sc_x[i * sc_stride] = dv;  // the face neighbour's ghost column
      if (sc_y) sc_y[i * sc_stride] = dv;
    }
  }
  if constexpr (VEC) {
    if constexpr (sizeof(TO) == 8) {
#pragma unroll
      for (int c = 0; c < 8; c += 2) *reinterpret_cast<double2 *>(fin_base + i0 + c) = make_double2(o[c], o[c + 1]);
    } else {
#pragma unroll
      for (int c = 0; c < 8; c += 4)
        *reinterpret_cast<float4 *>(fin_base + i0 + c) = make_float4(o[c], o[c + 1], o[c + 2], o[c + 3]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) fin_base[(long long)(i0 + c) * fin_stride] = o[c];
  }
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr));
}
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kProducers)); }

// Barrier of the 256 producer threads that also ORs a flag over them.
__device__ __forceinline__ bool producer_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kProducers));
  return r != 0;
}

struct TileCoord {
  int lb, q, b, t1, t2;
  bool valid;
};

// The tiles of this CTA: interleaved (tile = CTA + k * grid) or a contiguous run of
// tiles_per_cta (tile_order 1; neighbouring tiles share input rows in L2).
struct TileRange {
  int first, end, step;
};
__device__ __forceinline__ TileRange tile_range(const DenseParams &P) {
  TileRange r;
  if (P.tile_order) {
    r.first = blockIdx.x * P.tiles_per_cta;
    r.end = min(P.ntiles, r.first + P.tiles_per_cta);
    r.step = 1;
  } else {
    r.first = blockIdx.x;
    r.end = P.ntiles;
    r.step = gridDim.x;
  }
  return r;
}

__device__ __forceinline__ int dir_index_dev(int dz, int dy, int dx) {
  const int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
  return r > 13 ? r - 1 : r;
}

// pencil index p (within the block and field) of pencil `pencil` of a tile
// n / d for 0 <= n < 2^22 with inv = 1/d rounded to FP32: (n + 1/2) / d stays at least 1/(2d)
// away from an integer, more than the two roundings can move it
__device__ __forceinline__ int fdiv(int n, float inv) { return __float2int_rz(((float)n + 0.5f) * inv); }

__device__ __forceinline__ int tile_pencil(const DenseParams &P, int tile, int pencil) {
  const int job = fdiv(tile, P.inv_tpj), tj = tile - job * P.tiles_per_job;
  return tj * kTile + pencil;
}

__device__ __forceinline__ TileCoord tile_coord(const DenseParams &P, int tile, int pencil) {
  TileCoord c;
  const int job = fdiv(tile, P.inv_tpj), tj = tile - job * P.tiles_per_job;
  c.lb = fdiv(job, P.inv_nf);
  c.q = job - c.lb * P.nf;
  c.b = P.contig ? P.b0 + c.lb : P.blocks[c.lb];
  const int p = tj * kTile + pencil;
  c.valid = p < P.n1 * P.n2;
  c.t1 = c.valid ? fdiv(p, P.inv_n2) : 0;
  c.t2 = c.valid ? p - c.t1 * P.n2 : 0;
  return c;
}

// TFM = 1: the one-product TF32 form (S = 1, L = 0): A = the pencils scaled by tau and rounded
// to TF32, B = the TF32 image of D, one kind::tf32 MMA chain per pass, FP32 accumulators.
//
// ITER = 1: the final pass of an iterated stage (halo_in set), whose TMA-staged tiles take the
// neighbours' previous iterate as 4 extra columns.  A separate instantiation keeps that code out
// of the closed passes' producer loop (measured 5 % slower with it there).
//
// SPL = 1: a closed pass whose pencils fill an odd number of 8-value K chunks (E = N + 8 for
// N = 16, 32), the last chunk all padding.  The two producer threads of a pencil then split
// the last real chunk four values each instead of one of them taking it whole, so both do the
// same digit work.
template <typename TI, typename TO, int KP, int S, int L, int TFM, bool ITER, bool SPL>
__global__ void __launch_bounds__(kThreads, 1) k_dense(const __grid_constant__ DenseParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int EB = TFM ? 4 : 2;  // bytes per operand element (TF32 or BF16)
  constexpr int A_BYTES = S * kTile * KP * EB;
  // cp.async staging row pitch (elements): odd for the y/z axes (one element per thread and
  // copy, spread over the banks); for the x axis, where a pencil is a contiguous row copied in
  // 16-byte chunks, a pitch whose rows stay 16-byte aligned.
  constexpr int VE = 16 / sizeof(TI);  // elements per 16-byte chunk
  constexpr int XB = 128 / sizeof(TI); // elements per 128-byte swizzled TMA row (x rows)
  const bool xrow = P.xrow != 0;
  const int pitch = xrow ? KP + VE : KP + 1;
  constexpr int NCH = KP / 8;    // 8-value K chunks per pencil
  const int R = P.rows;
  const int B_PASS_BYTES = S * R * KP * EB;
  const int kind = P.tma_kind;
  uint16_t *sA = reinterpret_cast<uint16_t *>(smem);  // [2][S][128][KP] (32-bit elements for TF32)
  unsigned char *sB = smem + 2 * A_BYTES;
  // operands of the bias MMA (K = 16, canonical K-major): A = 1 in column 0 of all 128 rows,
  // B = kAccBias in column 0 of the (L + 1) R level rows
  uint16_t *sOne = reinterpret_cast<uint16_t *>(smem + 2 * A_BYTES + 2 * B_PASS_BYTES);
  uint16_t *sBias = sOne + kTile * 16;
  // staging, 1024-byte aligned (128-byte swizzle atoms)
  const int stg_off = (2 * A_BYTES + 2 * B_PASS_BYTES + kBiasBytes + 1023) & ~1023;
  TI *stg = reinterpret_cast<TI *>(smem + stg_off);
  const int stg_bytes = max(kTile * (KP + VE) * (int)sizeof(TI), P.tma_boxes * kTile * 128);
  int *s_rowexp = reinterpret_cast<int *>(smem + stg_off + stg_bytes);
  int *s_emax = s_rowexp + 2 * 48;   // [2 tiles][kParts][128]
  // Pencil scales of the last 8 tiles: producers run at most 5 tiles ahead of
  // the epilogue (two A buffers, three TMEM pass buffers), so a slot and its
  // mbarrier phase are never reused before the epilogue has read them.
  int *s_etau = s_emax + 2 * kParts * kTile;  // [8][128] ring
  uint64_t *bars = reinterpret_cast<uint64_t *>(s_etau + 8 * kTile);
  // bars: a_empty[2], t_full[3], t_empty[3], meta_full[8], a_full[2], stg_full, drain (thread 0
  // issues the MMAs after the a_full wait; the other producers go on to the next tile)
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 24);
  const uint32_t bar0 = smem_u32(bars);
  auto a_empty = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  auto t_full = [&](int i) { return bar0 + 8u * (uint32_t)(2 + i); };
  auto t_empty = [&](int i) { return bar0 + 8u * (uint32_t)(5 + i); };
  auto meta_full = [&](int i) { return bar0 + 8u * (uint32_t)(8 + i); };
  auto a_full = [&](int i) { return bar0 + 8u * (uint32_t)(16 + i); };
  const uint32_t stg_full = bar0 + 8u * 18u;
  const uint32_t drain = bar0 + 8u * 19u;  // the exit path's commit: every MMA this CTA issued has completed
  const long long WL = P.wait_limit;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = P.N, g = P.g, E = N + 2 * g;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) { mbar_init(a_empty(i), 1); mbar_init(a_full(i), kProducers); }
    for (int i = 0; i < kPassBufs; ++i) { mbar_init(t_full(i), 1); mbar_init(t_empty(i), kEpilogue); }
    for (int i = 0; i < 8; ++i) mbar_init(meta_full(i), kProducers);
    mbar_init(stg_full, 1);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const int SR = P.seg_rows;
  for (int ps = 0; ps < P.passes; ++ps) {
    for (int sg = 0; sg < P.nseg[ps]; ++sg) {
      const uint4 *src = reinterpret_cast<const uint4 *>(P.seg_img[ps][sg]);
      const int slice_u4 = SR * KP * EB / 16;
      for (int t = 0; t < S; ++t) {
        uint4 *dst = reinterpret_cast<uint4 *>(sB + (size_t)ps * B_PASS_BYTES + ((size_t)t * R * KP +
                                               (size_t)sg * SR * KP) * EB);
        const uint4 *sp = src + (size_t)t * slice_u4;
        for (int i = tid; i < slice_u4; i += kThreads) dst[i] = __ldg(sp + i);
      }
      for (int i = tid; i < SR; i += kThreads) s_rowexp[ps * 48 + sg * SR + i] = P.seg_exp[ps][sg][i];
    }
  }
  // index i of a 16-column canonical chunk: column (i >> 6 & 1) * 8 + (i & 7); column 0 iff (i & 0x47) == 0
  for (int i = tid; i < kTile * 16; i += kThreads) sOne[i] = (i & 0x47) == 0 ? 0x3F80 : 0;            // 1.0
  for (int i = tid; i < kBiasRows * 16; i += kThreads) sBias[i] = (i & 0x47) == 0 ? 0x4B40 : 0;      // 1.5 * 2^23
  // generic-proxy writes read by tcgen05.mma (async proxy)
  asm volatile("fence.proxy.async.shared::cta;");
  const long long is0 = (long long)P.in_dims[1] * P.in_dims[2], is1 = P.in_dims[2];
  const long long s_t1 = stride_of(P.t1, is0, is1), s_t2 = stride_of(P.t2, is0, is1), s_ax = stride_of(P.axis, is0, is1);
  const int in_s1 = P.t1 == 0 ? P.in_start[0] : (P.t1 == 1 ? P.in_start[1] : P.in_start[2]);
  const int in_s2 = P.t2 == 0 ? P.in_start[0] : (P.t2 == 1 ? P.in_start[1] : P.in_start[2]);
  const long long E3 = (long long)E * E * E;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  bool failed = false;

  if (warp < kProdWarps) {
    // ================================================================ producers
    // kParts threads per pencil; part `half` splits K chunks half, half + kParts, ...
    const int pl = (warp & 3) * 32 + lane, half = warp >> 2;
    constexpr int CPP = (NCH + kParts - 1) / kParts;  // K chunks per producer thread
    static_assert(!SPL || (!TFM && !ITER && kParts == 2 && NCH % 2 == 0), "split last chunk: two threads per pencil");
    const float inv_n2 = 1.0f / (float)P.n2;
    const int cpr = E / VE;  // 16-byte chunks per pencil row (x axis); E * sizeof(TI) is a multiple of 16
    const float inv_cpr = 1.0f / (float)cpr;
    // TMA: one thread posts the expected bytes and issues the box copies of a tile
    bool tma_pending = false;
    auto tma_issue = [&](int tile) {
      const int job = tile / P.tiles_per_job, tj = tile - job * P.tiles_per_job;
      const int t1_0 = tj * (kTile / P.n2);
      const uint64_t tmap = reinterpret_cast<uint64_t>(&P.tmap);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(stg_full), "r"(P.tma_bytes)
                   : "memory");
      // box origin in (x, y, z) of the tensor map: z also steps over the jobs
      const int cz = P.in_start[0] + job * P.tma_zstep + (P.t1 == 0 ? t1_0 : 0);
      const int cy = P.in_start[1] + (P.t1 == 1 ? t1_0 : 0);
      for (int bx = 0; bx < P.tma_boxes; ++bx) {
        const uint32_t dst = smem_u32(stg) + (uint32_t)(bx * kTile * 128);
        const int cx = P.in_start[2] + bx * XB;
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(dst),
            "l"(tmap), "r"(cx), "r"(cy), "r"(cz), "r"(stg_full)
            : "memory");
      }
      tma_pending = true;
    };
    auto prefetch = [&](int tile) {
      const int pp = tid & (kTile - 1), jq = tid >> 7;  // kParts threads per pencil
      const TileCoord c = tile_coord(P, tile, pp);
      if (xrow) {
        // x axis: the tile's pencil rows, 16-byte chunks, consecutive threads on consecutive
        // chunks (rows of consecutive pencils are adjacent in memory)
        const int job = tile / P.tiles_per_job, tj = tile - job * P.tiles_per_job;
        const int lb = job / P.nf, q = job - lb * P.nf, np = P.n1 * P.n2;
        const long long jb = !P.in_field ? (long long)job * (long long)P.in_box
                             : P.contig  ? (long long)P.nf * P.ext0 + (long long)job * E3
                                         : (long long)P.nf * P.extpre[P.blocks[lb]] + (long long)q * E3;
        const TI *in = static_cast<const TI *>(P.in) + jb;
        for (int ch = tid; ch < kTile * cpr; ch += kProducers) {
          // exact: the fractional parts stay >= 0.5 / divisor away from an integer
          const int cp = __float2int_rz(((float)ch + 0.5f) * inv_cpr), r = ch - cp * cpr;
          const int p = tj * kTile + cp;
          if (p < np) {
            const int t1 = __float2int_rz(((float)p + 0.5f) * inv_n2), t2 = p - t1 * P.n2;
            const TI *src = in + (long long)(in_s1 + t1) * s_t1 + (long long)(in_s2 + t2) * s_t2 + r * VE;
            cp_async16(stg + cp * pitch + r * VE, src);
          }
        }
      }
      if (c.valid) {
        if (!xrow) {
          long long ib = !P.in_field ? ((long long)c.lb * P.nf + c.q) * (long long)P.in_box
                         : P.contig  ? (long long)P.nf * P.ext0 + ((long long)c.lb * P.nf + c.q) * E3
                                     : (long long)P.nf * P.extpre[c.b] + (long long)c.q * E3;
          ib += (long long)(in_s1 + c.t1) * s_t1 + (long long)(in_s2 + c.t2) * s_t2;
          const TI *src = static_cast<const TI *>(P.in) + ib;
          for (int j = jq; j < E; j += kParts) {
            if constexpr (sizeof(TI) == 8) cp_async8(stg + pp * pitch + j, src + (long long)j * s_ax);
            else cp_async4(stg + pp * pitch + j, src + (long long)j * s_ax);
          }
        }
        if (P.halo_in && jq < 2) {
          // previous iterate of the neighbours at k^c: d_lo from the lower neighbour's row N-2,
          // d_hi from the upper neighbour's row 1 (same pencil), per degree
          const int ez = P.axis == 0, ey = P.axis == 1, ex = P.axis == 2;
          const int nb = P.nbr[c.b * 26 + dir_index_dev(jq ? ez : -ez, jq ? ey : -ey, jq ? ex : -ex)];
          const long long hp = ((long long)nb * P.nf + c.q) * (long long)(P.n1 * P.n2) +
                               (long long)(tile_pencil(P, tile, pp));
          for (int d = 0; d < 2; ++d) {
            const double hv = ((P.halo_deg_mask >> d) & 1) ? P.halo_in[hp * 4 + 2 * d + (jq ? 0 : 1)] : 0.0;
            stg[pp * pitch + E + 2 * d + jq] = TI(hv);
          }
        }
      }
      asm volatile("cp.async.commit_group;");
    };
    // staging address of element j of this thread's pencil, one formula for every staging kind
    // (j is a constant in the unrolled loads, so each is an XOR and two multiply-adds, with no
    // branch on the kind in the hot loop):
    //   kind 0 (cp.async rows):        pl * pitch + j
    //   kind 1 (TMA, 128-byte rows):   (j / XB) * 128 XB + pl * XB + ((j % XB) XOR (pl % 8) * VE),
    //                                  i.e. the 16-byte chunk index XOR (row mod 8)
    //   kinds 2, 3 (TMA boxes):        col_base + j * col_step
    const int n2 = P.n2;
    // (a kind-2 box is [t1][kext][x]: kext rows along y, the 4 halo columns of an iterated pass
    // included)
    const int col_base = kind == 2 ? (pl / n2) * P.kext * n2 + (pl % n2) : pl;  // kinds 2, 3
    const int col_step = kind == 2 ? n2 : kTile;
    constexpr int LVE = VE == 2 ? 1 : 2;  // log2(VE)
    static_assert(XB == 8 * VE && (VE == 2 || VE == 4), "a 128-byte row holds 8 chunks of 16 bytes");
    const int ib = kind == 0 ? pl * pitch : (kind == 1 ? pl * XB : col_base);
    const int ihi = kind == 0 ? XB : (kind == 1 ? kTile * XB : XB * col_step);
    const int ilo = kind <= 1 ? 1 : col_step;
    const int ixr = kind == 1 ? (pl & 7) << LVE : 0;
    auto stg_index = [&](int j) -> int { return ib + (j / XB) * ihi + ((j % XB) ^ ixr) * ilo; };
    const uint32_t lbo = 128, sbo = KP * 16;
    int it = 0, pit = 0;
    uint32_t last_bar = 0;  // thread 0: an MMA was issued
    const TileRange tr = tile_range(P);
    int tile = tr.first;
    if (tile < tr.end) {
      if (kind) { if (tid == 0) tma_issue(tile); }
      else prefetch(tile);
    }
    for (; tile < tr.end; tile += tr.step, ++it) {
      const int buf = it & 1, use = it >> 1;
      const TileCoord c = tile_coord(P, tile, pl);
      // An iterated pass staged by TMA: the neighbours' previous iterate goes into staging
      // columns E .. E+3 of this pencil (the box reads zeros or data it overwrites there).  Each
      // of the pencil's threads writes the columns of its own K chunks, which only it reads.
      double hq[4] = {0.0, 0.0, 0.0, 0.0};
      const bool tma_halo = ITER && kind && P.halo_in && c.valid;
      if (tma_halo) {
        const int ez = P.axis == 0, ey = P.axis == 1, ex = P.axis == 2;
        const long long pp = (long long)tile_pencil(P, tile, pl);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int d = m >> 1, jq = m & 1;
          if ((((E + m) >> 3) % kParts) != half || !((P.halo_deg_mask >> d) & 1)) continue;
          const int nb = P.nbr[c.b * 26 + dir_index_dev(jq ? ez : -ez, jq ? ey : -ey, jq ? ex : -ex)];
          hq[m] = P.halo_in[(((long long)nb * P.nf + c.q) * (long long)(P.n1 * P.n2) + pp) * 4 + 2 * d + (jq ? 0 : 1)];
        }
      }
      if (kind) {
        if (!mbar_wait_bounded(stg_full, (uint32_t)(it & 1), WL)) failed = true;
        else if (tid == 0) tma_pending = false;
      } else {
        asm volatile("cp.async.wait_all;");
        producer_sync();
      }
      if (tma_halo && !failed) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if ((((E + m) >> 3) % kParts) == half) stg[stg_index(E + m)] = TI(hq[m]);
      }
      TI v[CPP][8];
      int em = 0;
      const int kv = c.valid ? P.kext : 0;  // values of this pencil (none for a pencil past the end)
#pragma unroll
      for (int h = 0; h < CPP; ++h) {
        // the last slot of a split pass: values 4 half .. 4 half + 3 of chunk NCH - 2
        const bool sl = SPL && h == CPP - 1;
#pragma unroll
        for (int k = 0; k < (sl ? 4 : 8); ++k) {
          const int j = sl ? (NCH - 2) * 8 + 4 * half + k : (half + kParts * h) * 8 + k;
          v[h][k] = j < kv ? stg[stg_index(j)] : TI(0);
          em = max(em, biased_exp(v[h][k]));
        }
      }
      int *se = s_emax + (it & 1) * (kParts * kTile);
      se[half * kTile + pl] = em;
      // staging fully read, exponents exchanged; a failed wait anywhere ends every producer here
      if (producer_any(failed)) { failed = true; break; }
      int emax = se[pl];
#pragma unroll
      for (int q = 1; q < kParts; ++q) emax = max(emax, se[q * kTile + pl]);
      // a NaN or an infinity anywhere in the pencil: every output of the pencil is NaN (the
      // epilogue sees kBadTau); its digits are written as zeros
      const bool bad_pencil = emax >= nonfinite_exp(TI(0));
      if (tile + tr.step < tr.end) {
        if (kind) { if (tid == 0) tma_issue(tile + tr.step); }
        else prefetch(tile + tr.step);
      }
      // A[buf] must be free: the MMAs of its previous use have completed
      if (use > 0 && !mbar_wait_bounded(a_empty(buf), (uint32_t)((use - 1) & 1), WL)) failed = true;
      if (half == 0) s_etau[(it & 7) * kTile + pl] = bad_pencil ? kBadTau : tau_exp(emax, TI(0));
      // a non-finite pencil: every shift in fixed_of / tf32_of runs past the significand (zero digits)
      if (bad_pencil) emax = nonfinite_exp(TI(0)) + 128;
      uint16_t *Ab = sA + (size_t)buf * (A_BYTES / 2);
      const int row_group = pl >> 3, row_in = pl & 7;
      if constexpr (TFM) {
        // TF32 rows: chunk ch (8 values) fills core-matrix columns 2 ch and 2 ch + 1
        uint32_t *A32 = reinterpret_cast<uint32_t *>(Ab);
#pragma unroll
        for (int h = 0; h < CPP; ++h) {
          const int ch = half + kParts * h;
          if (ch >= NCH) break;
          uint32_t w[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) w[k] = ch * 8 < P.kext ? tf32_of(v[h][k], emax) : 0u;
#pragma unroll
          for (int q = 0; q < 2; ++q)
            *reinterpret_cast<uint4 *>(A32 + ((size_t)row_group * (KP / 4) + 2 * ch + q) * 32 + row_in * 4) =
                make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
      } else {
#pragma unroll
      for (int h = 0; h < CPP; ++h) {
        if (SPL && h == CPP - 1) {
          // half of chunk NCH - 2 (8-byte digit stores); the second thread also writes the
          // zero digits of the padding chunk NCH - 1
          uint32_t w2[S][2];
#pragma unroll
          for (int k = 0; k < 4; k += 2) {
            uint32_t d0[S], d1[S];
            digits_of<S>(fixed_of(v[h][k], emax), d0);
            digits_of<S>(fixed_of(v[h][k + 1], emax), d1);
#pragma unroll
            for (int t = 0; t < S; ++t) w2[t][k / 2] = __byte_perm(d0[t], d1[t], 0x7632);
          }
#pragma unroll
          for (int t = 0; t < S; ++t) {
            uint16_t *row = Ab + (size_t)t * kTile * KP + (size_t)row_group * NCH * 64 + row_in * 8;
            *reinterpret_cast<uint2 *>(row + (NCH - 2) * 64 + 4 * half) = make_uint2(w2[t][0], w2[t][1]);
            if (half) *reinterpret_cast<uint4 *>(row + (NCH - 1) * 64) = make_uint4(0u, 0u, 0u, 0u);
          }
          continue;
        }
        const int ch = half + kParts * h;
        if (ch >= NCH) break;
        uint32_t w[S][4];
        if (ch * 8 >= P.kext) {  // K padding: zero digits (warp-uniform branch)
#pragma unroll
          for (int t = 0; t < S; ++t) {
            uint4 *dst = reinterpret_cast<uint4 *>(Ab + (size_t)t * kTile * KP + ((size_t)row_group * NCH + ch) * 64 +
                                                   row_in * 8);
            *dst = make_uint4(0u, 0u, 0u, 0u);
          }
          continue;
        }
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          uint32_t d0[S], d1[S];
          digits_of<S>(fixed_of(v[h][k], emax), d0);
          digits_of<S>(fixed_of(v[h][k + 1], emax), d1);
#pragma unroll
          for (int t = 0; t < S; ++t) w[t][k / 2] = __byte_perm(d0[t], d1[t], 0x7632);
        }
#pragma unroll
        for (int t = 0; t < S; ++t) {
          uint4 *dst = reinterpret_cast<uint4 *>(Ab + (size_t)t * kTile * KP + ((size_t)row_group * NCH + ch) * 64 +
                                                 row_in * 8);
          *dst = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
        }
      }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      mbar_arrive(meta_full(it & 7));
      mbar_arrive(a_full(buf));  // A[buf] written by this thread
      if (tid == 0) {
        // MMA issue: once every producer has written A[buf] (the others go on to the next tile)
        if (!mbar_wait_bounded(a_full(buf), (uint32_t)(use & 1), WL)) failed = true;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(sA) + (uint32_t)(buf * A_BYTES);
        for (int ps = 0; ps < P.passes && !failed; ++ps, ++pit) {
          const int tb = pit % kPassBufs, tuse = pit / kPassBufs;
          if (tuse > 0 && !mbar_wait_bounded(t_empty(tb), (uint32_t)((tuse - 1) & 1), WL)) { failed = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t b0 = smem_u32(sB) + ps * B_PASS_BYTES;
          const uint32_t cbase = tmem + (uint32_t)(tb * kPassCols);
          if constexpr (TFM) {
            // one product: K steps of 8 TF32 values (32 bytes = two core matrices)
            const uint32_t idesc_t = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(R >> 3) << 17) |
                                     ((uint32_t)(kTile >> 4) << 24);
#pragma unroll
            for (int kk = 0; kk < KP / 8; ++kk)
              mma_tf32(cbase, smem_desc(a0 + (uint32_t)(kk * 256), 128, KP * 32),
                       smem_desc(b0 + (uint32_t)(kk * 256), 128, KP * 32), idesc_t, kk ? 1u : 0u);
          } else {
          {
            // every level column of the pass buffer starts at kAccBias (1 x kAccBias, K = 16)
            const uint32_t idesc_b = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(((L + 1) * R) >> 3) << 17) |
                                     ((uint32_t)(kTile >> 4) << 24);
            mma_bf16(cbase, smem_desc(smem_u32(sOne), 128, 256), smem_desc(smem_u32(sBias), 128, 256), idesc_b, 0u);
          }
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const int nt = (L - s + 1) < S ? (L - s + 1) : S;
            if (nt <= 0) continue;
            const uint32_t idesc_s = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((nt * R) >> 3) << 17) |
                                     ((uint32_t)(kTile >> 4) << 24);
#pragma unroll
            for (int kk = 0; kk < KP / 16; ++kk) {
              const uint64_t da = smem_desc(a0 + (uint32_t)(s * kTile * KP * 2 + kk * 256), lbo, sbo);
              const uint64_t db = smem_desc(b0 + (uint32_t)(kk * 256), lbo, sbo);
              mma_bf16(cbase + (uint32_t)(s * R), da, db, idesc_s, 1u);
            }
          }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              t_full(tb)));
          last_bar = 1;
        }
        if (!failed)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              a_empty(buf)));
      }
    }
    asm volatile("cp.async.wait_all;");
    if (tid == 0) {
      // a TMA copy still in flight after a failure completes before the CTA leaves, and every
      // MMA issued (also those of a tile left half-done by a failed wait) completes before TMEM
      // is released: one more commit tracks them all
      if (tma_pending) mbar_wait_bounded(stg_full, (uint32_t)(it & 1));
      if (last_bar) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain));
        mbar_wait_bounded(drain, 0u);
      }
    }
  } else {
    // ================================================================ epilogue
    const int quad = warp & 3, ehalf = (warp - kProdWarps) >> 2;
    const int pl = quad * 32 + lane;
    const long long n3 = (long long)N * N * N;
    const long long f_t1 = stride_of(P.t1, (long long)N * N, N), f_t2 = stride_of(P.t2, (long long)N * N, N),
                    f_ax = stride_of(P.axis, (long long)N * N, N);
    const long long ss0 = (long long)P.sc_dims[1] * P.sc_dims[2], ss1 = P.sc_dims[2];
    const long long c_t1 = stride_of(P.t1, ss0, ss1), c_t2 = stride_of(P.t2, ss0, ss1), c_ax = stride_of(P.axis, ss0, ss1);
    const int sc_s1 = P.t1 == 0 ? P.sc_start[0] : (P.t1 == 1 ? P.sc_start[1] : P.sc_start[2]);
    const int sc_s2 = P.t2 == 0 ? P.sc_start[0] : (P.t2 == 1 ? P.sc_start[1] : P.sc_start[2]);
    // range of the row exponents of each pass: with the pencil scale it decides whether every
    // output of a thread stays in the normal range (the unchecked conversion)
    int rlo0 = s_rowexp[0], rhi0 = rlo0, rlo1 = s_rowexp[48], rhi1 = rlo1;
    for (int i = 1; i < R; ++i) {
      rlo0 = min(rlo0, s_rowexp[i]);
      rhi0 = max(rhi0, s_rowexp[i]);
      rlo1 = min(rlo1, s_rowexp[48 + i]);
      rhi1 = max(rhi1, s_rowexp[48 + i]);
    }
    // unchecked conversion: Y * 2^E (|Y| < 2^55) or a * 2^E (an FP32 accumulator) stays normal
    constexpr int kExLo = sizeof(TO) == 8 ? (TFM ? -870 : -1022) : -126;
    constexpr int kExHi = sizeof(TO) == 8 ? (TFM ? 1000 : 969) : 127;
    // launch-invariant: this thread's rows of a pass, their segment, and per pass the segment's
    // mode and output slot
    const int RH = R / 2, r0 = ehalf * RH;  // the two warps of a quadrant split the rows
    const int sg = r0 / P.seg_rows, i0 = r0 - sg * P.seg_rows;
    const int mode0 = P.seg_mode[0][sg], mode1 = P.passes > 1 ? P.seg_mode[1][sg] : -1;
    const long long opoff0 = (long long)P.seg_op[0][sg] * n3,
                    opoff1 = P.passes > 1 ? (long long)P.seg_op[1][sg] * n3 : 0;
    int it = 0, pit = 0;
    const TileRange tr = tile_range(P);
    for (int tile = tr.first; tile < tr.end && !failed; tile += tr.step, ++it) {
      const TileCoord c = tile_coord(P, tile, pl);
      const bool interior = c.valid && P.int_lo1 <= c.t1 && c.t1 < P.int_hi1 && P.int_lo2 <= c.t2 && c.t2 < P.int_hi2;
      if (!mbar_wait_bounded(meta_full(it & 7), (uint32_t)((it >> 3) & 1), WL)) { failed = true; break; }
      const int etau = s_etau[(it & 7) * kTile + pl];
      const bool bad = etau == kBadTau;
      const int ebase = TFM ? etau : etau - 14 - 8 * L;
      // per tile: the output and intermediate addresses of this thread's pencil (the pass adds
      // its operator's output slot)
      TO *fb_tile = static_cast<TO *>(P.out);
      if (interior)
        fb_tile += (long long)P.nf * P.nops * (P.contig ? P.int0 + (long long)c.lb * n3 : P.intpre[c.b]) +
                   (long long)c.q * P.nops * n3 + (long long)(c.t1 - P.int_lo1) * f_t1 +
                   (long long)(c.t2 - P.int_lo2) * f_t2;
      double *sb = P.scratch_out;
      const bool any_sc = sb != nullptr && c.valid;
      if (any_sc)
        sb += ((long long)(P.sc_local ? P.sc_local[c.lb] : c.lb) * P.nf + c.q) * (long long)P.sc_box +
              (long long)(sc_s1 + c.t1) * c_t1 + (long long)(sc_s2 + c.t2) * c_t2;
      const long long sstr = c_ax;
      // interior pencils near an x (y) face also fill the neighbour's ghost column (row)
      double *gx = nullptr, *gyp = nullptr;
      if (any_sc && P.ghost_x) {
        const int xs = sc_s2 + c.t2;  // t2 is the x axis in the stages that write intermediates
        const long long jump = (long long)P.nf * (long long)P.sc_box;
        // (no write where the block has no such neighbour: it computes that strip itself)
        const int *nl = P.nl + c.lb * 4;
        if (xs < 2 * g) { if (nl[0] >= 0) gx = sb + (long long)(nl[0] - c.lb) * jump + N; }
        else if (xs >= N) { if (nl[1] >= 0) gx = sb + (long long)(nl[1] - c.lb) * jump - N; }
        if (P.ghost_y) {
          const int ys = sc_s1 + c.t1;  // t1 is the y axis (z stage)
          if (ys < 2 * g) { if (nl[2] >= 0) gyp = sb + (long long)(nl[2] - c.lb) * jump + (long long)N * ss1; }
          else if (ys >= N) { if (nl[3] >= 0) gyp = sb + (long long)(nl[3] - c.lb) * jump - (long long)N * ss1; }
        }
      }
      for (int ps = 0; ps < P.passes; ++ps, ++pit) {
        const int tb = pit % kPassBufs, tuse = pit / kPassBufs;
        if (!mbar_wait_bounded(t_full(tb), (uint32_t)(tuse & 1), WL)) { failed = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int mode = ps ? mode1 : mode0;
        const bool wf = (mode == 0 || mode == 3) && interior;
        const bool ws = (mode == 2 || mode == 3) && c.valid;
        TO *fb = fb_tile + (ps ? opoff1 : opoff0);
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tb * kPassCols + r0);
        const int *rexp = s_rowexp + ps * 48 + r0;
        // rows in groups of 8 (fewer live registers); the pass buffer is released after the last group.
        // A warp whose outputs all stay in the normal range takes the unchecked conversion.  The
        // groups run as a loop, not unrolled: one copy of the rebuild code per conversion keeps the
        // epilogue's hot loop small next to the producers' in each sub-partition's instruction cache.
        const int rlo = ps ? rlo1 : rlo0, rhi = ps ? rhi1 : rhi0;
        const bool safe = !(wf || ws) || (!bad && ebase + rlo >= kExLo && ebase + rhi <= kExHi);
        const bool vec = P.xvec != 0;
        const int ng = RH / 8;  // row groups; the last one releases the pass buffer
        // the common cases first: final outputs, with or without the intermediate (warp-uniform
        // choices: tcgen05.ld is a warp-wide instruction)
        const bool fast = safe && wf;
        if (__all_sync(0xffffffffu, fast && !ws)) {
#pragma unroll 1
          for (int gq = 0; gq < ng; ++gq) {
            const int o8 = gq * 8;
            const uint32_t rel = gq == ng - 1 ? t_empty(tb) : 0u;
            if (vec)
              epilogue_fast8<L + 1, TO, true, false, TFM>(taddr + o8, (uint32_t)R, ebase, rexp + o8, fb, f_ax, nullptr, 0,
                                                    nullptr, nullptr, i0 + o8, rel);
            else
              epilogue_fast8<L + 1, TO, false, false, TFM>(taddr + o8, (uint32_t)R, ebase, rexp + o8, fb, f_ax, nullptr, 0,
                                                     nullptr, nullptr, i0 + o8, rel);
          }
        } else if (sizeof(TO) == 8 && __all_sync(0xffffffffu, fast && ws)) {
#pragma unroll 1
          for (int gq = 0; gq < ng; ++gq) {
            const int o8 = gq * 8;
            const uint32_t rel = gq == ng - 1 ? t_empty(tb) : 0u;
            if (vec)
              epilogue_fast8<L + 1, TO, true, true, TFM>(taddr + o8, (uint32_t)R, ebase, rexp + o8, fb, f_ax, sb, sstr, gx,
                                                   gyp, i0 + o8, rel);
            else
              epilogue_fast8<L + 1, TO, false, true, TFM>(taddr + o8, (uint32_t)R, ebase, rexp + o8, fb, f_ax, sb, sstr, gx,
                                                    gyp, i0 + o8, rel);
          }
        } else if (__all_sync(0xffffffffu, safe)) {
#pragma unroll 1
          for (int gq = 0; gq < ng; ++gq) {
            const int o8 = gq * 8;
            epilogue_rows<8, L + 1, TO, false, TFM>(taddr + o8, (uint32_t)R, ebase, bad, rexp + o8, fb, f_ax, sb, sstr,
                                                    wf, ws, i0 + o8, gq == ng - 1 ? t_empty(tb) : 0u, vec, gx, gyp);
          }
        } else {
#pragma unroll 1
          for (int gq = 0; gq < ng; ++gq) {
            const int o8 = gq * 8;
            epilogue_rows<8, L + 1, TO, true, TFM>(taddr + o8, (uint32_t)R, ebase, bad, rexp + o8, fb, f_ax, sb, sstr,
                                                   wf, ws, i0 + o8, gq == ng - 1 ? t_empty(tb) : 0u, vec, gx, gyp);
          }
        }
      }
    }
  }

  if (failed) atomicExch(P.status, (int)CFD_ERR_TIMEOUT);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <typename TI, typename TO, int KP>
cfd_status launch_kp(const DenseParams &P, int S, int L, size_t smem, unsigned grid, cudaStream_t st) {
  void (*fn)(const __grid_constant__ DenseParams);
  const bool it = P.halo_in != nullptr;
  // the exact slices' closed passes whose last K chunk is all padding split the last real one,
  // except in the stages that also write an intermediate (measured 1-3 % slower there, 3 %
  // faster in the others)
  const bool spl = !it && P.scratch_out == nullptr && P.kext > KP - 16 && P.kext <= KP - 8;
  if (S == 5 && L == 4)
    fn = it ? k_dense<TI, TO, KP, 5, 4, 0, true, false>
            : (spl ? k_dense<TI, TO, KP, 5, 4, 0, false, true> : k_dense<TI, TO, KP, 5, 4, 0, false, false>);
  else if (S == 2 && L == 1) fn = it ? k_dense<TI, TO, KP, 2, 1, 0, true, false> : k_dense<TI, TO, KP, 2, 1, 0, false, false>;
  else if (S == 1 && L == 0) fn = it ? k_dense<TI, TO, KP, 1, 0, 1, true, false> : k_dense<TI, TO, KP, 1, 0, 1, false, false>;
  else { set_error("dense: unsupported slice configuration"); return CFD_ERR_UNSUPPORTED; }
  // The shared-memory opt-in is set once per device and instantiation (and raised when a
  // launch needs more), so that later calls issue nothing but the launch: a stream being
  // captured into a CUDA graph sees only kernel nodes.
  static size_t opted[7][64] = {};  // [slice configuration, iterated or split][device]
  const int v = (S == 5 ? 0 : (S == 2 ? 1 : 2)) + (it ? 3 : 0) + (S == 5 && spl ? 6 : 0);
  int dev = 0;
  cfd_status s = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
  if (s != CFD_OK) return s;
  if (dev < 0 || dev >= 64 || opted[v][dev] < smem) {
    s = cuda_fail(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                  "cudaFuncSetAttribute");
    if (s != CFD_OK) return s;
    if (dev >= 0 && dev < 64) opted[v][dev] = smem;
  }
  launch_begin(KF_DENSE, st);
  DenseParams Q = P;
  Q.wait_limit = dense_wait_limit();
  Q.inv_tpj = 1.0f / (float)Q.tiles_per_job;
  Q.inv_nf = 1.0f / (float)Q.nf;
  Q.inv_n2 = 1.0f / (float)Q.n2;
  fn<<<grid, kThreads, smem, st>>>(Q);
  launch_end(KF_DENSE, st);
  return cuda_fail(cudaGetLastError(), "k_dense launch");
}

template <typename TI, typename TO>
cfd_status launch_types(const DenseParams &P, int KP, int S, int L, size_t smem, unsigned grid, cudaStream_t st) {
  switch (KP) {
    case 32: return launch_kp<TI, TO, 32>(P, S, L, smem, grid, st);
    case 48: return launch_kp<TI, TO, 48>(P, S, L, smem, grid, st);
    default: set_error("dense: N + 2 ng must be 17..48"); return CFD_ERR_UNSUPPORTED;
  }
}

// ------------------------------------------------------------------ host planning

struct DenseOp {        // one (group, axis, degree) operator
  uint16_t *img = nullptr;    // device: kS x N x Kp digits
  uint32_t *img32 = nullptr;  // device: N x Kp TF32 values (the one-product TF32 form)
  int *rowexp = nullptr;      // device: N
  const void *image(bool tf32) const { return tf32 ? (const void *)img32 : (const void *)img; }
};

struct DenseGroup {
  int N = 0, Kp = 0;
  bool ok = false;
  bool iter_ok = false;  // iterated images built (E + 4 <= Kp)
  bool cyc[3] = {false, false, false};
  DenseOp op[3][2];      // [axis box index z,y,x][degree-1]: closed operator [0]D, dx-scaled
  DenseOp opI[3][2];     // iterated operator [D1 | c- | c+] with halo columns, dx-scaled
  // rows 1 and N-2 per degree of [0]D and of the iterated operator (unscaled), for the halo
  // passes on the CUDA cores
  HaloRows hr0[3], hrI[3];
  int *d_nl = nullptr;   // device [nblk][4]: local indices of the x-, x+, y-, y+ neighbours (-1: none)
  // blocks of the group without a same-size, reciprocal face neighbour on side x-, x+, y-, y+:
  // global ids and local indices (device), for the strips of intermediates they compute
  // themselves (their neighbours cannot write those ghost columns)
  int nmiss[4] = {0, 0, 0, 0};
  int *d_miss_b[4] = {nullptr, nullptr, nullptr, nullptr};
  int *d_miss_l[4] = {nullptr, nullptr, nullptr, nullptr};
  // biased first-degree operators ([box][0 left-biased S+, 1 right-biased S-]), dx-scaled:
  // closed (or cyclic) [0]D, iterated [D1 | coupling in halo column E (S+) or E+3 (S-)];
  // halo images (unscaled): row 1 = S+ row N-kc, row 2 = S- row kc-1
  bool biased = false;
  DenseOp bop[3][2], bopI[3][2];
  HaloRows bhr0[3], bhrI[3];
};

// Launch choices of the autotuner: per request (fields, ops, precision, iterations, entry
// point) and per launch of it, the staging of the input tiles (0 TMA where the tile is a box,
// 1 cp.async) and the tile order (0 interleaved, 1 contiguous runs), with the times measured.
struct TuneRec {
  int staging = 0, order = 0;
  float ms[4] = {-1, -1, -1, -1};  // [staging * 2 + order]
  std::string stage;
};
struct DenseState {
  std::vector<DenseGroup> groups;
  std::map<std::string, std::vector<TuneRec>> tuned;
  bool tuning = false;             // cfd_autotune in progress: every launch tries its candidates
  std::string key;                 // the request of the current call
  int launch = 0;                  // launches of the current call so far
};

DenseState *state_of(cfd_blocks_s *B) { return reinterpret_cast<DenseState *>(B->dense_state); }

}  // namespace

static cfd_status upload_op(cfd_blocks_s *B, const std::vector<ld> &D, int rows, int cols, int Kp, DenseOp &o) {
  std::vector<uint16_t> img;
  std::vector<uint32_t> img32;
  std::vector<int> rexp;
  digit_image(D, rows, cols, Kp, img, rexp);
  tf32_image(D, rows, cols, Kp, img32);
  cfd_status s = cuda_fail(cudaMalloc((void **)&o.img, img.size() * 2), "cudaMalloc");
  if (s == CFD_OK) s = cuda_fail(cudaMemcpy(o.img, img.data(), img.size() * 2, cudaMemcpyHostToDevice), "cudaMemcpy");
  if (s == CFD_OK) s = cuda_fail(cudaMalloc((void **)&o.img32, img32.size() * 4), "cudaMalloc");
  if (s == CFD_OK)
    s = cuda_fail(cudaMemcpy(o.img32, img32.data(), img32.size() * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  if (o.img32) B->d_dense_ptrs.push_back(o.img32);
  if (s == CFD_OK) s = cuda_fail(cudaMalloc((void **)&o.rowexp, rexp.size() * 4), "cudaMalloc");
  if (s == CFD_OK) s = cuda_fail(cudaMemcpy(o.rowexp, rexp.data(), rexp.size() * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  if (o.img) B->d_dense_ptrs.push_back(o.img);
  if (o.rowexp) B->d_dense_ptrs.push_back(o.rowexp);
  return s;
}

cfd_status dense_bind(cfd_blocks_s *B) {
  // The dense state lives in host memory; its device images are freed with the handle.
  DenseState *st = new (std::nothrow) DenseState();
  if (!st) { set_error("out of host memory"); return CFD_ERR_ALLOC; }
  B->dense_state = st;
  B->dense_free = [](void *p) { delete reinterpret_cast<DenseState *>(p); };
  const int g = B->ng;
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    DenseGroup G;
    G.N = B->sizes[gi];
    const int N = G.N, E = N + 2 * g;
    G.Kp = (E + 15) / 16 * 16;
    G.ok = G.Kp <= 48 && (N == 16 || N == 32);
    G.iter_ok = G.ok && E + 4 <= G.Kp;
    const int b0 = B->groups[gi][0];
    for (int b : B->groups[gi])
      for (int a = 0; a < 3; ++a)
        if (B->dx[b * 3 + a] != B->dx[b0 * 3 + a]) G.ok = false;
    for (int box = 0; box < 3 && G.ok; ++box) {
      const int ax = 2 - box;  // dx index (x, y, z)
      // cyclic along this axis if every block of the group is its own neighbour on both faces
      int ncyc = 0;
      const int ez = box == 0, ey = box == 1, ex = box == 2;
      for (int b : B->groups[gi]) {
        auto di = [](int dz, int dy, int dx) { int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1); return r > 13 ? r - 1 : r; };
        const int lo = B->nbr[b * 26 + di(-ez, -ey, -ex)], hi = B->nbr[b * 26 + di(ez, ey, ex)];
        if (lo == b && hi == b) ++ncyc;
      }
      const bool cyc = ncyc == (int)B->groups[gi].size();
      if (ncyc && !cyc) { G.ok = false; break; }
      G.cyc[box] = cyc;
      std::vector<ld> H0(16 * E, 0), HI(16 * G.Kp, 0);
      for (int d = 1; d <= 2; ++d) {
        if (!B->s[d - 1].present) continue;
        const ld h = B->dx[b0 * 3 + ax];
        const ld scale = 1.0L / (d == 1 ? h : h * h);
        std::vector<ld> D;
        if (cyc) cyclic_operator(B->s[d - 1], N, g, scale, D);
        else closed_operator(B->s[d - 1], N, g, scale, D);
        cfd_status s = upload_op(B, D, N, E, G.Kp, G.op[box][d - 1]);
        if (s != CFD_OK) return s;
        if (cyc || !G.iter_ok) continue;
        // closed operator without dx scaling: rows 1 and N-2 feed the first halo pass
        std::vector<ld> D0;
        closed_operator(B->s[d - 1], N, g, 1.0L, D0);
        for (int j = 0; j < E; ++j) {
          H0[(2 * (d - 1)) * E + j] = D0[1 * E + j];
          H0[(2 * (d - 1) + 1) * E + j] = D0[(N - 2) * E + j];
        }
        std::vector<ld> D1, cm, cp;
        iterated_operator(B->s[d - 1], N, g, D1, cm, cp);
        const int hc = E + 2 * (d - 1);  // halo columns of this degree
        std::vector<ld> F(N * G.Kp, 0);
        for (int i = 0; i < N; ++i) {
          for (int j = 0; j < E; ++j) F[i * G.Kp + j] = D1[i * E + j] * scale;
          F[i * G.Kp + hc] = cm[i] * scale;
          F[i * G.Kp + hc + 1] = cp[i] * scale;
        }
        if ((s = upload_op(B, F, N, G.Kp, G.Kp, G.opI[box][d - 1])) != CFD_OK) return s;
        const int rows[2] = {1, N - 2};
        for (int w = 0; w < 2; ++w) {
          const int r = 2 * (d - 1) + w, i = rows[w];
          for (int j = 0; j < E; ++j) HI[r * G.Kp + j] = D1[i * E + j];
          HI[r * G.Kp + hc] = cm[i];
          HI[r * G.Kp + hc + 1] = cp[i];
        }
      }
      if (!cyc && G.iter_ok) {
        halo_rows_from(H0, E, G.hr0[box]);
        halo_rows_from(HI, G.Kp, G.hrI[box]);
      }
      if (B->biased.present && B->biased.kc <= N) {
        const BiasedCoef &bc = B->biased;
        const ld scale = 1.0L / (ld)B->dx[b0 * 3 + ax];
        std::vector<ld> W, cp, BH0(16 * E, 0), BHI(16 * G.Kp, 0);
        for (int side = 0; side < 2; ++side) {
          const int sg = side == 0 ? 1 : -1;
          biased_operator(bc, N, g, sg, cyc ? 2 : 0, W, cp);
          std::vector<ld> D(W);
          for (auto &v : D) v *= scale;
          cfd_status s = upload_op(B, D, N, E, G.Kp, G.bop[box][side]);
          if (s != CFD_OK) return s;
          if (cyc || !G.iter_ok) continue;
          const int krow = sg > 0 ? N - bc.kc : bc.kc - 1;
          for (int j = 0; j < E; ++j) BH0[(1 + side) * E + j] = W[(size_t)krow * E + j];
          biased_operator(bc, N, g, sg, 1, W, cp);
          const int hcol = side == 0 ? E : E + 3;   // halo column the kernel fills for this side
          std::vector<ld> F((size_t)N * G.Kp, 0);
          for (int i = 0; i < N; ++i) {
            for (int j = 0; j < E; ++j) F[(size_t)i * G.Kp + j] = W[(size_t)i * E + j] * scale;
            F[(size_t)i * G.Kp + hcol] = cp[i] * scale;
          }
          if ((s = upload_op(B, F, N, G.Kp, G.Kp, G.bopI[box][side])) != CFD_OK) return s;
          for (int j = 0; j < E; ++j) BHI[(size_t)(1 + side) * G.Kp + j] = W[(size_t)krow * E + j];
          BHI[(size_t)(1 + side) * G.Kp + hcol] = cp[krow];
        }
        if (!cyc && G.iter_ok) {
          halo_rows_from(BH0, E, G.bhr0[box]);
          halo_rows_from(BHI, G.Kp, G.bhrI[box]);
        }
        G.biased = true;
      }
    }
    st->groups.push_back(G);
  }
  std::vector<int> lidx(B->nblocks, 0), gidx(B->nblocks, -1);
  for (size_t gi = 0; gi < B->groups.size(); ++gi)
    for (size_t k = 0; k < B->groups[gi].size(); ++k) {
      lidx[B->groups[gi][k]] = (int)k;
      gidx[B->groups[gi][k]] = (int)gi;
    }
  for (size_t gi = 0; gi < B->groups.size(); ++gi) {
    DenseGroup &G = st->groups[gi];
    if (!G.ok) continue;
    auto di = [](int dz, int dy, int dx) { int r = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1); return r > 13 ? r - 1 : r; };
    const std::vector<int> &gb = B->groups[gi];
    // per block and side: the local index of a same-group, reciprocal face neighbour, or -1
    const int sdy[4] = {0, 0, -1, 1}, sdx[4] = {-1, 1, 0, 0};
    std::vector<int> nl(gb.size() * 4, -1);
    std::vector<int> mb[4], ml[4];
    for (size_t k = 0; k < gb.size(); ++k) {
      const int b = gb[k];
      for (int sd = 0; sd < 4; ++sd) {
        const int nb = B->nbr[b * 26 + di(0, sdy[sd], sdx[sd])];
        const bool ok = nb >= 0 && gidx[nb] == (int)gi && B->nbr[nb * 26 + di(0, -sdy[sd], -sdx[sd])] == b;
        if (ok) {
          nl[k * 4 + sd] = lidx[nb];
        } else {
          mb[sd].push_back(b);
          ml[sd].push_back((int)k);
        }
      }
    }
    cfd_status s = cuda_fail(cudaMalloc((void **)&G.d_nl, nl.size() * 4), "cudaMalloc");
    if (G.d_nl) B->d_dense_ptrs.push_back(G.d_nl);
    if (s == CFD_OK) s = cuda_fail(cudaMemcpy(G.d_nl, nl.data(), nl.size() * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
    for (int sd = 0; sd < 4 && s == CFD_OK; ++sd) {
      G.nmiss[sd] = (int)mb[sd].size();
      if (mb[sd].empty()) continue;
      s = cuda_fail(cudaMalloc((void **)&G.d_miss_b[sd], mb[sd].size() * 4), "cudaMalloc");
      if (G.d_miss_b[sd]) B->d_dense_ptrs.push_back(G.d_miss_b[sd]);
      if (s == CFD_OK) s = cuda_fail(cudaMalloc((void **)&G.d_miss_l[sd], ml[sd].size() * 4), "cudaMalloc");
      if (G.d_miss_l[sd]) B->d_dense_ptrs.push_back(G.d_miss_l[sd]);
      if (s == CFD_OK)
        s = cuda_fail(cudaMemcpy(G.d_miss_b[sd], mb[sd].data(), mb[sd].size() * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
      if (s == CFD_OK)
        s = cuda_fail(cudaMemcpy(G.d_miss_l[sd], ml[sd].data(), ml[sd].size() * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    if (s != CFD_OK) return s;
  }
  return CFD_OK;
}

namespace {

// Digit slices S of the inputs and the highest level L kept: exact mode five slices and levels
// 0..4 (15 slice pairs), for FP32 fields too -- four slices and levels 0..3 measured ~1e-6 on
// second derivatives at fine spacing (the truncated fifth operator digit acts coherently on
// smooth data), ten times the FP32 rounding of the outputs.
int slices_of(cfd_precision p, int) { return p == CFD_TC_BF16_EXACT ? 5 : (p == CFD_TC_TF32 ? 1 : 2); }
int levels_of(cfd_precision p, int) { return p == CFD_TC_BF16_EXACT ? 4 : (p == CFD_TC_TF32 ? 0 : 1); }
bool tc_precision(cfd_precision p) { return p == CFD_TC_BF16_EXACT || p == CFD_TC_BF16X3 || p == CFD_TC_TF32; }

// Shared memory per CTA: two A digit buffers, B digits of two passes, the
// input staging tile, row exponents, exponent exchange, etau ring, barriers.  At least 116 KB so that
// one CTA (holding all 512 TMEM columns) occupies an SM.
size_t dense_smem(int KP, int S, int rows, size_t elem, int tma_boxes) {
  const size_t eb = S == 1 ? 4 : 2;  // TF32 or BF16 operands
  const size_t ab = 2 * (size_t)S * kTile * KP * eb + 2 * (size_t)S * rows * KP * eb;
  const size_t stg = std::max((size_t)kTile * (KP + 16 / elem) * elem, (size_t)tma_boxes * kTile * 128);
  const size_t need = ((ab + kBiasBytes + 1023) & ~(size_t)1023) + stg + (2 * 48 + 2 * kParts * kTile + 8 * kTile) * 4 +
                      24 * 8 + 64;
  return std::max(need, (size_t)116 * 1024);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// TMA staging for a stage whose 128-pencil tiles are boxes of the input: pencils along x
// (x rows, 128-byte swizzled boxes) or along y / z (one box of the whole columns).  Falls
// back to the cp.async path (tma_kind 0) when a box or alignment rule does not hold.
void plan_tma(DenseParams &P, size_t elem) {
  P.tma_kind = 0;
  P.tma_boxes = 0;
  // An iterated pass (halo_in) takes kext = E + 4 values per pencil: the boxes cover kext along
  // the pencil axis, and the producers write the 4 halo columns into the staged tile.
  const int n2 = P.n2, E = P.N + 2 * P.g, K = P.kext;
  if ((n2 != 16 && n2 != 32) || (P.n1 * n2) % kTile != 0) return;
  if (P.in_field && !P.contig) return;
  const int d0 = P.in_dims[0], d1 = P.in_dims[1], d2 = P.in_dims[2];
  if (P.in_dims[P.axis] != E) return;
  const char *base = static_cast<const char *>(P.in) + (P.in_field ? (size_t)P.nf * P.ext0 * elem : 0);
  if (((uintptr_t)base & 15) || ((size_t)d2 * elem) % 16 || ((size_t)d1 * d2 * elem) % 16) return;
  if (((size_t)P.in_start[2] * elem) % 16) return;
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return;
  const int njobs = P.nblk * P.nf;
  const cuuint64_t gdim[3] = {(cuuint64_t)d2, (cuuint64_t)d1, (cuuint64_t)d0 * njobs};
  const cuuint64_t gstr[2] = {(cuuint64_t)d2 * elem, (cuuint64_t)d1 * d2 * elem};
  const cuuint32_t estr[3] = {1, 1, 1};
  cuuint32_t box[3];
  int kind, boxes;
  CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE;
  const int xb = (int)(128 / elem);
  if (P.axis == 2) {  // t1 = z, t2 = y
    kind = 1;
    boxes = (K + xb - 1) / xb;
    box[0] = (cuuint32_t)xb; box[1] = (cuuint32_t)n2; box[2] = (cuuint32_t)(kTile / n2);
    swz = CU_TENSOR_MAP_SWIZZLE_128B;
  } else if (P.axis == 1) {  // t1 = z, t2 = x
    kind = 2;
    boxes = 1;
    box[0] = (cuuint32_t)n2; box[1] = (cuuint32_t)K; box[2] = (cuuint32_t)(kTile / n2);
  } else {  // t1 = y, t2 = x
    kind = 3;
    boxes = 1;
    box[0] = (cuuint32_t)n2; box[1] = (cuuint32_t)(kTile / n2); box[2] = (cuuint32_t)K;
  }
  const CUtensorMapDataType dt = elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (enc(&P.tmap, dt, 3, const_cast<char *>(base), gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return;
  P.tma_kind = kind;
  P.tma_boxes = boxes;
  P.tma_bytes = (int)(box[0] * box[1] * box[2] * elem) * boxes;
  P.tma_zstep = d0;
}

// Launch one stage with the choices the autotuner made for it (TMA staging and interleaved
// tiles by default); during cfd_autotune, launch every candidate three times, time the last two
// with events on the stream, and keep the fastest.  Repeated launches of a stage are idempotent
// (a stage never reads what it writes), and every candidate computes the same outputs.
cfd_status launch_stage(DenseState *ds, const DenseParams &P, int KP, int S, int L, size_t ein, bool f32,
                        unsigned grid, cudaStream_t st) {
  auto launch = [&](const DenseParams &Q) -> cfd_status {
    const size_t smem = dense_smem(KP, S, Q.rows, ein, Q.tma_boxes);
    if (!Q.in_field)
      return f32 ? launch_types<double, float>(Q, KP, S, L, smem, grid, st)
                 : launch_types<double, double>(Q, KP, S, L, smem, grid, st);
    return f32 ? launch_types<float, float>(Q, KP, S, L, smem, grid, st)
               : launch_types<double, double>(Q, KP, S, L, smem, grid, st);
  };
  auto configure = [&](int staging, int order) {
    DenseParams Q = P;
    Q.tile_order = order;
    Q.tiles_per_cta = (Q.ntiles + (int)grid - 1) / (int)grid;
    if (staging == 0) plan_tma(Q, ein);
    else { Q.tma_kind = 0; Q.tma_boxes = 0; }
    return Q;
  };
  const int idx = ds->launch++;
  std::vector<TuneRec> &recs = ds->tuned[ds->key];
  if (!ds->tuning) {
    const bool have = idx < (int)recs.size();
    return launch(configure(have ? recs[idx].staging : 0, have ? recs[idx].order : 0));
  }
  if ((int)recs.size() <= idx) recs.resize(idx + 1);
  TuneRec &r = recs[idx];
  const char axis = "zyx"[P.axis];
  r.stage = std::string(P.in_field ? "S_" : "T_") + axis;
  const int nstaging = configure(0, 0).tma_kind ? 2 : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cfd_status s = cuda_fail(cudaEventCreate(&e0), "cudaEventCreate");
  if (s == CFD_OK) s = cuda_fail(cudaEventCreate(&e1), "cudaEventCreate");
  float best = 1e30f;
  for (int stg = 0; stg < nstaging && s == CFD_OK; ++stg)
    for (int ord = 0; ord < 2 && s == CFD_OK; ++ord) {
      const DenseParams Q = configure(stg, ord);
      s = launch(Q);
      if (s == CFD_OK) s = cuda_fail(cudaEventRecord(e0, st), "cudaEventRecord");
      for (int k = 0; k < 2 && s == CFD_OK; ++k) s = launch(Q);
      if (s == CFD_OK) s = cuda_fail(cudaEventRecord(e1, st), "cudaEventRecord");
      if (s == CFD_OK) s = cuda_fail(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0;
      if (s == CFD_OK) s = cuda_fail(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (s != CFD_OK) break;
      r.ms[stg * 2 + ord] = ms / 2;
      if (ms < best) { best = ms; r.staging = stg; r.order = ord; }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return s;
}

}  // namespace

struct DensePlanSizes {
  size_t gy = 0, gz = 0;  // elements per group (max over groups) of the two intermediates
  size_t halo = 0;        // elements of one halo buffer (two are used, ping-pong)
};

static size_t bytes256(size_t elems) { return (elems * 8 + 255) & ~(size_t)255; }

static DensePlanSizes dense_sizes(const cfd_blocks_s *B, int nf, unsigned mask, int n_iter) {
  DensePlanSizes z;
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const size_t N = B->sizes[gi], E = N + 2 * B->ng, nb = B->groups[gi].size();
    if (mask & CFD_OP_DXY) z.gy = std::max(z.gy, nb * nf * N * N * E);
    if (mask & (CFD_OP_DXZ | CFD_OP_DYZ)) z.gz = std::max(z.gz, nb * nf * N * E * E);
    // halo values are indexed by global block id and the pencil of the stage (at most E^2 pencils)
    if (n_iter > 0) z.halo = std::max(z.halo, (size_t)B->nblocks * nf * E * E * 4);
  }
  return z;
}

cfd_status dense_workspace(cfd_blocks_s *B, int nf, unsigned mask, cfd_precision prec, int n_iter, size_t *bytes) {
  if (!tc_precision(prec)) {
    set_error("unknown precision");
    return CFD_ERR_ARG;
  }
  const DensePlanSizes z = dense_sizes(B, nf, mask, n_iter);
  *bytes = bytes256(z.gy) + bytes256(z.gz) + 2 * bytes256(z.halo) + 256;
  return CFD_OK;
}

cfd_status dense_apply(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, cfd_precision prec, int n_iter,
                       void *out, void *work, size_t work_bytes, cudaStream_t st) {
  size_t need = 0;
  cfd_status s = dense_workspace(B, nf, mask, prec, n_iter, &need);
  if (s != CFD_OK) return s;
  if (need > 256 && (!work || work_bytes < need)) {
    set_error("dense: workspace too small (see cfd_apply_workspace)");
    return CFD_ERR_ARG;
  }
  DenseState *ds = state_of(B);
  if (!ds) { set_error("dense: operators were not built at bind"); return CFD_ERR_UNSUPPORTED; }
  ds->key = "apply nf=" + std::to_string(nf) + " ops=" + std::to_string(mask) + " prec=" + std::to_string((int)prec) +
            " n_iter=" + std::to_string(n_iter);
  ds->launch = 0;
  const int S = slices_of(prec, B->dtype), L = levels_of(prec, B->dtype);
  const DensePlanSizes z = dense_sizes(B, nf, mask, n_iter);
  double *gy = (double *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  double *gz = gy + bytes256(z.gy) / 8;
  double *halo[2] = {gz + bytes256(z.gz) / 8, gz + bytes256(z.gz) / 8 + bytes256(z.halo) / 8};
  int bits[9], nops = 0;
  for (int i = 0; i < 9; ++i)
    if (mask & (1u << i)) bits[nops++] = i;
  auto opidx_of = [&](int bit) {
    for (int i = 0; i < nops; ++i)
      if (bits[i] == bit) return i;
    return -1;
  };
  const bool need1 = (mask & (CFD_OP_DX | CFD_OP_DY | CFD_OP_DZ | CFD_OP_DXY | CFD_OP_DXZ | CFD_OP_DYZ)) != 0;
  const bool need2 = (mask & (CFD_OP_DXX | CFD_OP_DYY | CFD_OP_DZZ)) != 0;
  if ((need1 && !B->s[0].present) || (need2 && !B->s[1].present)) {
    set_error("op needs a scheme that was not given");
    return CFD_ERR_ARG;
  }
  const int sms = B->num_sms > 0 ? B->num_sms : 148;
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const DenseGroup &G = ds->groups[gi];
    if (!G.ok) {
      set_error("dense: block group unsupported (N must be 16 or 32, uniform spacing, consistent cyclic axes)");
      return CFD_ERR_UNSUPPORTED;
    }
    const int N = G.N, g = B->ng, E = N + 2 * g;
    if (n_iter > 0 && !G.iter_ok) {
      set_error("dense: hybrid iteration needs N + 2 ng + 4 <= the padded K of the block size");
      return CFD_ERR_UNSUPPORTED;
    }
    DenseParams base;
    memset(&base, 0, sizeof(base));
    base.blocks = B->d_groups[gi];
    base.extpre = B->d_extpre;
    base.intpre = B->d_intpre;
    base.nblk = (int)B->groups[gi].size();
    base.nf = nf;
    base.nops = nops;
    base.N = N;
    base.g = g;
    base.status = B->d_status;
    base.out = out;
    base.seg_rows = N;
    base.kext = E;
    {
      const std::vector<int> &gb = B->groups[gi];
      bool contig = true;
      for (size_t k = 0; k < gb.size(); ++k)
        if (gb[k] != gb[0] + (int)k) contig = false;
      base.contig = contig ? 1 : 0;
      base.b0 = gb[0];
      base.ext0 = B->extpre[gb[0]];
      base.int0 = B->intpre[gb[0]];
    }
    base.nbr = B->d_nbr;
    base.halo_deg_mask = (B->s[0].present ? 1 : 0) | (B->s[1].present ? 2 : 0);
    // the intermediates and halo values are FP64 for every field dtype
    auto run = [&](DenseParams P) -> cfd_status {
      const int np = P.n1 * P.n2;
      const bool f32 = B->dtype == CFD_F32;
      const size_t ein = (P.in_field && f32) ? 4 : 8, eout = f32 ? 4 : 8;
      P.xrow = P.axis == 2 && (E * ein) % 16 == 0 && ((uintptr_t)P.in & 15) == 0;
      P.xvec = P.axis == 2 && (N * eout) % 16 == 0 && ((uintptr_t)P.out & 15) == 0;
      P.tiles_per_job = (np + kTile - 1) / kTile;
      P.ntiles = P.tiles_per_job * P.nblk * P.nf;
      const unsigned grid = (unsigned)std::min(P.ntiles, sms);
      return launch_stage(ds, P, G.Kp, S, L, ein, f32, grid, st);
    };
    // segments: (degree, mode, op); passes of at most 32 rows
    auto iterating = [&](int box) { return n_iter > 0 && !G.cyc[box]; };
    auto set_segments = [&](DenseParams &P, int box, int m1, int op1, int m2, int op2) {
      int deg[2], mode[2], op[2], n = 0;
      if (m1 >= 0) { deg[n] = 1; mode[n] = m1; op[n] = op1; ++n; }
      if (m2 >= 0) { deg[n] = 2; mode[n] = m2; op[n] = op2; ++n; }
      const int per_pass = (n * N <= 32) ? n : 1;
      P.passes = n / per_pass;
      P.rows = per_pass * N;
      for (int ps = 0; ps < P.passes; ++ps) {
        P.nseg[ps] = per_pass;
        for (int k = 0; k < per_pass; ++k) {
          const int sgi = ps * per_pass + k;
          const DenseOp &o = iterating(box) ? G.opI[box][deg[sgi] - 1] : G.op[box][deg[sgi] - 1];
          P.seg_img[ps][k] = o.image(prec == CFD_TC_TF32);
          P.seg_exp[ps][k] = o.rowexp;
          P.seg_mode[ps][k] = mode[sgi];
          P.seg_op[ps][k] = op[sgi];
        }
      }
      return n > 0;
    };
    // A stage along a decomposed axis with n_iter > 0 (Eq. iter_center_P): halo
    // passes compute rows 1 and N-2 of every block's iterate [0], [1], ...
    // [n_iter-1] (the values the neighbours need at their k^c nodes) into a
    // ping-pong buffer; the final pass applies the iterated operator with
    // those values as four extra K columns.  Each pass is one launch: all
    // blocks of iterate i are complete before any block reads them.  The halo
    // passes are four dot products per pencil and run on the CUDA cores in
    // compensated FP32 (halo_rows.cu), at a fraction of a tensor-core pass.
    auto run_stage = [&](DenseParams P, int box) -> cfd_status {
      if (!iterating(box)) return run(P);
      DenseParams H = P;
      H.scratch_out = nullptr;
      for (int it = 0; it < n_iter; ++it) {
        H.halo_in = it == 0 ? nullptr : halo[(it - 1) & 1];
        H.halo_out = halo[it & 1];
        H.kext = it == 0 ? E : E + 4;
        cfd_status r = halo_rows_launch(H, it == 0 ? G.hr0[box] : G.hrI[box],
                                        H.in_field && B->dtype == CFD_F32, st);
        if (r != CFD_OK) return r;
      }
      P.halo_in = halo[(n_iter - 1) & 1];
      P.kext = E + 4;
      return run(P);
    };
    auto field_stage = [&](int box, int t1, int t2, int lo1, int n1, int lo2, int n2) {
      DenseParams P = base;
      P.in = fields;
      P.in_field = 1;
      P.axis = box;
      P.t1 = t1;
      P.t2 = t2;
      for (int t = 0; t < 3; ++t) P.in_dims[t] = E;
      P.in_start[box] = 0;
      P.in_start[t1] = lo1;
      P.in_start[t2] = lo2;
      P.n1 = n1;
      P.n2 = n2;
      // final outputs: pencils whose transverse coordinates are interior
      P.int_lo1 = g - lo1; P.int_hi1 = g - lo1 + N;
      P.int_lo2 = g - lo2; P.int_hi2 = g - lo2 + N;
      return P;
    };
    const int odx = opidx_of(0), ody = opidx_of(1), odz = opidx_of(2);
    const int odxx = opidx_of(3), odyy = opidx_of(4), odzz = opidx_of(5);
    const int odxy = opidx_of(6), odxz = opidx_of(7), odyz = opidx_of(8);
    // S_x: D_x on interior (z, y) pencils -> d_x, d_xx
    if (odx >= 0 || odxx >= 0) {
      DenseParams P = field_stage(2, 0, 1, g, N, g, N);
      set_segments(P, 2, odx >= 0 ? 0 : -1, odx, odxx >= 0 ? 0 : -1, odxx);
      if ((s = run_stage(P, 2)) != CFD_OK) return s;
    }
    // Intermediates for the mixed derivatives: G_y = D_y f on the x-extended (z, x) pencils,
    // G_z = D_z f on the x- and y-extended (y, x) pencils (not the corners).  Each block
    // computes its interior pencils; the epilogue also writes each value within g of an x (y)
    // face into the face neighbour's ghost column (row), which is what local evaluation there
    // would give (same input data, same arithmetic).  A block without a same-size face
    // neighbour on a side computes that strip of ghost pencils itself, in a small launch over
    // the blocks missing that side.  (Blocks narrower than 2g take the extended pencils
    // directly.)
    auto strip = [&](DenseParams P, int sd, int lo1, int n1, int lo2, int n2) -> cfd_status {
      if (G.nmiss[sd] == 0) return CFD_OK;
      P.blocks = G.d_miss_b[sd];
      P.sc_local = G.d_miss_l[sd];
      P.nblk = G.nmiss[sd];
      P.contig = 0;
      P.in_start[P.t1] = lo1;
      P.in_start[P.t2] = lo2;
      P.n1 = n1;
      P.n2 = n2;
      P.sc_start[P.t2] = lo2;              // the x axis: scratch and input coordinates agree
      if (P.t1 == 1) P.sc_start[1] = lo1;  // the y axis of G_z likewise (z of G_y is interior only)
      P.ghost_x = P.ghost_y = 0;
      P.int_lo1 = P.int_hi1 = P.int_lo2 = P.int_hi2 = 0;
      set_segments(P, P.axis, 2, 0, -1, -1);  // the degree-1 operator, intermediate only
      return run(P);
    };
    // S_y: D_y on (z interior, x interior) -> d_y, d_yy, and G_y for d_xy
    if (ody >= 0 || odyy >= 0 || odxy >= 0) {
      const bool ext = odxy >= 0;
      const bool copy = ext && N >= 2 * g;  // interior pencils + ghost columns from the epilogue
      DenseParams P = field_stage(1, 0, 2, g, N, (ext && !copy) ? 0 : g, (ext && !copy) ? E : N);
      const int m1 = (ody >= 0 && ext) ? 3 : (ody >= 0 ? 0 : (ext ? 2 : -1));
      set_segments(P, 1, m1, ody, odyy >= 0 ? 0 : -1, odyy);
      if (ext) {
        P.scratch_out = gy;
        P.sc_box = (unsigned long long)N * N * E;
        P.sc_dims[0] = N; P.sc_dims[1] = N; P.sc_dims[2] = E;
        P.sc_start[0] = 0; P.sc_start[1] = 0; P.sc_start[2] = copy ? g : 0;
        P.ghost_x = copy ? 1 : 0;
        P.nl = G.d_nl;
      }
      if ((s = run_stage(P, 1)) != CFD_OK) return s;
      if (copy) {
        if ((s = strip(P, 0, g, N, 0, g)) != CFD_OK) return s;          // x- ghost columns
        if ((s = strip(P, 1, g, N, N + g, g)) != CFD_OK) return s;      // x+
      }
    }
    // S_z: D_z on (y, x) interior -> d_z, d_zz, and G_z for d_xz / d_yz
    if (odz >= 0 || odzz >= 0 || odxz >= 0 || odyz >= 0) {
      const bool ext = odxz >= 0 || odyz >= 0;
      const bool copy = ext && N >= 2 * g;
      const bool wide = ext && !copy;
      DenseParams P = field_stage(0, 1, 2, wide ? 0 : g, wide ? E : N, wide ? 0 : g, wide ? E : N);
      const int m1 = (odz >= 0 && ext) ? 3 : (odz >= 0 ? 0 : (ext ? 2 : -1));
      set_segments(P, 0, m1, odz, odzz >= 0 ? 0 : -1, odzz);
      if (ext) {
        P.scratch_out = gz;
        P.sc_box = (unsigned long long)N * E * E;
        P.sc_dims[0] = N; P.sc_dims[1] = E; P.sc_dims[2] = E;
        P.sc_start[0] = 0; P.sc_start[1] = copy ? g : 0; P.sc_start[2] = copy ? g : 0;
        P.ghost_x = P.ghost_y = copy ? 1 : 0;
        P.nl = G.d_nl;
      }
      if ((s = run_stage(P, 0)) != CFD_OK) return s;
      if (copy) {
        if ((s = strip(P, 0, g, N, 0, g)) != CFD_OK) return s;          // x- ghost columns
        if ((s = strip(P, 1, g, N, N + g, g)) != CFD_OK) return s;      // x+
        if ((s = strip(P, 2, 0, g, g, N)) != CFD_OK) return s;          // y- ghost rows
        if ((s = strip(P, 3, N + g, g, g, N)) != CFD_OK) return s;      // y+
      }
    }
    // T stages on the intermediates (one order of the mixed product: the closed
    // block operators of two axes commute, D_i D_j = D_j D_i)
    auto scratch_stage = [&](double *src, int d0, int d1, int d2, int box, int t1, int t2, int lo1, int lo2,
                             int op) {
      DenseParams P = base;
      P.in = src;
      P.in_field = 0;
      P.in_box = (unsigned long long)d0 * d1 * d2;
      P.in_dims[0] = d0; P.in_dims[1] = d1; P.in_dims[2] = d2;
      P.axis = box;
      P.t1 = t1;
      P.t2 = t2;
      P.in_start[box] = 0;
      P.in_start[t1] = lo1;
      P.in_start[t2] = lo2;
      P.n1 = N;
      P.n2 = N;
      P.int_lo1 = 0; P.int_hi1 = N; P.int_lo2 = 0; P.int_hi2 = N;
      set_segments(P, box, 0, op, -1, -1);
      P.halo_deg_mask = 1;  // the mixed products apply the degree-1 operator only
      return run_stage(P, box);
    };
    if (odxy >= 0 && (s = scratch_stage(gy, N, N, E, 2, 0, 1, 0, 0, odxy)) != CFD_OK) return s;
    if (odxz >= 0 && (s = scratch_stage(gz, N, E, E, 2, 0, 1, 0, g, odxz)) != CFD_OK) return s;
    if (odyz >= 0 && (s = scratch_stage(gz, N, E, E, 1, 0, 2, 0, g, odyz)) != CFD_OK) return s;
  }
  return CFD_OK;
}

// ------------------------------------------------------------------ biased operators

static size_t interior_points(const cfd_blocks_s *B) {
  size_t t = 0;
  for (size_t gi = 0; gi < B->sizes.size(); ++gi)
    t += B->groups[gi].size() * (size_t)B->sizes[gi] * B->sizes[gi] * B->sizes[gi];
  return t;
}

size_t dense_biased_workspace(const cfd_blocks_s *B, int nf, int n_iter, bool advect) {
  const size_t elem = B->dtype == CFD_F32 ? 4 : 8;
  const DensePlanSizes z = dense_sizes(B, nf, 0, n_iter);
  return (advect ? ((interior_points(B) * nf * 6 * elem + 255) & ~(size_t)255) : 0) + 2 * bytes256(z.halo) + 256;
}

// Biased first derivatives on the tensor cores: mode 0 (S+) or 1 (S-) of the axes in `axes`
// into `out` (one op per axis); mode 2: both sides of every axis (one stage per axis) into the
// workspace, then the upwind blend (advect_combine) into slot out_opidx of out_nops in `out`.
// (Blending in the k_dense epilogue instead reads the shift twice per axis and adds a
// read-modify-write of the output to the epilogue; measured slower, 9.5 vs 5.7 ms at 256^3.)
// The operators are
// the dense forms of the block systems of Eqs. closure_left_X / iter_left_X (bind time); the
// iteration runs the halo passes of the centred path (k_halo_rows) with the biased halo rows
// (slot 1: S+ at row N-kc, read by the upper neighbour; slot 2: S- at row kc-1, read by the
// lower one).
cfd_status dense_biased(cfd_blocks_s *B, const void *fields, int nf, const void *beta, const int *axes, int naxes,
                        int mode, cfd_precision prec, int n_iter, void *out, int out_nops, int out_opidx,
                        bool accum_all, void *work, size_t work_bytes, cudaStream_t st) {
  if (!tc_precision(prec)) {
    set_error("unknown precision");
    return CFD_ERR_ARG;
  }
  DenseState *ds = state_of(B);
  if (!ds) { set_error("dense: operators were not built at bind"); return CFD_ERR_UNSUPPORTED; }
  ds->key = "biased nf=" + std::to_string(nf) + " mode=" + std::to_string(mode) + " naxes=" + std::to_string(naxes) +
            " prec=" + std::to_string((int)prec) + " n_iter=" + std::to_string(n_iter);
  ds->launch = 0;
  const size_t need = dense_biased_workspace(B, nf, n_iter, mode == 2);
  if (!work || work_bytes < need) { set_error("biased path: workspace too small (see cfd_biased_workspace)"); return CFD_ERR_ARG; }
  const int S = slices_of(prec, B->dtype), L = levels_of(prec, B->dtype);
  const DensePlanSizes z = dense_sizes(B, nf, 0, n_iter);
  char *base_w = (char *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  void *tmp6 = nullptr;
  if (mode == 2) {
    tmp6 = base_w;
    base_w += (interior_points(B) * nf * 6 * (B->dtype == CFD_F32 ? 4 : 8) + 255) & ~(size_t)255;
  }
  double *halo[2] = {(double *)base_w, (double *)(base_w + bytes256(z.halo))};
  const int sms = B->num_sms > 0 ? B->num_sms : 148;
  cfd_status s;
  for (size_t gi = 0; gi < B->sizes.size(); ++gi) {
    const DenseGroup &G = ds->groups[gi];
    if (!G.ok || !G.biased) {
      set_error("dense biased: block group unsupported (N must be 16 or 32, uniform spacing, kc <= N)");
      return CFD_ERR_UNSUPPORTED;
    }
    const int N = G.N, g = B->ng, E = N + 2 * g;
    if (n_iter > 0 && !G.iter_ok) {
      set_error("dense: hybrid iteration needs N + 2 ng + 4 <= the padded K of the block size");
      return CFD_ERR_UNSUPPORTED;
    }
    DenseParams base;
    memset(&base, 0, sizeof(base));
    base.blocks = B->d_groups[gi];
    base.extpre = B->d_extpre;
    base.intpre = B->d_intpre;
    base.nblk = (int)B->groups[gi].size();
    base.nf = nf;
    base.nops = mode == 2 ? 6 : naxes;
    base.N = N;
    base.g = g;
    base.status = B->d_status;
    base.out = mode == 2 ? tmp6 : out;
    base.seg_rows = N;
    base.kext = E;
    {
      const std::vector<int> &gb = B->groups[gi];
      bool contig = true;
      for (size_t k = 0; k < gb.size(); ++k)
        if (gb[k] != gb[0] + (int)k) contig = false;
      base.contig = contig ? 1 : 0;
      base.b0 = gb[0];
      base.ext0 = B->extpre[gb[0]];
      base.int0 = B->intpre[gb[0]];
    }
    base.nbr = B->d_nbr;
    base.halo_deg_mask = 3;   // both halo slots pairs: S+ (columns E, E+1), S- (E+2, E+3)
    auto run = [&](DenseParams P) -> cfd_status {
      const int np = P.n1 * P.n2;
      const size_t eout = B->dtype == CFD_F32 ? 4 : 8;
      const bool f32 = B->dtype == CFD_F32;
      const size_t ein_b = f32 ? 4 : 8;
      P.xrow = P.axis == 2 && (E * ein_b) % 16 == 0 && ((uintptr_t)P.in & 15) == 0;
      P.xvec = P.axis == 2 && (N * eout) % 16 == 0 && ((uintptr_t)P.out & 15) == 0;
      P.tiles_per_job = (np + kTile - 1) / kTile;
      P.ntiles = P.tiles_per_job * P.nblk * P.nf;
      const unsigned grid = (unsigned)std::min(P.ntiles, sms);
      return launch_stage(ds, P, G.Kp, S, L, ein_b, f32, grid, st);
    };
    for (int i = 0; i < naxes; ++i) {
      const int box = axes[i];
      const bool iter = n_iter > 0 && !G.cyc[box];
      DenseParams P = base;
      P.in = fields;
      P.in_field = 1;
      P.axis = box;
      P.t1 = box == 0 ? 1 : 0;
      P.t2 = box == 2 ? 1 : 2;
      for (int t = 0; t < 3; ++t) P.in_dims[t] = E;
      P.in_start[box] = 0;
      P.in_start[P.t1] = g;
      P.in_start[P.t2] = g;
      P.n1 = N;
      P.n2 = N;
      P.int_lo1 = 0; P.int_hi1 = N; P.int_lo2 = 0; P.int_hi2 = N;
      // segments: (side, op); both sides of axis i go to ops 2i, 2i+1 of the workspace
      int side[2], op[2], n = 0;
      if (mode == 2) { side[0] = 0; op[0] = 2 * i; side[1] = 1; op[1] = 2 * i + 1; n = 2; }
      else { side[0] = mode; op[0] = i; n = 1; }
      const int per_pass = (n * N <= 32) ? n : 1;
      P.passes = n / per_pass;
      P.rows = per_pass * N;
      for (int ps = 0; ps < P.passes; ++ps) {
        P.nseg[ps] = per_pass;
        for (int k = 0; k < per_pass; ++k) {
          const int sgi = ps * per_pass + k;
          const DenseOp &o = iter ? G.bopI[box][side[sgi]] : G.bop[box][side[sgi]];
          P.seg_img[ps][k] = o.image(prec == CFD_TC_TF32);
          P.seg_exp[ps][k] = o.rowexp;
          P.seg_mode[ps][k] = 0;
          P.seg_op[ps][k] = op[sgi];
        }
      }
      if (iter) {
        // halo passes on the CUDA cores (halo_rows.cu), as for the centred operators
        DenseParams H = P;
        for (int it = 0; it < n_iter; ++it) {
          H.halo_in = it == 0 ? nullptr : halo[(it - 1) & 1];
          H.halo_out = halo[it & 1];
          H.kext = it == 0 ? E : E + 4;
          if ((s = halo_rows_launch(H, it == 0 ? G.bhr0[box] : G.bhrI[box], B->dtype == CFD_F32, st)) != CFD_OK)
            return s;
        }
        P.halo_in = halo[(n_iter - 1) & 1];
        P.kext = E + 4;
      }
      if ((s = run(P)) != CFD_OK) return s;
    }
  }
  if (mode == 2) return advect_combine(B, tmp6, beta, nf, out, out_nops, out_opidx, accum_all, st);
  return CFD_OK;
}

}  // namespace cfd

// Test hook (no counterpart in the paper): the main-loop wait limit of k_dense in clock cycles
// (<= 0 restores the default of ~2 s).  A tiny limit makes the first waits of a launch run out,
// so that the timeout path (status word, drained copies and MMAs, freed TMEM) can be checked.
extern "C" cfd_status cfd_debug_set_wait_limit(long long cycles) {
  cfd::g_wait_limit = cycles > 0 ? cycles : cfd::kWaitLimit;
  return CFD_OK;
}

namespace cfd {
// Autotuning hooks (api.cpp exposes them): switch the tuning mode of a handle, and describe the
// choices made so far as JSON.
void dense_set_tuning(cfd_blocks_s *B, bool on) {
  DenseState *ds = state_of(B);
  if (ds) ds->tuning = on;
}
std::string dense_tuning_report(cfd_blocks_s *B) {
  DenseState *ds = state_of(B);
  std::string o = "{";
  if (ds) {
    bool first = true;
    for (const auto &kv : ds->tuned) {
      o += std::string(first ? "" : ", ") + "\"" + kv.first + "\": [";
      first = false;
      for (size_t i = 0; i < kv.second.size(); ++i) {
        const TuneRec &r = kv.second[i];
        char buf[512];
        snprintf(buf, sizeof buf,
                 "%s{\"stage\": \"%s\", \"staging\": \"%s\", \"order\": \"%s\", \"ms\": {\"tma/interleaved\": %.5f, "
                 "\"tma/contiguous\": %.5f, \"cp.async/interleaved\": %.5f, \"cp.async/contiguous\": %.5f}}",
                 i ? ", " : "", r.stage.c_str(), r.staging ? "cp.async" : "tma", r.order ? "contiguous" : "interleaved",
                 r.ms[0], r.ms[1], r.ms[2], r.ms[3]);
        o += buf;
      }
      o += "]";
    }
  }
  return o + "}";
}
}  // namespace cfd
