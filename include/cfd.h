/*
 * cfd.h -- C ABI of the GB300 compact finite-difference (CFD) operator library.
 *
 * The library applies centred, tridiagonal compact finite-difference schemes
 * (arXiv 2302.14858, Eq. mdAnsatz with alpha^{(d)} = (a, 1, a)) to 3D fields
 * split into MeshBlocks with ghost layers.  Each block solves its own banded
 * system closed by explicit, error-matched closures (Eq. sch_cent_om), with
 * optional hybrid matching-communication iterations (Eq. iter_center_P).
 * It also applies biased (upwind) first-degree schemes with their
 * single-point closures (Eqs. defChenSchemes, closure_left_X, iter_left_X),
 * the upwinded shift-advection term built from them (Eq. biasderapproxadv),
 * and time steps of the wave, shifted-wave and advection systems.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All entry points return a cfd_status; nothing aborts or throws across
 *    the ABI.  cfd_last_error() gives a message for the last failure on the
 *    calling thread.
 *  - Host pointers (coefficients, tables) are read during the call and not
 *    retained.  Device pointers (fields, outputs, workspaces) are owned by the
 *    caller and must stay valid until the work queued on `stream` finishes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is asynchronous; errors detected on the device
 *    (bounded waits that ran out, failed self-checks) are latched in a status
 *    word of the blocks handle and reported by cfd_sync_status().
 *  - Field layout (device memory): blocks in bind order; block b holds
 *    nfields arrays of (N_b + 2 ng)^3 values, axes (z, y, x), x fastest.
 *    Interior index k = 0..N_b-1 of an axis sits at array index k + ng
 *    (cell-centred sampling, Eq. gridDisc CC).
 *  - Output layout: blocks in bind order; block b holds nfields x nops arrays
 *    of N_b^3 interior values (z, y, x), ops in increasing bit order of
 *    op_mask.  Outputs have the field dtype.
 */
#ifndef CFD_H
#define CFD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cfd_status {
  CFD_OK = 0,
  CFD_ERR_ARG = 1,            /* invalid argument (null pointer, size, layout) */
  CFD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  CFD_ERR_UNSUPPORTED = 3,    /* valid request outside what this build supports */
  CFD_ERR_NOT_CONVERGED = 4,  /* reserved: iteration did not reach a tolerance */
  CFD_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out */
  CFD_ERR_DEVICE_ASSERT = 6,  /* a device-side self-check failed */
  CFD_ERR_ALLOC = 7           /* host or device allocation failed */
} cfd_status;

/*
 * Arithmetic of cfd_apply.
 *
 * The tensor-core forms apply the dense block operator D = A^-1 B ([0]D of
 * Eq. iter_scheme) per pencil.  Number format of CFD_TC_BF16_EXACT (and of the
 * hi/lo split, which keeps fewer slices): each pencil (its N + 2 ng ghost-
 * extended inputs, plus the neighbour values of an iterated pass) is
 * quantised to 39-bit fixed point relative to its own largest magnitude
 * (rounded to nearest; a power-of-two scale per pencil), so
 *   - inputs below 2^-40 of the pencil maximum contribute nothing, and
 *     subnormal inputs are taken as zero;
 *   - the error of an output is bounded by ~2^-32 max_j |D_ij| max_j |f_j|
 *     of its pencil and is typically ~2^-37 sum_j |D_ij f_j|;
 *   - a NaN or an infinity anywhere in a pencil makes every output of that
 *     pencil NaN (the FP64 banded solve spreads non-finite values over the
 *     same pencils);
 *   - outputs that overflow become infinities; FP64 outputs below the normal
 *     range flush to zero, FP32 outputs round as IEEE.
 * With n_iter > 0 the values the neighbours read at their k^c nodes (the halo
 * rows of each iterate) are computed on the CUDA cores in compensated FP32
 * (~2^-46 of sum_j |c_j f_j|), then enter the final pass as four extra inputs of
 * each pencil in the format above.
 */
typedef enum cfd_precision {
  CFD_FP64_BANDED = 0,   /* FP64 right-hand side + Thomas solve per pencil */
  CFD_TC_BF16X3 = 1,     /* dense D on BF16 tensor cores, hi/lo split, 3 products */
  CFD_TC_BF16_EXACT = 2, /* dense D on BF16 tensor cores, exact integer slices (FP64-level result) */
  CFD_TC_TF32 = 3        /* dense D on TF32 tensor cores, one product, FP32 accumulation:
                            each pencil and D rounded to TF32 (same per-pencil scale);
                            measured max relative error against FP64 (tuned Q schemes,
                            smooth data): ~1e-2 for first and ~1e-1 for second and mixed
                            derivatives at 64^3, ~2e-2 / ~4e-1 at 128^3; at 256^3 second
                            derivatives are not resolved (cancellation ~ dx^-2) */
} cfd_precision;

typedef enum cfd_dtype { CFD_F64 = 0, CFD_F32 = 1 } cfd_dtype;

/* Derivative outputs (op_mask bits). Mixed ops are symmetrised (D_i D_j + D_j D_i)/2. */
#define CFD_OP_DX  (1u << 0)
#define CFD_OP_DY  (1u << 1)
#define CFD_OP_DZ  (1u << 2)
#define CFD_OP_DXX (1u << 3)
#define CFD_OP_DYY (1u << 4)
#define CFD_OP_DZZ (1u << 5)
#define CFD_OP_DXY (1u << 6)
#define CFD_OP_DXZ (1u << 7)
#define CFD_OP_DYZ (1u << 8)
#define CFD_OP_ALL 0x1FFu

/* Neighbour direction r of block b: (dz, dy, dx) in {-1,0,1}^3 without the
 * centre, lexicographic with dz slowest: r = 9(dz+1) + 3(dy+1) + (dx+1),
 * minus one when that exceeds 13. */
#define CFD_NDIRS 26

/*
 * One centred tridiagonal compact scheme of derivative degree `deriv`
 * (Eq. mdAnsatz with alpha^{(d)} = (lhs_offdiag, 1, lhs_offdiag) and
 * alpha^{(0)}_{-M..M}), together with its explicit closure C-bar_{p+1}
 * (Eq. sch_cent_om rows k = k*_+-), e.g. the appendix tables pade_deg_one,
 * pade_deg_two, num_deg_one and num_deg_two.
 *   order             formal order 2p of the interior scheme (4, 6, 8 or 10).
 *   M                 half-width of the interior right-hand side, 1 <= M <= 5.
 *   rhs               2M+1 host values alpha^{(0)}_{-M..M}.
 *   closure_halfwidth p+1, 2 <= p+1 <= 6 (ignored when closure is NULL).
 *   closure           2(p+1)+1 host values, or NULL: the library then builds
 *                     the closure of half-width order/2 + 1 whose eta^{2p}
 *                     error constant matches the interior's C_0 and whose
 *                     eta^{2p+1} term vanishes (the two conditions after
 *                     Eq. errelmodwavecentmatch).
 */
typedef struct cfd_scheme_desc {
  int deriv;
  int order;
  int M;
  double lhs_offdiag;
  const double *rhs;
  int closure_halfwidth;
  const double *closure;
} cfd_scheme_desc;

typedef struct cfd_scheme_s *cfd_scheme_t;
typedef struct cfd_blocks_s *cfd_blocks_t;

/*
 * Create a scheme pair: `first` (deriv = 1) for d_x, d_y, d_z and the mixed
 * ops, `second` (deriv = 2) for d_xx, d_yy, d_zz.  Either may be NULL if the
 * ops that need it are never requested.  Host-only; allocates host memory.
 * Errors: CFD_ERR_ARG (bad degree, widths, or a non-diagonally-dominant
 * system 2|a| >= 1), CFD_ERR_ALLOC.
 */
cfd_status cfd_scheme_create(const cfd_scheme_desc *first, const cfd_scheme_desc *second,
                             cfd_scheme_t *out);

/* Copy the closure in use for degree `deriv` (built or given) to `closure`
 * (room for 13 doubles); *halfwidth receives p+1. */
cfd_status cfd_scheme_closure(cfd_scheme_t scheme, int deriv, double *closure, int *halfwidth);

void cfd_scheme_destroy(cfd_scheme_t scheme);

/*
 * Bind a set of MeshBlocks (Sec. "Domain decomposition"; the communication
 * pattern of matrix G, Eq. example_G) to a scheme on the current CUDA device.
 *   nblocks    number of blocks, >= 1.
 *   block_n    host [nblocks]: interior points per axis N_b, 8 <= N_b <= 32,
 *              N_b >= ng.
 *   dx         host [nblocks][3]: grid spacing (dx, dy, dz) of each block.
 *   neighbors  host [nblocks][26]: neighbour block per direction (see
 *              CFD_NDIRS), -1 = the caller fills that ghost region itself
 *              (e.g. an interface to a block of another size).  A neighbour
 *              must have the same N as the block.  A block that is its own
 *              neighbour on both faces of an axis covers the whole periodic
 *              line: that axis uses the undecomposed cyclic scheme.
 *   ng         ghost layers, >= closure half-width and >= M + 1.
 *   dtype      CFD_F64 or CFD_F32 fields.
 * Builds per block size: the banded LU factors of the closed and iterated
 * systems and the dense operators D = A^-1 B ([0]D of Eq. iter_scheme) with
 * their tensor-core copies; uploads them with the neighbour tables.
 * Allocates device memory owned by the handle.
 */
cfd_status cfd_blocks_bind(cfd_scheme_t scheme, int nblocks, const int *block_n, const double *dx,
                           const int *neighbors, int ng, cfd_dtype dtype, cfd_blocks_t *out);

void cfd_blocks_destroy(cfd_blocks_t blocks);

/*
 * Ghost exchange (matrix G of Eq. example_G): for every block and every
 * direction with a neighbour >= 0, copy the neighbour's interior slab into
 * the block's ghost region (faces, edges and corners).  `fields` is the
 * device field buffer described above with `nfields` fields.  Exact copy.
 * CFD_ERR_UNSUPPORTED when the blocks of one size times nfields exceed 65535.
 */
cfd_status cfd_exchange_ghosts(cfd_blocks_t blocks, void *fields, int nfields, void *stream);

/* Device workspace cfd_apply needs for this request (bytes, 256-aligned). */
cfd_status cfd_apply_workspace(cfd_blocks_t blocks, int nfields, unsigned op_mask, cfd_precision prec,
                               int n_iter, size_t *bytes);

/*
 * Derivatives of ghost-filled fields.  For every block, field and op in
 * `op_mask`: d_i with the first-degree scheme, d_ii with the second-degree
 * scheme, d_ij (i != j) as (D_i[D_j f] + D_j[D_i f]) / 2 where the inner D_j
 * is evaluated on the ghost rows of axis i too (needs edge ghosts).
 *   n_iter     hybrid iterations (Eq. iter_center_P), 0 = closures only.
 *              n_iter > 0 needs same-size face neighbours on every
 *              decomposed axis.
 *   prec       arithmetic (see cfd_precision).
 *   work       device workspace of at least cfd_apply_workspace() bytes.
 * Errors: CFD_ERR_ARG, CFD_ERR_UNSUPPORTED, CFD_ERR_CUDA.
 */
cfd_status cfd_apply(cfd_blocks_t blocks, const void *fields, int nfields, unsigned op_mask,
                     cfd_precision prec, int n_iter, void *out, void *work, size_t work_bytes,
                     void *stream);

/*
 * Autotuner of the tensor-core form (no counterpart in the paper): runs the request
 * cfd_apply(blocks, fields, nfields, op_mask, prec, n_iter, out, work, ...) once, launching
 * each of its kernels under every candidate launch configuration -- the staging of the input
 * tiles (TMA boxes or cp.async) and the order in which the persistent CTAs take the tiles
 * (interleaved or contiguous runs) -- three times, timing the last two with CUDA events, and
 * keeps the fastest per kernel of the request in the handle; later cfd_apply calls of the same
 * request (fields, ops, precision, iterations) use those choices.  Synchronises the stream (not
 * for use during stream capture); `out` receives the request's results.  Errors: as cfd_apply,
 * CFD_ERR_ARG for the FP64 banded path (nothing to tune).
 */
cfd_status cfd_autotune(cfd_blocks_t blocks, const void *fields, int nfields, unsigned op_mask, cfd_precision prec,
                        int n_iter, void *out, void *work, size_t work_bytes, void *stream);

/* The autotuner's choices and measured times as a JSON object (request -> per-kernel list),
 * written to buf (len bytes, NUL-terminated, truncated if short); *needed = bytes required. */
cfd_status cfd_autotune_report(cfd_blocks_t blocks, char *buf, size_t len, size_t *needed);

/*
 * Order of the mixed derivatives on the FP64 banded path.  one_order = 0
 * (the default) evaluates the symmetrised form of Sec. "Z4c: system
 * description", (D_i[D_j f] + D_j[D_i f]) / 2; one_order = 1 evaluates
 * D_i[D_j f] only, half the work.  The two agree to rounding where the block
 * operators of the two axes commute: every block has same-size face
 * neighbours along every decomposed axis (closed or iterated systems, cyclic
 * axes) and its edge ghosts hold the neighbours' values (cfd_exchange_ghosts).
 * The tensor-core forms always evaluate one order.  Errors: CFD_ERR_ARG,
 * CFD_ERR_UNSUPPORTED (one order on blocks without face neighbours).
 */
cfd_status cfd_blocks_set_mixed_order(cfd_blocks_t blocks, int one_order);

/*
 * Allocation-free variant of cfd_apply for callers that cannot allocate
 * device memory when they call it (no counterpart in the paper).  Such
 * callers are typically host codes that give all device memory to their own
 * pool at start-up and forbid later cudaMalloc/cudaFree, solver loops under a
 * fixed memory budget, or loops that must not synchronise the device the way
 * cudaFree does.  They bind the blocks once at start-up (cfd_blocks_bind
 * allocates) and then call this instead of cfd_apply.
 *
 * It computes exactly what cfd_apply(blocks, fields, nfields, op_mask,
 * CFD_FP64_BANDED, 0, out, ...) computes -- closures only, no hybrid
 * iteration -- but takes no workspace: its scratch (the inner D_j of the mixed
 * derivatives, Sec. "Z4c: system description") is one file-scope device
 * array of 64 MiB that every GPU loading the library holds until the process
 * exits.  A request whose scratch would exceed 64 MiB (nfields x, per block,
 * (N+2ng) N^2 doubles when op_mask has a mixed op) fails with CFD_ERR_ARG and
 * a message; split the fields or blocks over several calls.  Single-axis ops
 * need no scratch.
 *
 * The first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and caches it; make that first
 * call before any stream capture.  On success the call allocates nothing,
 * host or device, and calls no allocating routine (with the profiling
 * diagnostics off, their default).  All calls share the one array, which keeps
 * the previous call's contents; nothing in it needs to start at zero.  Calls
 * whose device work overlaps in time (other streams, other host threads on
 * the same device) race on the array: order them on one stream or serialise
 * them.  Errors: as cfd_apply, plus CFD_ERR_ARG when the current device is
 * not the device the blocks were bound on.
 */
cfd_status cfd_apply_static(cfd_blocks_t blocks, const void *fields, int nfields, unsigned op_mask, void *out,
                            void *stream);

/* Device workspace of cfd_wave_rk_step (bytes). */
cfd_status cfd_wave_workspace(cfd_blocks_t blocks, cfd_precision prec, int n_iter, size_t *bytes);

/*
 * One classical RK4 step (ERK4 of Sec. "Two dimensional advection", fully
 * discrete) of the linear wave system d/dt Phi = K, d/dt K = sum_i D2_i Phi
 * (Eq. toyShiftWaveEqnSys with zero shift).  `phi` and `K` are single-field
 * buffers in the field layout; ghosts of Phi are exchanged before every
 * stage (blocks with -1 neighbours are not supported here).  Needs the
 * second-degree scheme.
 */
cfd_status cfd_wave_rk_step(cfd_blocks_t blocks, void *phi, void *K, double dt, cfd_precision prec,
                            int n_iter, void *work, size_t work_bytes, void *stream);

/*
 * Coefficients of a two-register (2S) low-storage Runge-Kutta method with
 * `stages` stages (1..8).  Per stage i, with S1 the state and S2 a second
 * register that is zero on entry:
 *     S2 <- S2 + delta[i] S1
 *     S1 <- gamma1[i] S1 + gamma2[i] S2 + beta[i] dt F(S1 before this stage)
 * The paper's host code evolves with the 4-stage 4th-order RK4()4[2S] method
 * of this form (Sec. "Z4c: system description"); it prints no coefficients,
 * so the caller supplies them.  The arrays are host memory, read during the
 * call only.
 */
typedef struct {
  int stages;
  const double *gamma1, *gamma2, *beta, *delta;
} cfd_lsrk_desc;

/* Device workspace of cfd_wave_lsrk_step (bytes). */
cfd_status cfd_wave_lsrk_workspace(cfd_blocks_t blocks, cfd_precision prec, int n_iter, size_t *bytes);

/*
 * One step of the 2S method above for the wave system of cfd_wave_rk_step
 * with Kreiss-Oliger dissipation (Eq. dissdef) added to the right-hand side of
 * both fields in each direction:
 *     F_Phi = K + sum_i Q_i[Phi],  F_K = sum_i D2_i Phi + sum_i Q_i[K],
 *     Q_i = -((-1)^r / 2^{2r}) sigma dx_i^{2r-1} (D_+)^r (D_-)^r along axis i.
 *   sigma >= 0; ko_r = r, 1 <= r <= ng (the stencil of (2r)E_r, Tab. diss_scheme,
 *   reads r ghosts; the ghosts of both fields are exchanged every stage when
 *   sigma > 0).  The dissipation sums run in FP64 for CFD_FP64_BANDED and in
 *   FP32 (added to the FP64 right-hand side) for the tensor-core precisions.
 * `phi`, `K`: single-field buffers in the field layout, advanced in place.
 * Errors: CFD_ERR_ARG (bad coefficients, sigma < 0, r out of range, workspace),
 * CFD_ERR_UNSUPPORTED (FP32 fields, -1 neighbours), CFD_ERR_CUDA.
 */
cfd_status cfd_wave_lsrk_step(cfd_blocks_t blocks, void *phi, void *K, double dt, const cfd_lsrk_desc *rk,
                              double sigma, int ko_r, cfd_precision prec, int n_iter, void *work,
                              size_t work_bytes, void *stream);

/*
 * Biased (upwind) first-degree compact scheme, Eq. defChenSchemes with a
 * two-point left side (Sec. "Domain decomposition: dispersion relation
 * preservation"), given in its left-biased form S_+ (Im eta~ <= 0; e.g. the
 * CCU schemes X_M^- of Tab. ccux_deg_one_col or Q^{1,0}_{3,4} of
 * Tab. num_deg_one).  On a block (local k = 0..N-1, k*_- = 0, k*_+ = N-1):
 *   interior rows k = 1..N-1 (Eq. closure_left_X):
 *     a d_{k-1} + d_k = dx^{-1} sum_{i<rhs_n} rhs[i] f_{k + rhs_lo + i}
 *   closure row k = k*_-:
 *     d_k + closure_sup d_{k+1} = dx^{-1} sum_{i<closure_n} closure[i] f_{k + closure_lo + i}
 * The right-biased scheme S_- is its mirror (the rule stated with
 * Tabs. ucd_slow and ccux_deg_one_col): alpha^{(1)}_m -> alpha^{(1)}_{-m},
 * alpha^{(0)}_m -> -alpha^{(0)}_{-m}, closed at k*_+.  Hybrid iteration
 * (Eq. iter_left_X) fixes the derivative at k^c_- = k*_- - kc (S_-:
 * k^c_+ = k*_+ + kc) to the neighbour's previous iterate and solves the
 * interior rows from there.
 *   order        formal order (informational, >= 1).
 *   a            alpha^{(1)}_{-1}, |a| < 1 (the bidiagonal solve then damps
 *                rounding); closure_sup with |closure_sup * a| < 1.
 *   rhs_lo/rhs_n, closure_lo/closure_n   offsets and lengths (<= 12 taps,
 *                offsets within -6..6); host arrays read during the call.
 *   kc           1, 2 or 3.
 * Stencil support of this build: ng = 4 with the interior offsets within
 * -4..4 and the closure's within -4..5 (Tab. ccux M = 1, 2; Q^{1,0}_{3,4}),
 * or ng = 6 with -5..5 and -5..6 (M = 3).
 */
typedef struct cfd_biased_desc {
  int order;
  double a;
  int rhs_lo, rhs_n;
  const double *rhs;
  double closure_sup;
  int closure_lo, closure_n;
  const double *closure;
  int kc;
} cfd_biased_desc;

/* Attach the biased scheme to a scheme handle (before cfd_blocks_bind, which
 * builds its per-block-size tables).  Errors: CFD_ERR_ARG. */
cfd_status cfd_scheme_set_biased(cfd_scheme_t scheme, const cfd_biased_desc *desc);

/* Device workspace of cfd_apply_biased / cfd_advect for this arithmetic (bytes; 0 for
 * CFD_FP64_BANDED without iteration; the tensor-core form keeps both biased derivatives of
 * every axis, 6 N^3 values per block and field, for the upwind blend). */
cfd_status cfd_biased_workspace(cfd_blocks_t blocks, int nfields, cfd_precision prec, int n_iter, size_t *bytes);

/*
 * Biased first derivatives of ghost-filled fields: for every block, field
 * and axis in `axis_mask` (CFD_OP_DX | CFD_OP_DY | CFD_OP_DZ), D_i[S_+] f
 * (side = +1) or D_i[S_-] f (side = -1), solved per pencil in FP64 as the
 * bidiagonal block system above (n_iter = 0) or its iteration (n_iter > 0,
 * Jacobi: every block reads its neighbours' iterate i-1).  An axis along
 * which a block is its own neighbour on both faces uses the undecomposed
 * cyclic scheme.  Output layout as cfd_apply (axes in bit order).
 *   prec   CFD_FP64_BANDED: per-pencil FP64 bidiagonal solves;
 *          CFD_TC_BF16_EXACT / CFD_TC_BF16X3: the dense operators
 *          D = A^-1 B of the same block systems on the tensor cores (exact
 *          integer digit slices, or BF16 hi/lo), with the iteration as
 *          d = D_1 f + c d^c (blocks of 16^3 or 32^3, uniform spacing).
 * Errors: CFD_ERR_ARG (no biased scheme bound, bad mask/side, workspace),
 * CFD_ERR_UNSUPPORTED (stencil support, iteration without face neighbours,
 * TF32, block sizes the tensor-core form does not cover), CFD_ERR_CUDA.
 */
cfd_status cfd_apply_biased(cfd_blocks_t blocks, const void *fields, int nfields, unsigned axis_mask, int side,
                            cfd_precision prec, int n_iter, void *out, void *work, size_t work_bytes,
                            void *stream);

/*
 * Upwinded shift-advection term beta^i d_i f as it appears on a right-hand
 * side (u_t = beta^i d_i u + ..., Sec. "Z4c: system description"): it
 * transports with velocity c = -beta^i, and Eq. biasderapproxadv takes the
 * scheme with Im eta~ <= 0 (S_+, left-biased) where c > 0.  For every block
 * and field
 *     out = sum_{i = x, y, z} beta^i_+ D_i[S_-] f + beta^i_- D_i[S_+] f,
 *     beta_+- = (beta +- |beta|) / 2,
 * i.e. the right-biased scheme where beta^i > 0 and the left-biased one
 * where beta^i < 0 (for u_t + c . grad u = 0 pass beta = -c).  With this
 * choice the semi-discrete operator has no growing mode; the opposite one
 * is anti-dissipative.  `beta` holds three fields (beta^x,
 * beta^y, beta^z) in the field layout (ghosts unused); `out` one N^3 array
 * per block and field.  Arithmetic as cfd_apply_biased; the three axis terms
 * are added in the order x, y, z (the tensor-core form writes both biased
 * derivatives of every axis to the workspace and blends them in one pass).
 */
cfd_status cfd_advect(cfd_blocks_t blocks, const void *fields, int nfields, const void *beta, cfd_precision prec,
                      int n_iter, void *out, void *work, size_t work_bytes, void *stream);

/* Device workspace of cfd_shifted_wave_lsrk_step (bytes). */
cfd_status cfd_shifted_wave_workspace(cfd_blocks_t blocks, cfd_precision prec, int n_iter, size_t *bytes);

/*
 * One step of the 2S method (cfd_lsrk_desc) for the shifted wave system of
 * Eq. toyShiftWaveEqnSys with a flat background (gamma^{ij} = delta^{ij}):
 *     F_Phi = beta^j d_j Phi + K + sum_i Q_i[Phi],
 *     F_K   = beta^j d_j K + sum_i D2_i Phi + sum_i Q_i[K],
 * where the advective terms beta^j d_j are the upwinded biased operators of
 * cfd_advect (Eq. biasderapproxadv with c -> beta^j, as Sec. "Shifted wave
 * equation" prescribes for biased schemes), the Laplacian uses the
 * second-degree scheme, both with arithmetic `prec`, and Q_i
 * is the Kreiss-Oliger term of cfd_wave_lsrk_step.  `beta`: three fields
 * (beta^x, beta^y, beta^z) in the field layout, constant during the step
 * (ghosts unused).  Needs a biased scheme (cfd_scheme_set_biased) and the
 * second-degree scheme; n_iter applies to both.  Errors as
 * cfd_wave_lsrk_step, plus the checks of cfd_advect.
 */
cfd_status cfd_shifted_wave_lsrk_step(cfd_blocks_t blocks, void *phi, void *K, const void *beta, double dt,
                                      const cfd_lsrk_desc *rk, double sigma, int ko_r, cfd_precision prec,
                                      int n_iter, void *work, size_t work_bytes, void *stream);

/* Device workspace of cfd_advect_lsrk_step (bytes). */
cfd_status cfd_advect_lsrk_workspace(cfd_blocks_t blocks, int nfields, cfd_precision prec, int n_iter,
                                     size_t *bytes);

/*
 * One step of the 2S method (cfd_lsrk_desc) for the advection equation of
 * every field, u_t = beta^i d_i u + sum_i Q_i[u] (Eq. tr2pde of Sec. "Two
 * dimensional advection" with c = -beta, and the shift-advection term of
 * Sec. "Z4c: system description"): the advective term is cfd_advect (upwinded
 * biased operators, arithmetic `prec`), Q_i the Kreiss-Oliger term of
 * cfd_wave_lsrk_step (FP64; none when sigma = 0).  `u`: nfields fields in the
 * field layout, advanced in place (ghosts are exchanged every stage); `beta`:
 * three fields as for cfd_advect, constant during the step.  Needs a biased
 * scheme (cfd_scheme_set_biased).  FP64 fields, every ghost region with a
 * neighbour.  Errors as cfd_advect plus CFD_ERR_ARG for the coefficients.
 */
cfd_status cfd_advect_lsrk_step(cfd_blocks_t blocks, void *u, int nfields, const void *beta, double dt,
                                const cfd_lsrk_desc *rk, double sigma, int ko_r, cfd_precision prec, int n_iter,
                                void *work, size_t work_bytes, void *stream);

/*
 * Ghost regions between processes.  When the MeshBlocks of one problem are
 * split over several processes (one GPU each), a process binds its own
 * blocks with -1 for the directions whose neighbour lives elsewhere, fills
 * the local ghosts with cfd_exchange_ghosts, and moves the remote ones with
 * these plans (the remote part of matrix G, Eq. example_G); the transport
 * between processes (e.g. NCCL send/recv of the buffers) is the caller's.
 *   items  host [n][2] = (local block, direction r, numbered as CFD_NDIRS).
 *          In a pack plan the block is the one that owns the data and r is
 *          the direction of the ghost region as seen from the receiving
 *          neighbour: pack copies the owner's interior slab that fills that
 *          region (ghost cell c of the receiver takes the owner's value at
 *          c - d N, d the unit offset of r).  In an unpack plan the block is
 *          the receiver and r its ghost region.
 *  Buffer: the items in order; per item nfields slabs of the region's shape
 *  (g or N per axis), (z, y, x) order, field dtype.  A pack plan on the owner
 *  and an unpack plan on the receiver that list the same regions in the same
 *  order move exactly the values cfd_exchange_ghosts would copy.
 * The plan keeps a device copy of the items (freed by cfd_halo_plan_destroy).
 */
typedef struct cfd_halo_plan_s *cfd_halo_plan_t;
cfd_status cfd_halo_plan_create(cfd_blocks_t blocks, const int *items, int n, cfd_halo_plan_t *out);
/* Buffer bytes for `nfields` fields. */
cfd_status cfd_halo_plan_bytes(cfd_halo_plan_t plan, int nfields, size_t *bytes);
cfd_status cfd_halo_pack(cfd_halo_plan_t plan, const void *fields, int nfields, void *buf, void *stream);
cfd_status cfd_halo_unpack(cfd_halo_plan_t plan, void *fields, int nfields, const void *buf, void *stream);
void cfd_halo_plan_destroy(cfd_halo_plan_t plan);

/* Wait for `stream`, then read and clear the device status word of the
 * handle: CFD_OK, CFD_ERR_TIMEOUT or CFD_ERR_DEVICE_ASSERT. */
cfd_status cfd_sync_status(cfd_blocks_t blocks, void *stream);

/* Message for the last failed call on this thread ("" if none). */
const char *cfd_last_error(void);

/*
 * Diagnostics (no counterpart in the paper).  Kernel families:
 * 0 ghost exchange, 1 banded line solve, 2 RK4 combine, 3 dense tensor-core
 * operator, 4 halo rows of the hybrid iteration on the tensor-core path
 * (CUDA cores), 5 biased line solve (cfd_apply_biased,
 * cfd_advect).  cfd_kernel_launches() counts every kernel the
 * library has launched in this process.  With profiling on, every launch is
 * bracketed by CUDA events recorded on its own stream; cfd_profile_read()
 * (after the stream has finished) returns the number of launches and their
 * summed device time for one family since profiling was last enabled.
 * cfd_profile_enable(0) stops recording; enabling resets the sums.
 */
unsigned long long cfd_kernel_launches(void);
cfd_status cfd_profile_enable(int on);
cfd_status cfd_profile_read(int family, unsigned long long *launches, double *ms);

/*
 * Test hook (no counterpart in the paper): the number of clock cycles a wait
 * inside the tensor-core kernel's main loop may take before the kernel gives
 * up, latches CFD_ERR_TIMEOUT in the handle's status word and ends (after
 * draining its own copies and MMAs and freeing its tensor memory).
 * cycles <= 0 restores the default (~2 s).  Process-wide; read at each launch.
 */
cfd_status cfd_debug_set_wait_limit(long long cycles);

#ifdef __cplusplus
}
#endif

#endif /* CFD_H */
