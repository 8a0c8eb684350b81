// Dense per-block operator D = A^-1 B on the tensor cores (see dense_tc.cu).
#pragma once
#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's driver entry point)

#include <vector>

#include "cfd_internal.h"

namespace cfd {

// One stage of the dense path over a group of same-size blocks: a GEMM of
// 128-pencil tiles against the digit images of up to two operators per pass.
struct DenseParams {
  const void *in;            // field buffer (dtype) or FP64 scratch
  void *out;                 // final output buffer (dtype): block b, field q, op -> N^3 box
  double *scratch_out;       // FP64 scratch box of this stage (or null)
  const int *blocks;         // [nblk] global block ids
  const long long *extpre, *intpre;
  int nblk, nf, nops, N, g;
  int in_field;              // 1: in is the field buffer
  unsigned long long in_box, sc_box;  // scratch box sizes (elements per block and field)
  int axis, t1, t2;          // box axes (0 z, 1 y, 2 x); t2 fastest
  int in_dims[3], in_start[3];        // input box and the start of the pencil range
  int sc_dims[3], sc_start[3];        // scratch output box and offset of pencil (t1, t2)
  int n1, n2;                // transverse pencil counts
  int int_lo1, int_hi1, int_lo2, int_hi2;  // pencils that write final outputs (interior)
  int passes, rows;          // MMA passes per tile, output rows per pass (16 or 32)
  int nseg[2];               // operators (segments of N rows) per pass
  const void *seg_img[2][2];  // operator images of the pass's segments (BF16 digits or TF32)
  const int *seg_exp[2][2];
  int seg_mode[2][2];        // -1 skip, 0 final (interior pencils), 2 scratch, 3 both
  int seg_op[2][2];          // op index in the output for final stores
  int tiles_per_job, ntiles; // 128-pencil tiles per (block, field); all tiles of the stage
  int tile_order, tiles_per_cta;  // 0: tile = CTA + k grid; 1: contiguous runs of tiles_per_cta
  int seg_rows;              // operator rows per segment (N, or 16 for a halo pass)
  int kext;                  // K values loaded per pencil: N + 2g, or N + 2g + 4 with halo columns
  const double *halo_in;     // [nblocks][nf][n1 n2][4]: previous iterate at rows 1, N-2 per degree (x dx^d)
  double *halo_out;          // same layout, written by a halo pass (k_halo_rows)
  const int *nbr;            // [nblocks][26] neighbour table
  int halo_deg_mask;         // degrees whose halo columns are filled (bit d-1)
  int xrow;                  // x-axis stage with 16-byte aligned pencil rows: chunked row copies
  int xvec;                  // x-axis stage with a 16-byte aligned output: vector stores
  // Consecutive block ids (blocks[lb] = b0 + lb): offsets follow from the job index
  // (no dependent table loads in the tile loop)
  int contig, b0;
  long long ext0, int0;      // extpre[b0], intpre[b0]
  // TMA staging of the tile's pencils (0: cp.async path): 1 x rows (SWIZZLE_128B boxes of 128
  // bytes along x), 2 y columns (box [t1][y][x]), 3 z columns (box [z][t1][x])
  int tma_kind, tma_boxes, tma_bytes, tma_zstep;  // zstep: z planes per job in the tensor map
  // Intermediate written on interior pencils only: each value within g of an x (and, with
  // ghost_y, a y) face is also written into the face neighbour's ghost column of the same box.
  // nl: [nblk][4] local indices of the x-, x+, y-, y+ face neighbours.
  int ghost_x, ghost_y;
  const int *nl;
  // Scratch block index of each block of the launch (null: its position in blocks): a strip
  // launch over some blocks of a group writes into the group's intermediate boxes.
  const int *sc_local;
  CUtensorMap tmap;          // (the type carries its own 128-byte alignment)
  int *status;
  long long wait_limit;      // clock cycles a main-loop wait may take before it latches CFD_ERR_TIMEOUT
  float inv_tpj, inv_nf, inv_n2;  // 1 / tiles_per_job, 1 / nf, 1 / n2 (set at launch)
};

// The four operator rows of one halo pass of the hybrid iteration (Eq. iter_center_P: rows 1
// and N-2 per degree; Eq. iter_left_X: the biased rows the neighbours read), each coefficient
// as an FP32 pair c = h + l (to ~2^-48 relative), for the compensated CUDA-core kernel of
// halo_rows.cu.  Columns: the N + 2g pencil values, then the 4 halo columns of the previous
// iterate (zero in the first pass).
struct HaloRows {
  float h[48][4], l[48][4];  // [column][row]
};
// rows 0..3 of the row-major rows x cols matrix M (cols <= 48)
void halo_rows_from(const std::vector<long double> &M, int cols, HaloRows &R);
// One halo pass of a dense stage on the CUDA cores: for every pencil of the stage (the
// addressing of P, as k_dense reads it), the 4 rows of R applied to the pencil (and, with
// P.halo_in, to the neighbours' previous iterate), written to P.halo_out.
cfd_status halo_rows_launch(const DenseParams &P, const HaloRows &R, bool f32_in, cudaStream_t st);

cfd_status dense_bind(cfd_blocks_s *B);
void dense_set_tuning(cfd_blocks_s *B, bool on);
std::string dense_tuning_report(cfd_blocks_s *B);
cfd_status dense_workspace(cfd_blocks_s *B, int nf, unsigned mask, cfd_precision prec, int n_iter, size_t *bytes);
cfd_status dense_apply(cfd_blocks_s *B, const void *fields, int nf, unsigned mask, cfd_precision prec, int n_iter,
                       void *out, void *work, size_t work_bytes, cudaStream_t st);
}  // namespace cfd
