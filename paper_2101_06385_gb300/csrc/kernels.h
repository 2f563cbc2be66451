// Host-side launch interface of the SP2 kernels (internal to libsp2.so).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sp2 {

// Arguments shared by the squaring kernels (FFMA and tcgen05).
//
// Storage of instance b (0 <= b < batch) with size n_b = Ns[b]:
//   Y      FP32 iterate, element (r, c) at Y + b*slot_y + r*ld_y + c
//   planes FP16 planes of Y (tensor-core path: hp = 2^s hi and lo' for the
//          split product, hi for plain FP16), b*slot_h + r*ld_h + c; the
//          region [n_b, ld) of every row and rows >= n_b stay zero
//   Dptr   per-instance final outputs [n_b, n_b] (ld n_b), used by OUT_D
// Tiles: tiles[t] packs (b, I, J, h); the tiles of one instance are
// contiguous, starting at tile_off[b], tile_cnt[b] of them.
struct SqArgs {
  const float* Yin;        // FFMA path: operand and old value (read-only)
  float* Yout;             // updated iterate (may equal Yin on the tensor-core path)
  long long ld_y, slot_y;
  __half* hi_out;          // FP16 planes of the updated iterate, each written when set:
  __half* lo_out;          //   hi = fp16(Y'), lo' = fp16(2^s (Y' - hi)),
  __half* hp_out;          //   hp = 2^s hi (single-accumulator kernels: split writes hp_out
                           //   and lo_out, plain FP16 hi_out and lo_out)
  long long ld_h, slot_h;
  float* const* Dptr;      // [batch] device array of output pointers (OUT_D)
  const int* Ns;           // [batch]
  const uint32_t* tiles;   // [ntiles]
  int ntiles;
  const int* tile_off;     // [batch]
  const int* tile_cnt;     // [batch]
  Ctl* ctl;                // [batch] control blocks, or nullptr
  const LayerParams* lp;   // coefficients when ctl == nullptr
  int lp_per_instance;     // 1: lp[b] per instance, 0: lp[0] shared by the batch
  double2* tile_part;      // [ntiles] per-tile (tr, sq) partials
  unsigned* inst_done;     // [batch] tile-completion counters (zero between launches)
  double* traces_out;      // [batch][2] when ctl == nullptr, or nullptr
  const double* rn;        // [batch][ld_rn] FP64 row norms sum_k Y[r][k]^2 = (Y^2)_rr of the input
  long long ld_rn;
  // Row norms carried between launches (single-accumulator kernels): FP32
  // sums of squares of 32-column segments, rnp[b][seg][row] at
  // b * slot_rnp + seg * ld_rnp + row.  rnp_out receives those of Y' (every
  // (row, segment) once: the direct part of an upper tile or the column sums
  // of its mirror); rnp_in, when set, holds those of the input Y and replaces
  // rn: (Y^2)_rr = sum over segments in FP64.
  float* rnp_out;
  const float* rnp_in;
  long long ld_rnp, slot_rnp;
  int fused_ctl;           // 1: the last tile of an instance runs its control step with
                           //    (tr Y', ||Y'||_F^2) from the tiles (no row-norm launch)
  int nseg;                // 1: P = Y Y (one operand); 2: P = A B^T + B A^T (second map set)
  float* R;                // readout accumulator R = sum_i c_i X_i (layout of Y), or nullptr
  const float* const* Hobs; // [batch] N x N matrices A: the launch that writes D (OUT_D) also
                            // accumulates Tr[D A] per instance into dots_out[3 b] (or nullptr)
  const float* aux;        // adjoint mode: Y_n, same layout as Yin; dots <P, aux>, <Yin, aux>
  double* tile_dots;       // [ntiles][3] per-tile (tr Yin, <Yin, aux>, <P, aux>) in adjoint mode
  double* dots_out;        // [batch][3] per-instance sums of tile_dots
  int tri_planes;          // 1: the operand planes too are kept as upper super tiles (the
                           //    mirror plane stores are skipped); only for the CTA-pair kernel,
                           //    whose operand reads use the upper super tiles alone
  int tri_y;               // 1: Y' is kept as its upper triangle: off-diagonal tiles skip the
                           //    mirror store of Y' (the next launch reads the old values of
                           //    the upper tiles only); the operand planes and the D of the
                           //    final launch are stored whole
  float lo_scale;          // 2^s
  float lo_unscale;        // 2^-s
  int* err;                // device error word (SP2_ERR_DEVICE_TIMEOUT on a timed-out wait)
  unsigned long long wait_ns;  // bound of every mbarrier wait of the tcgen05 kernels (0: 4 s)
  int stall;               // fault injection: the MMA issuer first waits on a barrier that
                           // nothing arrives on, so that wait runs out after wait_ns
  // Soft synchronisation of the CTA pairs' K progress (CTA-pair kernel, one
  // instance): every sync_stages K stages a pair publishes the epoch it
  // finished in wave_ctr[epoch] and, before loading further, waits (bounded;
  // it stops waiting for the rest of the launch after one time-out) until
  // every pair has finished the epoch before that one.  Pairs that share an
  // operand panel then read it within a short time of each other, while it
  // is still in L2.  wave_ctr: zeroed counters of this launch; nullptr = off.
  unsigned* wave_ctr;
  int sync_stages;
  int wide;                // CTA-pair kernel: 1 = units of two super tiles (I, J), (I, J + 1) of a
                           //    row (tile list with four entries per unit; a unit without a second
                           //    tile has a null second entry, rows past N), A loaded once per stage
  int snake;               // 1: a pair walks K backwards on its odd-numbered tiles, so that a
                           //    wave starts on the K slices the previous wave left in L2
};

// tensor-core tile geometry
constexpr int kTcBM = 128;   // rows per CTA tile (TMEM lanes)
constexpr int kTcBN = 256;   // columns per CTA tile; 256 x 256 "super tiles" hold two CTA tiles
constexpr int kSimtB = 128;  // FFMA tile

// nan_row >= 0 (fault injection): that row of the stacked instances is
// treated as holding a NaN.
cudaError_t launch_gershgorin(const float* H, int N, long long ld, long long slot, int B, double2* partials,
                              unsigned* ticket, Ctl* ctl, double* bounds_out, int grid, cudaStream_t st,
                              long long nan_row = -1);
cudaError_t launch_gershgorin_batched(const float* const* Hs, const int* Ns, Ctl* ctl, int batch, double2* partials,
                                     unsigned* tickets, int grid_x, cudaStream_t st);
cudaError_t launch_input_layer(const float* const* Hs, const int* Ns, long long ld_in, float* Y, long long ld_y,
                               long long slot_y, __half* hi, __half* lo, __half* hp, long long ld_h, long long slot_h,
                               int rows_pad, int cols_pad, float lo_scale, Ctl* ctl, const double* bounds, double2* partials, unsigned* tickets,
                               int shift, int ctl_step, int batch, int grid_x, cudaStream_t st);
cudaError_t launch_split(const float* X, long long n, float lo_scale, __half* hi, __half* lo, int grid,
                         cudaStream_t st);
cudaError_t launch_split_pad(const float* X, long long ld_x, long long slot_x, int N, int B, float lo_scale,
                             __half* hi, __half* lo, __half* hp, long long ld_h, long long slot_h, int grid,
                             cudaStream_t st);
// R[b] = s Y[b] + d[b] I (diagonal in FP64): the readout of the input layer.
cudaError_t launch_readout_init(const float* Y, long long ld_y, long long slot_y, int N, int B, float s,
                                const double* d, float* R, int grid_x, cudaStream_t st);
cudaError_t launch_materialize(const float* Y, long long ld_y, long long slot_y, int N, int B, const double* alpha,
                               float* out, long long ld_o, long long slot_o, int grid_x, cudaStream_t st);
cudaError_t launch_observable(const float* D, const float* A, long long n, double* block_out, int grid,
                              cudaStream_t st);

// rn[b][i] = sum_k Y[b][i][k]^2 in FP64 for every row of every instance.
// With ctl: instances whose next launch is inactive are skipped, and the
// last block of an instance runs its control step with (trY_new, sum rn).
cudaError_t launch_rownorm(const float* Y, long long ld_y, long long slot_y, const int* Ns, int batch, int max_rows,
                           double* rn, long long ld_rn, Ctl* ctl, double2* partials, unsigned* tickets, int grid_x,
                           cudaStream_t st);

// Single-accumulator split squaring (tcgen05, double-buffered TMEM): the
// three products hp hp + lo' hp + hp lo' = 2^(2s) (hi hi + lo hi + hi lo)
// go into one FP32 accumulator (hp = 2^s hi, lo' = 2^s lo).  tmaps: {p0(A),
// p1(A), p0(B), p1(B)} with p0 = hp, p1 = lo'; split = false: plain FP16
// with p0 = hi (p1 unused).  The epilogue writes the planes whose output
// pointers are set (hp_out and lo_out for split, hi_out for plain).
cudaError_t launch_syrk_tc1(const SqArgs& a, const CUtensorMap* tmaps, bool split, int grid, cudaStream_t st);
size_t syrk_tc1_smem_bytes(bool split);
// The same product run by CTA pairs (clusters of 2) whose MMAs span both CTAs
// (M = 256 per super tile, each CTA holding 128 rows of A and of B): tiles
// come in (h = 0, h = 1) pairs of one super tile, a.ntiles = 2 x super tiles,
// and the B maps have 128-row boxes.  tmaps holds
// six maps: the four above and {p0, p1} with 64 x 64 boxes, through which the
// K blocks left of the diagonal are read transposed from the upper tiles.
cudaError_t launch_syrk_tc2(const SqArgs& a, const CUtensorMap* tmaps, bool split, int grid, cudaStream_t st);
size_t syrk_tc2_smem_bytes(bool split);

cudaError_t launch_syrk_simt(const SqArgs& a, int grid, cudaStream_t st);

// Tensor-core squaring.  tmaps: {hi(A box), lo(A box), hi(B box), lo(B box)}
// over the current split buffers, followed (nseg == 2) by the four maps of
// the second K segment.  split = false: plain FP16 (hi only).
cudaError_t launch_syrk_tc(const SqArgs& a, const CUtensorMap* tmaps, bool split, int grid, cudaStream_t st);
size_t syrk_tc_smem_bytes(bool split);

// Encodes a 3D tensor map over FP16 [batch][rows][ld] with box {box_k, box_rows, 1}.
bool make_tmap_f16(CUtensorMap* out, const void* base, int cols, int rows, int batch, long long ld, long long slot,
                   int box_k, int box_rows);

}  // namespace sp2
