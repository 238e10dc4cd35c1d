// Tensor-core (tcgen05) GEMM paths: split-fp16 operands, FP32 accumulators in TMEM.
#pragma once
#include <vector>

#include "internal.h"

// True when the tcgen05 kernels are compiled in and the current device is sm_103.
bool fg_tc_available();
// True when the pair assembly's launch (K = 2 L_max powers, resident coefficients, staging
// buffers, two ring stages) fits in the shared memory of the current device.
bool fg_tc_pair_fits(int L_max);
// Rows of the signal split planes for B signals in the given number of groups
// (padded so that every TMA box row stays inside the buffer).
int64_t fg_tc_signal_rows(int64_t B, int64_t groups);
// Device scratch (tile tables, partial sums) of one call.
size_t fg_tc_scratch_bytes(int64_t N, int64_t B, int64_t groups, int nblk);

// Y[:, group g] = Q_g X[:, group g] for consecutive column groups (assembled path).
struct TcGroupedArgs {
  int64_t N, Np, plane_elems;
  const __half* Qs;        // [groups][4][plane_elems] split operators (scaled by 2^FG_SPLIT_SHIFT)
  int64_t groups;
  const int64_t* gstart;   // host: first column of each group
  const int64_t* gcount;   // host: columns of each group
  const void* X;           // B x N c64 signals (real float32 with x_real)
  float2* Y;               // B x N c64 outputs (real float32 with y_real)
  __half* Xs;              // work: [4][xs_rows][Np] split signals
  int64_t xs_rows;
  int* col_exp;            // work: [xs_rows]
  int64_t B;
  void* scratch;
  size_t scratch_bytes;
  uint32_t* status;
  bool real_a;             // every Q_g is real (imaginary planes zero): 6 MMAs per k16 step
  int* bimag;              // work: one word, 0 after the split when every signal is real
  const int4* tiles_dev;   // optional: the tile table (fg_tc_grouped_tiles) already on the device
  int64_t ntiles;
  bool x_split_done;       // Xs, col_exp and bimag already hold this X (a second GEMM on it)
  bool x_real;             // X is real float32
  bool y_real;             // write only the real parts (the caller knows the products are real)
  bool pair;               // Qs came from the pair assembly: left of each row tile's diagonal
                           // block, Q_g[i][k] is read from planes 2, 3 at (k, i) (real_a only)
};
cudaError_t fg_tc_grouped_apply(const TcGroupedArgs& a, cudaStream_t s);
// Column-tile width of the grouped GEMM (256 for real operators, else 128) and its tile table:
// {row tile, plane base of Q_g, first column, end column}.
int fg_tc_grouped_bn(bool real_a);
void fg_tc_grouped_tiles(int64_t N, int64_t groups, const int64_t* gstart, const int64_t* gcount, int bn,
                         std::vector<int4>& tiles);

// Y[:, j] = sum_b coef[b][j] A_b X[:, j] over the stored blocks (stacked path),
// D likewise with coefd (dual accumulator, may be NULL).
struct TcStackedArgs {
  int64_t N, Np, plane_elems;
  const __half* stack;     // [nblk_total][4][plane_elems]
  int b0, nb_pow, p_blk;
  const void* X;           // B x N c64 signals (real float32 with x_real)
  float2* Y;
  float2* D;
  const float2* coef;      // [nb_pow + 1][B]
  const float2* coefd;
  int64_t B;
  __half* Xs;
  int64_t xs_rows;
  int* col_exp;
  void* scratch;
  size_t scratch_bytes;
  uint32_t* status;
  bool real_a;             // every stored block is real (real F)
  int* bimag;              // work: one word, 0 after the split when every signal is real
  bool x_real;             // X is real float32
  float2* Ysplit;          // work: [splits][B][N] partial sums (splits > 1)
  float2* Dsplit;          // work: the same for D
};
cudaError_t fg_tc_stacked_apply(const TcStackedArgs& a, cudaStream_t s);
// Block splits of a stacked launch (1, or more when the tiles are fewer than the SMs).
int fg_tc_stacked_splits(int64_t N, int64_t B, int nblk);

// Fused multi-order assembly on the tensor cores: Q_a = sum_k C[a][k] S_k over all
// stored blocks k (zero coefficients outside -L..L), from the entry-major split stack and
// the split coefficient planes Cs (filled by fg_coeff_planes).
struct TcAssembleArgs {
  // chunk-major fp16 (scaled by 2^FG_SPLIT_SHIFT): [4 planes][Kp / 32][planeT][32], then
  // the tail [4 planes][planeT][Kp mod 32]
  const __half* entry_stack;
  int64_t entries;            // N * N
  int64_t K;                  // stored blocks (2 L_max + 2)
  int64_t Kp;                 // K rounded up to 8
  int64_t planeT;             // entries per chunk plane (N * N padded to 128)
  int64_t A;
  const __half* Cs;           // [4][A][Kp] split coefficients
  const int* col_exp;         // [A] their exponents
  float2* Qc;                 // c64 output [A][N*N] (when Qs is NULL)
  __half* Qs;                 // split output [A][4][plane_elems] or NULL
  int64_t N, Np, plane_elems;
  void* scratch;
  size_t scratch_bytes;
  uint32_t* status;
  bool real_a;                // the stored blocks are real (real F)
  bool skip_im;               // split output whose imaginary part is zero (real F, no -1 eigenvalue)
  bool re_only;               // real blocks and a real result: form only the real accumulator
  // pair assembly (real F without a -1 eigenvalue, split output, A <= 64, N % 128 == 0):
  // pair_stack != NULL selects it; Cs is then [4][128][K2] (rows a: c_l(alpha_a), rows 64 + a:
  // c_{-l}(alpha_a), over the stored powers l != 0) and Qs receives Q_a in planes 0, 1 on and
  // right of the diagonal blocks, Q_a^T in planes 2, 3 left of them (see fg_pair_stack)
  const __half* pair_stack;   // chunk-major [2 planes][K2 / 32][pair_rows][32]
  int64_t pair_rows;          // 128 * (pair tiles)
  int64_t K2;                 // 2 L_max
  const float* diag;          // [A]: c_0(alpha_a) at the accumulator scale
};
cudaError_t fg_tc_assemble(const TcAssembleArgs& a, cudaStream_t s);
size_t fg_tc_assemble_scratch_bytes(int64_t entries, int64_t A);
