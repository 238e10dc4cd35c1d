// Internal declarations shared by the libfgfrft translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fgfrft.h"

// ---------------------------------------------------------------------------
// plan record (host side; the device memory it points into belongs to the caller)
// ---------------------------------------------------------------------------
struct fgfrft_plan_s {
  int64_t N;
  int L_max;
  int storage;
  int nblk;            // 2 * L_max + 2: M_{-L_max} .. M_{L_max}, then P
  int64_t blk_elems;   // c64 entries per block (N*N padded to 32)
  int64_t Np;          // fp16 row pitch in elements (N rounded up to 8, 16-byte rows)
  int64_t plane_elems; // fp16 entries per plane (N * Np, padded to 128)
  int64_t qplane;      // fp16 entries per plane of the assembled split operators (work buffers)
  size_t bytes;
  uint32_t* dstatus;   // device status word (bit set of kernel error codes)
  float2* c64;         // [nblk][blk_elems] or NULL
  __half* f16;         // [nblk][4][plane_elems] or NULL; planes re_hi, re_lo, im_hi, im_lo
  __half* f16T;        // entry-major copy (chunk-major, see fg_entry_major) or NULL
  float* h32;          // half stack [L_max + 2][re, im][hplane]: M_0 .. M_L_max, then P; or NULL
  int nt;              // 64 x 64 tiles per dimension of the half stack
  int64_t hplane;      // floats per half-stack plane (nt * nt * 4096)
  int64_t Kp;          // entry-major row pitch (nblk rounded up to 8)
  int64_t planeT;      // entries per chunk plane of the entry-major copy (N * N padded to 128)
  int r_neg1;
  double proj_residual;
  int squarings;
  double min_gap_lo, min_gap_hi;  // bracket of min_{k not in I} |lambda_k + 1| (inf when r_neg1 = N)
  double neg1_tol;                // 0: adaptive classification
  bool real;           // F (hence every stored block) is real: tensor paths skip the imaginary planes
  // pair stack (fg_pair_stack) for the fused multi-order assembly of split operators: built
  // when F is real without a -1 eigenvalue (M_{-l} = M_l^T, M_0 = I), N % 128 == 0 and
  // L_max % 16 == 0, in the entry-major storage's imaginary planes (unused for a real F)
  bool pair;
  __half* pairS;
  int64_t pair_rows;
};

// Index of the stored block holding M_l (l in -L_max..L_max) and of P.
static inline int blk_of_power(const fgfrft_plan_s* p, int l) { return p->L_max + l; }
static inline int blk_of_P(const fgfrft_plan_s* p) { return 2 * p->L_max + 1; }

// Scale applied to stored entries before the fp16 hi/lo split (exact power of two):
// entries of the partial isometries F^l P_c and of Q are at most ~1.2 in magnitude,
// so 2^12 keeps hi below the fp16 maximum and lo in the normal range for typical
// entries (~N^{-1/2}).
#define FG_SPLIT_SHIFT 12
// Signals are scaled per column by 2^e so that max |x| * 2^e lies in [2^13, 2^14).
#define FG_X_TARGET_EXP 13
// The fused assembly's coefficients (modulus at most 1) are all scaled by 2^FG_COEF_EXP.
#define FG_COEF_EXP 14

// Device status codes (OR-ed into the plan's status word).
#define FG_STATUS_WAIT_TIMEOUT 1u
#define FG_STATUS_LAUNCH_MISMATCH 2u  // a kernel found its launch sizing unusable and did nothing

// Bounded waits give up after this many nanoseconds of %globaltimer.
#define FG_WAIT_LIMIT_NS 2000000000ull

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same test, suspending the thread until the phase completes or about hint_ns have passed
// (the retry of a bounded wait: a waiting warp then takes no issue slots from working ones).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most
// FG_WAIT_LIMIT_NS.  On timeout, record it in *status and return false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > FG_WAIT_LIMIT_NS) {
      atomicOr(status, FG_STATUS_WAIT_TIMEOUT);
      return false;
    }
  }
}

// 1-D bulk copy global -> shared, completion counted in bytes on *bar.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_g2s_evict_first(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                     uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
      "%4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 3-D tensor-map tile load (global -> shared), completion counted in bytes on *bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Pair tiles (the pair stack of a real F without a -1 eigenvalue, N a multiple of 128): tile t
// holds the 128 entries (i, 128 kt + r), r < 128, of the block-upper region kt >= i / 128, in
// the order of row blocks I = i / 128, each 128 rows of nbt - I tiles (nbt = N / 128).
__host__ __device__ __forceinline__ void pair_tile(int64_t t, int nbt, int& i, int& kt) {
  int I = 0;
  int64_t base = 0;
  while (I < nbt - 1 && base + 128 * (int64_t)(nbt - I) <= t) {
    base += 128 * (int64_t)(nbt - I);
    ++I;
  }
  const int w = nbt - I;
  const int64_t local = t - base;
  i = 128 * I + (int)(local / w);
  kt = I + (int)(local % w);
}
__host__ __device__ __forceinline__ int64_t pair_tiles(int nbt) { return 128 * (int64_t)nbt * (nbt + 1) / 2; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
#endif  // __CUDACC__

// ---------------------------------------------------------------------------
// instrumentation (timing.cu): per-class launch counters and optional event timing
// ---------------------------------------------------------------------------
void fg_note_launch(int cls, int n = 1);

// 3-D fp16 tensor map {cols (contiguous), rows (pitch elements apart), planes (plane_elems
// apart)} with a box_cols x box_rows x 1 box; swizzle_bytes is 0, 32, 64 or 128.  Out-of-range
// elements of a box read as zero.  False if the driver rejects the map.
bool fg_make_map_f16(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t pitch, int64_t nplanes,
                     int64_t plane_elems, int box_cols, int box_rows, int swizzle_bytes);

// Host-to-device copy of a small per-call table, staged through pinned memory so that the
// call stays asynchronous (the source may be reused as soon as this returns).
cudaError_t fg_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s);
// A pinned copy of a small table that kernels read directly from host memory: returns a
// token (and the device-readable address in *dev), or -1 when the caller must copy instead.
// fg_stage_done(token, s) must follow once every kernel that reads it is enqueued on s.
int fg_stage(const void* src, size_t bytes, const void** dev);
void fg_stage_done(int token, cudaStream_t s);
// True while s is being captured into a CUDA graph.
bool fg_capturing(cudaStream_t s);
// dst (device) <- src (host), bytes carried in the parameters of small kernels: what a graph
// captures keeps the bytes (used for the host tables of a call under capture).
cudaError_t fg_upload(void* dst, const void* src, size_t bytes, cudaStream_t s);
// An auxiliary stream of the current device for work of a call that may run beside the
// rest of it: fg_fork makes it wait for everything queued on s so far and returns it
// (nullptr: run everything on s); fg_join makes s wait for everything queued on it so far.
cudaStream_t fg_fork(cudaStream_t s);
cudaError_t fg_join(cudaStream_t aux, cudaStream_t s);
struct FgTimed {  // records a CUDA event pair around its scope when timing is enabled
  FgTimed(int cls, cudaStream_t s);
  ~FgTimed();
  FgTimed(const FgTimed&) = delete;
  FgTimed& operator=(const FgTimed&) = delete;

 private:
  int cls_;
  cudaStream_t s_;
  long slot_;
};

// ---------------------------------------------------------------------------
// launchers (one translation unit each)
// ---------------------------------------------------------------------------
// offline.cu
// real: A and B real (zero imaginary parts), alpha and beta real; a quarter of the FP64
// work, the same real parts, zero imaginary parts in C.
cudaError_t fg_zgemm(bool transA, bool transB, int M, int N, int K, double2 alpha, const double2* A, int lda,
                     const double2* B, int ldb, double2 beta, double2* C, int ldc, cudaStream_t s,
                     bool real = false);
cudaError_t fg_zaxpby_identity(int64_t N, double2 a, const double2* X, double2 b, double2 d, double2* Y,
                               cudaStream_t s);  // Y = a*X + b*Y + d*I
cudaError_t fg_zherm_sym(int64_t N, double2* S, cudaStream_t s);  // S <- (S + S^H)/2
cudaError_t fg_zmcweeny(int64_t N, const double2* P2, const double2* P3, double2* P, cudaStream_t s);
cudaError_t fg_ztrace_fro(int64_t N, const double2* S, const double2* Sub, double* out, cudaStream_t s);
cudaError_t fg_zimag_sq(int64_t N, const double2* F, double* out, cudaStream_t s);  // out[0] = sum Im(F)^2
cudaError_t fg_store_block(int64_t N, const double2* M, bool conj_transpose, float2* c64, __half* f16,
                           int64_t Np, int64_t plane_elems, cudaStream_t s);
// Entry-major copy of the split stack for the fused multi-order assembly: for plane p,
// entry e = i * N + k and stored block b < Kp (blocks nblk..Kp-1 zero), chunk-major so that
// every 32-block chunk of 128 entries is one contiguous 8 KB tile:
//   b < 32 * (Kp / 32):  T[((p * (Kp / 32) + b / 32) * planeT + e) * 32 + b % 32]
//   else (the tail):     T[4 * (Kp / 32) * planeT * 32 + (p * planeT + e) * (Kp % 32) + b % 32]
cudaError_t fg_entry_major(const __half* f16, int nblk, int64_t N, int64_t Np, int64_t plane_elems, __half* T,
                           int64_t Kp, int64_t planeT, cudaStream_t s);
// Pair stack of a real plan without a -1 eigenvalue (N % 128 == 0, L_max % 16 == 0): row
// r < 128 of pair tile t = (i, kt) (pair_tile) holds, at column c < K2 = 2 L_max, split plane
// p (0: hi, 1: lo) of M_l[i][128 kt + r], l = c - L_max for c < L_max, else c - L_max + 1 (M_0 = I
// is not stored).  Tile-contiguous, as the MMA operand image a ring stage holds: tile t at
// PS + t * 2 K2 * 128, then per 32-column chunk, per plane, 128 rows of 64 bytes whose 16-byte
// pieces j sit at j ^ ((r >> 1) & 3) (the 64-byte swizzle); R = 128 * pair_tiles(N / 128) rows.
cudaError_t fg_pair_stack(const __half* f16, int L_max, int64_t N, int64_t Np, int64_t plane_elems, __half* PS,
                          int64_t R, cudaStream_t s);
// One half-stack block (FP32 re/im planes of 64 x 64 swizzled tiles) from an FP64 matrix.
cudaError_t fg_store_half(int64_t N, const double2* M, float* planes, int nt, int64_t hplane, cudaStream_t s);

// assemble.cu
// One order from the half stack (blocks M_0..M_L_max and P, FP32 tiled planes): Q = e^{j pi a} P
// + sum_{|l| <= L} c_l M_l with M_{-l} = M_l^H read as transposed tiles.  coef = [2L+2] as
// fg_coeffs writes it.  c64 output Q [N][N] or split output Qs (pitch Np, plane stride q_plane).
cudaError_t fg_assemble_half(const float* planes, int64_t hplane, int nt, int L_max, int L, bool cplx, bool has_p,
                             int64_t N, int64_t Np, const float2* coef, float2* Q, __half* Qs, int64_t q_plane,
                             bool write_im, uint32_t* status, cudaStream_t s);
// Q (c64, [NN]) or, with Qs != NULL, split fp16 planes of N rows x Np (plane stride plane_elems).
cudaError_t fg_assemble_single(const float2* stack, int64_t blk_elems, int b0, int nb_pow, int p_blk,
                               int64_t NN, const float2* coef, float2* Q, uint32_t* status, cudaStream_t s,
                               __half* Qs = nullptr, int64_t N = 0, int64_t Np = 0, int64_t plane_elems = 0);
// Real F: one order from the two real split planes of each stored block (blk_stride halves
// between blocks, plane_elems between planes); output c64 Q [N*N] or split planes Qs with
// the stored pitch (imaginary planes only when write_im).
cudaError_t fg_assemble_single_real(const __half* planes, int64_t blk_stride, int64_t plane_elems, int b0,
                                    int nb_pow, int p_blk, int64_t N, int64_t Np, const float2* coef, float2* Q,
                                    __half* Qs, int64_t q_plane, bool write_im, uint32_t* status, cudaStream_t s);
// Multi-order: Q_a = sum_b coef[b * A + a] * block_b for a < A; output c64 (Qc) or split fp16 (Qs).
cudaError_t fg_assemble_multi(const float2* stack, int64_t blk_elems, int b0, int nb_pow, int p_blk,
                              int64_t N, int A, const float2* coef, float2* Qc, __half* Qs, int64_t Np,
                              int64_t plane_elems, uint32_t* status, cudaStream_t s);

// gemm_simt.cu: Y[j][i] (+)= sum_b coef[b][j] * sum_k A_b[i][k] X[j][k]   (FP32 CUDA cores)
struct SimtStackArgs {
  const float2* A;       // block b starts at A + blk_index(b) * blk_elems, rows of lda entries
  int64_t blk_elems;
  int lda;
  int b0, nb_pow, p_blk; // blocks b0 .. b0+nb_pow-1, then p_blk (p_blk < 0: none)
  int N;                 // rows of A and length of each signal
  int ncols;             // columns (signals) handled
  const float2* X;       // signal j at X + j * N
  float2* Y;             // output signal j at Y + j * N
  float2* D;             // dual output or NULL
  const float2* coef;    // [nblk][ldcoef] or NULL (unscaled single block)
  const float2* coefd;   // [nblk][ldcoef] for D
  int ldcoef;
  // plain batched mode (coef == NULL): group g = blockIdx.z multiplies A + g * group_stride by
  // columns groups[g].x .. groups[g].x + groups[g].y - 1 (device table); NULL = one group
  const int2* groups;
  int64_t group_stride;
  int max_group_cols;
  int ngroups;
};
cudaError_t fg_simt_stacked(const SimtStackArgs& a, cudaStream_t s);

// reduce.cu
// coefficient (b, j) at b * ldb + j * ldj; blocks b = 0..2L are the powers -L..L, b = 2L+1 is P
cudaError_t fg_coeffs(const double* alpha, int B, int L, bool adjoint, float2* coef, float2* coefd, int64_t ldb,
                      int64_t ldj, cudaStream_t s);
int fg_grad_chunks(int64_t N);
// out = sum over s < splits of parts[s][0 .. count), float2 entries, in split order
cudaError_t fg_sum_splits(const float2* parts, int splits, int64_t count, float2* out, cudaStream_t s);
// out[j] = Re sum_i conj(G_ji) D_ji (FP64 partials per 1024-entry chunk, summed in a fixed
// order); sum_all: out[0] = the sum over all j (one order shared by every column).
cudaError_t fg_grad_alpha(const float2* G, const float2* D, int64_t B, int64_t N, float* out, double* partials,
                          cudaStream_t s, bool sum_all = false);
// Split each signal (row of X) into fp16 planes with a per-signal power-of-two scale.
// bimag (may be NULL) is cleared first and set nonzero when some signal has a nonzero
// imaginary part.  X is B x N c64, or B x N real float32 when x_real.
cudaError_t fg_split_signals(const void* X, int64_t B, int64_t N, int64_t Np, int64_t rows_pad, __half* planes,
                             int* col_exp, cudaStream_t s, int* bimag = nullptr, bool x_real = false);
// Split coefficient planes [4][A][Kp] (and per-order exponents) of the fused multi-order
// assembly: order a's column holds c_l(alpha_a) at stored position L_max + l for |l| <= L,
// e^{j pi alpha_a} at the P position 2 L_max + 1, zeros elsewhere.  alpha: the orders on the
// device; alpha_host (optional, the same values): with at most 64 orders they travel in the
// launch's parameters, so the kernel does not wait on a read of the table.
cudaError_t fg_coeff_planes(const double* alpha, int64_t A, int L, int L_max, int64_t Kp, __half* planes,
                            int* col_exp, cudaStream_t s, const double* alpha_host = nullptr);
// Coefficient planes of the pair assembly (A <= 64 orders): [4][128][2 L_max], row a < A holding
// c_l(alpha_a) and row 64 + a holding c_{-l}(alpha_a) at the pair stack's column of each power
// l != 0 (zero for |l| > L), other rows zero; col_exp[0 .. 127] = FG_COEF_EXP; diag[a] = c_0(alpha_a)
// * 2^(FG_SPLIT_SHIFT + FG_COEF_EXP).
cudaError_t fg_coeff_planes_pair(const double* alpha, int64_t A, int L, int L_max, __half* planes, int* col_exp,
                                 float* diag, cudaStream_t s, const double* alpha_host = nullptr);
