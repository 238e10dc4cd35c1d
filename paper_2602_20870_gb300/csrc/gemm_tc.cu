// Tensor-core (tcgen05) complex GEMM over stacked blocks, split-fp16 operands.
//
//   T_b = A_b[rows, :] X[cols, :]^T            (complex, K = N; Def. 2 x~ = Q x)
//   Y[j] (+)= coef[b][j] T_b[:, j]              (Def. 1 per column; or Y = T when
//   D[j] (+)= coefd[b][j] T_b[:, j]              there is one block per tile, Prop. 3)
//
// Operands are stored as four fp16 planes {re_hi, re_lo, im_hi, im_lo}: A scaled by
// 2^FG_SPLIT_SHIFT, signal column j by 2^{e_j}; hi = fp16(v), lo = fp16(v - hi).
// Each complex product keeps the three significant split products
// (hi*hi + hi*lo + lo*hi), so every K=16 step issues 12 MMAs:
//   acc_re += Ar*Xr - Ai*Xi ,  acc_im += Ar*Xi + Ai*Xr   (3 split products each term)
// with FP32 accumulation in tensor memory (TMEM).
//
// CTA layout (one CTA per SM, persistent over a tile list):
//   warp 0      TMA producer: 3-D tensor-map loads of the A planes (+ the X planes unless
//               B is resident) per stage (32 k-values, 64-byte swizzled rows) into a ring
//               sized to the shared memory left;
//   warp 1      allocates the TMEM columns; one thread issues tcgen05.mma and
//               tcgen05.commit; accumulators in 2..8 buffers of [re BN | im BN];
//   warps 2..   epilogue, groups of four warps (one per TMEM lane quadrant; 2 groups, 4 for
//               the fused assembly): tcgen05.ld the finished block, undo the power-of-two
//               scales, apply the per-column coefficients, and accumulate into Y/D in
//               global memory (each output tile is owned by one CTA, blocks in order,
//               so the sums are deterministic), or write the split operators.
// Every mbarrier wait is bounded; on a timeout the CTA records it in the status word,
// stops issuing work, waits (bounded) for its copies and MMAs in flight, frees TMEM and
// returns.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "tc.h"

namespace {

constexpr int TC_BM = 128;                 // rows per tile (TMEM lanes)
// k per chunk: 32 fp16 = 64-byte rows (64-byte swizzle), or KC = 64 = 128-byte rows
// (128-byte swizzle), which the tensor-map loads serve from L2 at a higher rate
constexpr int TC_KC = 32;
constexpr int TC_EPI_WARP0 = 2;  // warps before the epilogue: the producer and the MMA issuer
constexpr int TC_MAXBUF = 8;     // TMEM accumulator buffers at most
constexpr int TC_BN_MAX = 256;
constexpr int TC_BN_STD = 128;  // column-tile width of the stacked and complex grouped GEMMs

// Column-tile width BN (complex columns per tile): 128, or 64 for few columns.
// RB ("resident B"): every tile uses the same B columns (one column tile), so all k-chunks
// of B are loaded once per CTA into shared memory and the ring stages carry A only.
constexpr int TC_RB_MAXCH = 5;  // resident-B mode: at most 5 k-chunks (K <= 160)
// RA ("real A"): the A operand is real (its imaginary planes are zero), so only the two
// real planes are loaded and each k16 step issues 6 MMAs (Ar*Xr, Ar*Xi) instead of 12.
template <int BN, bool RB = false, bool RA = false, int KC = TC_KC>
struct TcCfg {
  static constexpr int PLANE_A = TC_BM * KC * 2;
  static constexpr int PLANE_B = BN * KC * 2;
  static constexpr int A_PLANES = RA ? 2 : 4;
  // Epilogue warps: 8, or 16 for the resident-B launch (the fused assembly), whose few MMAs
  // per tile leave the epilogue (TMEM -> fp16 hi/lo -> global) as the critical path: four
  // warp groups take turns on the tiles, so twice the warps hide its latencies.
  static constexpr int EPI_WARPS = RB ? 16 : 8;
  static constexpr int THREADS = 32 * TC_EPI_WARP0 + 32 * EPI_WARPS;
  // accumulator columns an epilogue warp loads at a time (16 keeps 18 warps within the
  // register file without spills)
  static constexpr int CW = RB ? 16 : 32;
  // 2 buffers x [re BN | im BN]; BN = 256 has 512 columns: 2 real-only buffers or 1 complex;
  // the resident-B launch takes all 512 columns (up to 8 buffers for its four warp groups)
  static constexpr int TMEM_COLS = RB ? 512 : (4 * BN > 512 ? 512 : 4 * BN);
  // kind::f16 instruction descriptor: D f32, A/B f16, both K-major, N = BN, M = 128.
  static constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
  static constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);
  // N = 2 BN: the hi and lo planes of B are adjacent in shared memory (BN rows each, a
  // whole number of 8-row swizzle atoms), so one MMA forms A*B_hi and A*B_lo side by side
  static constexpr uint32_t IDESC_2N = (1u << 4) | ((uint32_t)(2 * BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
  // merged split products for a real product on the resident-B launch (BN = 64):
  // acc[0:BN] = A_hi*B_hi + A_lo*B_hi, acc[BN:2BN] = A_hi*B_lo, 2 MMAs per k16 step instead of 3
  // (the 128-column pair launch keeps 3 MMAs, so that four accumulator buffers fit in TMEM)
  static constexpr bool MERGE = RB && BN == 64;
};

// Shared memory: this control block, then the resident B operand (RB: k-chunks x 4 planes),
// then as many ring stages as fit in the rest (at most TC_MAXST).  A stage holds the A
// planes and the B planes the launch needs (2 for a real B, else 4), so a launch with a
// real operand gets a deeper ring from the same shared memory.
constexpr int TC_MAXST = 16;
struct __align__(1024) TcCtl {
  uint64_t full[TC_MAXST];
  uint64_t empty[TC_MAXST];
  uint64_t bfull;
  uint64_t tfull[TC_MAXBUF];
  uint64_t tempty[TC_MAXBUF];
  uint64_t drain;
  uint32_t tmem_base;
  volatile int abort;
  float scale[TC_BN_MAX];
};
// the smallest ring the kernel runs with
constexpr int TC_MIN_STAGES = 2;

struct TcParams {
  const int4* tiles;  // {row tile, A plane base (grouped), first column, end column}; NULL: tile t
                      // is row tile t of the single column tile [0, arith_cols)
  int ntiles;
  int arith_cols;
  int nblk;           // blocks per tile
  int grouped;        // 1: A plane base from the tile, one block; 0: stacked blocks
  int b0, nb_pow, p_blk;
  int64_t rows;       // rows of A (M extent) and the stride of output columns
  int kchunks;
  int kvalid;         // k range with data (0: kchunks * 32); k16 steps at or past it are all zero
  // split output (fused assembly): column j, row r -> Qs[j][plane][r / qN][r % qN] (pitch qNp),
  // value scaled by 2^FG_SPLIT_SHIFT and split into fp16 hi/lo
  __half* Qs;
  int64_t qN, qNp, qplane;
  int skip_im;        // split output: the imaginary planes are zero and not written
  int re_only;        // real A and a real product: only the real accumulator is formed
  int smem_bytes;     // dynamic shared memory usable from the 1024-aligned base
  float uscale;       // nonzero: every column has this output scale (no per-column exponents)
  int y_real;         // grouped output: Y is real float32 (only the real parts are written)
  int cps;            // k-chunks per ring stage (one mbarrier handshake per group of chunks)
  // chunk-major A (the entry-major stack): k-chunk kc < a_nfull of plane q is plane
  // q * a_nfull + kc of the A map (32 columns each); the last chunk, narrower, is plane q
  // of the tail map (its missing columns read as zeros)
  int a_chunked;
  int a_nfull;
  // narrow tail (chunk-major A with the resident B and every chunk of a tile in one stage):
  // the tail chunk is a 16-column box with 32-byte swizzle (4 KB per plane, one k16 step)
  // instead of a 32-column one, so a stage holds no zero-filled columns
  int a_tail16;
  int stage_bytes;    // nonzero: the stage size the host computed for this layout
  // stacked tiles split over the stored blocks: tile.y = s takes blocks [s * bps, (s + 1) * bps)
  // and writes its partial sums at Y + s * split_stride (D likewise); bps = 0: no split
  int bps;
  int64_t split_stride;
  // pair assembly (real F, no -1 eigenvalue): A rows are entry pairs of the pair stack, tile t
  // holds entries (i, 128 kt + r), r < 128, of the block-upper region (kt >= i / 128); columns
  // j < 64 are the orders' Q[i][k], columns 64 + j their Q[k][i] (mirror), written at the same
  // position (i, k) of planes 2, 3 (the transposed store) when kt > i / 128.  pair_nbt = N / 128
  // (0: not a pair launch); diag[j] is added to Q[i][i] (c_0 of order j, accumulator scale).
  int pair_nbt;
  int pair_A;
  const float* diag;
  // A operand stored as ring-stage images (the pair stack): tile t's stage is one bulk copy of
  // stage_bytes from a_img + t * stage_bytes (streamed once: L2 evict-first)
  const uint8_t* a_img;
  // pair assembly output through shared memory: each epilogue group stages a 16-column chunk
  // (16 orders x 2 planes x 128 entries, 8 KB) and one 4-D tensor store (tmT: {k, i, plane,
  // order}) writes it; out_bytes = the staging area (out_bufs 8 KB buffers per group: two when
  // they fit beside two ring stages, else one), 0: direct stores
  int out_bytes;
  int out_bufs;
  int out_pairs;      // 1: two 16-order chunks per tensor store (one 16 KB buffer per group)
  // grouped GEMM over pair-structured operators: k-chunks left of the row tile's diagonal
  // block come from the transposed store (planes 2, 3 of the group), read MN-major
  int pair_lower;
  const int* bimag;   // NULL, or a device word that is 0 when every B column is real
  const float2* coef;
  const float2* coefd;
  int64_t ldcoef;
  float2* Y;
  float2* D;
  const int* col_exp;
  uint32_t* status;
};

__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;            // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)4 << 61;                     // 64-byte swizzle
  return d;
}

// K-major operand with 32-byte rows and 32-byte swizzle (8-row atoms of 256 bytes)
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(256 >> 4) << 32;            // stride byte offset: 8 rows x 32 B
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)6 << 61;                     // 32-byte swizzle
  return d;
}

// K-major operand with 128-byte rows and 128-byte swizzle (8-row atoms of 1 KB)
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// MN-major operand, 128-byte swizzle: 8 k-rows of 128 bytes (64 MN values) per 1 KB atom;
// the two 64-value halves of the 128 MN values are 4 KB apart (leading byte offset), the
// 8-row k groups 1 KB apart (stride byte offset)
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)(4096 >> 4) << 16;           // leading byte offset: the next 64 MN values
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: the next 8 k-rows
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

template <int KC>
__device__ __forceinline__ uint64_t desc_kc(uint32_t saddr) {
  return KC == 64 ? desc_sw128(saddr) : desc_sw64(saddr);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&v)[32]) { tmem_ld32(taddr, v); }
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&v)[16]) { tmem_ld16(taddr, v); }

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bounded wait that also gives up at once when another role already aborted.
// The retries suspend in the barrier (up to 20 us each, woken when the phase completes), so
// the many waiting roles of a CTA do not crowd out the issue slots of the working ones.
template <class Smem>
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, Smem& sm, uint32_t* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    if (sm.abort) return false;
    if (global_timer_ns() - t0 > FG_WAIT_LIMIT_NS) {
      sm.abort = 1;
      atomicOr(status, FG_STATUS_WAIT_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ int4 tile_of(const TcParams& p, int t) {
  return p.tiles ? p.tiles[t] : make_int4(t, 0, 0, p.arith_cols);
}

// the blocks a tile accumulates: all of them, or its split's range
__device__ __forceinline__ int2 blk_range(const TcParams& p, const int4& tl) {
  if (p.grouped || p.bps == 0) return make_int2(0, p.nblk);
  const int b0 = tl.y * p.bps;
  return make_int2(b0, min(b0 + p.bps, p.nblk));
}

// Split-output epilogue of one CW-column chunk: column j0 + c of this thread's row goes to
// Qs + (j0 + c) * 4 * qplane + qoff as fp16 hi/lo planes (re_hi, re_lo, im_hi, im_lo).
// UNIFORM: every column has the scale p.uscale (no per-column table).
template <bool UNIFORM, int CW>
__device__ __forceinline__ void split_out_cols(const uint32_t (&vr)[CW], const uint32_t (&vi)[CW], const TcParams& p,
                                               const float* scale, int cc, int j0, int ncol, int64_t qoff) {
  const int64_t pl = p.qplane, cs = 4 * pl;
  __half* qp = p.Qs + (int64_t)j0 * cs + qoff;
  const bool write_im = !p.skip_im;
  if (!write_im) {  // real operators: the real planes only
    // two columns per packed conversion (cvt.rn.f16x2.f32): half the conversion instructions
    // of one conversion per value, which otherwise bound this epilogue
#pragma unroll
    for (int c = 0; c < CW; c += 2) {
      const float r0 = __uint_as_float(vr[c]) * (UNIFORM ? p.uscale : scale[cc * CW + c]);
      const float r1 = __uint_as_float(vr[c + 1]) * (UNIFORM ? p.uscale : scale[cc * CW + c + 1]);
      const __half2 hi = __floats2half2_rn(r0, r1);
      const float2 hf = __half22float2(hi);
      const __half2 lo = __floats2half2_rn(r0 - hf.x, r1 - hf.y);
      if (c < ncol) {
        qp[0] = __low2half(hi);
        qp[pl] = __low2half(lo);
      }
      if (c + 1 < ncol) {
        qp[cs] = __high2half(hi);
        qp[cs + pl] = __high2half(lo);
      }
      qp += 2 * cs;
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < CW; ++c) {
    if (c < ncol) {
      const float sc = UNIFORM ? p.uscale : scale[cc * CW + c];
      const float re = __uint_as_float(vr[c]) * sc, im = __uint_as_float(vi[c]) * sc;
      const __half2 hi = __floats2half2_rn(re, im);
      const float2 hf = __half22float2(hi);
      const __half2 lo = __floats2half2_rn(re - hf.x, im - hf.y);
      qp[0] = __low2half(hi);
      qp[pl] = __low2half(lo);
      if (write_im) {
        qp[2 * pl] = __high2half(hi);
        qp[3 * pl] = __high2half(lo);
      }
    }
    qp += cs;
  }
}

template <int EPI_WARPS>
__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory");
}

// the four warps of one epilogue group (named barrier 2 + group)
__device__ __forceinline__ void grp_bar(int grp) { asm volatile("bar.sync %0, 128;" ::"r"(2 + grp) : "memory"); }

__device__ __forceinline__ void sts16(uint32_t a, __half v) {
  asm volatile("st.shared.b16 [%0], %1;" ::"r"(a), "h"(__half_as_ushort(v)) : "memory");
}

// 16 columns of this thread's row as fp16 hi/lo into a staging buffer laid out as the output
// box {128 entries, 1 row, 2 planes, 16 orders}: column c, plane q at ((2 c + q) * 128 + row) * 2
__device__ __forceinline__ void stage_split16(const uint32_t (&vr)[16], float uscale, uint32_t buf, int row) {
  const uint32_t a = buf + 2u * (uint32_t)row;
#pragma unroll
  for (int c = 0; c < 16; c += 2) {
    const float r0 = __uint_as_float(vr[c]) * uscale, r1 = __uint_as_float(vr[c + 1]) * uscale;
    const __half2 hi = __floats2half2_rn(r0, r1);
    const float2 hf = __half22float2(hi);
    const __half2 lo = __floats2half2_rn(r0 - hf.x, r1 - hf.y);
    sts16(a + (2 * c + 0) * 256, __low2half(hi));
    sts16(a + (2 * c + 1) * 256, __low2half(lo));
    sts16(a + (2 * c + 2) * 256, __high2half(hi));
    sts16(a + (2 * c + 3) * 256, __high2half(lo));
  }
}

// shared -> global tensor store of one box; completion tracked in this thread's bulk groups
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// wait until at most one of this thread's bulk stores still reads shared memory
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// wait until none of this thread's bulk stores still reads shared memory
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until every bulk store of this thread has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int BN, bool RB, bool RA, int KC>
__global__ void __launch_bounds__(TcCfg<BN, RB, RA, KC>::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmT, TcParams p) {
  using Cfg = TcCfg<BN, RB, RA, KC>;
  static_assert(KC == 32 || (KC == 64 && !RB), "128-byte k-chunks: streamed B only");
  constexpr int PLANE_A = Cfg::PLANE_A;
  constexpr int A_PLANES = Cfg::A_PLANES;
  constexpr int TC_BN = BN;
  constexpr int TC_PLANE_B = Cfg::PLANE_B;
  constexpr int TC_TMEM_COLS = Cfg::TMEM_COLS;
  constexpr uint32_t kIdesc = Cfg::IDESC;
  constexpr uint32_t kIdescNegA = Cfg::IDESC_NEG_A;
  constexpr int EPI_WARPS = Cfg::EPI_WARPS;
  constexpr int NGRP = EPI_WARPS / 4;  // epilogue warp groups (each covers the 128 TMEM lanes)
  constexpr int CW = Cfg::CW;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* const sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  TcCtl& sm = *reinterpret_cast<TcCtl*>(sbase);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // A real B (no column with an imaginary part) needs only its two real planes; with a
  // real A the product is then real and only the real accumulator is formed.  The skipped
  // products are exact zeros, so the results do not change.
  const bool breal = p.bimag != nullptr && *p.bimag == 0;
  const bool re_only = RA && (p.re_only || breal);
  const int nbp = (re_only || breal) ? 2 : 4;  // B planes loaded
  uint8_t* const bres = sbase + sizeof(TcCtl);  // resident B: [chunk][nbp planes][BN rows x 64 B]
  const int res_bytes = RB ? p.kchunks * nbp * TC_PLANE_B : 0;
  uint8_t* const obuf = bres + res_bytes;  // pair output staging: [group][2][16 x 2 x 128 fp16]
  const int out_bytes = RB ? p.out_bytes : 0;
  uint8_t* const stages = obuf + out_bytes;
  const int chunk_bytes = A_PLANES * PLANE_A + (RB ? 0 : nbp * TC_PLANE_B);
  const int cps = p.cps > 1 ? p.cps : 1;
  // narrow tail: chunk c < a_nfull at c * chunk_bytes, the tail after them, TAIL_PLANE apart
  constexpr int TAIL_PLANE = TC_BM * 32;
  const bool tail16 = RB && p.a_chunked && p.a_tail16 && cps >= p.kchunks;
  const int stage_bytes = p.stage_bytes ? p.stage_bytes : cps * chunk_bytes;
  const int nst = min(TC_MAXST, (p.smem_bytes - (int)sizeof(TcCtl) - res_bytes - out_bytes) / stage_bytes);
  // a launch sized for real signals whose split reports an imaginary part (or any other
  // mismatch of the host's sizing): record it and return before anything is set up
  if (nst < 1 || (p.stage_bytes && !tail16 && cps * chunk_bytes > p.stage_bytes) ||
      (p.pair_nbt && (!RB || out_bytes == 0))) {
    if (threadIdx.x == 0) atomicOr(p.status, FG_STATUS_LAUNCH_MISMATCH);
    return;
  }
  // TMEM columns of one accumulator buffer, and how many buffers fit (2: the epilogue of one
  // block overlaps the MMAs of the next)
  const bool merged = Cfg::MERGE && re_only;
  const uint32_t acc_w = (re_only && !merged ? 1u : 2u) * (uint32_t)BN;
  // ping-pong epilogue (one block per tile and one output scale, as in the fused assembly):
  // the epilogue warp groups take turns on the tiles, with up to 2 buffers per group so the
  // MMAs run ahead of all of them
  const int nbuf_fit = (int)((uint32_t)Cfg::TMEM_COLS / acc_w);
  const bool pingpong = p.nblk == 1 && p.uscale != 0.f && nbuf_fit >= NGRP;
  const int nbuf = pingpong ? min(2 * NGRP, nbuf_fit) / NGRP * NGRP : (nbuf_fit >= 2 ? 2 : 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < TC_MAXBUF; ++b) {
      mbar_init(&sm.tfull[b], 1);
      mbar_init(&sm.tempty[b], pingpong ? 4 : EPI_WARPS);
    }
    mbar_init(&sm.drain, 1);
    mbar_init(&sm.bfull, 1);
    sm.abort = 0;
    fence_barrier_init();
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    if (p.a_chunked || p.pair_lower || out_bytes)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmT)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_tc_before();
  __syncthreads();
  fence_tc_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int s_cur = 0;  // ring position and phase of the next stage
      uint32_t ph_cur = 0;
      uint32_t issued[TC_MAXST] = {};
      bool ok = true;
      int4 next = blockIdx.x < p.ntiles ? tile_of(p, blockIdx.x) : make_int4(0, 0, 0, 0);
      bool b_issued = false;
      const uint64_t l2_first = policy_evict_first();
      if (RB && blockIdx.x < p.ntiles) {  // all k-chunks of B, once
        mbar_arrive_expect_tx(&sm.bfull, (uint32_t)(p.kchunks * nbp * TC_PLANE_B));
        for (int kc = 0; kc < p.kchunks; ++kc)
          for (int q = 0; q < nbp; ++q)
            tma_load_3d(bres + (kc * nbp + q) * TC_PLANE_B, &tmB, kc * KC, next.z, q, &sm.bfull);
        b_issued = true;
      }
      for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x) {
        const int4 tile = next;
        if (t + (int)gridDim.x < p.ntiles) next = tile_of(p, t + gridDim.x);  // prefetch
        const int2 br = blk_range(p, tile);
        for (int b = br.x; ok && b < br.y; ++b) {
          const int zA = p.grouped ? tile.y : 4 * (b < p.nb_pow ? p.b0 + b : p.p_blk);
          for (int kc0 = 0; kc0 < p.kchunks; kc0 += cps) {
            const int s = s_cur;
            const uint32_t ph = ph_cur;
            if (++s_cur == nst) {
              s_cur = 0;
              ph_cur ^= 1u;
            }
            if (!tc_wait(&sm.empty[s], ph ^ 1, sm, p.status)) {
              ok = false;
              break;
            }
            const int nc = min(cps, p.kchunks - kc0);
            mbar_arrive_expect_tx(&sm.full[s], (uint32_t)(tail16 || p.a_img ? stage_bytes : nc * chunk_bytes));
            issued[s]++;
            if (RB && p.a_img) {  // the stage's image, one contiguous copy (one stage per tile)
              bulk_g2s_evict_first(stages + s * stage_bytes, p.a_img + (int64_t)tile.x * stage_bytes,
                                   (uint32_t)stage_bytes, &sm.full[s], l2_first);
              continue;
            }
            for (int c = 0; c < nc; ++c) {
              uint8_t* st = stages + s * stage_bytes + c * chunk_bytes;
              const int k0 = (kc0 + c) * KC;
              if (p.a_chunked) {  // chunk-major A: full 32-column chunk planes, then the tail
                const int kc = kc0 + c;
#pragma unroll
                for (int q = 0; q < A_PLANES; ++q) {
                  if (kc < p.a_nfull)
                    tma_load_3d(st + q * PLANE_A, &tmA, 0, tile.x * TC_BM, q * p.a_nfull + kc, &sm.full[s]);
                  else
                    tma_load_3d(st + q * (tail16 ? TAIL_PLANE : PLANE_A), &tmT, 0, tile.x * TC_BM, q, &sm.full[s]);
                }
              } else if (RA && p.pair_lower && k0 < tile.x * TC_BM) {
                // left of the diagonal block: Q[i][k] = S'[k][i], rows k0 .. k0 + 31 of the
                // transposed store (planes 2, 3 of the group), 64 i-values per box
#pragma unroll
                for (int q = 0; q < A_PLANES; ++q)
#pragma unroll
                  for (int h = 0; h < 2; ++h)
                    tma_load_3d(st + q * PLANE_A + h * (PLANE_A / 2), &tmT, tile.x * TC_BM + 64 * h, k0, zA + 2 + q,
                                &sm.full[s]);
              } else {
#pragma unroll
                for (int q = 0; q < A_PLANES; ++q)
                  tma_load_3d(st + q * PLANE_A, &tmA, k0, tile.x * TC_BM, zA + q, &sm.full[s]);
              }
              if (!RB) {
                for (int q = 0; q < nbp; ++q)
                  tma_load_3d(st + A_PLANES * PLANE_A + q * TC_PLANE_B, &tmB, k0, tile.z, q, &sm.full[s]);
              }
            }
          }
        }
      }
      if (!ok) {  // wait (bounded) until every issued copy has landed
        if (b_issued) {
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&sm.bfull, 0) && global_timer_ns() - t0 < FG_WAIT_LIMIT_NS) {
          }
        }
        for (int s = 0; s < nst; ++s) {
          if (!issued[s]) continue;
          const uint32_t par = (issued[s] - 1) & 1;
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&sm.full[s], par) && global_timer_ns() - t0 < FG_WAIT_LIMIT_NS) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s_cur = 0;
      uint32_t ph_cur = 0, bc = 0;
      bool ok = true;
      if (RB && blockIdx.x < p.ntiles) ok = tc_wait(&sm.bfull, 0, sm, p.status);
      // grouped tiles may be narrower than BN (ragged groups, halved last-wave tiles): each
      // tile's MMAs take N = its columns rounded up to 16 (the rest of B is not read)
      const bool tile_n = p.tiles != nullptr && p.grouped;
      int4 next = tile_n && blockIdx.x < p.ntiles ? tile_of(p, blockIdx.x) : make_int4(0, 0, 0, 0);
      for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x) {
        uint32_t idesc = kIdesc, idesc_neg = kIdescNegA;
        // pair-structured operators: k-chunks left of this row tile's diagonal block are MN-major
        int lower_k = 0;
        if (tile_n) {
          const int4 tl = next;
          if (t + (int)gridDim.x < p.ntiles) next = tile_of(p, t + gridDim.x);  // prefetch
          if (RA && p.pair_lower) lower_k = tl.x * TC_BM;
          const int n16 = min(TC_BN, max(16, (tl.w - tl.z + 15) / 16 * 16));
          idesc = (kIdesc & ~(0x3Fu << 17)) | ((uint32_t)(n16 >> 3) << 17);
          idesc_neg = idesc | (1u << 13);
        }
        const int2 br = blk_range(p, p.bps && !p.grouped ? tile_of(p, t) : make_int4(0, 0, 0, 0));
        for (int b = br.x; ok && b < br.y; ++b, ++bc) {
          const uint32_t buf = bc % (uint32_t)nbuf, tph = (bc / (uint32_t)nbuf) & 1;
          if (!tc_wait(&sm.tempty[buf], tph ^ 1, sm, p.status)) {
            ok = false;
            break;
          }
          fence_tc_after();
          const uint32_t d_re = tmem + buf * acc_w;
          const uint32_t d_im = d_re + TC_BN;
          for (int kc0 = 0; kc0 < p.kchunks; kc0 += cps) {
            const int s = s_cur;
            const uint32_t ph = ph_cur;
            if (++s_cur == nst) {
              s_cur = 0;
              ph_cur ^= 1u;
            }
            if (!tc_wait(&sm.full[s], ph, sm, p.status)) {
              ok = false;
              break;
            }
            fence_tc_after();
            const int nc = min(cps, p.kchunks - kc0);
            for (int c = 0; c < nc; ++c) {
            const int kc = kc0 + c;
            const uint32_t sa = smem_u32(stages + s * stage_bytes + c * chunk_bytes);
            const uint32_t sb = RB ? smem_u32(bres + kc * nbp * TC_PLANE_B) : sa + A_PLANES * PLANE_A;
            // the narrow tail: 32-byte rows (one k16 step), 32-byte swizzle
            const bool is_tail = tail16 && kc >= p.a_nfull;
            const uint32_t apl = is_tail ? (uint32_t)TAIL_PLANE : (uint32_t)PLANE_A;
            // MN-major A (left of a pair-structured operator's diagonal block): k16 step kk is
            // 16 rows of 128 bytes further; the instruction reads A transposed
            const bool mn = kc * KC < lower_k;
            const uint32_t idesc_c = mn ? (idesc | (1u << 15)) : idesc;
            const uint32_t idesc_neg_c = mn ? (idesc_neg | (1u << 15)) : idesc_neg;
            auto adesc = [&](uint32_t a) { return mn ? desc_mn_sw128(a) : is_tail ? desc_sw32(a) : desc_kc<KC>(a); };
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              if (is_tail && kk > 0) continue;
              const uint32_t off = kk * 32;  // 16 fp16 along k
              const uint32_t offa = mn ? kk * 2048 : off;
              const uint64_t arh = adesc(sa + 0 * apl + offa), arl = adesc(sa + 1 * apl + offa);
              const uint64_t brh = desc_kc<KC>(sb + 0 * TC_PLANE_B + off), brl = desc_kc<KC>(sb + 1 * TC_PLANE_B + off);
              const uint64_t bih = desc_kc<KC>(sb + 2 * TC_PLANE_B + off), bil = desc_kc<KC>(sb + 3 * TC_PLANE_B + off);
              if (p.kvalid > 0 && kc * KC + kk * 16 >= p.kvalid) continue;  // all-zero k16 step
              const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
              if (merged) {  // [A_hi*B_hi | A_hi*B_lo], then A_lo*B_hi into the first half
                umma(d_re, arh, brh, Cfg::IDESC_2N, acc);
                umma(d_re, arl, brh, idesc_c, 1);
                continue;
              }
              // real part: Ar*Xr - Ai*Xi
              umma(d_re, arh, brh, idesc_c, acc);
              umma(d_re, arh, brl, idesc_c, 1);
              umma(d_re, arl, brh, idesc_c, 1);
              if (re_only) continue;  // real product: no imaginary accumulator
              if (breal) {            // complex A, real X: Im = Ai*Xr only
                if (!RA) {
                  const uint64_t aih = adesc(sa + 2 * apl + offa), ail = adesc(sa + 3 * apl + offa);
                  umma(d_im, aih, brh, idesc_c, acc);
                  umma(d_im, aih, brl, idesc_c, 1);
                  umma(d_im, ail, brh, idesc_c, 1);
                }
                continue;
              }
              // imaginary part: Ar*Xi + Ai*Xr
              umma(d_im, arh, bih, idesc_c, acc);
              umma(d_im, arh, bil, idesc_c, 1);
              umma(d_im, arl, bih, idesc_c, 1);
              if (!RA) {
                const uint64_t aih = adesc(sa + 2 * apl + offa), ail = adesc(sa + 3 * apl + offa);
                umma(d_re, aih, bih, idesc_neg_c, 1);
                umma(d_re, aih, bil, idesc_neg_c, 1);
                umma(d_re, ail, bih, idesc_neg_c, 1);
                umma(d_im, aih, brh, idesc_c, 1);
                umma(d_im, aih, brl, idesc_c, 1);
                umma(d_im, ail, brh, idesc_c, 1);
              }
            }
            }                           // chunks of the stage
            umma_commit(&sm.empty[s]);  // stage s is free once these MMAs complete
          }
          if (!ok) break;
          umma_commit(&sm.tfull[buf]);  // block done: accumulators ready for the epilogue
        }
      }
      // wait (bounded) for every MMA this thread issued before TMEM is released
      umma_commit(&sm.drain);
      const uint64_t t0 = global_timer_ns();
      while (!mbar_try_wait(&sm.drain, 0) && global_timer_ns() - t0 < FG_WAIT_LIMIT_NS) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // NGRP groups of 4 warps; the warps of a group read the four TMEM lane quadrants
    // (warp w may access quadrant w mod 4).  Ping-pong: group g takes the tiles li = g mod
    // NGRP whole; otherwise the groups take alternate 32-column chunks of every tile.
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const int grp = (warp - TC_EPI_WARP0) >> 2;
    const int row = 32 * q + lane;
    const int et = threadIdx.x - TC_EPI_WARP0 * 32;  // 0 .. 32 * EPI_WARPS - 1
    const bool split_out = p.Qs != nullptr;
    uint32_t bc = 0;
    bool ok = true;
    // one scale per column: undo 2^{e_j} and the operator scale; the next tile's
    // descriptor and scales are loaded while the current tile is processed
    auto col_scale = [&](const int4& tl) -> float {
      if (et >= TC_BN || p.uscale != 0.f) return 0.f;  // one output scale: no per-column table
      const int j = tl.z + et;
      const int e = j < tl.w ? p.col_exp[j] : 0;
      return ldexpf(1.0f, split_out ? -e : -(FG_SPLIT_SHIFT + e));
    };
    int4 next = blockIdx.x < p.ntiles ? tile_of(p, blockIdx.x) : make_int4(0, 0, 0, 0);
    float next_scale = blockIdx.x < p.ntiles ? col_scale(next) : 0.f;
    int64_t li = 0;  // local tile index (ping-pong: group grp takes the tiles li = grp mod NGRP)
    // staged pair output: the group's first warp, lane 0, issues its tensor stores
    const bool staged = RB && out_bytes > 0 && pingpong;
    const bool leader = staged && warp == TC_EPI_WARP0 + 4 * grp && lane == 0;
    const uint32_t obufs = p.out_bufs == 1 ? 1u : 2u;
    const bool opairs = p.out_pairs != 0;
    const uint32_t gbuf = smem_u32(obuf) + (uint32_t)grp * (opairs ? 16384u : obufs * 8192u);
    uint32_t nstaged = 0;
    for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++li) {
      const bool mine = !pingpong || (int)(li % NGRP) == grp;
      const int4 tile = next;
      const float my_scale = next_scale;
      if (t + (int)gridDim.x < p.ntiles) {
        next = tile_of(p, t + gridDim.x);
        next_scale = col_scale(next);
      }
      if (p.uscale == 0.f) {  // per-column scales: publish this tile's table
        epi_bar<EPI_WARPS>();
        if (et < TC_BN) sm.scale[et] = my_scale;
        epi_bar<EPI_WARPS>();
      }
      const int64_t gi = (int64_t)tile.x * TC_BM + row;
      const bool row_ok = gi < p.rows;
      int64_t qoff = 0;
      if (split_out && !p.pair_nbt) {
        const int64_t qi = gi / p.qN;
        qoff = qi * p.qNp + (gi - qi * p.qN);
      }
      // pair tile: this row is entry (i, 128 kt + row); its mirror (128 kt + row, i) is written at
      // the same position of the transposed store unless the tile is in a diagonal block
      bool mirror_ok = false, diag_lane = false;
      int pi = 0, pkt = 0;
      if (p.pair_nbt && mine) {
        pair_tile(tile.x, p.pair_nbt, pi, pkt);
        qoff = (int64_t)pi * p.qNp + 128 * (int64_t)pkt + row;
        mirror_ok = pkt != pi / 128;
        diag_lane = 128 * pkt + row == pi;
      }

      const int2 br = blk_range(p, tile);
      const int64_t split_off = (p.bps && !p.grouped) ? (int64_t)tile.y * p.split_stride : 0;
      for (int b = br.x; b < br.y; ++b, ++bc) {
        if (!mine) continue;  // the other group's tile (its buffer index still counts)
        const uint32_t buf = bc % (uint32_t)nbuf, tph = (bc / (uint32_t)nbuf) & 1;
        if (!tc_wait(&sm.tfull[buf], tph, sm, p.status)) {
          ok = false;
          break;
        }
        fence_tc_after();
        const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + buf * acc_w;
        if (staged) {
          // the pair launch's output: chunks of 16 columns, the first 64 the orders' Q[i][k],
          // the rest their mirrors (skipped in a diagonal block); every test here is uniform
          // over the group, and only the warp holding the diagonal entry adds c_0
          const bool diag_warp = __any_sync(0xffffffffu, diag_lane);
#pragma unroll 1
          for (int cc = 0; cc < TC_BN / CW; ++cc) {
            const bool mir = cc >= 4;
            const int jo = (cc & 3) * CW;
            if (jo >= p.pair_A || (mir && !mirror_ok)) continue;
            uint32_t vr[CW];
            __syncwarp();
            tmem_ld(base + cc * CW, vr);
            tmem_wait_ld();
            if (diag_warp && !mir) {
              if (diag_lane) {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                  if (jo + c < p.pair_A) vr[c] = __float_as_uint(__uint_as_float(vr[c]) + __ldg(p.diag + jo + c));
              }
              __syncwarp();
            }
            if (opairs) {
              // two chunks (32 orders) per tensor store: the first half of a pair waits until
              // the group's buffer has been read by the previous store; the store follows the
              // pair's last chunk in range (orders past A are outside the tensor, not written)
              const int h = cc & 1;
              if (h == 0) {
                if (leader) bulk_wait_read0();
                grp_bar(grp);
              }
              stage_split16(reinterpret_cast<const uint32_t(&)[16]>(vr), p.uscale, gbuf + (uint32_t)h * 8192u, row);
              if (h == 1 || jo + CW >= p.pair_A) {
                fence_proxy_async_smem();
                grp_bar(grp);
                if (leader) tma_store_4d(&tmT, gbuf, 128 * pkt, pi, mir ? 2 : 0, jo - CW * h);
              }
            } else {
              // one chunk per store: this buffer's previous store must have read it, then the
              // group fills it and one tensor store writes the 16 orders x 2 planes
              const uint32_t sbuf = gbuf + (obufs == 2u ? (nstaged & 1u) * 8192u : 0u);
              if (leader) {
                if (obufs == 2u)
                  bulk_wait_read1();
                else
                  bulk_wait_read0();
              }
              grp_bar(grp);
              stage_split16(reinterpret_cast<const uint32_t(&)[16]>(vr), p.uscale, sbuf, row);
              fence_proxy_async_smem();
              grp_bar(grp);
              if (leader) tma_store_4d(&tmT, sbuf, 128 * pkt, pi, mir ? 2 : 0, jo);
              ++nstaged;
            }
          }
        }
#pragma unroll 1
        for (int cc = pingpong ? 0 : grp; !staged && cc < TC_BN / CW; cc += pingpong ? 1 : NGRP) {
          const int j0 = tile.z + cc * CW;
          if (j0 >= tile.w) break;  // uniform: no column of this chunk is in range
          const int ncol = min(CW, tile.w - j0);
          uint32_t vr[CW], vi[CW];
          __syncwarp();  // tcgen05.ld is warp-collective: the whole warp converged
          tmem_ld(base + cc * CW, vr);
          if (re_only && !merged) {  // the imaginary accumulator was not formed: the product is real
#pragma unroll
            for (int c = 0; c < CW; ++c) vi[c] = 0u;
          } else {
            tmem_ld(base + TC_BN + cc * CW, vi);
          }
          tmem_wait_ld();
          if (merged) {  // real product: the two halves of the merged split products
#pragma unroll
            for (int c = 0; c < CW; ++c) {
              vr[c] = __float_as_uint(__uint_as_float(vr[c]) + __uint_as_float(vi[c]));
              vi[c] = 0u;
            }
          }
          if (!row_ok) {
            // rows past the end: nothing to store
          } else if (split_out) {
            // value * 2^FG_SPLIT_SHIFT as fp16 hi + lo, four planes per column
            if (p.uscale != 0.f)
              split_out_cols<true, CW>(vr, vi, p, sm.scale, cc, j0, ncol, qoff);
            else
              split_out_cols<false, CW>(vr, vi, p, sm.scale, cc, j0, ncol, qoff);
          } else if (p.coef == nullptr && p.y_real) {
            float* yp = reinterpret_cast<float*>(p.Y) + (int64_t)j0 * p.rows + gi;
#pragma unroll
            for (int c = 0; c < CW; ++c) {
              if (c < ncol) *yp = __uint_as_float(vr[c]) * sm.scale[cc * CW + c];
              yp += p.rows;
            }
          } else if (p.coef == nullptr) {
            float2* yp = p.Y + (int64_t)j0 * p.rows + gi;
            const bool uni = p.uscale != 0.f;
#pragma unroll
            for (int c = 0; c < CW; ++c) {
              if (c < ncol) {
                const float sc = uni ? p.uscale : sm.scale[cc * CW + c];
                *yp = make_float2(__uint_as_float(vr[c]) * sc, __uint_as_float(vi[c]) * sc);
              }
              yp += p.rows;
            }
          } else {
            // Y (may be absent: the dual alone) and D accumulate block by block; the first
            // block of the tile's range starts them
            float2* yp = p.Y ? p.Y + split_off + (int64_t)j0 * p.rows + gi : nullptr;
            float2* dp = p.D ? p.D + split_off + (int64_t)j0 * p.rows + gi : nullptr;
            const float2* cfp = p.coef + (int64_t)b * p.ldcoef + j0;
            const float2* cdp = p.D ? p.coefd + (int64_t)b * p.ldcoef + j0 : nullptr;
            const bool first = b == br.x;
            // groups of 4 columns: the partial sums of a group are loaded first and then
            // updated and stored, so their loads are in flight together (a load after the
            // previous column's store would wait for it: the compiler cannot tell that they do
            // not alias).  Only the stacked launches (streamed B) take this path.
            if constexpr (!RB) {
              constexpr int CG = 4;
#pragma unroll
              for (int c0 = 0; c0 < CW; c0 += CG) {
                float2 yv[CG], dv[CG];
#pragma unroll
                for (int u = 0; u < CG; ++u) {
                  const bool ld = c0 + u < ncol && !first;
                  yv[u] = yp && ld ? yp[(int64_t)(c0 + u) * p.rows] : make_float2(0.f, 0.f);
                  dv[u] = dp && ld ? dp[(int64_t)(c0 + u) * p.rows] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < CG; ++u) {
                  const int c = c0 + u;
                  if (c >= ncol) continue;
                  const float sc = sm.scale[cc * CW + c];
                  const float tr = __uint_as_float(vr[c]) * sc, ti = __uint_as_float(vi[c]) * sc;
                  if (yp) {
                    const float2 cf = __ldg(cfp + c);
                    float2 y = yv[u];
                    y.x = fmaf(cf.x, tr, fmaf(-cf.y, ti, y.x));
                    y.y = fmaf(cf.x, ti, fmaf(cf.y, tr, y.y));
                    yp[(int64_t)c * p.rows] = y;
                  }
                  if (dp) {
                    const float2 cd = __ldg(cdp + c);
                    float2 d = dv[u];
                    d.x = fmaf(cd.x, tr, fmaf(-cd.y, ti, d.x));
                    d.y = fmaf(cd.x, ti, fmaf(cd.y, tr, d.y));
                    dp[(int64_t)c * p.rows] = d;
                  }
                }
              }
            }
          }
        }
        fence_tc_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.tempty[buf]);
      }
    }
    if (leader) bulk_wait_all();  // the staged stores have left shared memory and completed
  }
  fence_tc_before();
  __syncthreads();
  fence_tc_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D fp16 map: dim0 = k (N, contiguous), dim1 = rows (pitch Np), dim2 = planes (stride plane_elems);
// kc k x box_rows boxes, 2 kc-byte swizzle (the MMA operand layout of a kc-wide k-chunk).
bool make_map(CUtensorMap* m, const void* base, int64_t N, int64_t rows, int64_t Np, int64_t nplanes,
              int64_t plane_elems, int box_rows, int kc = TC_KC) {
  return fg_make_map_f16(m, base, N, rows, Np, nplanes, plane_elems, kc, box_rows, 2 * kc);
}

}  // namespace

bool fg_make_map_f16(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t pitch, int64_t nplanes,
                     int64_t plane_elems, int box_cols, int box_rows, int swizzle_bytes) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)plane_elems * 2};
  cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

int smem_optin() {
  static int n = 0;
  if (!n) {
    int d = 0, v = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    n = v > 0 ? v : 48 * 1024;
  }
  return n;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int d = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
    if (n < 1) n = 1;
  }
  return n;
}

template <int BN, bool RB, bool RA, int KC = TC_KC>
cudaError_t launch_bn(const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mT, int ntiles,
                      const TcParams& p, cudaStream_t s, int kclass) {
  // all the shared memory a CTA may have (one CTA per SM); the kernel sizes its ring to it
  const int smem = smem_optin();
  using Cfg = TcCfg<BN, RB, RA, KC>;
  // resident B: the planes the kernel loads (2 when the product is real by construction; a
  // real B found on the device only leaves more room for the ring)
  const int res_bytes = RB ? p.kchunks * ((RA && p.re_only) ? 2 : 4) * Cfg::PLANE_B : 0;
  const int worst_stage =
      p.stage_bytes ? p.stage_bytes
                    : (p.cps > 1 ? p.cps : 1) * (Cfg::A_PLANES * Cfg::PLANE_A + (RB ? 0 : 4 * Cfg::PLANE_B));
  TcParams q = p;
  q.smem_bytes = smem - 1024;  // the kernel aligns its base up to 1024 bytes
  const int out_bytes = RB ? p.out_bytes : 0;
  if (q.smem_bytes - (int)sizeof(TcCtl) - res_bytes - out_bytes < TC_MIN_STAGES * worst_stage)
    return cudaErrorInvalidValue;
  int smem_req = smem;
  if (RB) {
    // resident B: a stage holds A only, so the ring depth is known here; ask for just that
    // much, leaving the rest of the SM's shared memory to kernels running beside this one
    const int nst = std::min(TC_MAXST, (q.smem_bytes - (int)sizeof(TcCtl) - res_bytes - out_bytes) / worst_stage);
    q.smem_bytes = (int)sizeof(TcCtl) + res_bytes + out_bytes + nst * worst_stage;
    smem_req = q.smem_bytes + 1024;
  }
  cudaError_t e =
      cudaFuncSetAttribute(tc_gemm_kernel<BN, RB, RA, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_req);
  if (e != cudaSuccess) return e;
  const int grid = std::min<int>(ntiles, sm_count());
  FgTimed timed(kclass, s);
  tc_gemm_kernel<BN, RB, RA, KC><<<grid, Cfg::THREADS, smem_req, s>>>(mA, mB, mT, q);
  fg_note_launch(kclass);
  return cudaGetLastError();
}

// bn: column-tile width (64 or 128); the B tensor map's box must have bn rows.
// resident_b: every tile has the same columns (needs bn == 64 and kchunks <= TC_RB_MAXCH).
cudaError_t launch(const CUtensorMap& mA, const CUtensorMap& mB, const std::vector<int4>& tiles, TcParams p,
                   void* scratch, size_t scratch_bytes, cudaStream_t s, int kclass = FGFRFT_KC_TC_GEMM,
                   int bn = 128, bool resident_b = false, bool real_a = false, const CUtensorMap* mTail = nullptr,
                   int kc = TC_KC) {
  const CUtensorMap& mT = mTail ? *mTail : mA;  // the tail map is read only with p.a_chunked
  if (p.a_chunked && !mTail) return cudaErrorInvalidValue;
  if (tiles.empty()) {
    // a table already on the device (p.tiles), or arithmetic tiles (p.tiles == NULL)
    if (p.ntiles <= 0 || (!p.tiles && p.arith_cols <= 0)) return cudaSuccess;
  } else {
    const size_t tbytes = tiles.size() * sizeof(int4);
    if (tbytes > scratch_bytes) return cudaErrorInvalidValue;
    cudaError_t e = fg_h2d(scratch, tiles.data(), tbytes, s);
    if (e != cudaSuccess) return e;
    p.tiles = (const int4*)scratch;
    p.ntiles = (int)tiles.size();
  }
  if (resident_b) {
    if (p.kchunks > TC_RB_MAXCH) return cudaErrorInvalidValue;
    if (bn == 128) {  // the pair assembly (64 orders and their mirrors): real blocks only
      if (!real_a) return cudaErrorInvalidValue;
      return launch_bn<128, true, true>(mA, mB, mT, p.ntiles, p, s, kclass);
    }
    if (bn != 64) return cudaErrorInvalidValue;
    return real_a ? launch_bn<64, true, true>(mA, mB, mT, p.ntiles, p, s, kclass)
                  : launch_bn<64, true, false>(mA, mB, mT, p.ntiles, p, s, kclass);
  }
  if (kc == 64) {  // 128-byte k-chunks (the caller checked that two stages fit)
    if (bn == 256) {
      if (!real_a) return cudaErrorInvalidValue;
      return launch_bn<256, false, true, 64>(mA, mB, mT, p.ntiles, p, s, kclass);
    }
    if (bn == 64)
      return real_a ? launch_bn<64, false, true, 64>(mA, mB, mT, p.ntiles, p, s, kclass)
                    : launch_bn<64, false, false, 64>(mA, mB, mT, p.ntiles, p, s, kclass);
    return real_a ? launch_bn<128, false, true, 64>(mA, mB, mT, p.ntiles, p, s, kclass)
                  : launch_bn<128, false, false, 64>(mA, mB, mT, p.ntiles, p, s, kclass);
  }
  if (bn == 256) {  // real A only (a complex A at BN = 256 leaves too few stages)
    if (!real_a) return cudaErrorInvalidValue;
    return launch_bn<256, false, true>(mA, mB, mT, p.ntiles, p, s, kclass);
  }
  if (bn == 64)
    return real_a ? launch_bn<64, false, true>(mA, mB, mT, p.ntiles, p, s, kclass)
                  : launch_bn<64, false, false>(mA, mB, mT, p.ntiles, p, s, kclass);
  return real_a ? launch_bn<128, false, true>(mA, mB, mT, p.ntiles, p, s, kclass)
                : launch_bn<128, false, false>(mA, mB, mT, p.ntiles, p, s, kclass);
}

// k-chunk width of a streamed-B launch: 64 (128-byte rows, which the tensor-map loads serve
// from L2 faster than 64-byte rows) when two ring stages of it fit in shared memory, else 32.
// b_real: every B column is known to be real (real float32 signals), so a stage needs only
// the two real B planes; *stage_bytes then receives that stage size (0 otherwise).  Used by
// the stacked GEMM, whose tiles stream every stored block against one signal tile (measured
// 18% faster than 32-wide chunks at N = 1024); the grouped GEMM keeps 32-wide chunks (its
// 256-column tiles fit four 48 KB stages instead of two 96 KB ones, measured 8% faster).
int pick_kc(int bn, bool real_a, bool b_real, int* stage_bytes) {
  const int st = (real_a ? 2 : 4) * TC_BM * 64 * 2 + (b_real ? 2 : 4) * bn * 64 * 2;
  *stage_bytes = 0;
  if (TC_MIN_STAGES * st + (int)sizeof(TcCtl) + 1024 > smem_optin()) return TC_KC;
  if (b_real) *stage_bytes = st;
  return 64;
}

}  // namespace

bool fg_tc_available() {
  static int avail = -1;
  if (avail < 0) {
    int d = 0, major = 0, minor = 0;
    avail = 0;
    if (cudaGetDevice(&d) == cudaSuccess &&
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, d) == cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, d) == cudaSuccess)
      avail = (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
  }
  return avail == 1;
}

int64_t fg_tc_signal_rows(int64_t B, int64_t) { return B; }


size_t fg_tc_scratch_bytes(int64_t N, int64_t B, int64_t groups, int nblk) {
  const int64_t row_tiles = (N + TC_BM - 1) / TC_BM;
  const int64_t col_tiles = (B + 63) / 64 + groups;  // each group may add a ragged tile (tiles >= 64 wide)
  // stacked tiles repeat once per block split
  const int64_t splits = nblk > 1 ? fg_tc_stacked_splits(N, B, nblk) : 1;
  return (size_t)(row_tiles * col_tiles * splits) * sizeof(int4) + 256;
}

int fg_tc_grouped_bn(bool real_a) { return real_a ? 256 : TC_BN_STD; }

void fg_tc_grouped_tiles(int64_t N, int64_t groups, const int64_t* gstart, const int64_t* gcount, int bn,
                         std::vector<int4>& tiles) {
  tiles.clear();
  const int row_tiles = (int)((N + TC_BM - 1) / TC_BM);
  for (int64_t g = 0; g < groups; ++g) {
    const int64_t c0 = gstart[g], c1 = gstart[g] + gcount[g];
    for (int rt = 0; rt < row_tiles; ++rt)
      for (int64_t c = c0; c < c1; c += bn)
        tiles.push_back(make_int4(rt, (int)(4 * g), (int)c, (int)std::min<int64_t>(c + bn, c1)));
  }
  // Persistent CTAs take tiles t, t + P, ...: a last wave of R <= P/2 tiles would leave most
  // SMs idle for a whole tile, so its tiles are halved along the columns (the kernel sizes
  // each tile's MMAs to its columns) and the wave takes half as long.
  const int64_t P = sm_count(), T = (int64_t)tiles.size(), R = T % P;
  if (T > P && R > 0 && 2 * R <= P) {
    std::vector<int4> tail(tiles.end() - R, tiles.end());
    tiles.resize((size_t)(T - R));
    for (const int4& t : tail) {
      const int half = ((t.w - t.z + 1) / 2 + 15) / 16 * 16;  // a multiple of 16 columns
      if (t.w - t.z > 16 && t.z + half < t.w) {
        tiles.push_back(make_int4(t.x, t.y, t.z, t.z + half));
        tiles.push_back(make_int4(t.x, t.y, t.z + half, t.w));
      } else {
        tiles.push_back(t);
      }
    }
  }
}

cudaError_t fg_tc_grouped_apply(const TcGroupedArgs& a, cudaStream_t s) {
  if (a.N > (1 << 24) || a.B > (1 << 30)) return cudaErrorInvalidValue;
  if (!a.x_split_done) {
    cudaError_t e = fg_split_signals(a.X, a.B, a.N, a.Np, a.xs_rows, a.Xs, a.col_exp, s, a.bimag, a.x_real);
    if (e != cudaSuccess) return e;
  }
  // real operators: 256-column tiles halve the re-reads of each operator tile from L2
  const int bn = fg_tc_grouped_bn(a.real_a);
  const int kc = TC_KC, stage_bytes = 0;
  CUtensorMap mA, mB, mT;
  if (!make_map(&mA, a.Qs, a.N, a.N, a.Np, 4 * a.groups, a.plane_elems, TC_BM, kc) ||
      !make_map(&mB, a.Xs, a.N, a.xs_rows, a.Np, 4, a.xs_rows * a.Np, bn, kc))
    return cudaErrorInvalidValue;
  // pair-structured operators: the transposed store (planes 2, 3) read as 64 x 32 MN-major boxes
  if (a.pair && (!a.real_a || a.N % 128 ||
                 !fg_make_map_f16(&mT, a.Qs, a.N, a.N, a.Np, 4 * a.groups, a.plane_elems, 64, 32, 128)))
    return cudaErrorInvalidValue;
  std::vector<int4> tiles;
  TcParams p{};
  if (a.tiles_dev) {  // uploaded by the caller at the start of the call (built with the same bn)
    p.tiles = a.tiles_dev;
    p.ntiles = (int)a.ntiles;
  } else {
    fg_tc_grouped_tiles(a.N, a.groups, a.gstart, a.gcount, bn, tiles);
  }
  p.nblk = 1;
  p.grouped = 1;
  p.rows = a.N;
  p.kchunks = (int)((a.N + kc - 1) / kc);
  p.stage_bytes = stage_bytes;
  p.Y = a.Y;
  p.col_exp = a.col_exp;
  p.status = a.status;
  p.bimag = a.bimag;
  p.y_real = a.y_real ? 1 : 0;
  p.pair_lower = a.pair ? 1 : 0;
  return launch(mA, mB, tiles, p, a.scratch, a.scratch_bytes, s, FGFRFT_KC_TC_GEMM, bn, false, a.real_a,
                a.pair ? &mT : nullptr, kc);
}

cudaError_t fg_tc_stacked_apply(const TcStackedArgs& a, cudaStream_t s) {
  if (a.N > (1 << 24) || a.B > (1 << 30)) return cudaErrorInvalidValue;
  cudaError_t e = fg_split_signals(a.X, a.B, a.N, a.Np, a.xs_rows, a.Xs, a.col_exp, s, a.bimag, a.x_real);
  if (e != cudaSuccess) return e;
  CUtensorMap mA, mB;
  const int64_t nplanes = 4 * (int64_t)(std::max(a.b0 + a.nb_pow, a.p_blk + 1));
  int stage_bytes = 0;
  const int kc = pick_kc(TC_BN_STD, a.real_a, a.x_real, &stage_bytes);
  if (!make_map(&mA, a.stack, a.N, a.N, a.Np, nplanes, a.plane_elems, TC_BM, kc) ||
      !make_map(&mB, a.Xs, a.N, a.xs_rows, a.Np, 4, a.xs_rows * a.Np, TC_BN_STD, kc))
    return cudaErrorInvalidValue;
  std::vector<int4> tiles;
  const int row_tiles = (int)((a.N + TC_BM - 1) / TC_BM);
  const int nblk = a.nb_pow + (a.p_blk >= 0 ? 1 : 0);
  // few tiles (small batches): each tile's blocks are split over several CTAs, whose partial
  // sums are added in a fixed order afterwards (deterministic)
  const int splits = fg_tc_stacked_splits(a.N, a.B, nblk);
  const int bps = (nblk + splits - 1) / splits;
  if (splits > 1 && (!a.Ysplit || (a.D && !a.Dsplit))) return cudaErrorInvalidValue;
  for (int sp = 0; sp < splits; ++sp)
    for (int rt = 0; rt < row_tiles; ++rt)
      for (int64_t c = 0; c < a.B; c += TC_BN_STD)
        tiles.push_back(make_int4(rt, sp, (int)c, (int)std::min<int64_t>(c + TC_BN_STD, a.B)));
  TcParams p{};
  p.nblk = nblk;
  p.bps = splits > 1 ? bps : 0;
  p.split_stride = a.B * a.N;
  p.grouped = 0;
  p.b0 = a.b0;
  p.nb_pow = a.nb_pow;
  p.p_blk = a.p_blk;
  p.rows = a.N;
  p.kchunks = (int)((a.N + kc - 1) / kc);
  p.stage_bytes = stage_bytes;
  p.coef = a.coef;
  p.coefd = a.coefd;
  p.ldcoef = a.B;
  p.Y = splits > 1 && a.Y ? a.Ysplit : a.Y;
  p.D = splits > 1 && a.D ? a.Dsplit : a.D;
  p.col_exp = a.col_exp;
  p.status = a.status;
  p.bimag = a.bimag;
  e = launch(mA, mB, tiles, p, a.scratch, a.scratch_bytes, s, FGFRFT_KC_TC_GEMM, 128, false, a.real_a, nullptr, kc);
  if (e != cudaSuccess || splits == 1) return e;
  if (a.Y && (e = fg_sum_splits(a.Ysplit, splits, a.B * a.N, a.Y, s)) != cudaSuccess) return e;
  if (a.D) e = fg_sum_splits(a.Dsplit, splits, a.B * a.N, a.D, s);
  return e;
}

int fg_tc_stacked_splits(int64_t N, int64_t B, int nblk) {
  const int64_t tiles = ((N + TC_BM - 1) / TC_BM) * ((B + TC_BN_STD - 1) / TC_BN_STD);
  const int64_t want = sm_count() / std::max<int64_t>(tiles, 1);
  if (want < 2 || nblk < 2) return 1;
  const int s0 = (int)std::min<int64_t>(want, nblk);
  const int bps = (nblk + s0 - 1) / s0;
  return (nblk + bps - 1) / bps;
}

// Staging buffers per epilogue group of the pair launch for this L_max: 2 when they fit beside
// two ring stages and the resident coefficients, else 1, else 0 (the launch does not fit).
static int pair_out_bufs(int L_max) {
  const int nch = 2 * L_max / TC_KC;
  const int stage = nch * 2 * TC_BM * TC_KC * 2;         // A hi, lo per chunk
  const int res = nch * 2 * 128 * TC_KC * 2;             // the resident coefficients, 2 planes
  const int avail = smem_optin() - 1024 - (int)sizeof(TcCtl) - res;
  for (int b = 2; b >= 1; --b)
    if (avail - 4 * b * 8192 >= TC_MIN_STAGES * stage) return b;
  return 0;
}
// Two chunks per tensor store (a 16 KB buffer per group) when that keeps four ring stages.
static bool pair_out_pairs(int L_max) {
  const int nch = 2 * L_max / TC_KC;
  const int stage = nch * 2 * TC_BM * TC_KC * 2;
  const int res = nch * 2 * 128 * TC_KC * 2;
  return smem_optin() - 1024 - (int)sizeof(TcCtl) - res - 4 * 16384 >= 4 * stage;
}

bool fg_tc_pair_fits(int L_max) {
  return fg_tc_available() && L_max % 16 == 0 && L_max >= 16 && 2 * L_max / TC_KC <= TC_RB_MAXCH &&
         pair_out_bufs(L_max) > 0;
}

// Pair assembly (real F without a -1 eigenvalue): one GEMM row per entry pair (i, k) of the
// block-upper region, K = the 2 L_max powers M_l, l != 0 (M_0 = I and P = 0 are not stored);
// columns: the orders' coefficients c_l and, 64 columns on, the mirror coefficients c_{-l},
// so one pass gives Q[i][k] and Q[k][i] = sum_l c_{-l} M_l[i][k] (M_{-l} = M_l^T).
static cudaError_t tc_assemble_pair(const TcAssembleArgs& a, cudaStream_t s) {
  if (!a.real_a || !a.Qs || a.A < 1 || a.A > 64 || a.N % 128 || a.K2 % TC_KC || a.K2 < TC_KC ||
      a.K2 / TC_KC > TC_RB_MAXCH || a.pair_rows % TC_BM || a.pair_rows / TC_BM > INT32_MAX)
    return cudaErrorInvalidValue;
  const int nch = (int)(a.K2 / TC_KC);
  CUtensorMap mB, mO;
  if (!make_map(&mB, a.Cs, a.K2, 128, a.K2, 4, 128 * a.K2, 128)) return cudaErrorInvalidValue;
  // the operators as a 4-D tensor {k, i, plane, order} for the staged stores: box = 128 entries
  // of one row, 2 planes, 16 orders (the box's orders past A are not written)
  {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorInvalidValue;
    cuuint64_t dims[4] = {(cuuint64_t)a.N, (cuuint64_t)a.N, 4, (cuuint64_t)a.A};
    cuuint64_t strides[3] = {(cuuint64_t)a.Np * 2, (cuuint64_t)a.plane_elems * 2, (cuuint64_t)a.plane_elems * 8};
    cuuint32_t box[4] = {128, 1, 2, pair_out_pairs((int)(a.K2 / 2)) ? 32u : 16u};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&mO, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, a.Qs, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  TcParams p{};
  p.ntiles = (int)(a.pair_rows / TC_BM);
  p.arith_cols = 128;
  p.nblk = 1;
  p.grouped = 1;
  p.rows = a.pair_rows;
  p.kchunks = nch;
  p.kvalid = (int)a.K2;
  p.cps = nch;  // every chunk of a tile in one ring stage, copied from its image
  p.a_img = reinterpret_cast<const uint8_t*>(a.pair_stack);
  p.stage_bytes = nch * 2 * TC_BM * TC_KC * 2;
  p.Qs = a.Qs;
  p.qN = a.N;
  p.qNp = a.Np;
  p.qplane = a.plane_elems;
  p.col_exp = a.col_exp;
  p.status = a.status;
  p.skip_im = 1;
  p.re_only = 1;
  p.uscale = ldexpf(1.0f, -FG_COEF_EXP);
  p.pair_nbt = (int)(a.N / 128);
  p.pair_A = (int)a.A;
  p.diag = a.diag;
  p.out_bufs = pair_out_bufs((int)(a.K2 / 2));
  if (p.out_bufs == 0) return cudaErrorNotSupported;
  p.out_pairs = pair_out_pairs((int)(a.K2 / 2)) ? 1 : 0;
  // staging buffers of the four epilogue groups: one 16 KB buffer (two chunks per store), or
  // out_bufs 8 KB buffers
  p.out_bytes = p.out_pairs ? 4 * 16384 : 4 * p.out_bufs * 8192;
  std::vector<int4> none;
  return launch(mB, mB, none, p, a.scratch, a.scratch_bytes, s, FGFRFT_KC_ASSEMBLE_MULTI, 128, true, true, &mO);
}

cudaError_t fg_tc_assemble(const TcAssembleArgs& a, cudaStream_t s) {
  if (a.pair_stack) return tc_assemble_pair(a, s);
  // Fused multi-order assembly as one complex GEMM: rows = the N*N entries of the
  // entry-major split stack (K = all stored blocks), columns = the orders, whose
  // "signals" are their coefficient vectors over the stored blocks.
  if (a.entries > ((int64_t)1 << 37) || a.A > (1 << 20)) return cudaErrorInvalidValue;
  const int bn = a.A <= 64 ? 64 : 128;
  // the entry-major stack is chunk-major: per plane, Kp / 32 full chunk planes of 32
  // columns (64-byte rows: a TMA box is 8 KB of contiguous, aligned memory), then a
  // tail plane of Kp mod 32 columns
  const int64_t nfull = a.Kp / TC_KC, wtail = a.Kp % TC_KC;
  if (a.Kp % 8 || a.Kp < a.K) return cudaErrorInvalidValue;
  CUtensorMap mA, mB, mT;
  const __half* tail = a.entry_stack + 4 * nfull * a.planeT * TC_KC;
  // one column tile (A <= 64): the coefficient operand stays resident in shared memory
  const bool rb = bn == 64 && (a.K + TC_KC - 1) / TC_KC <= TC_RB_MAXCH;
  // a tail of at most 16 columns is read as a 16-column box with 32-byte swizzle (the box
  // carries no more than 8 zero-filled columns, 4 KB per plane instead of 8 KB)
  const bool tail16 = rb && wtail > 0 && wtail <= 16;
  if ((nfull > 0 && !fg_make_map_f16(&mA, a.entry_stack, TC_KC, a.entries, TC_KC, 4 * nfull, a.planeT * TC_KC,
                                      TC_KC, TC_BM, 64)) ||
      (wtail > 0 && !fg_make_map_f16(&mT, tail, wtail, a.entries, wtail, 4, a.planeT * wtail, tail16 ? 16 : TC_KC,
                                     TC_BM, tail16 ? 32 : 64)) ||
      !make_map(&mB, a.Cs, a.K, a.A, a.Kp, 4, a.A * a.Kp, bn))
    return cudaErrorInvalidValue;
  if (nfull == 0) mA = mT;
  if (wtail == 0) mT = mA;
  std::vector<int4> tiles;
  const int64_t row_tiles = (a.entries + TC_BM - 1) / TC_BM;
  if (row_tiles > INT32_MAX) return cudaErrorInvalidValue;
  TcParams p{};
  if (a.A <= bn) {  // one column tile: tile t is row tile t, no table
    p.ntiles = (int)row_tiles;
    p.arith_cols = (int)a.A;
  } else {
    for (int64_t c = 0; c < a.A; c += bn)
      for (int64_t rt = 0; rt < row_tiles; ++rt)
        tiles.push_back(make_int4((int)rt, 0, (int)c, (int)std::min<int64_t>(c + bn, a.A)));
  }
  p.nblk = 1;
  p.grouped = 1;
  p.rows = a.entries;
  p.kchunks = (int)((a.K + TC_KC - 1) / TC_KC);
  p.kvalid = (int)a.K;
  p.a_chunked = 1;
  p.a_nfull = (int)nfull;
  p.Y = a.Qc;
  p.Qs = a.Qs;
  p.qN = a.N;
  p.qNp = a.Np;
  p.qplane = a.plane_elems;
  p.col_exp = a.col_exp;
  p.status = a.status;
  p.skip_im = a.skip_im ? 1 : 0;
  p.re_only = a.re_only && a.real_a ? 1 : 0;
  // one exponent for every coefficient column (FG_COEF_EXP)
  p.uscale = ldexpf(1.0f, a.Qs ? -FG_COEF_EXP : -(FG_SPLIT_SHIFT + FG_COEF_EXP));
  // the k-chunks of a tile are few (K = 2L+2 stored blocks): group them into one ring stage,
  // as many as leave room for two stages (all of them with the narrow tail)
  if (tail16) {
    const int ap = a.real_a ? 2 : 4;
    p.a_tail16 = 1;
    p.cps = p.kchunks;
    p.stage_bytes = (int)nfull * ap * TC_BM * TC_KC * 2 + ap * TC_BM * 32;
  } else {
    const int plane_b = bn * TC_KC * 2;
    const int chunk = (a.real_a ? 2 : 4) * TC_BM * TC_KC * 2 + (rb ? 0 : 4 * plane_b);
    const int res = rb ? p.kchunks * 4 * plane_b : 0;
    const int avail = smem_optin() - 1024 - (int)sizeof(TcCtl) - res;
    p.cps = std::max(1, std::min(p.kchunks, avail / (2 * chunk)));
  }
  return launch(mA, mB, tiles, p, a.scratch, a.scratch_bytes, s, FGFRFT_KC_ASSEMBLE_MULTI, bn, rb, a.real_a, &mT);
}

size_t fg_tc_assemble_scratch_bytes(int64_t entries, int64_t A) {
  const int64_t row_tiles = (entries + TC_BM - 1) / TC_BM;
  const int64_t col_tiles = (A + 63) / 64;
  return (size_t)(row_tiles * col_tiles) * sizeof(int4) + 256;
}
