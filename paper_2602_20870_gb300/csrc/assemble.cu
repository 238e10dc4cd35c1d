// Online operator assembly (Def. 1; Algorithm 1, online part):
//   Q = e^{j pi a} P + sum_{l=-L}^{L} c_l(a) M_l
// is a streaming linear combination of 2L + 2 stored N x N blocks, bound by HBM
// bandwidth.  Each CTA owns a contiguous chunk of entries and walks the blocks in
// order; one thread stages (chunk, block) tiles into a shared-memory ring with 1-D
// bulk copies (cp.async.bulk, completion on an mbarrier), so the loads in flight per
// SM are bounded by the ring size rather than by registers.
#include <algorithm>

#include "internal.h"

namespace {

// ---------------------------------------------------------------------------
// K1: one order.  CHUNK complex entries per tile, STAGES ring slots.
// ---------------------------------------------------------------------------
constexpr int K1_THREADS = 256;
constexpr int K1_CHUNK = 2048;                      // 16 KB of c64 per tile
constexpr int K1_STAGES = 6;                        // 96 KB ring per CTA
constexpr int K1_PER_THREAD = K1_CHUNK / K1_THREADS;  // 8 entries (4 x float4)
constexpr int K1_MAXBLK = 1024;

struct K1Smem {
  float4 ring[K1_STAGES][K1_CHUNK / 2];
  float2 coef[K1_MAXBLK];
  uint64_t full[K1_STAGES];
};

// SPLIT: Q is written as four fp16 planes (scaled by 2^FG_SPLIT_SHIFT, hi/lo) of N rows
// with pitch Np instead of c64.
template <bool SPLIT>
__global__ void __launch_bounds__(K1_THREADS) assemble_single_kernel(const float2* __restrict__ stack,
                                                                     int64_t blk_elems, int b0, int nb_pow,
                                                                     int p_blk, int64_t NN,
                                                                     const float2* __restrict__ coef,
                                                                     float2* __restrict__ Q, __half* __restrict__ Qs,
                                                                     int64_t N, int64_t Np, int64_t plane_elems,
                                                                     uint32_t* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  K1Smem& sm = *reinterpret_cast<K1Smem*>(smem_raw);
  const int nblk = nb_pow + (p_blk >= 0 ? 1 : 0);
  const int tid = threadIdx.x;
  for (int b = tid; b < nblk; b += K1_THREADS) sm.coef[b] = coef[b];
  if (tid == 0) {
    for (int s = 0; s < K1_STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();

  const int64_t ntiles = (NN + K1_CHUNK - 1) / K1_CHUNK;
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_tiles * nblk;
  uint64_t policy = 0;
  if (tid == 0) policy = policy_evict_first();

  auto issue = [&](int64_t item) {
    const int s = (int)(item % K1_STAGES);
    const int64_t t = blockIdx.x + (item / nblk) * gridDim.x;
    const int b = (int)(item % nblk);
    const int blk = b < nb_pow ? b0 + b : p_blk;
    const int64_t e0 = t * K1_CHUNK;
    const int64_t cnt = (NN - e0) < K1_CHUNK ? (NN - e0) : K1_CHUNK;
    // byte count rounded up to 16: the block stride is padded to 32 entries, so
    // the over-read stays inside the block's padding.
    const uint32_t bytes = (uint32_t)(((cnt * 8) + 15) & ~int64_t(15));
    mbar_arrive_expect_tx(&sm.full[s], bytes);
    bulk_g2s_evict_first(&sm.ring[s][0], stack + (int64_t)blk * blk_elems + e0, bytes, &sm.full[s], policy);
  };

  if (tid == 0) {
    const int64_t pre = items < K1_STAGES ? items : K1_STAGES;
    for (int64_t it = 0; it < pre; ++it) issue(it);
  }

  float2 acc[K1_PER_THREAD];
#pragma unroll
  for (int e = 0; e < K1_PER_THREAD; ++e) acc[e] = make_float2(0.f, 0.f);

  bool ok = true;
  for (int64_t it = 0; it < items; ++it) {
    const int s = (int)(it % K1_STAGES);
    const uint32_t parity = (uint32_t)((it / K1_STAGES) & 1);
    const int b = (int)(it % nblk);
    if (ok) ok = mbar_wait(&sm.full[s], parity, status);
    const float2 c = sm.coef[b];
    if (ok) {
#pragma unroll
      for (int v = 0; v < K1_PER_THREAD / 2; ++v) {
        const float4 x = sm.ring[s][tid + v * K1_THREADS];
        // entries 2*(tid + v*256) and +1
        acc[2 * v].x = fmaf(c.x, x.x, fmaf(-c.y, x.y, acc[2 * v].x));
        acc[2 * v].y = fmaf(c.x, x.y, fmaf(c.y, x.x, acc[2 * v].y));
        acc[2 * v + 1].x = fmaf(c.x, x.z, fmaf(-c.y, x.w, acc[2 * v + 1].x));
        acc[2 * v + 1].y = fmaf(c.x, x.w, fmaf(c.y, x.z, acc[2 * v + 1].y));
      }
    }
    __syncthreads();  // every thread is done with slot s
    if (tid == 0 && ok && it + K1_STAGES < items) issue(it + K1_STAGES);
    if (b == nblk - 1) {
      const int64_t t = blockIdx.x + (it / nblk) * gridDim.x;
      const int64_t e0 = t * K1_CHUNK;
#pragma unroll
      for (int v = 0; v < K1_PER_THREAD / 2; ++v) {
        const int64_t e = e0 + 2 * (tid + (int64_t)v * K1_THREADS);
        if (!SPLIT) {
          if (e < NN) Q[e] = acc[2 * v];
          if (e + 1 < NN) Q[e + 1] = acc[2 * v + 1];
        } else {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int64_t g = e + u;
            if (g < NN) {
              const int64_t i = g / N, k = g - (g / N) * N;
              const float sc = (float)(1 << FG_SPLIT_SHIFT);
              const float re = acc[2 * v + u].x * sc, im = acc[2 * v + u].y * sc;
              const __half2 hi = __floats2half2_rn(re, im);
              const float2 hf = __half22float2(hi);
              const __half2 lo = __floats2half2_rn(re - hf.x, im - hf.y);
              __half* q = Qs + i * Np + k;
              q[0] = __low2half(hi);
              q[plane_elems] = __low2half(lo);
              q[2 * plane_elems] = __high2half(hi);
              q[3 * plane_elems] = __high2half(lo);
            }
          }
        }
        acc[2 * v] = make_float2(0.f, 0.f);
        acc[2 * v + 1] = make_float2(0.f, 0.f);
      }
    }
  }
  // drain: if a wait failed, the copies already issued may still land; wait for
  // each outstanding slot (bounded) before the CTA's shared memory is released.
  if (!ok && tid == 0) {
    for (int s = 0; s < K1_STAGES; ++s) {
      const uint64_t t0 = global_timer_ns();
      while (!mbar_try_wait(&sm.full[s], 0) && !mbar_try_wait(&sm.full[s], 1)) {
        if (global_timer_ns() - t0 > FG_WAIT_LIMIT_NS) break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K1 for real F: the stored blocks are real, so the assembly streams only their two real
// split planes (fp16 hi/lo of 2^12 M, 4 bytes per entry instead of 8):
//   Re Q = sum_l c_l M_l + cos(pi a) P,   Im Q = sin(pi a) P.
// The planes are N rows of pitch Np; the kernel streams all N * Np slots of a plane and
// skips the padding columns on output.
// ---------------------------------------------------------------------------
constexpr int KR_CHUNK = 4096;  // entries per tile: 2 planes x 8 KB per block
constexpr int KR_STAGES = 6;
constexpr int KR_EPT = KR_CHUNK / K1_THREADS;  // 16 entries per thread

struct KRSmem {
  uint4 ring[KR_STAGES][2][KR_CHUNK / 8];  // [stage][hi, lo][8 halves]
  float2 coef[K1_MAXBLK];
  uint64_t full[KR_STAGES];
};

template <bool SPLIT>
__global__ void __launch_bounds__(K1_THREADS) assemble_single_real_kernel(
    const __half* __restrict__ planes, int64_t blk_stride, int64_t plane_elems, int b0, int nb_pow, int p_blk,
    int64_t N, int64_t Np, const float2* __restrict__ coef, float2* __restrict__ Q, __half* __restrict__ Qs,
    int64_t q_plane, int write_im, uint32_t* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  KRSmem& sm = *reinterpret_cast<KRSmem*>(smem_raw);
  const int nblk = nb_pow + (p_blk >= 0 ? 1 : 0);
  const int tid = threadIdx.x;
  for (int b = tid; b < nblk; b += K1_THREADS) sm.coef[b] = coef[b];
  if (tid == 0) {
    for (int s = 0; s < KR_STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  const int64_t total = N * Np;  // slots per plane (N rows of pitch Np)
  const int64_t ntiles = (total + KR_CHUNK - 1) / KR_CHUNK;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_tiles * nblk;
  uint64_t policy = 0;
  if (tid == 0) policy = policy_evict_first();
  auto issue = [&](int64_t item) {
    const int s = (int)(item % KR_STAGES);
    const int64_t t = blockIdx.x + (item / nblk) * gridDim.x;
    const int b = (int)(item % nblk);
    const int blk = b < nb_pow ? b0 + b : p_blk;
    const int64_t e0 = t * KR_CHUNK;
    const int64_t cnt = (total - e0) < KR_CHUNK ? (total - e0) : KR_CHUNK;
    // plane_elems is padded to 128 slots, so rounding the byte count up to 16 stays inside it
    const uint32_t bytes = (uint32_t)(((cnt * 2) + 15) & ~int64_t(15));
    mbar_arrive_expect_tx(&sm.full[s], 2 * bytes);
    const __half* src = planes + (int64_t)blk * blk_stride + e0;
    bulk_g2s_evict_first(&sm.ring[s][0][0], src, bytes, &sm.full[s], policy);
    bulk_g2s_evict_first(&sm.ring[s][1][0], src + plane_elems, bytes, &sm.full[s], policy);
  };
  if (tid == 0) {
    const int64_t pre = items < KR_STAGES ? items : KR_STAGES;
    for (int64_t it = 0; it < pre; ++it) issue(it);
  }
  const float inv = 1.0f / (float)(1 << FG_SPLIT_SHIFT);
  float acc[KR_EPT];
  float accp[KR_EPT];  // the P block (real), kept apart for its complex coefficient
#pragma unroll
  for (int e = 0; e < KR_EPT; ++e) acc[e] = accp[e] = 0.f;
  bool ok = true;
  for (int64_t it = 0; it < items; ++it) {
    const int s = (int)(it % KR_STAGES);
    const uint32_t parity = (uint32_t)((it / KR_STAGES) & 1);
    const int b = (int)(it % nblk);
    if (ok) ok = mbar_wait(&sm.full[s], parity, status);
    if (ok) {
      const float c = b < nb_pow ? sm.coef[b].x * inv : 0.f;
#pragma unroll
      for (int v = 0; v < KR_EPT / 8; ++v) {
        const uint4 hv = sm.ring[s][0][tid + v * K1_THREADS];
        const uint4 lv = sm.ring[s][1][tid + v * K1_THREADS];
        const __half2* h2 = reinterpret_cast<const __half2*>(&hv);
        const __half2* l2 = reinterpret_cast<const __half2*>(&lv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 hf = __half22float2(h2[q]), lf = __half22float2(l2[q]);
          const float x0 = hf.x + lf.x, x1 = hf.y + lf.y;
          if (b < nb_pow) {
            acc[8 * v + 2 * q] = fmaf(c, x0, acc[8 * v + 2 * q]);
            acc[8 * v + 2 * q + 1] = fmaf(c, x1, acc[8 * v + 2 * q + 1]);
          } else {
            accp[8 * v + 2 * q] = x0 * inv;
            accp[8 * v + 2 * q + 1] = x1 * inv;
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && ok && it + KR_STAGES < items) issue(it + KR_STAGES);
    if (b == nblk - 1) {
      const int64_t t = blockIdx.x + (it / nblk) * gridDim.x;
      const float2 cp = p_blk >= 0 ? sm.coef[nb_pow] : make_float2(0.f, 0.f);
#pragma unroll
      for (int v = 0; v < KR_EPT / 8; ++v) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e_loc = 8 * (tid + v * K1_THREADS) + u;  // slot within the tile
          const int64_t slot = t * KR_CHUNK + e_loc;
          const float re = acc[8 * v + u] + cp.x * accp[8 * v + u];
          const float im = cp.y * accp[8 * v + u];
          if (slot < total) {
            const int64_t i = slot / Np, k = slot - (slot / Np) * Np;
            if (k < N) {
              if (!SPLIT) {
                Q[i * N + k] = make_float2(re, im);
              } else {
                const float sc = (float)(1 << FG_SPLIT_SHIFT);
                const __half2 hi = __floats2half2_rn(re * sc, im * sc);
                const float2 hf = __half22float2(hi);
                const __half2 lo = __floats2half2_rn(re * sc - hf.x, im * sc - hf.y);
                __half* qq = Qs + slot;  // same pitch as the stored planes
                qq[0] = __low2half(hi);
                qq[q_plane] = __low2half(lo);
                if (write_im) {
                  qq[2 * q_plane] = __high2half(hi);
                  qq[3 * q_plane] = __high2half(lo);
                }
              }
            }
          }
          acc[8 * v + u] = 0.f;
          accp[8 * v + u] = 0.f;
        }
      }
    }
  }
  if (!ok && tid == 0) {
    for (int s = 0; s < KR_STAGES; ++s) {
      const uint64_t t0 = global_timer_ns();
      while (!mbar_try_wait(&sm.full[s], 0) && !mbar_try_wait(&sm.full[s], 1)) {
        if (global_timer_ns() - t0 > FG_WAIT_LIMIT_NS) break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K2: up to 128 orders in one pass over the stack.  The orders form n_og groups of
// 32; CTA c serves order group c mod n_og, and the n_og CTAs of a group walk the
// same tile sequence at the same pace, so each stored tile is fetched from HBM once
// and served to the other CTAs from L2.  Thread t of a CTA accumulates entry t of
// the 256-entry tile for the 32 orders of its group (64 FP32 accumulators in
// registers).  Each ring slot holds K2_GB consecutive blocks of the tile (one bulk
// copy per block), so one barrier round covers K2_GB blocks.  Real coefficients of
// the powers [nb_pow][32] and the complex coefficients of P live in shared memory and
// are read as warp-wide broadcasts.
// ---------------------------------------------------------------------------
constexpr int K2_CHUNK = 256;
constexpr int K2_GB = 4;
constexpr int K2_STAGES = 6;
constexpr int K2_AC = 32;

template <bool SPLIT>
__global__ void __launch_bounds__(256, 1) assemble_multi_kernel(
    const float2* __restrict__ stack, int64_t blk_elems, int b0, int nb_pow, int p_blk, int64_t N, int A, int a0,
    const float2* __restrict__ coef, float2* __restrict__ Qc, __half* __restrict__ Qs, int64_t Np,
    int64_t plane_elems, int n_og, uint32_t* status) {
  constexpr int NT = 256;
  constexpr int NA = K2_AC;  // orders per CTA
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* ring = reinterpret_cast<float2*>(smem_raw);        // [STAGES][GB][CHUNK]
  float2* cpx = ring + K2_STAGES * K2_GB * K2_CHUNK;         // [NA]
  float* cre = reinterpret_cast<float*>(cpx + NA);           // [nb_pow][NA]
  uint64_t* full = reinterpret_cast<uint64_t*>(cre + (size_t)nb_pow * NA);
  const bool has_p = p_blk >= 0;
  const int nblk = nb_pow + (has_p ? 1 : 0);
  const int ngrp = (nblk + K2_GB - 1) / K2_GB;
  const int tid = threadIdx.x;
  const int e_loc = tid;
  const int og = (int)(blockIdx.x % n_og);
  const int cta = (int)(blockIdx.x / n_og), ncta = (int)(gridDim.x / n_og);
  const int oa0 = a0 + og * K2_AC;  // first order of this CTA
  const int na = (A - oa0) < NA ? (A - oa0) : NA;
  for (int t = tid; t < nb_pow * NA; t += NT) {
    const int b = t / NA, a = t % NA;
    cre[t] = a < na ? coef[(size_t)b * A + oa0 + a].x : 0.f;
  }
  for (int a = tid; a < NA; a += NT)
    cpx[a] = (has_p && a < na) ? coef[(size_t)nb_pow * A + oa0 + a] : make_float2(0.f, 0.f);
  if (tid == 0) {
    for (int s = 0; s < K2_STAGES; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  const int64_t NN = N * N;
  const int64_t ntiles = (NN + K2_CHUNK - 1) / K2_CHUNK;
  const int64_t my_tiles = ntiles > cta ? (ntiles - 1 - cta) / ncta + 1 : 0;
  const int64_t items = my_tiles * ngrp;
  auto issue = [&](int64_t item) {
    const int s = (int)(item % K2_STAGES);
    const int64_t t = cta + (item / ngrp) * ncta;
    const int g = (int)(item % ngrp);
    const int64_t e0 = t * K2_CHUNK;
    const int64_t cnt = (NN - e0) < K2_CHUNK ? (NN - e0) : K2_CHUNK;
    const uint32_t bytes = (uint32_t)(((cnt * 8) + 15) & ~int64_t(15));
    const int bmax = (nblk - g * K2_GB) < K2_GB ? (nblk - g * K2_GB) : K2_GB;
    mbar_arrive_expect_tx(&full[s], bytes * (uint32_t)bmax);
    for (int q = 0; q < bmax; ++q) {
      const int b = g * K2_GB + q;
      const int blk = b < nb_pow ? b0 + b : p_blk;
      bulk_g2s(ring + ((size_t)s * K2_GB + q) * K2_CHUNK, stack + (int64_t)blk * blk_elems + e0, bytes, &full[s]);
    }
  };
  if (tid == 0) {
    const int64_t pre = items < K2_STAGES ? items : K2_STAGES;
    for (int64_t it = 0; it < pre; ++it) issue(it);
  }
  float2 acc[K2_AC];
#pragma unroll
  for (int a = 0; a < K2_AC; ++a) acc[a] = make_float2(0.f, 0.f);
  bool ok = true;
  for (int64_t it = 0; it < items; ++it) {
    const int s = (int)(it % K2_STAGES);
    const uint32_t parity = (uint32_t)((it / K2_STAGES) & 1);
    const int g = (int)(it % ngrp);
    if (ok) ok = mbar_wait(&full[s], parity, status);
    if (ok) {
      const int bmax = (nblk - g * K2_GB) < K2_GB ? (nblk - g * K2_GB) : K2_GB;
      for (int q = 0; q < bmax; ++q) {
        const int b = g * K2_GB + q;
        const float2 x = ring[((size_t)s * K2_GB + q) * K2_CHUNK + e_loc];
        if (b < nb_pow) {  // real coefficient: 2 FMAs per entry and order
          const float4* cb = reinterpret_cast<const float4*>(cre + (size_t)b * NA);
#pragma unroll
          for (int a4 = 0; a4 < K2_AC / 4; ++a4) {
            const float4 c = cb[a4];
            acc[4 * a4 + 0].x = fmaf(c.x, x.x, acc[4 * a4 + 0].x);
            acc[4 * a4 + 0].y = fmaf(c.x, x.y, acc[4 * a4 + 0].y);
            acc[4 * a4 + 1].x = fmaf(c.y, x.x, acc[4 * a4 + 1].x);
            acc[4 * a4 + 1].y = fmaf(c.y, x.y, acc[4 * a4 + 1].y);
            acc[4 * a4 + 2].x = fmaf(c.z, x.x, acc[4 * a4 + 2].x);
            acc[4 * a4 + 2].y = fmaf(c.z, x.y, acc[4 * a4 + 2].y);
            acc[4 * a4 + 3].x = fmaf(c.w, x.x, acc[4 * a4 + 3].x);
            acc[4 * a4 + 3].y = fmaf(c.w, x.y, acc[4 * a4 + 3].y);
          }
        } else {  // the P block: complex coefficient e^{j pi a} (or its derivative)
#pragma unroll
          for (int a = 0; a < K2_AC; ++a) cmac(acc[a], cpx[a], x);
        }
      }
    }
    __syncthreads();  // every thread is done with slot s
    if (tid == 0 && ok && it + K2_STAGES < items) issue(it + K2_STAGES);
    if (g == ngrp - 1) {
      const int64_t t = cta + (it / ngrp) * ncta;
      const int64_t e = t * K2_CHUNK + e_loc;
      if (e < NN) {
        const int64_t i = e / N, k = e - (e / N) * N;
        if (!SPLIT) {
          float2* q = Qc + (int64_t)oa0 * NN + e;
#pragma unroll
          for (int a = 0; a < K2_AC; ++a) {
            if (a < na) __stcs(q, acc[a]);
            q += NN;
          }
        } else {
          const float sc = (float)(1 << FG_SPLIT_SHIFT);
          __half* q = Qs + (int64_t)oa0 * 4 * plane_elems + i * Np + k;
#pragma unroll
          for (int a = 0; a < K2_AC; ++a) {
            if (a < na) {
              const float re = acc[a].x * sc, im = acc[a].y * sc;
              const __half rh = __float2half_rn(re), ih = __float2half_rn(im);
              q[0] = rh;
              q[plane_elems] = __float2half_rn(re - __half2float(rh));
              q[2 * plane_elems] = ih;
              q[3 * plane_elems] = __float2half_rn(im - __half2float(ih));
            }
            q += 4 * plane_elems;
          }
        }
      }
#pragma unroll
      for (int a = 0; a < K2_AC; ++a) acc[a] = make_float2(0.f, 0.f);
    }
  }
  if (!ok && tid == 0) {
    for (int s = 0; s < K2_STAGES; ++s) {
      const uint64_t t0 = global_timer_ns();
      while (!mbar_try_wait(&full[s], 0) && !mbar_try_wait(&full[s], 1)) {
        if (global_timer_ns() - t0 > FG_WAIT_LIMIT_NS) break;
      }
    }
  }
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <bool SPLIT>
cudaError_t launch_multi(const float2* stack, int64_t blk_elems, int b0, int nb_pow, int p_blk, int64_t N, int A,
                         int a0, int n_og, const float2* coef, float2* Qc, __half* Qs, int64_t Np,
                         int64_t plane_elems, uint32_t* status, cudaStream_t s) {
  const size_t smem = (size_t)K2_STAGES * K2_GB * K2_CHUNK * sizeof(float2) + K2_AC * sizeof(float2) +
                      (size_t)nb_pow * K2_AC * sizeof(float) + K2_STAGES * sizeof(uint64_t) + 16;
  auto kern = assemble_multi_kernel<SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t NN = N * N;
  const int64_t ntiles = (NN + K2_CHUNK - 1) / K2_CHUNK;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t ncta = (int64_t)num_sms() * per_sm / n_og;  // CTAs per order group
  if (ncta > ntiles) ncta = ntiles;
  if (ncta < 1) ncta = 1;
  kern<<<(unsigned)(ncta * n_og), 256, smem, s>>>(stack, blk_elems, b0, nb_pow, p_blk, N, A, a0, coef, Qc, Qs, Np,
                                                  plane_elems, n_og, status);
  fg_note_launch(FGFRFT_KC_ASSEMBLE_MULTI);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// K1h: one order from the half stack.  Only M_0..M_L and P are stored; a negative power
// is the conjugate transpose of the positive one, M_{-l} = M_l^H (Prop. 2; Algorithm 1
// forms M_n^H the same way).  Q is cut into 64 x 64 tiles and a CTA takes the pair
// (I, K), (K, I), I <= K, reading both tiles of every stored block once:
//   Q[I,K] += c_l M_l[I,K] + c_{-l} (M_l[K,I])^H,   Q[K,I] += c_l M_l[K,I] + c_{-l} (M_l[I,K])^H,
// so each stored entry serves one positive and one negative power and the stack streams
// half the bytes of a full one.  The stack holds FP32 tiles of 16 KB per plane, each row r
// permuted by c -> c ^ (r & 31): one bulk copy brings a tile into shared memory, and a
// warp reading one row (lanes = columns) or one column (lanes = rows) of it touches 32
// different banks.  Warp w owns rows 8w..8w+7 of a tile; lane t its columns t and t + 32.
// A producer warp keeps the ring full; consumer warps release each stage on an mbarrier.
// P (stored once) comes last with its complex coefficient.
// ---------------------------------------------------------------------------
constexpr int KH_T = 64;
constexpr int KH_WARPS = 8;                      // consumer warps
constexpr int KH_THREADS = 32 * (KH_WARPS + 1);  // + one producer warp
constexpr int KH_TILE = KH_T * KH_T * 4;         // bytes of one FP32 plane of one tile

template <bool CPLX>
struct KHCfg {
  static constexpr int PLANES = CPLX ? 2 : 1;        // re (, im)
  static constexpr int STAGE = 2 * PLANES * KH_TILE;  // both tiles of a pair
  static constexpr int STAGES = CPLX ? 3 : 6;
};

struct KHCtl {
  uint64_t full[8];   // stage loaded (bulk-copy bytes)
  uint64_t empty[8];  // stage consumed (one arrival per consumer warp)
  float cpos[K1_MAXBLK];  // c_l, l = 0..L
  float cneg[K1_MAXBLK];  // c_{-l} (0 for l = 0)
  float2 cp;              // e^{j pi a}
};

// (I, K) of pair p: row I of the upper triangle holds nt - I pairs, K = I .. nt-1.  A
// single-precision estimate of the row (FP64 is a slow pipe here), corrected exactly.
__device__ __forceinline__ void kh_pair(int64_t p, int nt, int& I, int& K) {
  auto start = [&](int64_t i) { return i * nt - i * (i - 1) / 2; };
  const float b = 2.0f * (float)nt + 1.0f;
  int64_t i = (int64_t)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)p, 0.f))) * 0.5f);
  if (i < 0) i = 0;
  if (i > nt - 1) i = nt - 1;
  while (i < nt - 1 && start(i + 1) <= p) ++i;
  while (i > 0 && start(i) > p) --i;
  I = (int)i;
  K = (int)(i + (p - start(i)));
}

template <bool CPLX, bool SPLIT>
__global__ void __launch_bounds__(KH_THREADS, 1) assemble_half_kernel(
    const float* __restrict__ stack, int64_t hplane, int nt, int L, int blk_P, int has_p,
    const float2* __restrict__ coef, int64_t N, float2* __restrict__ Q, __half* __restrict__ Qs, int64_t Np,
    int64_t q_plane, int write_im, uint32_t* status) {
  using Cfg = KHCfg<CPLX>;
  constexpr int PL = Cfg::PLANES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* const base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  KHCtl& sm = *reinterpret_cast<KHCtl*>(base + Cfg::STAGES * Cfg::STAGE);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j = tid; j <= L; j += KH_THREADS) {
    sm.cpos[j] = coef[L + j].x;
    sm.cneg[j] = j > 0 ? coef[L - j].x : 0.f;
  }
  if (tid == 0) {
    sm.cp = has_p ? coef[2 * L + 1] : make_float2(0.f, 0.f);
    for (int s = 0; s < Cfg::STAGES; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], KH_WARPS);
    }
    fence_barrier_init();
  }
  __syncthreads();

  const int64_t npairs = (int64_t)nt * (nt + 1) / 2;
  const int nbi = L + 1 + (has_p ? 1 : 0);  // items per pair: blocks 0..L, then P
  const int64_t my_pairs = npairs > blockIdx.x ? (npairs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_pairs * nbi;

  if (warp == KH_WARPS) {
    // ---------------------------------------------------------------- producer warp
    if (lane == 0) {
      int ps = 0, pj = 0, pI = 0, pK = 0;
      int64_t ppr = blockIdx.x;
      if (my_pairs > 0) kh_pair(ppr, nt, pI, pK);
      uint32_t issued[Cfg::STAGES] = {};
      uint32_t eph = 1;  // a fresh barrier's preceding phase counts as complete
      bool pok = true;
      uint64_t policy = policy_evict_first();
      for (int64_t it = 0; pok && it < items; ++it) {
        const int s = ps;
        if (!mbar_wait(&sm.empty[s], eph, status)) {
          pok = false;
          break;
        }
        const int blk = pj <= L ? pj : blk_P;
        const bool diag = pI == pK;
        uint8_t* st = base + s * Cfg::STAGE;
        mbar_arrive_expect_tx(&sm.full[s], (uint32_t)(PL * KH_TILE * (diag ? 1 : 2)));
        const float* bb = stack + (int64_t)blk * 2 * hplane;
#pragma unroll
        for (int q = 0; q < PL; ++q) {
          bulk_g2s_evict_first(st + q * KH_TILE, bb + q * hplane + ((int64_t)pI * nt + pK) * 4096, KH_TILE,
                               &sm.full[s], policy);
          if (!diag)
            bulk_g2s_evict_first(st + (PL + q) * KH_TILE, bb + q * hplane + ((int64_t)pK * nt + pI) * 4096, KH_TILE,
                                 &sm.full[s], policy);
        }
        issued[s]++;
        if (++ps == Cfg::STAGES) {
          ps = 0;
          eph ^= 1u;
        }
        if (++pj == nbi) {
          pj = 0;
          ppr += gridDim.x;
          if (ppr < npairs) kh_pair(ppr, nt, pI, pK);
        }
      }
      if (!pok) {  // wait (bounded) until every issued copy has landed
        for (int s = 0; s < Cfg::STAGES; ++s) {
          if (!issued[s]) continue;
          const uint32_t par = (issued[s] - 1) & 1;
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&sm.full[s], par) && global_timer_ns() - t0 < FG_WAIT_LIMIT_NS) {
          }
        }
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumer warps
  // accumulators: [tile (I,K) / (K,I)][row of the warp][column half]
  float re[2][8][2], im[2][8][2];
#pragma unroll
  for (int o = 0; o < 2; ++o)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) re[o][r][h] = im[o][r][h] = 0.f;
  // element offsets in a swizzled tile, the same for every stage: (row 8w + r, column
  // lane + 32h) read directly, and the transposed element (lane + 32h, 8w + r)
  int offD[8][2], offT[8][2];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = 8 * warp + r, col = lane + 32 * h;
      offD[r][h] = row * KH_T + (col ^ (row & 31));
      offT[r][h] = col * KH_T + (row ^ (col & 31));
    }

  bool ok = true;
  int cs_ = 0, cj = 0, I = 0, K = 0;
  uint32_t parity = 0;
  int64_t cpr = blockIdx.x;
  if (my_pairs > 0) kh_pair(cpr, nt, I, K);
  for (int64_t it = 0; it < items; ++it) {
    const int s = cs_;
    const int j = cj;
    const bool diag = I == K;
    if (ok) ok = mbar_wait(&sm.full[s], parity, status);
    if (!ok) break;  // the producer gives up on its own bounded wait
    const float* tA = reinterpret_cast<const float*>(base + s * Cfg::STAGE);
    const float* tB = diag ? tA : tA + PL * (KH_TILE / 4);
    const int no = diag ? 1 : 2;
    if (j <= L) {
      const float c = sm.cpos[j], cm = sm.cneg[j];
      for (int o = 0; o < no; ++o) {
        // o = 0: Q[I,K] from D = M[I,K] and T = M[K,I] read transposed; o = 1: Q[K,I] from B and A
        const float* tD = o ? tB : tA;
        const float* tT = o ? tA : tB;
        float d[8][2], t[8][2];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            d[r][h] = tD[offD[r][h]];
            t[r][h] = tT[offT[r][h]];  // c_{-l} = 0 only for l = 0: the read is cheaper than a branch
          }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float& a = o ? re[1][r][h] : re[0][r][h];
            a = fmaf(c, d[r][h], fmaf(cm, t[r][h], a));
          }
        if (CPLX) {  // imaginary planes; the transposed term is conjugated
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              d[r][h] = tD[KH_TILE / 4 + offD[r][h]];
              t[r][h] = tT[KH_TILE / 4 + offT[r][h]];
            }
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float& a = o ? im[1][r][h] : im[0][r][h];
              a = fmaf(c, d[r][h], fmaf(-cm, t[r][h], a));
            }
        }
      }
    } else {  // P with e^{j pi a} = cr + j ci
      const float cr = sm.cp.x, ci = sm.cp.y;
      for (int o = 0; o < no; ++o) {
        const float* tD = o ? tB : tA;
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float dr = tD[offD[r][h]];
            const float di = CPLX ? tD[KH_TILE / 4 + offD[r][h]] : 0.f;
            float& a = o ? re[1][r][h] : re[0][r][h];
            float& b = o ? im[1][r][h] : im[0][r][h];
            a += cr * dr - ci * di;
            b += cr * di + ci * dr;
          }
      }
    }
    __syncwarp();  // the warp is done with slot s
    if (lane == 0) mbar_arrive(&sm.empty[s]);
    if (++cs_ == Cfg::STAGES) {
      cs_ = 0;
      parity ^= 1u;
    }
    if (j == nbi - 1) {
      // the pair is complete: write Q[I,K] and Q[K,I]
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        if (o == 1 && diag) continue;
        const int64_t R0 = (int64_t)(o ? K : I) * KH_T, C0 = (int64_t)(o ? I : K) * KH_T;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t row = R0 + 8 * warp + r;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int64_t col = C0 + lane + 32 * h;
            if (row < N && col < N) {
              if (!SPLIT) {
                Q[row * N + col] = make_float2(re[o][r][h], im[o][r][h]);
              } else {
                // Qs planes (pitch Np, scaled by 2^FG_SPLIT_SHIFT)
                const float sc = (float)(1 << FG_SPLIT_SHIFT);
                const float x = re[o][r][h] * sc, y = im[o][r][h] * sc;
                const __half2 hi = __floats2half2_rn(x, y);
                const float2 hf = __half22float2(hi);
                const __half2 lo = __floats2half2_rn(x - hf.x, y - hf.y);
                __half* qq = Qs + row * Np + col;
                qq[0] = __low2half(hi);
                qq[q_plane] = __low2half(lo);
                if (write_im) {
                  qq[2 * q_plane] = __high2half(hi);
                  qq[3 * q_plane] = __high2half(lo);
                }
              }
            }
            re[o][r][h] = im[o][r][h] = 0.f;
          }
        }
      }
      cj = 0;
      cpr += gridDim.x;
      if (cpr < npairs) kh_pair(cpr, nt, I, K);
    } else {
      ++cj;
    }
  }
}

}  // namespace

cudaError_t fg_assemble_single(const float2* stack, int64_t blk_elems, int b0, int nb_pow, int p_blk, int64_t NN,
                               const float2* coef, float2* Q, uint32_t* status, cudaStream_t s, __half* Qs,
                               int64_t N, int64_t Np, int64_t plane_elems) {
  const int nblk = nb_pow + (p_blk >= 0 ? 1 : 0);
  if (nblk > K1_MAXBLK) return cudaErrorInvalidValue;
  const size_t smem = sizeof(K1Smem);
  auto kern = Qs ? assemble_single_kernel<true> : assemble_single_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K1_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (NN + K1_CHUNK - 1) / K1_CHUNK;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > ntiles) grid = ntiles;
  FgTimed timed(FGFRFT_KC_ASSEMBLE_SINGLE, s);
  kern<<<(unsigned)grid, K1_THREADS, smem, s>>>(stack, blk_elems, b0, nb_pow, p_blk, NN, coef, Q, Qs, N, Np,
                                                plane_elems, status);
  fg_note_launch(FGFRFT_KC_ASSEMBLE_SINGLE);
  return cudaGetLastError();
}

cudaError_t fg_assemble_multi(const float2* stack, int64_t blk_elems, int b0, int nb_pow, int p_blk, int64_t N,
                              int A, const float2* coef, float2* Qc, __half* Qs, int64_t Np, int64_t plane_elems,
                              uint32_t* status, cudaStream_t s) {
  FgTimed timed(FGFRFT_KC_ASSEMBLE_MULTI, s);
  // passes of at most 4 order groups of 32 (one pass over the stack per 128 orders)
  constexpr int kPass = 4 * K2_AC;
  for (int a0 = 0; a0 < A; a0 += kPass) {
    const int na = (A - a0) < kPass ? (A - a0) : kPass;
    const int n_og = (na + K2_AC - 1) / K2_AC;
    cudaError_t e = Qs != nullptr ? launch_multi<true>(stack, blk_elems, b0, nb_pow, p_blk, N, A, a0, n_og, coef, Qc,
                                                       Qs, Np, plane_elems, status, s)
                                  : launch_multi<false>(stack, blk_elems, b0, nb_pow, p_blk, N, A, a0, n_og, coef, Qc,
                                                        Qs, Np, plane_elems, status, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t fg_assemble_single_real(const __half* planes, int64_t blk_stride, int64_t plane_elems, int b0,
                                    int nb_pow, int p_blk, int64_t N, int64_t Np, const float2* coef, float2* Q,
                                    __half* Qs, int64_t q_plane, bool write_im, uint32_t* status, cudaStream_t s) {
  const int nblk = nb_pow + (p_blk >= 0 ? 1 : 0);
  if (nblk > K1_MAXBLK) return cudaErrorInvalidValue;
  const size_t smem = sizeof(KRSmem);
  auto kern = Qs ? assemble_single_real_kernel<true> : assemble_single_real_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K1_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (N * Np + KR_CHUNK - 1) / KR_CHUNK;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > ntiles) grid = ntiles;
  FgTimed timed(FGFRFT_KC_ASSEMBLE_SINGLE, s);
  kern<<<(unsigned)grid, K1_THREADS, smem, s>>>(planes, blk_stride, plane_elems, b0, nb_pow, p_blk, N, Np, coef, Q, Qs,
                                                q_plane, write_im ? 1 : 0, status);
  fg_note_launch(FGFRFT_KC_ASSEMBLE_SINGLE);
  return cudaGetLastError();
}

cudaError_t fg_assemble_half(const float* planes, int64_t hplane, int nt, int L_max, int L, bool cplx, bool has_p,
                             int64_t N, int64_t Np, const float2* coef, float2* Q, __half* Qs, int64_t q_plane,
                             bool write_im, uint32_t* status, cudaStream_t s) {
  if (L + 1 > K1_MAXBLK || L > L_max || N < 1 || nt < 1 || (int64_t)nt * KH_T < N) return cudaErrorInvalidValue;
  const int64_t npairs = (int64_t)nt * (nt + 1) / 2;
  const int blk_P = L_max + 1;
  auto pick = [&](auto kern, size_t smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(npairs, num_sms());
    FgTimed timed(FGFRFT_KC_ASSEMBLE_SINGLE, s);
    kern<<<(unsigned)grid, KH_THREADS, smem, s>>>(planes, hplane, nt, L, blk_P, has_p ? 1 : 0, coef, N, Q, Qs, Np,
                                                  q_plane, write_im ? 1 : 0, status);
    fg_note_launch(FGFRFT_KC_ASSEMBLE_SINGLE);
    return cudaGetLastError();
  };
  if (cplx) {
    const size_t smem = KHCfg<true>::STAGES * KHCfg<true>::STAGE + sizeof(KHCtl) + 1024;
    return Qs ? pick(assemble_half_kernel<true, true>, smem) : pick(assemble_half_kernel<true, false>, smem);
  }
  const size_t smem = KHCfg<false>::STAGES * KHCfg<false>::STAGE + sizeof(KHCtl) + 1024;
  return Qs ? pick(assemble_half_kernel<false, true>, smem) : pick(assemble_half_kernel<false, false>, smem);
}
