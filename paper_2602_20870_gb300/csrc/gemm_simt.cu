// FP32 CUDA-core complex GEMM over stacked blocks (the "plain" path and the FP32
// stacked path):
//   T_b[i][j] = sum_k A_b[i][k] X[j][k]                     (Def. 2: x~ = Q x)
//   Y[j][i]  = sum_b coef[b][j] T_b[i][j]                     (Def. 1 per column)
//   D[j][i]  = sum_b coefd[b][j] T_b[i][j]                    (Prop. 3, dual)
// With coef == NULL there is one block and Y = T (an assembled Q times X).
// 64 x 64 output tile per 256-thread CTA, 4 x 4 complex entries per thread.
#include "internal.h"

namespace {

constexpr int SBM = 64, SBN = 64, SBK = 16;

template <bool SCALED, bool DUAL>
__global__ void __launch_bounds__(256) simt_stacked_kernel(SimtStackArgs a) {
  __shared__ float2 As[SBK][SBM + 1];
  __shared__ float2 Bs[SBK][SBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // tx -> rows i (coalesced output), ty -> columns j
  const int i0 = blockIdx.x * SBM, j0 = blockIdx.y * SBN;
  const int N = a.N;
  const int nblk = SCALED ? a.nb_pow + (a.p_blk >= 0 ? 1 : 0) : 1;

  float2 T[4][4], Yc[4][4], Dc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Yc[r][c] = make_float2(0.f, 0.f);
      if (DUAL) Dc[r][c] = make_float2(0.f, 0.f);
    }

  for (int b = 0; b < nblk; ++b) {
    const int blk = (!SCALED || b < a.nb_pow) ? a.b0 + b : a.p_blk;
    const float2* __restrict__ Ab = a.A + (int64_t)blk * a.blk_elems;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) T[r][c] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < N; k0 += SBK) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = tid + e * 256;
        const int kk = idx & 15, rr = idx >> 4;  // 16 consecutive k per row segment
        const int gk = k0 + kk;
        {
          const int gi = i0 + rr;
          As[kk][rr] = (gi < N && gk < N) ? Ab[(int64_t)gi * a.lda + gk] : make_float2(0.f, 0.f);
        }
        {
          const int gj = j0 + rr;
          Bs[kk][rr] = (gj < a.ncols && gk < N) ? a.X[(int64_t)gj * N + gk] : make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < SBK; ++kk) {
        float2 av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = As[kk][tx + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][ty + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) cmac(T[r][c], av[r], bv[c]);
      }
      __syncthreads();
    }
    // fold this block into the per-column combinations
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + ty + 16 * c;
      if (SCALED) {
        float2 cf = make_float2(0.f, 0.f), cd = make_float2(0.f, 0.f);
        if (gj < a.ncols) {
          cf = a.coef[(int64_t)b * a.ldcoef + gj];
          if (DUAL) cd = a.coefd[(int64_t)b * a.ldcoef + gj];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          cmac(Yc[r][c], cf, T[r][c]);
          if (DUAL) cmac(Dc[r][c], cd, T[r][c]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) Yc[r][c] = T[r][c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gj = j0 + ty + 16 * c;
    if (gj >= a.ncols) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int gi = i0 + tx + 16 * r;
      if (gi < N) {
        if (a.Y) a.Y[(int64_t)gj * N + gi] = Yc[r][c];
        if (DUAL) a.D[(int64_t)gj * N + gi] = Dc[r][c];
      }
    }
  }
}

// Plain Y = A X (one block, no coefficients): 128 x 64 output tile, 8 x 4 complex per thread
// (rows strided by 16 so that a warp's stores along i are contiguous), the next k-tile
// prefetched into registers while the current one is multiplied from shared memory.
constexpr int PBM = 128, PBN = 64, PBK = 16;

__global__ void __launch_bounds__(256) cgemm_plain_kernel(SimtStackArgs a) {
  __shared__ float2 As[PBK][PBM + 1];
  __shared__ float2 Bs[PBK][PBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * PBM, j0 = blockIdx.y * PBN;
  const int N = a.N;
  const float2* __restrict__ A = a.A;
  if (a.groups) {  // batched over column groups: this CTA's group
    const int2 gr = a.groups[blockIdx.z];
    if (j0 >= gr.y) return;
    A += (int64_t)blockIdx.z * a.group_stride;
    a.X += (int64_t)gr.x * N;
    a.Y += (int64_t)gr.x * N;
    a.ncols = gr.y;
  }
  float2 acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
  float2 ra[8], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int idx = tid + e * 256;
      const int kk = idx & 15, rr = idx >> 4;
      const int gi = i0 + rr, gk = k0 + kk;
      ra[e] = (gi < N && gk < N) ? __ldg(A + (int64_t)gi * a.lda + gk) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * 256;
      const int kk = idx & 15, rr = idx >> 4;
      const int gj = j0 + rr, gk = k0 + kk;
      rb[e] = (gj < a.ncols && gk < N) ? __ldg(a.X + (int64_t)gj * N + gk) : make_float2(0.f, 0.f);
    }
  };
  load(0);
  for (int k0 = 0; k0 < N; k0 += PBK) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int idx = tid + e * 256;
      As[idx & 15][idx >> 4] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * 256;
      Bs[idx & 15][idx >> 4] = rb[e];
    }
    __syncthreads();
    if (k0 + PBK < N) load(k0 + PBK);
#pragma unroll
    for (int kk = 0; kk < PBK; ++kk) {
      float2 av[8], bv[4];
#pragma unroll
      for (int r = 0; r < 8; ++r) av[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac(acc[r][c], av[r], bv[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gj = j0 + ty + 16 * c;
    if (gj >= a.ncols) continue;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int gi = i0 + tx + 16 * r;
      if (gi < N) a.Y[(int64_t)gj * N + gi] = acc[r][c];
    }
  }
}

}  // namespace

cudaError_t fg_simt_stacked(const SimtStackArgs& a, cudaStream_t s) {
  if (a.ncols <= 0 || a.N <= 0) return cudaSuccess;
  dim3 grid((a.N + SBM - 1) / SBM, (a.ncols + SBN - 1) / SBN);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  const bool scaled = a.coef != nullptr;
  const bool dual = a.D != nullptr;
  FgTimed timed(FGFRFT_KC_SIMT_GEMM, s);
  fg_note_launch(FGFRFT_KC_SIMT_GEMM);
  if (!scaled) {
    const int cols = a.groups ? a.max_group_cols : a.ncols;
    dim3 pg((a.N + PBM - 1) / PBM, (cols + PBN - 1) / PBN, a.groups ? a.ngroups : 1);
    if (pg.y > 65535 || pg.z > 65535) return cudaErrorInvalidValue;
    cgemm_plain_kernel<<<pg, 256, 0, s>>>(a);
  } else if (!dual)
    simt_stacked_kernel<true, false><<<grid, 256, 0, s>>>(a);
  else
    simt_stacked_kernel<true, true><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
