// Offline part of Algorithm 1 in FP64 on the GPU: complex GEMM, the lambda = -1
// projector iteration helpers, and the rounding of FP64 blocks into the stored
// c64 / split-fp16 formats.  Not on the timed online path.
#include "internal.h"

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// C[M x N] = alpha * op(A) op(B) + beta * C, row-major complex128.
// op(A)[i][k] = A[i][k] or conj(A[k][i]); op(B)[k][j] = B[k][j] or conj(B[j][k]).
// 64 x 64 output tile per 256-thread block, 4 x 4 entries per thread, k step 16.
// REAL: A and B have zero imaginary parts and alpha, beta are real; only the real
// products are formed (a quarter of the FP64 work) and C gets zero imaginary parts.
// The real parts are the same FP64 values the complex kernel produces (its extra
// terms are exact zeros).
constexpr int ZBM = 64, ZBN = 64, ZBK = 16;

template <bool TA, bool TB, bool REAL>
__global__ void __launch_bounds__(256) zgemm_kernel(int M, int N, int K, double2 alpha, const double2* __restrict__ A,
                                                    int lda, const double2* __restrict__ B, int ldb, double2 beta,
                                                    double2* __restrict__ C, int ldc) {
  __shared__ double2 As[ZBK][ZBM + 1];
  __shared__ double2 Bs[ZBK][ZBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * ZBM, j0 = blockIdx.x * ZBN;
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < K; k0 += ZBK) {
    // 1024 entries of each tile, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + e * 256;
      // A tile: op(A)[i0 + ii][k0 + kk]
      {
        int ii, kk;
        if (!TA) { kk = idx & 15; ii = idx >> 4; } else { ii = idx & 63; kk = idx >> 6; }
        const int gi = i0 + ii, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gi < M && gk < K) v = TA ? zconj(A[(int64_t)gk * lda + gi]) : A[(int64_t)gi * lda + gk];
        As[kk][ii] = v;
      }
      // B tile: op(B)[k0 + kk][j0 + jj]
      {
        int jj, kk;
        if (!TB) { jj = idx & 63; kk = idx >> 6; } else { kk = idx & 15; jj = idx >> 4; }
        const int gj = j0 + jj, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gj < N && gk < K) v = TB ? zconj(B[(int64_t)gj * ldb + gk]) : B[(int64_t)gk * ldb + gj];
        Bs[kk][jj] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < ZBK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[r][c].x = fma(a[r].x, b[c].x, acc[r][c].x);
          if (REAL) continue;
          acc[r][c].x = fma(-a[r].y, b[c].y, acc[r][c].x);
          acc[r][c].y = fma(a[r].x, b[c].y, acc[r][c].y);
          acc[r][c].y = fma(a[r].y, b[c].x, acc[r][c].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < M && gj < N) {
        double2* dst = C + (int64_t)gi * ldc + gj;
        if (REAL) {
          double v = alpha.x * acc[r][c].x;
          if (beta.x != 0.0) v += beta.x * dst->x;
          *dst = make_double2(v, 0.0);
          continue;
        }
        double2 v = zmul(alpha, acc[r][c]);
        if (beta.x != 0.0 || beta.y != 0.0) {
          const double2 o = zmul(beta, *dst);
          v.x += o.x;
          v.y += o.y;
        }
        *dst = v;
      }
    }
}

// Y = a X + b Y + d I   (X may equal NULL, meaning 0)
__global__ void zaxpby_identity_kernel(int64_t N, double2 a, const double2* __restrict__ X, double2 b, double2 d,
                                       double2* __restrict__ Y) {
  const int64_t total = N * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (X) v = zmul(a, X[t]);
    if (b.x != 0.0 || b.y != 0.0) {
      const double2 o = zmul(b, Y[t]);
      v.x += o.x;
      v.y += o.y;
    }
    if (t / N == t % N) {
      v.x += d.x;
      v.y += d.y;
    }
    Y[t] = v;
  }
}

// S <- (S + S^H)/2, one thread per pair (i <= j)
__global__ void zherm_sym_kernel(int64_t N, double2* S) {
  const int64_t total = N * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / N, j = t % N;
    if (i > j) continue;
    const double2 a = S[i * N + j], b = S[j * N + i];
    const double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    S[i * N + j] = m;
    S[j * N + i] = zconj(m);
  }
}

// P <- 3 P2 - 2 P3
__global__ void zmcweeny_kernel(int64_t total, const double2* __restrict__ P2, const double2* __restrict__ P3,
                                double2* __restrict__ P) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    P[t] = make_double2(3.0 * P2[t].x - 2.0 * P3[t].x, 3.0 * P2[t].y - 2.0 * P3[t].y);
  }
}

// out[0] = Re tr(S); out[1] = ||S - Sub||_F^2 (Sub may be NULL); out[2] = Im tr(S).
// One block, fixed reduction order (deterministic).
__global__ void __launch_bounds__(1024) ztrace_fro_kernel(int64_t N, const double2* __restrict__ S,
                                                          const double2* __restrict__ Sub, double* out) {
  __shared__ double red[3][32];
  double tr = 0.0, tri = 0.0, fro = 0.0;
  const int64_t total = N * N;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    double2 v = S[t];
    if (t / N == t % N) {
      tr += v.x;
      tri += v.y;
    }
    if (Sub) {
      v.x -= Sub[t].x;
      v.y -= Sub[t].y;
    }
    fro += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    tri += __shfl_xor_sync(0xffffffffu, tri, o);
    fro += __shfl_xor_sync(0xffffffffu, fro, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = tr;
    red[1][w] = fro;
    red[2][w] = tri;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    tr = lane < nw ? red[0][lane] : 0.0;
    fro = lane < nw ? red[1][lane] : 0.0;
    tri = lane < nw ? red[2][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
      fro += __shfl_xor_sync(0xffffffffu, fro, o);
      tri += __shfl_xor_sync(0xffffffffu, tri, o);
    }
    if (lane == 0) {
      out[0] = tr;
      out[1] = fro;
      out[2] = tri;
    }
  }
}

// Round one FP64 block (optionally conjugate-transposed) into the stored formats.
// c64: float2 [N*N]; f16: 4 planes of N rows x Np, plane stride plane_elems,
// hi = fp16(v * 2^s), lo = fp16(v * 2^s - hi), s = FG_SPLIT_SHIFT.
__global__ void __launch_bounds__(256) store_block_kernel(int64_t N, const double2* __restrict__ M, int conjT,
                                                          float2* __restrict__ c64, __half* __restrict__ f16,
                                                          int64_t Np, int64_t plane_elems) {
  __shared__ double2 tile[32][33];
  const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  // load tile of the source: rows (conjT ? bj : bi), cols (conjT ? bi : bj)
  const int64_t sr0 = conjT ? bj : bi, sc0 = conjT ? bi : bj;
  for (int r = ty; r < 32; r += 8) {
    const int64_t sr = sr0 + r, sc = sc0 + tx;
    tile[r][tx] = (sr < N && sc < N) ? M[sr * N + sc] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const double scale = (double)(1 << FG_SPLIT_SHIFT);
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bi + r, j = bj + tx;
    if (i >= N || j >= N) continue;
    const double2 v = conjT ? zconj(tile[tx][r]) : tile[r][tx];
    if (c64) c64[i * N + j] = make_float2((float)v.x, (float)v.y);
    if (f16) {
      const double re = v.x * scale, im = v.y * scale;
      const __half rh = __double2half(re), ih = __double2half(im);
      const __half rl = __double2half(re - (double)__half2float(rh));
      const __half il = __double2half(im - (double)__half2float(ih));
      const int64_t o = i * Np + j;
      f16[o] = rh;
      f16[plane_elems + o] = rl;
      f16[2 * plane_elems + o] = ih;
      f16[3 * plane_elems + o] = il;
    }
  }
}

// Half-stack block in FP32 64 x 64 tiles: planes re, im of [nt x nt tiles][64][64], tiles in
// row-major order, element (r, c) of a tile at r * 64 + (c ^ (r & 31)) so that a warp reading
// one row or one column of a tile hits 32 different banks.  Entries past N are zero.
__global__ void __launch_bounds__(256) store_half_kernel(int64_t N, const double2* __restrict__ M, int nt,
                                                         float* __restrict__ planes, int64_t hplane) {
  const int ti = blockIdx.y, tk = blockIdx.x;
  float* re = planes + ((int64_t)ti * nt + tk) * 4096;
  float* im = re + hplane;
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    const int64_t i = (int64_t)ti * 64 + r, k = (int64_t)tk * 64 + c;
    const double2 v = (i < N && k < N) ? M[i * N + k] : make_double2(0.0, 0.0);
    const int o = r * 64 + (c ^ (r & 31));
    re[o] = (float)v.x;
    im[o] = (float)v.y;
  }
}

// Entry-major copy of the split stack: entry e = i * N + k of block b < nblk of plane p
// is F16[b][p][e / N][e % N], stored at the chunk-major position fg_entry_major describes.
// 32 entries x 32 blocks per tile, staged in shared memory so both the reads (along
// entries) and the writes (along blocks) are contiguous.
__global__ void __launch_bounds__(256) entry_major_kernel(const __half* __restrict__ f16, int nblk, int64_t N,
                                                          int64_t Np, int64_t plane_elems, __half* __restrict__ T,
                                                          int64_t Kp, int64_t planeT) {
  __shared__ __half tile[32][33];
  const int64_t e0 = (int64_t)blockIdx.x * 32;
  const int b0 = blockIdx.y * 32;
  const int p = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t NN = N * N;
  for (int r = ty; r < 32; r += 8) {  // r: block offset, tx: entry offset
    const int b = b0 + r;
    const int64_t e = e0 + tx;
    __half v = __float2half(0.f);
    if (b < nblk && e < NN) {
      const int64_t i = e / N, k = e - (e / N) * N;
      v = f16[(int64_t)b * 4 * plane_elems + (int64_t)p * plane_elems + i * Np + k];
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {  // r: entry offset, tx: block offset
    const int64_t e = e0 + r;
    const int b = b0 + tx;
    if (e < NN && b < Kp) {
      const int64_t nfull = Kp / 32, wtail = Kp % 32;
      const int64_t c = b / 32;
      const int64_t at = c < nfull ? ((p * nfull + c) * planeT + e) * 32 + (b & 31)
                                   : 4 * nfull * planeT * 32 + (p * planeT + e) * wtail + (b & 31);
      T[at] = tile[tx][r];
    }
  }
}

// Pair stack (fg_pair_stack): 32 rows of one pair tile x 32 columns per CTA, transposed in
// shared memory so the reads (along k of one row of M_l) and the writes (along the columns of
// one pair row) are both contiguous.
__global__ void __launch_bounds__(256) pair_stack_kernel(const __half* __restrict__ f16, int L_max, int nbt,
                                                         int64_t Np, int64_t plane_elems, __half* __restrict__ PS,
                                                         int64_t R) {
  __shared__ __half tile[32][33];
  const int64_t rho0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int p = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int i = 0, kt = 0;
  pair_tile(rho0 / 128, nbt, i, kt);
  const int64_t k0 = 128 * (int64_t)kt + rho0 % 128;
  for (int r = ty; r < 32; r += 8) {  // r: column offset, tx: row offset
    const int c = c0 + r;
    const int l = c < L_max ? c - L_max : c - L_max + 1;
    const int64_t blk = L_max + l;
    tile[r][tx] = f16[blk * 4 * plane_elems + (int64_t)p * plane_elems + (int64_t)i * Np + k0 + tx];
  }
  __syncthreads();
  // tile t's image: [chunk][plane][128 rows x 32 halves], each row's 16-byte pieces placed as
  // the 64-byte swizzle puts them in shared memory (piece j of row r at j ^ ((r >> 1) & 3))
  const int nch = L_max / 16;  // K2 / 32
  const int64_t t = rho0 / 128;
  __half* img = PS + ((t * nch + blockIdx.y) * 2 + p) * (128 * 32);
  for (int r = ty; r < 32; r += 8) {  // r: row offset, tx: column offset
    const int rr = (int)(rho0 % 128) + r;
    img[rr * 32 + (tx ^ (((rr >> 1) & 3) << 3))] = tile[tx][r];
  }
}

// out[0] = sum of Im(F_ik)^2 (one block, fixed order): zero iff F is real.
__global__ void __launch_bounds__(1024) zimag_sq_kernel(int64_t total, const double2* __restrict__ F, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) acc += F[t].y * F[t].y;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[0] = s;
  }
}

inline int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <bool REAL>
void zgemm_launch(bool transA, bool transB, dim3 grid, int M, int N, int K, double2 alpha, const double2* A, int lda,
                  const double2* B, int ldb, double2 beta, double2* C, int ldc, cudaStream_t s) {
  if (!transA && !transB)
    zgemm_kernel<false, false, REAL><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (transA && !transB)
    zgemm_kernel<true, false, REAL><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!transA && transB)
    zgemm_kernel<false, true, REAL><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else
    zgemm_kernel<true, true, REAL><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

cudaError_t fg_zgemm(bool transA, bool transB, int M, int N, int K, double2 alpha, const double2* A, int lda,
                     const double2* B, int ldb, double2 beta, double2* C, int ldc, cudaStream_t s, bool real) {
  if (real && (alpha.y != 0.0 || beta.y != 0.0)) return cudaErrorInvalidValue;
  dim3 grid((N + ZBN - 1) / ZBN, (M + ZBM - 1) / ZBM);
  if (real)
    zgemm_launch<true>(transA, transB, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  else
    zgemm_launch<false>(transA, transB, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_zaxpby_identity(int64_t N, double2 a, const double2* X, double2 b, double2 d, double2* Y,
                               cudaStream_t s) {
  zaxpby_identity_kernel<<<grid_for(N * N), 256, 0, s>>>(N, a, X, b, d, Y);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_zherm_sym(int64_t N, double2* S, cudaStream_t s) {
  zherm_sym_kernel<<<grid_for(N * N), 256, 0, s>>>(N, S);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_zmcweeny(int64_t N, const double2* P2, const double2* P3, double2* P, cudaStream_t s) {
  zmcweeny_kernel<<<grid_for(N * N), 256, 0, s>>>(N * N, P2, P3, P);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_ztrace_fro(int64_t N, const double2* S, const double2* Sub, double* out, cudaStream_t s) {
  ztrace_fro_kernel<<<1, 1024, 0, s>>>(N, S, Sub, out);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_store_block(int64_t N, const double2* M, bool conj_transpose, float2* c64, __half* f16, int64_t Np,
                           int64_t plane_elems, cudaStream_t s) {
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((N + 31) / 32));
  store_block_kernel<<<grid, 256, 0, s>>>(N, M, conj_transpose ? 1 : 0, c64, f16, Np, plane_elems);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_store_half(int64_t N, const double2* M, float* planes, int nt, int64_t hplane, cudaStream_t s) {
  dim3 grid((unsigned)nt, (unsigned)nt);
  store_half_kernel<<<grid, 256, 0, s>>>(N, M, nt, planes, hplane);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_pair_stack(const __half* f16, int L_max, int64_t N, int64_t Np, int64_t plane_elems, __half* PS,
                          int64_t R, cudaStream_t s) {
  if (N % 128 || L_max % 16 || L_max < 16 || R != pair_tiles((int)(N / 128)) * 128) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(R / 32), (unsigned)(L_max / 16), 2);
  pair_stack_kernel<<<grid, 256, 0, s>>>(f16, L_max, (int)(N / 128), Np, plane_elems, PS, R);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_entry_major(const __half* f16, int nblk, int64_t N, int64_t Np, int64_t plane_elems, __half* T,
                           int64_t Kp, int64_t planeT, cudaStream_t s) {
  dim3 grid((unsigned)((N * N + 31) / 32), (unsigned)((Kp + 31) / 32), 4);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  entry_major_kernel<<<grid, 256, 0, s>>>(f16, nblk, N, Np, plane_elems, T, Kp, planeT);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}

cudaError_t fg_zimag_sq(int64_t N, const double2* F, double* out, cudaStream_t s) {
  zimag_sq_kernel<<<1, 1024, 0, s>>>(N * N, F, out);
  fg_note_launch(FGFRFT_KC_OFFLINE);
  return cudaGetLastError();
}
