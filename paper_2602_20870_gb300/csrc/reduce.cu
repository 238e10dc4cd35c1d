// Small kernels around the GEMMs:
//  - per-column transform coefficients (Sec. III-A, Prop. 3) in FP64 on the device,
//  - the alpha-gradient reduction g_j = Re sum_i conj(G_ij) D_ij (chain rule on Prop. 3),
//  - the fp16 hi/lo split of signal columns for the tensor-core paths.
#include "internal.h"

namespace {

// d/du (sin u / u) by its Taylor series sum_{k>=1} (-1)^k 2k u^{2k-1} / (2k+1)!
__device__ double dsinc_series(double u) {
  const double u2 = u * u;
  double term = -u / 3.0;  // k = 1
  double sum = term;
  for (int k = 2; k <= 6; ++k) {
    // ratio of consecutive terms: -u^2 * (2k) / ((2k-2) * (2k) * (2k+1))
    term *= -u2 * (double)(2 * k) / ((double)(2 * k - 2) * (double)(2 * k) * (double)(2 * k + 1));
    sum += term;
  }
  return sum;
}

// coef[b][j] (and coefd[b][j]) for blocks b = 0..2L (power l = b - L) and b = 2L+1 (P):
//   powers: c_l(a) = sin(pi (a - l)) / (pi (a - l)), c_l'(a);  P: e^{j pi a}, j pi e^{j pi a}.
// sign = -1 evaluates at -a (the adjoint, Prop. 2).
// Entry (b, j) is stored at b * ldb + j * ldj.
// Block b is stored at position b + pos_off for the powers and at p_pos for P.
__global__ void coeffs_kernel(const double* __restrict__ alpha, int B, int L, double sign,
                              float2* __restrict__ coef, float2* __restrict__ coefd, int64_t ldb, int64_t ldj,
                              int pos_off, int p_pos) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (j >= B) return;
  const double a = sign * alpha[j];
  const double pi = 3.14159265358979323846;
  const double sa = sinpi(a), ca = cospi(a);
  float2 c, cd;
  if (b == 2 * L + 1) {
    c = make_float2((float)ca, (float)sa);
    cd = make_float2((float)(-pi * sa), (float)(pi * ca));
  } else {
    const int l = b - L;
    const double d = a - (double)l;
    double v, dv;
    if (d == 0.0) {
      v = 1.0;
      dv = 0.0;
    } else {
      // sin(pi (a - l)) = (-1)^l sin(pi a), cos(pi (a - l)) = (-1)^l cos(pi a)
      const double sgn = (l & 1) ? -1.0 : 1.0;
      v = sgn * sa / (pi * d);
      if (fabs(d) < 1e-2)
        dv = pi * dsinc_series(pi * d);
      else
        dv = sgn * (pi * d * ca - sa) / (pi * d * d);
    }
    c = make_float2((float)v, 0.f);
    cd = make_float2((float)dv, 0.f);
  }
  const int64_t pos = b == 2 * L + 1 ? p_pos : b + pos_off;
  coef[pos * ldb + (int64_t)j * ldj] = c;
  if (coefd) coefd[pos * ldb + (int64_t)j * ldj] = cd;
}

constexpr int GR_CHUNK = 4096;

// level 1: partial[j][chunk] = Re sum_{i in chunk} conj(G_ji) D_ji   (FP64)
__global__ void __launch_bounds__(256) grad_partial_kernel(const float2* __restrict__ G,
                                                           const float2* __restrict__ D, int64_t N, int nchunks,
                                                           double* __restrict__ partial, float* __restrict__ out) {
  const int64_t j = blockIdx.y;
  const int ch = blockIdx.x;
  const int64_t i0 = (int64_t)ch * GR_CHUNK;
  const int64_t i1 = (i0 + GR_CHUNK) < N ? (i0 + GR_CHUNK) : N;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float2 g = G[j * N + i], d = D[j * N + i];
    acc += (double)g.x * (double)d.x + (double)g.y * (double)d.y;
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    if (nchunks == 1)
      out[j] = (float)s;
    else
      partial[j * nchunks + ch] = s;
  }
}

// level 2: out[j] = sum_c partial[j][c] in a fixed order
__global__ void grad_final_kernel(const double* __restrict__ partial, int nchunks, int64_t B,
                                  float* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= B) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[j * nchunks + c];
  out[j] = (float)s;
}

// One CTA per signal column j: e_j such that max(|re|, |im|) * 2^e_j lies in
// [2^13, 2^14); planes[p][j][k] for p = re_hi, re_lo, im_hi, im_lo of x * 2^e_j.
// Each thread handles 4 consecutive entries per round (8-byte plane stores); entries
// k in [N, Np) are written as zeros.
__global__ void __launch_bounds__(256) split_signals_kernel(const float2* __restrict__ X, int64_t B, int64_t N,
                                                            int64_t Np, int64_t rows_pad, __half* __restrict__ planes,
                                                            int* __restrict__ col_exp) {
  const int64_t j = blockIdx.x;
  const int64_t plane = rows_pad * Np;
  __half* r_hi = planes + j * Np;
  __half* r_lo = r_hi + plane;
  __half* i_hi = r_hi + 2 * plane;
  __half* i_lo = r_hi + 3 * plane;
  const float2* x = X + j * N;
  if (j >= B) {  // padding rows are zero
    for (int64_t k = threadIdx.x; k < Np; k += blockDim.x) {
      r_hi[k] = r_lo[k] = i_hi[k] = i_lo[k] = __float2half(0.f);
    }
    return;
  }
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < N; k += blockDim.x) {
    const float2 v = x[k];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  __shared__ float red[8];
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  int e = 0;
  if (m > 0.f && isfinite(m)) {
    int E;
    frexpf(m, &E);  // m in [2^(E-1), 2^E)
    e = (FG_X_TARGET_EXP + 1) - E;
  }
  if (threadIdx.x == 0) col_exp[j] = e;
  // Np is a multiple of 8, so groups of 4 entries never straddle the row end
  for (int64_t k0 = 4 * (int64_t)threadIdx.x; k0 < Np; k0 += 4 * (int64_t)blockDim.x) {
    __align__(8) __half rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = k0 + u;
      float re = 0.f, im = 0.f;
      if (k < N) {
        const float2 v = x[k];
        re = ldexpf(v.x, e);
        im = ldexpf(v.y, e);
      }
      const __half2 hi = __floats2half2_rn(re, im);
      const float2 hf = __half22float2(hi);
      const __half2 lo = __floats2half2_rn(re - hf.x, im - hf.y);
      rh[u] = __low2half(hi);
      ih[u] = __high2half(hi);
      rl[u] = __low2half(lo);
      il[u] = __high2half(lo);
    }
    *reinterpret_cast<uint2*>(r_hi + k0) = *reinterpret_cast<const uint2*>(rh);
    *reinterpret_cast<uint2*>(r_lo + k0) = *reinterpret_cast<const uint2*>(rl);
    *reinterpret_cast<uint2*>(i_hi + k0) = *reinterpret_cast<const uint2*>(ih);
    *reinterpret_cast<uint2*>(i_lo + k0) = *reinterpret_cast<const uint2*>(il);
  }
}

}  // namespace

cudaError_t fg_coeffs(const double* alpha, int B, int L, bool adjoint, float2* coef, float2* coefd, int64_t ldb,
                      int64_t ldj, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  dim3 grid((B + 127) / 128, 2 * L + 2);
  FgTimed timed(FGFRFT_KC_COEFFS, s);
  fg_note_launch(FGFRFT_KC_COEFFS);
  coeffs_kernel<<<grid, 128, 0, s>>>(alpha, B, L, adjoint ? -1.0 : 1.0, coef, coefd, ldb, ldj, 0, 2 * L + 1);
  return cudaGetLastError();
}

cudaError_t fg_coeffs_stored(const double* alpha, int B, int L, int L_max, bool adjoint, float2* coef, int64_t ldb,
                             int64_t ldj, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  dim3 grid((B + 127) / 128, 2 * L + 2);
  FgTimed timed(FGFRFT_KC_COEFFS, s);
  fg_note_launch(FGFRFT_KC_COEFFS);
  coeffs_kernel<<<grid, 128, 0, s>>>(alpha, B, L, adjoint ? -1.0 : 1.0, coef, nullptr, ldb, ldj, L_max - L,
                                     2 * L_max + 1);
  return cudaGetLastError();
}

int fg_grad_chunks(int64_t N) { return (int)((N + GR_CHUNK - 1) / GR_CHUNK); }

cudaError_t fg_grad_alpha(const float2* G, const float2* D, int64_t B, int64_t N, float* out, double* partials,
                          cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int nch = fg_grad_chunks(N);
  if (B > 65535) return cudaErrorInvalidValue;
  dim3 grid(nch, (unsigned)B);
  FgTimed timed(FGFRFT_KC_GRAD_REDUCE, s);
  fg_note_launch(FGFRFT_KC_GRAD_REDUCE, nch == 1 ? 1 : 2);
  grad_partial_kernel<<<grid, 256, 0, s>>>(G, D, N, nch, partials, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nch == 1) return e;
  grad_final_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(partials, nch, B, out);
  return cudaGetLastError();
}

cudaError_t fg_split_signals(const float2* X, int64_t B, int64_t N, int64_t Np, int64_t rows_pad, __half* planes,
                             int* col_exp, cudaStream_t s) {
  if (rows_pad <= 0) return cudaSuccess;
  FgTimed timed(FGFRFT_KC_SPLIT_SIGNALS, s);
  fg_note_launch(FGFRFT_KC_SPLIT_SIGNALS);
  split_signals_kernel<<<(unsigned)rows_pad, 256, 0, s>>>(X, B, N, Np, rows_pad, planes, col_exp);
  return cudaGetLastError();
}
