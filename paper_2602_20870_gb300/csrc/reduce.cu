// Small kernels around the GEMMs:
//  - per-column transform coefficients (Sec. III-A, Prop. 3) in FP64 on the device,
//  - the alpha-gradient reduction g_j = Re sum_i conj(G_ij) D_ij (chain rule on Prop. 3),
//  - the fp16 hi/lo split of signal columns for the tensor-core paths.
#include <algorithm>

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

// Coefficients of one stored block at order a (sa = sin(pi a), ca = cos(pi a)):
//   power l: c_l(a) = sin(pi (a - l)) / (pi (a - l)) and c_l'(a) (real);
//   P (is_p): e^{j pi a} and j pi e^{j pi a}.
__device__ __forceinline__ void block_coef(double a, double sa, double ca, int l, bool is_p, float2& c, float2& cd) {
  const double pi = 3.14159265358979323846;
  if (is_p) {
    c = make_float2((float)ca, (float)sa);
    cd = make_float2((float)(-pi * sa), (float)(pi * ca));
    return;
  }
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

// coef[b][j] (and coefd[b][j]) for blocks b = 0..2L (power l = b - L) and b = 2L+1 (P).
// sign = -1 evaluates at -a (the adjoint, Prop. 2).
// Entry (b, j) is stored at b * ldb + j * ldj.
// Block b is stored at position b + pos_off for the powers and at p_pos for P.
// A CTA covers 32 columns x 8 blocks; sin(pi a) and cos(pi a) are evaluated once per column
// (FP64 is a slow pipe on this part).
__global__ void __launch_bounds__(256) coeffs_kernel(const double* __restrict__ alpha, int B, int L, double sign,
                                                     float2* __restrict__ coef, float2* __restrict__ coefd,
                                                     int64_t ldb, int64_t ldj, int pos_off, int p_pos) {
  __shared__ double s_a[32], s_sa[32], s_ca[32];
  const int jl = threadIdx.x & 31, bl = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + jl;
  if (bl == 0 && j < B) {
    const double a = sign * alpha[j];
    s_a[jl] = a;
    s_sa[jl] = sinpi(a);
    s_ca[jl] = cospi(a);
  }
  __syncthreads();
  const int b = blockIdx.y * 8 + bl;
  if (j >= B || b > 2 * L + 1) return;
  float2 c, cd;
  block_coef(s_a[jl], s_sa[jl], s_ca[jl], b - L, b == 2 * L + 1, c, cd);
  const int64_t pos = b == 2 * L + 1 ? p_pos : b + pos_off;
  coef[pos * ldb + (int64_t)j * ldj] = c;
  if (coefd) coefd[pos * ldb + (int64_t)j * ldj] = cd;
}

// ---------------------------------------------------------------------------------
// fp16 hi/lo split of a column v (one signal, or one order's coefficient vector):
// e such that max(|re|, |im|) * 2^e lies in [2^13, 2^14) (0 for an all-zero column), then
// planes re_hi, re_lo, im_hi, im_lo of v * 2^e with hi = fp16(x), lo = fp16(x - hi).
__device__ __forceinline__ int split_exponent(float m) {
  int e = 0;
  if (m > 0.f && isfinite(m)) {
    int E;
    frexpf(m, &E);  // m in [2^(E-1), 2^E)
    e = (FG_X_TARGET_EXP + 1) - E;
  }
  return e;
}

// Four consecutive entries k0..k0+3 of one column into the four planes (8-byte stores);
// RE_ONLY: the real planes only (the caller knows the imaginary parts are zero and that no
// reader loads the imaginary planes).
template <bool RE_ONLY = false>
__device__ __forceinline__ void split_store4(const float2 (&v)[4], int e, __half* r_hi, int64_t plane,
                                             int64_t k0) {
  __align__(8) __half rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float re = ldexpf(v[u].x, e), im = ldexpf(v[u].y, e);
    const __half2 hi = __floats2half2_rn(re, im);
    const float2 hf = __half22float2(hi);
    const __half2 lo = __floats2half2_rn(re - hf.x, im - hf.y);
    rh[u] = __low2half(hi);
    ih[u] = __high2half(hi);
    rl[u] = __low2half(lo);
    il[u] = __high2half(lo);
  }
  *reinterpret_cast<uint2*>(r_hi + k0) = *reinterpret_cast<const uint2*>(rh);
  *reinterpret_cast<uint2*>(r_hi + plane + k0) = *reinterpret_cast<const uint2*>(rl);
  if (!RE_ONLY) {
    *reinterpret_cast<uint2*>(r_hi + 2 * plane + k0) = *reinterpret_cast<const uint2*>(ih);
    *reinterpret_cast<uint2*>(r_hi + 3 * plane + k0) = *reinterpret_cast<const uint2*>(il);
  }
}

// Block-wide max over 256 threads (every thread gets the result).
__device__ __forceinline__ float block_max256(float m, float* red) {
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  return m;
}

// Split coefficient planes of the fused multi-order assembly, one CTA per order a:
// column a holds, at stored-block position q, c_l(alpha_a) for q = L_max + l with
// |l| <= L, e^{j pi alpha_a} at q = 2 L_max + 1 (P) and zero elsewhere (q < Kp).  Every
// coefficient has modulus at most 1, so all columns share the exponent FG_COEF_EXP
// (values at most 2^14 in fp16).  FP64 is a slow pipe on this part, so it only reduces
// the order exactly, a = n0 + d with n0 = rint(a), |d| <= 1/2, and forms n0 - l; then in FP32
//   sin(pi a) = (-1)^n0 sinpi(d),  cos(pi a) = (-1)^n0 cospi(d),
//   c_l = (-1)^l sin(pi a) / (pi (d + (n0 - l)))   (c_l = 1 at a = l),
// within a few ulp of FP32, below the 22-bit resolution of the hi/lo split it feeds.
constexpr int COEF_PARAM_ORDERS = 64;
struct CoefOrders {  // orders passed by value in the launch parameters
  double a[COEF_PARAM_ORDERS];
};
__global__ void __launch_bounds__(256) coeff_planes_kernel(const double* __restrict__ alpha, const CoefOrders orders,
                                                           int L, int L_max, int64_t A, int64_t Kp,
                                                           __half* __restrict__ planes, int* __restrict__ col_exp) {
  const int64_t a_idx = blockIdx.x;
  const double a = alpha ? alpha[a_idx] : orders.a[a_idx];
  const double n0d = rint(a);
  const float d = (float)(a - n0d);  // exact difference, rounded once
  const float sgn0 = fmod(n0d, 2.0) != 0.0 ? -1.f : 1.f;
  const float sa = sgn0 * sinpif(d), ca = sgn0 * cospif(d);
  const float pi_f = 3.14159265358979323846f;
  if (threadIdx.x == 0) col_exp[a_idx] = FG_COEF_EXP;
  __half* r_hi = planes + a_idx * Kp;
  for (int64_t k0 = 4 * (int64_t)threadIdx.x; k0 < Kp; k0 += 4 * (int64_t)blockDim.x) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t q = k0 + u;
      float2 c = make_float2(0.f, 0.f);
      if (q == 2 * L_max + 1) {
        c = make_float2(ca, sa);
      } else if (q <= 2 * L_max && q >= L_max - L && q <= L_max + L) {
        const int l = (int)(q - L_max);
        const float dl = d + (float)(n0d - (double)l);  // a - l (n0 - l exact in FP64)
        if (dl == 0.f)
          c.x = 1.f;
        else
          c.x = ((l & 1) ? -sa : sa) / (pi_f * dl);
      }
      v[u] = c;
    }
    split_store4(v, FG_COEF_EXP, r_hi, A * Kp, k0);  // Kp is a multiple of 8
  }
}

// Pair assembly coefficients (fg_coeff_planes_pair), one CTA per row b < 128 of the resident
// operator: b = a < A gives order a's c_l, b = 64 + a its mirror coefficients c_{-l}, at column
// c of the pair stack (power l = c - L_max below L_max, c - L_max + 1 from it); the same FP32
// evaluation as coeff_planes_kernel.
__global__ void __launch_bounds__(128) coeff_planes_pair_kernel(const double* __restrict__ alpha,
                                                                const CoefOrders orders, int L, int L_max, int64_t A,
                                                                __half* __restrict__ planes,
                                                                int* __restrict__ col_exp, float* __restrict__ diag) {
  const int b = blockIdx.x;
  const int64_t a_idx = b < 64 ? b : b - 64;
  const bool live = a_idx < A;
  const double a = live ? (alpha ? alpha[a_idx] : orders.a[a_idx]) : 0.0;
  const double n0d = rint(a);
  const float d = (float)(a - n0d);
  const float sgn0 = fmod(n0d, 2.0) != 0.0 ? -1.f : 1.f;
  const float sa = sgn0 * sinpif(d);
  const float pi_f = 3.14159265358979323846f;
  auto coef = [&](int l) -> float {  // c_l(a) for |l| <= L, else 0
    if (l > L || l < -L) return 0.f;
    const float dl = d + (float)(n0d - (double)l);
    return dl == 0.f ? 1.f : ((l & 1) ? -sa : sa) / (pi_f * dl);
  };
  if (threadIdx.x == 0) {
    col_exp[b] = FG_COEF_EXP;
    if (live && b < 64) diag[a_idx] = coef(0) * (float)(1 << (FG_SPLIT_SHIFT + FG_COEF_EXP));
  }
  const int64_t K2 = 2 * (int64_t)L_max;
  __half* r_hi = planes + (int64_t)b * K2;
  for (int64_t k0 = 4 * (int64_t)threadIdx.x; k0 < K2; k0 += 4 * (int64_t)blockDim.x) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = (int)(k0 + u);
      const int l = c < L_max ? c - L_max : c - L_max + 1;
      v[u] = make_float2(live ? coef(b < 64 ? l : -l) : 0.f, 0.f);
    }
    split_store4(v, FG_COEF_EXP, r_hi, 128 * K2, k0);  // K2 is a multiple of 32
  }
}

constexpr int GR_CHUNK = 4096;

// level 1: partial[j][chunk] = Re sum_{i in chunk} conj(G_ji) D_ji   (FP64)
// (one CTA per (signal j = blockIdx.x, chunk = blockIdx.y); with out != NULL and one chunk
// the value goes to out[j] directly)
__global__ void __launch_bounds__(256) grad_partial_kernel(const float2* __restrict__ G,
                                                           const float2* __restrict__ D, int64_t N, int nchunks,
                                                           double* __restrict__ partial, float* __restrict__ out) {
  const int64_t j = blockIdx.x;
  const int ch = blockIdx.y;
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
    if (nchunks == 1 && out)
      out[j] = (float)s;
    else
      partial[j * nchunks + ch] = s;
  }
}

// shared order: out[0] = the sum of all B * nchunks partials, one CTA in a fixed order
// (thread t adds entries t, t + 1024, ...; then a fixed tree), so the result is
// deterministic
__global__ void __launch_bounds__(1024) grad_sum_kernel(const double* __restrict__ partial, int64_t count,
                                                        float* __restrict__ out) {
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) acc += partial[t];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[0] = (float)acc;
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

// One CTA (256 threads) per signal column j: planes[p][j][k] of x_j * 2^{e_j} (see
// split_exponent); entries k in [N, Np) are written as zeros and rows j in [B, rows_pad)
// are all zero.  bimag (may be NULL) is set to 1 when the signal has a nonzero (or NaN)
// imaginary part.
// G > 0: each thread keeps its G groups of 4 consecutive entries in registers between
// the max and the split (one read of the column; needs Np <= 1024 G).  G == 0: any Np,
// the column is read twice.  XR: the signals are real float32 (B x N); the imaginary planes
// are not written (the flag stays 0, so the GEMM reads only the real planes).
template <int G, bool XR>
__global__ void __launch_bounds__(256) split_signals_kernel(const void* __restrict__ Xv, int64_t B, int64_t N,
                                                            int64_t Np, int64_t rows_pad, __half* __restrict__ planes,
                                                            int* __restrict__ col_exp, int* __restrict__ bimag) {
  const int64_t j = blockIdx.x;
  const int64_t plane = rows_pad * Np;
  __half* r_hi = planes + j * Np;
  const float2* x = static_cast<const float2*>(Xv) + j * N;
  const float* xr = static_cast<const float*>(Xv) + j * N;
  auto load = [&](int64_t k) -> float2 { return XR ? make_float2(xr[k], 0.f) : x[k]; };
  if (j >= B) {  // padding rows are zero
    for (int64_t k = threadIdx.x; k < Np; k += blockDim.x) {
      r_hi[k] = r_hi[plane + k] = r_hi[2 * plane + k] = r_hi[3 * plane + k] = __float2half(0.f);
    }
    return;
  }
  __shared__ float red[8];
  float m = 0.f;
  bool im = false;
  if constexpr (G > 0) {
    float2 v[G][4];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t k0 = 4 * ((int64_t)threadIdx.x + (int64_t)g * blockDim.x);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[g][u] = k0 + u < N ? load(k0 + u) : make_float2(0.f, 0.f);
        m = fmaxf(m, fmaxf(fabsf(v[g][u].x), fabsf(v[g][u].y)));
        im |= !(v[g][u].y == 0.f);
      }
    }
    const int any_im = __syncthreads_or(im ? 1 : 0);
    m = block_max256(m, red);
    const int e = split_exponent(m);
    if (threadIdx.x == 0) {
      col_exp[j] = e;
      if (any_im && bimag) *bimag = 1;  // every writer stores the same value
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t k0 = 4 * ((int64_t)threadIdx.x + (int64_t)g * blockDim.x);
      if (k0 < Np) split_store4<XR>(v[g], e, r_hi, plane, k0);  // Np is a multiple of 8
    }
  } else {
    for (int64_t k = threadIdx.x; k < N; k += blockDim.x) {
      const float2 v = load(k);
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      im |= !(v.y == 0.f);
    }
    const int any_im = __syncthreads_or(im ? 1 : 0);
    m = block_max256(m, red);
    const int e = split_exponent(m);
    if (threadIdx.x == 0) {
      col_exp[j] = e;
      if (any_im && bimag) *bimag = 1;
    }
    for (int64_t k0 = 4 * (int64_t)threadIdx.x; k0 < Np; k0 += 4 * (int64_t)blockDim.x) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = k0 + u < N ? load(k0 + u) : make_float2(0.f, 0.f);
      split_store4<XR>(v, e, r_hi, plane, k0);
    }
  }
}

// The same split with one warp per column (Np <= 1024, SPLIT_WARPS columns per CTA): lane l
// holds the groups 4(l + 32g) .. +3, g < 8, so the max needs only warp shuffles and each
// group's plane stores are 8 bytes, 256 contiguous bytes per warp instruction.  Small CTAs
// fit beside a CTA of the operator assembly, which the split runs next to.
constexpr int SPLIT_WARPS = 4;
template <bool XR>
__global__ void __launch_bounds__(32 * SPLIT_WARPS) split_signals_warp_kernel(const void* __restrict__ Xv, int64_t B, int64_t N,
                                                                 int64_t Np, int64_t rows_pad,
                                                                 __half* __restrict__ planes,
                                                                 int* __restrict__ col_exp, int* __restrict__ bimag) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * SPLIT_WARPS + (threadIdx.x >> 5);
  if (j >= rows_pad) return;
  const int64_t plane = rows_pad * Np;
  __half* r_hi = planes + j * Np;
  if (j >= B) {  // padding rows are zero
    for (int64_t k = lane; k < Np; k += 32) {
      r_hi[k] = r_hi[plane + k] = r_hi[2 * plane + k] = r_hi[3 * plane + k] = __float2half(0.f);
    }
    return;
  }
  const float2* x = static_cast<const float2*>(Xv) + j * N;
  const float* xr = static_cast<const float*>(Xv) + j * N;
  float2 v[8][4];
  float m = 0.f;
  bool im = false;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const int64_t k0 = 4 * ((int64_t)lane + 32 * g);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = k0 + u;
      v[g][u] = k < N ? (XR ? make_float2(xr[k], 0.f) : x[k]) : make_float2(0.f, 0.f);
      m = fmaxf(m, fmaxf(fabsf(v[g][u].x), fabsf(v[g][u].y)));
      im |= !(v[g][u].y == 0.f);
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const bool any_im = __any_sync(0xffffffffu, im);
  const int e = split_exponent(m);
  if (lane == 0) {
    col_exp[j] = e;
    if (any_im && bimag) *bimag = 1;  // every writer stores the same value
  }
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const int64_t k0 = 4 * ((int64_t)lane + 32 * g);
    if (k0 < Np) split_store4<XR>(v[g], e, r_hi, plane, k0);  // Np is a multiple of 8
  }
}

}  // namespace

cudaError_t fg_coeffs(const double* alpha, int B, int L, bool adjoint, float2* coef, float2* coefd, int64_t ldb,
                      int64_t ldj, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  dim3 grid((B + 31) / 32, (2 * L + 2 + 7) / 8);
  FgTimed timed(FGFRFT_KC_COEFFS, s);
  fg_note_launch(FGFRFT_KC_COEFFS);
  coeffs_kernel<<<grid, 256, 0, s>>>(alpha, B, L, adjoint ? -1.0 : 1.0, coef, coefd, ldb, ldj, 0, 2 * L + 1);
  return cudaGetLastError();
}

// out[i] = sum over s of parts[s * count + i], the splits in order (a fixed order, so the sum
// is deterministic)
__global__ void __launch_bounds__(256) sum_splits_kernel(const float4* __restrict__ parts, int splits, int64_t count4,
                                                         float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 acc = parts[i];
    for (int sp = 1; sp < splits; ++sp) {
      const float4 v = parts[(int64_t)sp * count4 + i];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    out[i] = acc;
  }
}

__global__ void __launch_bounds__(256) sum_splits_tail_kernel(const float2* __restrict__ parts, int splits,
                                                              int64_t count, int64_t from, float2* __restrict__ out) {
  const int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  float2 acc = parts[i];
  for (int sp = 1; sp < splits; ++sp) {
    const float2 v = parts[(int64_t)sp * count + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  out[i] = acc;
}

int fg_grad_chunks(int64_t N) { return (int)((N + GR_CHUNK - 1) / GR_CHUNK); }

cudaError_t fg_sum_splits(const float2* parts, int splits, int64_t count, float2* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  // float4 pairs when every split starts 16-byte aligned (count even, 16-byte bases)
  const bool vec = (count % 2 == 0) && ((uintptr_t)parts % 16 == 0) && ((uintptr_t)out % 16 == 0);
  const int64_t done = vec ? count : 0;
  if (vec) {
    const int64_t c4 = count / 2;
    const int64_t g = std::min<int64_t>((c4 + 255) / 256, 152 * 8);
    sum_splits_kernel<<<(unsigned)g, 256, 0, s>>>((const float4*)parts, splits, c4, (float4*)out);
  } else {
    sum_splits_tail_kernel<<<(unsigned)((count - done + 255) / 256), 256, 0, s>>>(parts, splits, count, done, out);
  }
  fg_note_launch(FGFRFT_KC_TC_GEMM);
  return cudaGetLastError();
}

cudaError_t fg_grad_alpha(const float2* G, const float2* D, int64_t B, int64_t N, float* out, double* partials,
                          cudaStream_t s, bool sum_all) {
  if (B <= 0) return cudaSuccess;
  const int nch = fg_grad_chunks(N);
  if (B > 2147483647LL || nch > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)B, (unsigned)nch);
  FgTimed timed(FGFRFT_KC_GRAD_REDUCE, s);
  fg_note_launch(FGFRFT_KC_GRAD_REDUCE, (nch == 1 && !sum_all) ? 1 : 2);
  grad_partial_kernel<<<grid, 256, 0, s>>>(G, D, N, nch, partials, sum_all ? nullptr : out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (sum_all) {
    grad_sum_kernel<<<1, 1024, 0, s>>>(partials, B * nch, out);
    return cudaGetLastError();
  }
  if (nch == 1) return cudaSuccess;
  grad_final_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(partials, nch, B, out);
  return cudaGetLastError();
}

cudaError_t fg_split_signals(const void* X, int64_t B, int64_t N, int64_t Np, int64_t rows_pad, __half* planes,
                             int* col_exp, cudaStream_t s, int* bimag, bool x_real) {
  if (rows_pad <= 0) return cudaSuccess;
  if (bimag) {
    const cudaError_t e = cudaMemsetAsync(bimag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  FgTimed timed(FGFRFT_KC_SPLIT_SIGNALS, s);
  fg_note_launch(FGFRFT_KC_SPLIT_SIGNALS);
  const unsigned grid = (unsigned)rows_pad;
  auto go = [&](auto kern) { kern<<<grid, 256, 0, s>>>(X, B, N, Np, rows_pad, planes, col_exp, bimag); };
  if (Np <= 1024) {  // a warp per column
    const unsigned gw = (unsigned)((rows_pad + SPLIT_WARPS - 1) / SPLIT_WARPS);
    if (x_real)
      split_signals_warp_kernel<true><<<gw, 32 * SPLIT_WARPS, 0, s>>>(X, B, N, Np, rows_pad, planes, col_exp, bimag);
    else
      split_signals_warp_kernel<false><<<gw, 32 * SPLIT_WARPS, 0, s>>>(X, B, N, Np, rows_pad, planes, col_exp, bimag);
    return cudaGetLastError();
  }
  if (x_real) {
    if (Np <= 2048) go(split_signals_kernel<2, true>);
    else if (Np <= 4096) go(split_signals_kernel<4, true>);
    else go(split_signals_kernel<0, true>);
  } else {
    if (Np <= 2048) go(split_signals_kernel<2, false>);
    else if (Np <= 4096) go(split_signals_kernel<4, false>);
    else go(split_signals_kernel<0, false>);
  }
  return cudaGetLastError();
}

cudaError_t fg_coeff_planes(const double* alpha, int64_t A, int L, int L_max, int64_t Kp, __half* planes,
                            int* col_exp, cudaStream_t s, const double* alpha_host) {
  if (A <= 0) return cudaSuccess;
  if (A > INT32_MAX || Kp < 2 * (int64_t)L_max + 2 || Kp % 8) return cudaErrorInvalidValue;
  FgTimed timed(FGFRFT_KC_COEFFS, s);
  fg_note_launch(FGFRFT_KC_COEFFS);
  CoefOrders ord{};
  if (alpha_host && A <= COEF_PARAM_ORDERS) {
    for (int64_t i = 0; i < A; ++i) ord.a[i] = alpha_host[i];
    alpha = nullptr;
  }
  coeff_planes_kernel<<<(unsigned)A, 256, 0, s>>>(alpha, ord, L, L_max, A, Kp, planes, col_exp);
  return cudaGetLastError();
}

cudaError_t fg_coeff_planes_pair(const double* alpha, int64_t A, int L, int L_max, __half* planes, int* col_exp,
                                 float* diag, cudaStream_t s, const double* alpha_host) {
  if (A <= 0 || A > 64 || L_max % 16 || L > L_max) return cudaErrorInvalidValue;
  FgTimed timed(FGFRFT_KC_COEFFS, s);
  fg_note_launch(FGFRFT_KC_COEFFS);
  CoefOrders ord{};
  if (alpha_host) {
    for (int64_t i = 0; i < A; ++i) ord.a[i] = alpha_host[i];
    alpha = nullptr;
  }
  coeff_planes_pair_kernel<<<128, 128, 0, s>>>(alpha, ord, L, L_max, A, planes, col_exp, diag);
  return cudaGetLastError();
}
