// Zero-allocation variant of the alpha-gradient reduction.
//
// Some callers cannot allocate device memory at the point where they need the
// gradient: code running inside a framework whose allocator must not be
// re-entered, a real-time section that forbids cudaMalloc /
// cudaFree (they synchronise the device), or an embedding host that only hands
// over input and output buffers.  fgfrft_grad_alpha_noalloc serves them: its FP64
// partial sums live in a fixed array in this library's device memory instead of a
// caller-provided work buffer.
#include <mutex>

#include "internal.h"

namespace {

// Fixed scratch: one FP64 partial sum per (signal, 1024-entry chunk).  Every GPU
// that loads the library holds these 512 KiB until the process exits.
constexpr int64_t kNoallocMaxPartials = FGFRFT_NOALLOC_MAX_PARTIALS;
constexpr int kNoallocChunk = 1024;
static __device__ __align__(256) double g_grad_partials[kNoallocMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};

// level 1: partial[j][c] = Re sum_{i in chunk c} conj(G_ji) D_ji (FP64), always written
__global__ void __launch_bounds__(256) noalloc_partial_kernel(const float2* __restrict__ G,
                                                              const float2* __restrict__ D, int64_t N, int nchunks,
                                                              double* __restrict__ partial) {
  const int64_t j = blockIdx.x;
  const int c = blockIdx.y;
  const int64_t i0 = (int64_t)c * kNoallocChunk;
  const int64_t i1 = (i0 + kNoallocChunk) < N ? (i0 + kNoallocChunk) : N;
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
    partial[j * nchunks + c] = s;
  }
}

// level 2: out[j] = sum over the chunks of column j, in chunk order
__global__ void noalloc_final_kernel(const double* __restrict__ partial, int nchunks, int64_t B,
                                     float* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= B) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[j * nchunks + c];
  out[j] = (float)s;
}

// Device address of the fixed scratch on the current device, looked up once per device
// and kept for the life of the process (a device reset in between would leave it stale;
// the header tells callers not to call this entry point after one).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FGFRFT_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_grad_partials) != cudaSuccess || !p) return FGFRFT_ERR_CUDA;
    g_dev_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_dev_ptr[dev];
  return FGFRFT_OK;
}

}  // namespace

extern "C" int fgfrft_grad_alpha_noalloc(const void* G_dev, const void* D_dev, int64_t B, int64_t N,
                                         float* gradalpha_dev, void* stream) {
  if (!G_dev || !D_dev || !gradalpha_dev || B < 1 || N < 1) return FGFRFT_ERR_INVALID_ARG;
  const int64_t nchunks = (N + kNoallocChunk - 1) / kNoallocChunk;
  if (nchunks > 65535 || B > 2147483647LL || B * nchunks > kNoallocMaxPartials) return FGFRFT_ERR_UNSUPPORTED;
  double* partial = nullptr;
  const int rc = scratch_for_current_device(&partial);
  if (rc != FGFRFT_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid((unsigned)B, (unsigned)nchunks);
  noalloc_partial_kernel<<<grid, 256, 0, s>>>((const float2*)G_dev, (const float2*)D_dev, N, (int)nchunks, partial);
  if (cudaGetLastError() != cudaSuccess) return FGFRFT_ERR_CUDA;
  noalloc_final_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(partial, (int)nchunks, B, gradalpha_dev);
  if (cudaGetLastError() != cudaSuccess) return FGFRFT_ERR_CUDA;
  fg_note_launch(FGFRFT_KC_GRAD_REDUCE, 2);
  return FGFRFT_OK;
}
