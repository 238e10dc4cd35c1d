// Pinned staging of the small per-call host tables (orders, tile lists, group tables), and
// the auxiliary stream of each device (fg_fork / fg_join).
//
// A stream being captured into a CUDA graph takes neither: a graph replays long after the
// call, when the slots hold other calls' tables, so under capture the tables are written
// into the caller's work buffer by small kernels whose parameters carry the bytes
// (fg_upload), and the graph keeps them with its kernel nodes.
//
// cudaMemcpyAsync from pageable host memory returns only once the copy has been staged,
// which waits for the stream to reach it: every call would then hold the host until the
// device has drained the work queued before it, and the device would idle while the host
// enqueues the rest of the call.  The tables therefore go to a ring of fixed pinned slots
// per device, and the kernels read them there directly (fg_stage): a copy on the stream
// would also queue, on the copy engine, behind large signal transfers of other streams.
// A slot is reused only after the work that reads it has run (one event per slot, recorded
// by fg_stage_done or after fg_h2d's copy).  A table larger than a slot, or any table when
// pinned memory is unavailable, takes a stream copy.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr int kSlots = 64;
constexpr size_t kSlotBytes = 256 * 1024;
constexpr int kMaxDevices = 64;

struct Aux {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool failed = false;
};

struct Ring {
  char* base = nullptr;
  char* dbase = nullptr;  // device address of base
  cudaEvent_t ev[kSlots] = {};
  bool used[kSlots] = {};
  bool held[kSlots] = {};  // reserved by fg_stage until fg_stage_done
  int next = 0;
  bool failed = false;
};

std::mutex g_mu;
Ring g_ring[kMaxDevices];
std::mutex g_aux_mu;
Aux g_aux[kMaxDevices];

bool aux_init(Aux& a, cudaStream_t s) {
  if (a.stream) return true;
  if (a.failed) return false;
  // no stream or event is created while s is being captured into a graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  if (cudaStreamCreateWithFlags(&a.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    a.failed = true;
    a.stream = nullptr;
    return false;
  }
  return true;
}

bool ring_init(Ring& r) {
  if (r.base) return true;
  if (r.failed) return false;
  void* p = nullptr;
  if (cudaHostAlloc(&p, (size_t)kSlots * kSlotBytes, cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess || !p) {
    cudaGetLastError();
    r.failed = true;
    return false;
  }
  for (int i = 0; i < kSlots; ++i) {
    if (cudaEventCreateWithFlags(&r.ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaEventDestroy(r.ev[j]);
      cudaFreeHost(p);
      r.failed = true;
      return false;
    }
  }
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess || !d) {
    cudaGetLastError();
    d = nullptr;  // fg_stage falls back to stream copies
  }
  r.base = static_cast<char*>(p);
  r.dbase = static_cast<char*>(d);
  return true;
}

// Next free slot of the ring (waiting for its previous reader if needed), or -1.
int take_slot(Ring& r) {
  for (int tries = 0; tries < kSlots; ++tries) {
    const int k = r.next;
    r.next = (k + 1) % kSlots;
    if (r.held[k]) continue;
    if (r.used[k] && cudaEventSynchronize(r.ev[k]) != cudaSuccess) return -1;
    return k;
  }
  return -1;
}

constexpr int kUploadBytes = 3072;  // payload per upload kernel (kernel parameters <= 4 KB)
struct UploadChunk {
  unsigned char b[kUploadBytes];
};
__global__ void upload_kernel(unsigned char* __restrict__ dst, const UploadChunk chunk, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = chunk.b[i];
}

}  // namespace

bool fg_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

cudaError_t fg_upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  const unsigned char* in = static_cast<const unsigned char*>(src);
  unsigned char* out = static_cast<unsigned char*>(dst);
  UploadChunk chunk;
  for (size_t off = 0; off < bytes; off += kUploadBytes) {
    const int n = (int)std::min<size_t>(kUploadBytes, bytes - off);
    std::memcpy(chunk.b, in + off, (size_t)n);
    upload_kernel<<<(n + 255) / 256, 256, 0, s>>>(out + off, chunk, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t fg_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  if (fg_capturing(s)) return fg_upload(dst, src, bytes, s);
  int dev = 0;
  if (bytes <= kSlotBytes && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices) {
    std::lock_guard<std::mutex> g(g_mu);
    Ring& r = g_ring[dev];
    if (ring_init(r)) {
      const int k = take_slot(r);
      if (k < 0) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
      char* slot = r.base + (size_t)k * kSlotBytes;
      std::memcpy(slot, src, bytes);
      cudaError_t e = cudaMemcpyAsync(dst, slot, bytes, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return e;
      e = cudaEventRecord(r.ev[k], s);
      if (e != cudaSuccess) return e;
      r.used[k] = true;
      return cudaSuccess;
    }
  }
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

int fg_stage(const void* src, size_t bytes, const void** dev) {
  *dev = nullptr;
  int d = 0;
  if (bytes == 0 || bytes > kSlotBytes || cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  std::lock_guard<std::mutex> g(g_mu);
  Ring& r = g_ring[d];
  if (!ring_init(r) || !r.dbase) return -1;
  const int k = take_slot(r);
  if (k < 0) return -1;
  std::memcpy(r.base + (size_t)k * kSlotBytes, src, bytes);
  r.held[k] = true;
  *dev = r.dbase + (size_t)k * kSlotBytes;
  return d * kSlots + k;
}

void fg_stage_done(int token, cudaStream_t s) {
  if (token < 0) return;
  const int d = token / kSlots, k = token % kSlots;
  if (d >= kMaxDevices) return;
  std::lock_guard<std::mutex> g(g_mu);
  Ring& r = g_ring[d];
  if (!r.held[k]) return;
  r.used[k] = cudaEventRecord(r.ev[k], s) == cudaSuccess;
  if (!r.used[k]) {  // no event: wait for the work that reads the slot before releasing it
    cudaGetLastError();
    cudaStreamSynchronize(s);
  }
  r.held[k] = false;
}

cudaStream_t fg_fork(cudaStream_t s) {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> g(g_aux_mu);
  Aux& a = g_aux[d];
  if (!aux_init(a, s)) return nullptr;
  if (cudaEventRecord(a.fork, s) != cudaSuccess || cudaStreamWaitEvent(a.stream, a.fork, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.stream;
}

cudaError_t fg_join(cudaStream_t aux, cudaStream_t s) {
  if (!aux) return cudaSuccess;
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return e;
  if (d < 0 || d >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_aux_mu);
  e = cudaEventRecord(g_aux[d].join, aux);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, g_aux[d].join, 0);
}
