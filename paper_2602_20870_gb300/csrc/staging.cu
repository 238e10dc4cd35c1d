// Pinned staging of the small per-call host tables (orders, tile lists, group tables).
//
// cudaMemcpyAsync from pageable host memory returns only once the copy has been staged,
// which waits for the stream to reach it: every call would then hold the host until the
// device has drained the work queued before it, and the device would idle while the host
// enqueues the rest of the call.  Copying through pinned memory keeps the call
// asynchronous.  The pinned memory is a ring of fixed slots per device; a slot is reused
// only after the copy that last read from it has run (one event per slot).  A copy larger
// than a slot, or any copy when pinned memory is unavailable, takes the pageable route.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr int kSlots = 64;
constexpr size_t kSlotBytes = 256 * 1024;
constexpr int kMaxDevices = 64;

struct Ring {
  char* base = nullptr;
  cudaEvent_t ev[kSlots] = {};
  bool used[kSlots] = {};
  int next = 0;
  bool failed = false;
};

std::mutex g_mu;
Ring g_ring[kMaxDevices];

bool ring_init(Ring& r) {
  if (r.base) return true;
  if (r.failed) return false;
  void* p = nullptr;
  if (cudaHostAlloc(&p, (size_t)kSlots * kSlotBytes, cudaHostAllocPortable) != cudaSuccess || !p) {
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
  r.base = static_cast<char*>(p);
  return true;
}

}  // namespace

cudaError_t fg_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  int dev = 0;
  if (bytes <= kSlotBytes && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices) {
    std::lock_guard<std::mutex> g(g_mu);
    Ring& r = g_ring[dev];
    if (ring_init(r)) {
      const int k = r.next;
      r.next = (k + 1) % kSlots;
      if (r.used[k]) {
        const cudaError_t e = cudaEventSynchronize(r.ev[k]);  // the slot's previous copy has run
        if (e != cudaSuccess) return e;
      }
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
