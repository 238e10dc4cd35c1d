// Kernel-class launch counters and optional CUDA-event timing of every launch.
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

constexpr size_t kMaxPairs = 1 << 16;        // recorded launches per class between resets
constexpr size_t kPrecreatedPairs = 512;     // event pairs per class created when timing is enabled

struct ClassLog {
  std::vector<cudaEvent_t> start, stop;  // event pool, reused after a reset
  size_t used = 0;
  int64_t launches = 0;
  int64_t timed = 0;
};

struct Timing {
  std::mutex mu;
  bool enabled = false;
  ClassLog cls[FGFRFT_KC_COUNT];
};

Timing& T() {
  static Timing t;
  return t;
}

}  // namespace

void fg_note_launch(int cls, int n) {
  if (cls < 0 || cls >= FGFRFT_KC_COUNT) return;
  std::lock_guard<std::mutex> g(T().mu);
  T().cls[cls].launches += n;
}

FgTimed::FgTimed(int cls, cudaStream_t s) : cls_(cls), s_(s), slot_(-1) {
  Timing& t = T();
  std::lock_guard<std::mutex> g(t.mu);
  if (!t.enabled || cls < 0 || cls >= FGFRFT_KC_COUNT) return;
  if (fg_capturing(s)) return;  // an event pair inside a graph has no elapsed time
  ClassLog& c = t.cls[cls];
  if (c.used >= kMaxPairs) return;
  if (c.used == c.start.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    c.start.push_back(a);
    c.stop.push_back(b);
  }
  slot_ = (long)c.used++;
  cudaEventRecord(c.start[(size_t)slot_], s);
}

FgTimed::~FgTimed() {
  if (slot_ < 0) return;
  Timing& t = T();
  std::lock_guard<std::mutex> g(t.mu);
  cudaEventRecord(t.cls[cls_].stop[(size_t)slot_], s_);
  t.cls[cls_].timed++;
}

extern "C" {

int fgfrft_timing_enable(int on) {
  std::lock_guard<std::mutex> g(T().mu);
  T().enabled = on != 0;
  // create the event pool now, so that timed calls only record events (creating one inside
  // a timed loop costs host time that would show up as gaps between launches)
  if (on) {
    for (auto& c : T().cls) {
      while (c.start.size() < kPrecreatedPairs) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) break;
        if (cudaEventCreate(&b) != cudaSuccess) {
          cudaEventDestroy(a);
          break;
        }
        c.start.push_back(a);
        c.stop.push_back(b);
      }
    }
  }
  return FGFRFT_OK;
}

int fgfrft_timing_reset(void) {
  std::lock_guard<std::mutex> g(T().mu);
  for (auto& c : T().cls) {
    c.used = 0;
    c.timed = 0;
    c.launches = 0;
  }
  return FGFRFT_OK;
}

int fgfrft_timing_read(int kernel_class, int64_t* launches, int64_t* timed, double* total_ms) {
  if (kernel_class < 0 || kernel_class >= FGFRFT_KC_COUNT) return FGFRFT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(T().mu);
  ClassLog& c = T().cls[kernel_class];
  double sum = 0.0;
  for (size_t i = 0; i < c.used; ++i) {
    if (cudaEventSynchronize(c.stop[i]) != cudaSuccess) return FGFRFT_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c.start[i], c.stop[i]) != cudaSuccess) return FGFRFT_ERR_CUDA;
    sum += ms;
  }
  if (launches) *launches = c.launches;
  if (timed) *timed = (int64_t)c.used;
  if (total_ms) *total_ms = sum;
  return FGFRFT_OK;
}

}  // extern "C"
