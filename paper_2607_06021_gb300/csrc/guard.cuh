// Ordering of CUDA stream capture against device setup across host threads.
//
// A plan's iteration graphs are captured in thread-local mode on the plan's own
// non-blocking stream.  Allocation, freeing, legacy-stream work and device-wide
// synchronisation issued by another host thread while such a capture is open
// can fail ("operation not permitted when stream is capturing") or invalidate
// the capture.  Every capture therefore holds this mutex shared, and every
// library path that allocates, frees or synchronises the device holds it
// exclusively.  Lock order: a plan's own mutex (if taken) before this one; the
// mutex is not recursive.
#pragma once
#include <mutex>
#include <shared_mutex>

namespace lrp {

std::shared_mutex& setup_mutex();

struct SetupGuard {
  std::unique_lock<std::shared_mutex> lk;
  SetupGuard() : lk(setup_mutex()) {}
};

struct CaptureGuard {
  std::shared_lock<std::shared_mutex> lk;
  CaptureGuard() : lk(setup_mutex()) {}
};

}  // namespace lrp
