// Launch state cached per device ordinal.
//
// A kernel's raised shared-memory limit (cudaFuncSetAttribute), its
// occupancy and the SM count all belong to one device: a process that
// uploads clouds to two GPUs must set the attribute in each device's
// context and size each grid from that device's own figures. PerDevice<T>
// keeps one T per ordinal, filled on first use with that device current.
// Host code only, no CUDA types, so the table logic is testable on a CPU.
#pragma once
#include <mutex>

namespace mknn {

constexpr int kMaxDevices = 64;

template <class T>
class PerDevice {
 public:
  // Runs fn(T&) under the table's lock on device dev's entry (value-
  // initialised before its first use) and returns fn's result; returns
  // `bad` without calling fn when dev is outside [0, kMaxDevices).
  template <class R, class F>
  R with(int dev, R bad, F&& fn) {
    if (dev < 0 || dev >= kMaxDevices) return bad;
    std::lock_guard<std::mutex> lk(mu_);
    return fn(v_[dev]);
  }

 private:
  std::mutex mu_;
  T v_[kMaxDevices] = {};
};

}  // namespace mknn
