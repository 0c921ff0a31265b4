// A value computed once per device and cached, safe to query from several host threads at once.
// Plain C++ (no CUDA): the library's launchers use it through PerDevice (ds_internal.cuh) for
// launch settings that belong to a device (kernel attributes, occupancies, the SM count).
#pragma once

#include <atomic>
#include <mutex>

namespace ds {

constexpr int kMaxDevices = 64;

class PerDeviceValue {
 public:
  // The cached value of device `dev`, or, the first time it is asked for there, compute()'s
  // result, computed by one thread while the others wait. compute() returns a positive value, or
  // <= 0 on failure; a failure is returned but not cached, so the next query computes again.
  // A device id outside [0, kMaxDevices) returns 0 without calling compute().
  template <typename F>
  int get(int dev, F&& compute) {
    if (dev < 0 || dev >= kMaxDevices) return 0;
    int v = val_[dev].load(std::memory_order_acquire);
    if (v > 0) return v;
    std::lock_guard<std::mutex> lock(mu_);
    v = val_[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    v = compute();
    if (v > 0) val_[dev].store(v, std::memory_order_release);
    return v;
  }

 private:
  std::mutex mu_;
  std::atomic<int> val_[kMaxDevices] = {};
};

}  // namespace ds
