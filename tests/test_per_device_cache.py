"""The launchers' per-device cache of launch settings (csrc/per_device.h), exercised on the CPU:
several host threads asking for the same devices' values at once compute each device's value
exactly once, every thread sees it, devices do not share values, and a failed computation is not
cached.  The header is plain C++; this test compiles a small driver for it with g++."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2007_08576_gb300", "csrc")

DRIVER = r"""
#include <chrono>
#include <cstdio>
#include <thread>
#include <vector>
#include "per_device.h"

int main() {
  ds::PerDeviceValue cache;
  std::atomic<int> calls[4] = {};
  std::vector<std::thread> th;
  std::atomic<int> bad{0};
  for (int t = 0; t < 16; ++t)
    th.emplace_back([&, t] {
      for (int rep = 0; rep < 100; ++rep) {
        const int dev = (t + rep) % 4;
        const int v = cache.get(dev, [&] {
          calls[dev]++;
          std::this_thread::sleep_for(std::chrono::milliseconds(5));
          return 10 + dev;
        });
        if (v != 10 + dev) bad++;
      }
    });
  for (auto& x : th) x.join();
  for (int d = 0; d < 4; ++d)
    if (calls[d] != 1) { std::printf("device %d computed %d times\n", d, (int)calls[d]); return 1; }
  if (bad) { std::printf("%d wrong values\n", (int)bad); return 2; }
  // a failure is returned and computed again next time; then the success is cached
  ds::PerDeviceValue c2;
  int n = 0;
  if (c2.get(1, [&] { ++n; return 0; }) != 0) return 3;
  if (c2.get(1, [&] { ++n; return 7; }) != 7) return 4;
  if (c2.get(1, [&] { ++n; return 9; }) != 7) return 5;
  if (n != 2) return 6;
  // an out-of-range device id is refused without computing
  if (c2.get(-1, [&] { ++n; return 1; }) != 0 || c2.get(ds::kMaxDevices, [&] { ++n; return 1; }) != 0)
    return 7;
  if (n != 2) return 8;
  std::printf("ok\n");
  return 0;
}
"""


def test_per_device_cache_threads(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "driver.cc"
    src.write_text(DRIVER)
    exe = tmp_path / "driver"
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
