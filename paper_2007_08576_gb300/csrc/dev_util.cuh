// Device helpers shared by the factorisation and the solve kernels: the global timer, bounded
// waits on counters written by other CTAs (polling with sleeps, or with acquire loads),
// release stores, L2-only loads.
#pragma once
#include <cuda_runtime.h>

namespace ds {

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *p >= v. Returns false (and raises *err) on timeout or if *err is set.
__device__ __forceinline__ bool wait_ge(const int* p, int v, int* err,
                                        unsigned long long budget_ns) {
  const volatile int* vp = p;
  const volatile int* ve = err;
  if (*vp >= v) return true;
  unsigned long long t0 = globaltimer();
  int it = 0;
  while (*vp < v) {
    if (*ve) return false;
    if ((++it & 31) == 0 && globaltimer() - t0 > budget_ns) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// GPU-scope acquire load / release store of a flag word.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait until *p >= v with acquire loads and no sleep between polls (for waits on a
// critical path). False (and *err raised) on timeout or if *err is set.
__device__ __forceinline__ bool wait_flag(const int* p, int v, int* err,
                                          unsigned long long budget_ns) {
  if (ld_acquire(p) >= v) return true;
  const volatile int* ve = err;
  const unsigned long long t0 = globaltimer();
  int it = 0;
  while (ld_acquire(p) < v) {
    if (*ve) return false;
    if ((++it & 63) == 0 && globaltimer() - t0 > budget_ns) {
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

}  // namespace ds
