// Failure-detection self-test of the bounded device-side waits (the declaration in defsolve.h
// states the contract). Every cross-CTA hand-off of the factorisation and of the triangular
// solves waits through wait_flag (acquire polling) or wait_ge (polling with sleeps); here one
// thread waits with the same helpers for a flag that nothing sets, so the wait has to give up
// after its budget, raise the error word and return: the failure is made without a GPU fault and
// the context stays usable.
#include <cuda_runtime.h>

#include "dev_util.cuh"
#include "ds_internal.cuh"

namespace ds {
namespace {

// word[0] the flag (never set), word[1] the error word, word[2] 1 iff the wait saw the flag;
// *waited_ns the device time the wait took.
__global__ void k_wait_probe(int kind, int* __restrict__ word, unsigned long long budget_ns,
                             unsigned long long* __restrict__ waited_ns) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long t0 = globaltimer();
  const bool ok = kind == 0 ? wait_flag(&word[0], 1, &word[1], budget_ns)
                            : wait_ge(&word[0], 1, &word[1], budget_ns);
  *waited_ns = globaltimer() - t0;
  word[2] = ok ? 1 : 0;
}

}  // namespace
}  // namespace ds

extern "C" int ds_selftest_bounded_wait(int32_t kind, int64_t budget_ns, int32_t peer_error,
                                        double* waited_ms) {
  if ((kind != 0 && kind != 1) || budget_ns < 1000 || budget_ns > 100000000 ||
      (peer_error != 0 && peer_error != 1))
    return DS_ERR_ARG;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return DS_ERR_CUDA;
  int* word = nullptr;
  unsigned long long* dt = nullptr;
  int rc = DS_OK;
  if (cudaMalloc((void**)&word, 4 * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&dt, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    rc = DS_ERR_OOM;
  }
  int host[4] = {0, peer_error, 0, 0};
  unsigned long long waited = 0;
  if (!rc) {
    cudaMemcpyAsync(word, host, sizeof(host), cudaMemcpyHostToDevice, s);
    ds::k_wait_probe<<<1, 32, 0, s>>>(kind, word, (unsigned long long)budget_ns, dt);
    ++ds::g_launches;
    ds::count_kernels(1);
    cudaMemcpyAsync(host, word, sizeof(host), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&waited, dt, sizeof(waited), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = DS_ERR_CUDA;
  }
  if (word) cudaFree(word);
  if (dt) cudaFree(dt);
  cudaStreamDestroy(s);
  if (rc) return rc;
  if (waited_ms) *waited_ms = (double)waited * 1e-6;
  if (host[2]) return DS_OK;
  return host[1] ? DS_ERR_TIMEOUT : DS_ERR_CUDA;
}
