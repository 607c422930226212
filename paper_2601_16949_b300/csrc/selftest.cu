// Self-test of the bounded device waits (failure detection without a fault).
//
// The tensor-core kernels wait on mbarriers with a wall-clock limit read from
// %globaltimer; when a wait runs out they record an error code that the host
// reads (RTTDA_E_TIMEOUT) and return, leaving the context usable.  This file
// exercises the same pattern on a flag that nothing ever sets.
#include <cuda_runtime.h>

#include <string>

#include "../../include/rttda.h"
#include "engine_internal.h"

namespace {

// One thread waits for *flag != 0 for at most limit_ns, then reports:
// *status = 1 (ran out) or 2 (flag seen).
__global__ void k_wait_flag(const volatile int* flag, int* status, unsigned long long limit_ns) {
  if (threadIdx.x != 0) return;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (*flag == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      *status = 1;
      return;
    }
    __nanosleep(1000);
  }
  *status = 2;
}

}  // namespace

extern "C" rttda_status rttda_selftest_wait(double limit_s) {
  rttda::g_last_error.clear();
  if (!(limit_s >= 1e-3 && limit_s <= 2.0))
    return rttda::set_error(RTTDA_E_ARG, "rttda_selftest_wait: limit must be in [1e-3, 2] s");
  int* d = nullptr;
  cudaError_t e = cudaMalloc((void**)&d, 2 * sizeof(int));
  if (e != cudaSuccess) return rttda::set_error(RTTDA_E_CUDA, std::string("rttda_selftest_wait: ") + cudaGetErrorString(e));
  int h[2] = {0, 0};
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_flag<<<1, 32, 0, s>>>(d, d + 1, (unsigned long long)(limit_s * 1e9));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (s) cudaStreamDestroy(s);
  cudaFree(d);
  if (e != cudaSuccess) return rttda::set_error(RTTDA_E_CUDA, std::string("rttda_selftest_wait: ") + cudaGetErrorString(e));
  if (h[1] == 1) return rttda::set_error(RTTDA_E_TIMEOUT, "rttda_selftest_wait: the device wait ran out (expected)");
  return RTTDA_OK;
}
