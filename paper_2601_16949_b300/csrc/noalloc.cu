// Allocation-free Coulomb term: rttda_coulomb_noalloc.
//
// For callers that must not allocate device memory while they run: code
// executing inside a memory pool or arena that another component owns, an
// allocator-free real-time loop, or a host program whose device memory
// budget is fixed up front.  Such a caller cannot let the library call
// cudaMalloc behind its back, so this entry point keeps its only scratch
// buffer in a fixed-size array that is part of the loaded library.
//
// The array is a file-scope __device__ variable.  Every GPU on which the
// library is loaded holds it (kMaxScratch doubles) until the process exits.
// In host code its name is only a host-side stand-in; the device address
// is looked up once per device with cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/rttda.h"
#include "engine_internal.h"

namespace {

// Scratch for w[P][col] = sum_jb B^P_jb c_jb,col: naux * 2 * ntraj doubles.
constexpr long long kMaxScratch = 1LL << 20;  // 8 MiB of doubles

__device__ __align__(256) double g_noalloc_scratch[kMaxScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device, then cached).
rttda_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return rttda::set_error(RTTDA_E_CUDA, std::string("rttda_coulomb_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return rttda::set_error(RTTDA_E_ARG, "rttda_coulomb_noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return rttda::set_error(RTTDA_E_CUDA, std::string("rttda_coulomb_noalloc: cudaGetSymbolAddress: ") +
                                                cudaGetErrorString(e));
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return RTTDA_OK;
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  return x;
}

// w[p][2t+q] = sum_ia B[p][ia] c[t][1+ia][q]; one block per (p, t); fixed
// reduction order.  Every element of w that k_na_sigma reads is written here.
__global__ void __launch_bounds__(256) k_na_w(long long ov, long long n, int ntraj, const double* __restrict__ B,
                                              const double* __restrict__ c, double* __restrict__ w) {
  __shared__ double red[2][8];
  const int p = blockIdx.x, t = blockIdx.y;
  const double* Brow = B + (size_t)p * ov;
  const double* ct = c + ((size_t)t * n + 1) * 2;
  double sr = 0.0, si = 0.0;
  for (long long ia = threadIdx.x; ia < ov; ia += blockDim.x) {
    const double b = Brow[ia];
    sr = fma(b, ct[2 * ia], sr);
    si = fma(b, ct[2 * ia + 1], si);
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = sr;
    red[1][wid] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      ar += red[0][k];
      ai += red[1][k];
    }
    w[(size_t)p * 2 * ntraj + 2 * t] = ar;
    w[(size_t)p * 2 * ntraj + 2 * t + 1] = ai;
  }
}

// sigma[t][0] = 0, sigma[t][1+ia][q] = 2 sum_p B[p][ia] w[p][2t+q]
__global__ void __launch_bounds__(256) k_na_sigma(int naux, long long ov, long long n, int ntraj,
                                                  const double* __restrict__ B, const double* __restrict__ w,
                                                  double* __restrict__ sigma) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (k >= n) return;
  double* out = sigma + ((size_t)t * n + k) * 2;
  if (k == 0) {
    out[0] = 0.0;
    out[1] = 0.0;
    return;
  }
  const long long ia = k - 1;
  double sr = 0.0, si = 0.0;
  for (int p = 0; p < naux; ++p) {
    const double b = B[(size_t)p * ov + ia];
    sr = fma(b, w[(size_t)p * 2 * ntraj + 2 * t], sr);
    si = fma(b, w[(size_t)p * 2 * ntraj + 2 * t + 1], si);
  }
  out[0] = 2.0 * sr;
  out[1] = 2.0 * si;
}

}  // namespace

extern "C" rttda_status rttda_coulomb_noalloc(int nocc, int nvirt, int naux, const double* B_ov_dev,
                                              const double* c_dev, int ntraj, double* sigma_dev, void* stream) {
  rttda::g_last_error.clear();
  if (nocc < 1 || nvirt < 1 || naux < 1 || ntraj < 1)
    return rttda::set_error(RTTDA_E_ARG, "rttda_coulomb_noalloc: nocc, nvirt, naux, ntraj must be >= 1");
  if (!B_ov_dev || !c_dev || !sigma_dev) return rttda::set_error(RTTDA_E_ARG, "rttda_coulomb_noalloc: NULL pointer");
  const long long need = (long long)naux * 2 * ntraj;
  if (need > kMaxScratch)
    return rttda::set_error(RTTDA_E_ARG, "rttda_coulomb_noalloc: naux*2*ntraj = " + std::to_string(need) +
                                             " exceeds the fixed scratch of " + std::to_string(kMaxScratch) +
                                             " doubles");
  if ((long long)ntraj > 65535) return rttda::set_error(RTTDA_E_ARG, "rttda_coulomb_noalloc: ntraj too large");
  double* w = nullptr;
  rttda_status st = scratch_address(&w);
  if (st != RTTDA_OK) return st;
  const long long ov = (long long)nocc * nvirt, n = 1 + ov;
  cudaStream_t s = (cudaStream_t)stream;
  k_na_w<<<dim3(naux, ntraj), 256, 0, s>>>(ov, n, ntraj, B_ov_dev, c_dev, w);
  k_na_sigma<<<dim3((unsigned)((n + 255) / 256), ntraj), 256, 0, s>>>(naux, ov, n, ntraj, B_ov_dev, w, sigma_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return rttda::set_error(RTTDA_E_CUDA, std::string("rttda_coulomb_noalloc: launch: ") + cudaGetErrorString(e));
  return RTTDA_OK;
}
