// Coulomb term on the CUDA cores, FP32 arithmetic on FP32 or BF16 factors.
//
//   pass 1  w[P][col]    = sum_ia B^P_ia c_(ia),col        (K = ov)
//   pass 2  J[ia][col]   = 2 sum_P B^P_ia w[P][col]        (K = naux)
//
// (the Coulomb part 2(ia|jb) c_jb of the A matrix elements, Sec. 2.2, with
// (ia|jb) = sum_P B^P_ia B^P_jb).  Both passes stream B_ov once with a few
// multiply-adds per element, so they are bound by HBM bandwidth.  What keeps
// them there on this GPU:
//   * no FP64 arithmetic in the stream: the stage's amplitudes are converted
//     to FP32 once per stage (k_prep_xf), and the FP64 pipe is a small
//     fraction of the FP32 rate;
//   * 16-byte loads with eight of them in flight per thread and three CTAs
//     per SM for up to six columns (two above), so that 64-96 KB per SM are
//     in flight;
//   * pass 1 stages its slice of FP32 amplitudes in shared memory once per
//     CTA and reuses it for 32 factor rows.
// Partial sums (pass 1 over ia slices, pass 2 over chunks of P) are added in
// a fixed order by their consumers, so results are deterministic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels_simt.cuh"

namespace rttda {
namespace stream {

constexpr int kThreads = 256;
constexpr int kW1Rows = 32;              // pass 1: factor rows per CTA (4 per warp)
// CTAs per SM the register budget is sized for: three (85 registers) for
// up to six columns, two (128 registers) above, where the per-thread
// accumulators grow with C
template <int C>
constexpr int min_blocks_w() { return C <= 6 ? 3 : 2; }
template <int C>
constexpr int min_blocks_j() { return C <= 6 ? 3 : 2; }
constexpr int kW1SmemBytes = 48 * 1024;  // pass 1 amplitude slice

template <typename TF>
__device__ __forceinline__ float to_f(TF x);
template <>
__device__ __forceinline__ float to_f<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

template <typename TF>
__device__ __forceinline__ void unpack16(const uint4& u, float (&b)[16 / sizeof(TF)]) {
  const TF* e = reinterpret_cast<const TF*>(&u);
#pragma unroll
  for (int k = 0; k < (int)(16 / sizeof(TF)); ++k) b[k] = to_f<TF>(e[k]);
}

// Amplitudes of the stage as FP32, [ia][col] (row 0, the ground state, is
// not needed by the Coulomb term).
__global__ void __launch_bounds__(256) k_prep_xf(long long n, int C, const double* __restrict__ X,
                                                 float* __restrict__ Xf) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    Xf[e] = (float)X[C + e];
}

// ---------------------------------------------------------------------------
// Pass 1.  grid (ceil(P / 32), nslice).  CTA (x, s): rows p0 = 32x .. +31 of
// B_ov over the ia slice [s*slice, s*slice + slice); the slice's FP32
// amplitudes (slice x C) sit in shared memory.  Warp w owns rows 4w..4w+3;
// lane l the V-element groups l, l + 32, ... (two groups per iteration, so
// eight 16-byte factor loads are in flight).  wpart[s][p][col] receives the
// slice's partial sums.  Requires ov % V == 0, slice % V == 0 and
// slice * C * 4 <= kW1SmemBytes.
// ---------------------------------------------------------------------------
template <typename TF, int C>
__global__ void __launch_bounds__(kThreads, min_blocks_w<C>())
    k_coul_w_stream(const TF* __restrict__ Bov, const float* __restrict__ Xf, int P, long long ov, int slice,
                    float* __restrict__ wpart) {
  constexpr int V = 16 / sizeof(TF);
  static_assert(C % 2 == 0 && C <= 12, "C = 2T <= 12");
  extern __shared__ __align__(16) float xs[];  // [slice][C]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = blockIdx.x * kW1Rows;
  const long long ia0 = (long long)blockIdx.y * slice;
  const int len = (int)min((long long)slice, ov - ia0);
  {
    const float4* src = reinterpret_cast<const float4*>(Xf + (size_t)ia0 * C);
    float4* dst = reinterpret_cast<float4*>(xs);
    for (int e = threadIdx.x; e < len * C / 4; e += kThreads) dst[e] = __ldg(src + e);
  }
  __syncthreads();
  const TF* rowp[4];
  bool rok[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = p0 + warp * 4 + r;
    rok[r] = p < P;
    rowp[r] = Bov + (size_t)(rok[r] ? p : 0) * ov + ia0;
  }
  float acc[4][C];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[r][c] = 0.0f;
  auto fma_group = [&](const uint4(&u)[4], int k) {
    float x[V * C];
    const float4* xp = reinterpret_cast<const float4*>(xs + k * C);
#pragma unroll
    for (int e = 0; e < V * C / 4; ++e) {
      const float4 d = xp[e];
      x[4 * e] = d.x;
      x[4 * e + 1] = d.y;
      x[4 * e + 2] = d.z;
      x[4 * e + 3] = d.w;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float b[V];
      unpack16<TF>(u[r], b);
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = fmaf(b[v], x[v * C + c], acc[r][c]);
    }
  };
  int k = lane * V;
  for (; k + 32 * V < len; k += 64 * V) {
    uint4 u0[4], u1[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      u0[r] = rok[r] ? __ldg(reinterpret_cast<const uint4*>(rowp[r] + k)) : make_uint4(0, 0, 0, 0);
      u1[r] = rok[r] ? __ldg(reinterpret_cast<const uint4*>(rowp[r] + k + 32 * V)) : make_uint4(0, 0, 0, 0);
    }
    fma_group(u0, k);
    fma_group(u1, k + 32 * V);
  }
  if (k < len) {
    uint4 u0[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
      u0[r] = rok[r] ? __ldg(reinterpret_cast<const uint4*>(rowp[r] + k)) : make_uint4(0, 0, 0, 0);
    fma_group(u0, k);
  }
  float* w = wpart + (size_t)blockIdx.y * P * C;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float sum = warp_sum(acc[r][c]);
      if (lane == 0 && rok[r]) w[(size_t)(p0 + warp * 4 + r) * C + c] = sum;
    }
  }
}

// ---------------------------------------------------------------------------
// Pass 2.  grid (ceil(ov / (256 V)), nsplit).  CTA (x, s): thread t owns
// ia = 256 V x + V t .. +V and the rows P of chunk s [s*pchunk, +pchunk),
// eight rows per iteration (eight 16-byte loads in flight).  w (the sum of
// the nw pass-1 partials) for the chunk sits in shared memory.
// Jpart[s][ia][col] = 2 x partial sum.  Requires ov % V == 0.
// ---------------------------------------------------------------------------
template <typename TF, int C>
__global__ void __launch_bounds__(kThreads, min_blocks_j<C>())
    k_coul_J_stream(const TF* __restrict__ Bov, const float* __restrict__ wpart, int nw, int P, long long ov,
                    int pchunk, float* __restrict__ Jpart) {
  constexpr int V = 16 / sizeof(TF);
  constexpr int U = 8;
  static_assert(C % 2 == 0 && C <= 12, "C = 2T <= 12");
  extern __shared__ __align__(16) float ws[];  // [pchunk][C]
  const int p0 = blockIdx.y * pchunk, p1 = min(P, p0 + pchunk);
  const int nrows = max(0, p1 - p0);
  for (int e = threadIdx.x; e < nrows * C; e += kThreads) {
    float a = wpart[(size_t)p0 * C + e];
    for (int k = 1; k < nw; ++k) a += wpart[(size_t)k * P * C + (size_t)p0 * C + e];
    ws[e] = a;
  }
  __syncthreads();
  const long long ia = ((long long)blockIdx.x * kThreads + threadIdx.x) * V;
  if (ia >= ov) return;
  const TF* bp = Bov + (size_t)p0 * ov + ia;
  float acc[V][C];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[v][c] = 0.0f;
  auto fma_row = [&](const uint4& u, int r) {
    float b[V];
    unpack16<TF>(u, b);
    float wv[C];
#pragma unroll
    for (int c = 0; c < C; ++c) wv[c] = ws[r * C + c];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[v][c] = fmaf(b[v], wv[c], acc[v][c]);
  };
  int r = 0;
  for (; r + U <= nrows; r += U) {
    uint4 u[U];
#pragma unroll
    for (int q = 0; q < U; ++q) u[q] = __ldg(reinterpret_cast<const uint4*>(bp + (size_t)(r + q) * ov));
#pragma unroll
    for (int q = 0; q < U; ++q) fma_row(u[q], r + q);
  }
  for (; r < nrows; ++r) fma_row(__ldg(reinterpret_cast<const uint4*>(bp + (size_t)r * ov)), r);
  float* dst = Jpart + ((size_t)blockIdx.y * ov + ia) * C;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int c = 0; c < C; ++c) dst[v * C + c] = 2.0f * acc[v][c];
}

}  // namespace stream
}  // namespace rttda
