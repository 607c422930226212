// Device helpers shared by the library's kernel translation units: pulse
// shapes, type conversions, double-float arithmetic, fixed-order reductions
// and the fixed-order sum of split-K partials.  Only inline device functions
// and types live here, so every .cu file may include it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rttda {

// ---------------------------------------------------------------------------
// Pulses (Sec. 2.2, Eqs. (18a)-(18d), plus sin^2)
// ---------------------------------------------------------------------------
struct PulseDev {
  int kind;                       // 0 kick, 1 CW, 2 Gaussian TL, 3 chirp, 4 sin^2
  double E0, omega, t0, sigma, beta, duration;
};

__device__ __forceinline__ double pulse_field(const PulseDev& p, double t) {
  switch (p.kind) {
    case 1:
      return p.E0 * sin(p.omega * t);
    case 2:
    case 3: {
      const double tau = t - p.t0;
      const double env = exp(-tau * tau / (2.0 * p.sigma * p.sigma));
      const double w = p.omega + (p.kind == 3 ? 0.5 * p.beta * tau : 0.0);
      return p.E0 * env * sin(w * tau);
    }
    case 4: {
      if (t < 0.0 || t > p.duration) return 0.0;
      const double s = sin(3.14159265358979323846 * t / p.duration);
      return p.E0 * s * s * sin(p.omega * t);
    }
    default:
      return 0.0;  // a kick acts only at t = 0+
  }
}

// ---------------------------------------------------------------------------
// Conversions and reductions
// ---------------------------------------------------------------------------
template <typename TC, typename TS>
__device__ __forceinline__ TC cvt(TS x) { return static_cast<TC>(x); }
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

// Double-float ("float-float") numbers for the field product of the
// observables in the FP32 modes: a value is the unevaluated sum hi + lo of
// two floats (about 48 significant bits).  A multiply-add uses Dekker's exact
// product (p + e = a.hi b.hi, e from one FMA) and Knuth's two-sum for the
// addition of p to the running hi part; the remaining error terms are summed
// into lo.  The accumulator is not renormalised after every addition (lo
// only collects rounding errors, so its own rounding stays below 2^-24 of
// them).  Every step uses the _rn intrinsics so that the compiler neither
// contracts nor reorders the error-free transformations.  On B300 this runs
// on the FP32 pipe at about five times the rate of FP64 multiply-adds.
struct df32 {
  float hi, lo;
  df32() = default;
  __device__ __forceinline__ explicit df32(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ __forceinline__ df32(int x) : hi((float)x), lo(0.0f) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ df32 operator-() const {
    df32 r;
    r.hi = -hi;
    r.lo = -lo;
    return r;
  }
};

// the built-in float and double overloads stay visible beside this one
using ::fma;

// a * b + c in double-float
__device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);          // exact: a.hi b.hi = p + e
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float sh = __fadd_rn(p, c.hi);          // two-sum of p and c.hi
  const float bb = __fsub_rn(sh, p);
  const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(sh, bb)), __fsub_rn(c.hi, bb));
  df32 r;
  r.hi = sh;
  r.lo = __fadd_rn(__fadd_rn(err, e), c.lo);
  return r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  return x;
}

// Fixed-order block sum (deterministic); result valid in thread 0.
// scratch must hold blockDim.x/32 elements.
template <typename T>
__device__ __forceinline__ T block_sum(T x, T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  x = warp_sum(x);
  __syncthreads();
  if (lane == 0) scratch[wid] = x;
  __syncthreads();
  T r = 0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? scratch[lane] : T(0);
    r = warp_sum(r);
  }
  return r;
}

// sum_{p < np} x[p * stride] in the partials' own type, fixed order:
// partial p is added to accumulator p % 4, the accumulators are added last
// as (a0 + a1) + (a2 + a3).  FP32 partials are summed in FP32 (the FP64 pipe
// of this GPU is a small fraction of its FP32 rate).
template <typename TC>
__device__ __forceinline__ double sum_partials(const TC* __restrict__ x, size_t stride, int np) {
  TC a[4] = {TC(0), TC(0), TC(0), TC(0)};
  int p = 0;
  for (; p + 8 <= np; p += 8) {
    TC r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = x[(size_t)(p + u) * stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u & 3] += r[u];
  }
  for (; p < np; ++p) a[p & 3] += x[(size_t)p * stride];
  return (double)((a[0] + a[1]) + (a[2] + a[3]));
}

}  // namespace rttda
