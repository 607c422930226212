// Grouped serving step: one persistent kernel advances every active small
// request of the server together.
//
// A request of the serving pattern is one trajectory (one pulse) of its own
// molecule.  For small molecules the per-request step graph is launch-bound
// (about forty kernels per RK4 step, a few microseconds of work each), so
// the requests of a group are stepped by a single cooperative launch per
// chunk of steps instead: the kernel runs every phase of every RK4 stage of
// every request, with a grid-wide barrier between phases, and its CTAs take
// the work units of all requests of a phase from one shared list.
//
// Numerics are those of the library's plain BF16 path (the BF16 precision):
// factors and the amplitudes fed to the two-electron contractions rounded to
// BF16, products accumulated in FP32, the sigma assembly and the RK4 update
// in FP64, the field product of each step's start (which also gives the
// dipole expectation) in double-float arithmetic and the other stages' field
// products in FP32.  The contractions run on the warp-level tensor-core
// instruction mma.sync (m16n8k16, BF16 in, FP32 accumulate); the tiles of a
// small molecule are too small to feed the tcgen05 pipeline.
//
// Per RK4 stage s (stage input X = the engine's Xs / Xs2):
//   phase A  field F = M_d X (rows; stage 0 and pulses with a field), its
//            ground row F_0, Coulomb pass 1 w_P = sum_ia B^P_ia X_ia, and the
//            exchange intermediate Z^P_(col,i),b = sum_j B^P_ij X_(j,b),col
//   phase B  Coulomb pass 2 J_ia = 2 sum_P B^P_ia w_P, the exchange main
//            contraction K_(col,i),a = sum_{P,b} Z^P_(col,i),b B^P_ab
//            (fixed split-K partials), and at stage 0 the observables of
//            the step's start
//   phase C  sigma = (e_a - e_i) X + J - c_x K - E(t_s) F and the RK4 stage
//            update (k_combine's arithmetic), which also writes the BF16
//            copy X^T of the next stage input for the next phase A.
// Every work unit reduces in a fixed order that depends only on its own
// request's shape, so a request's results are bitwise the same whichever
// requests share the group and however the units fall on the CTAs.
//
// The grid barrier is a counter and a generation number in global memory;
// every wait on it is bounded by a wall-clock limit, after which the CTA
// records an error flag and the kernel ends (the host reports
// RTTDA_E_TIMEOUT for the group's requests).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/rttda.h"
#include "../../include/rttda_server.h"
#include "engine_internal.h"
#include "group_internal.h"

namespace rttda {
namespace grp {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per barrier wait
constexpr int kMainBM = 64, kMainBN = 64, kKC = 64;          // main contraction tile, K chunk
constexpr int kLd = kKC + 8;                                 // padded smem row (bf16): conflict-free fragments
constexpr long long kMainK = 1024;                           // K elements per main-contraction unit (split-K)
constexpr int kMainStages = 3;                               // cp.async pipeline depth of the main contraction
constexpr int kZP = kThreads / 32;                           // P values per Z-build unit (one per warp)
constexpr int kC1Rows = 8;                                   // P rows per Coulomb pass-1 unit
constexpr int kRowsPerUnit = 128;                            // amplitude rows per combine unit (2 columns)
constexpr size_t kSmemBytes = 64 * 1024;
constexpr int kMaxPhaseTicks = 4096;

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier: counter + generation; bounded spin.  Returns false when
// a wait ran out anywhere (the error flag is set).
__device__ bool grid_barrier(Barrier* b, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == nblocks - 1) {
      b->count = 0;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = gtimer();
      while (*vgen == g) {
        if (*(volatile int*)&b->err != 0) break;
        if (gtimer() - t0 > kWaitLimitNs) {
          atomicCAS(&b->err, 0, 1);
          break;
        }
      }
    }
    __threadfence();
    s_ok = *(volatile int*)&b->err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 16-byte global -> shared copy (L2 only, coherent with this kernel's own
// earlier writes); src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// all but the newest kMainStages - 2 commit groups complete
__device__ __forceinline__ void cp_wait_stages() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Loads of data that other CTAs wrote earlier in the same launch (state,
// field product, partial sums): from L2 (ld.global.cg), never through the
// non-coherent or L1 paths.
__device__ __forceinline__ double ldx(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldx(const float* p) { return __ldcg(p); }

// sum_{p < np} x[p * stride] in FP32 with k_combine's fixed order (partial p
// into accumulator p % 4, then (a0 + a1) + (a2 + a3)), from L2.
__device__ __forceinline__ double sum_parts(const float* x, size_t stride, int np) {
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  for (int p = 0; p < np; ++p) a[p & 3] += ldx(x + (size_t)p * stride);
  return (double)((a[0] + a[1]) + (a[2] + a[3]));
}

// Fixed-order block sum of nv values per thread (result in thread 0's out).
template <typename T, int NV>
__device__ void block_sums(T (&x)[NV], T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    T v = x[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    x[k] = v;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[wid * NV + k] = x[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T s = red[k];
      for (int w = 1; w < kWarps; ++w) s += red[w * NV + k];
      x[k] = s;
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Work units per phase
// ---------------------------------------------------------------------------
enum Phase : int {
  PH_KICK_INIT = 0,  // term = Xn (fresh kicked requests)
  PH_KICK_F = 1,     // F = M_d term (double-float) and its ground row (FP64)
  PH_KICK_ADD = 2,   // term = (i kappa / k) F, Xn += term
  PH_START = 3,      // Xs = Xn and its BF16 copy X^T
  PH_A = 4,
  PH_B = 5,
  PH_C = 6,
  PH_OBS_F = 7,      // the last step's field product (double-float)
  PH_OBS = 8         // the last step's observables
};

__device__ __forceinline__ int field_units(const Req& r) { return ((r.o + 7) / 8) * ((r.v + 31) / 32); }
__device__ __forceinline__ int row_units(const Req& r) { return (r.N + kRowsPerUnit - 1) / kRowsPerUnit; }
__device__ __forceinline__ int c1_units(const Req& r) { return (r.P + kC1Rows - 1) / kC1Rows; }
__device__ __forceinline__ int c2_units(const Req& r) { return (r.ov + kThreads / 8 - 1) / (kThreads / 8); }
__device__ __forceinline__ int z_units(const Req& r) { return 2 * ((r.P + kZP - 1) / kZP); }
__device__ __forceinline__ int main_units(const Req& r) {
  return r.S * ((2 * r.o + kMainBM - 1) / kMainBM) * ((r.v + kMainBN - 1) / kMainBN);
}

// Does request r take part in this phase at loop index k (step or kick term)?
__device__ __forceinline__ bool active(const Req& r, int ph, int k) {
  switch (ph) {
    case PH_KICK_INIT:
      return r.kick_terms > 0;
    case PH_KICK_F:
    case PH_KICK_ADD:
      return k < r.kick_terms;
    case PH_START:
    case PH_OBS_F:
    case PH_OBS:
      return true;
    default:
      return k < r.nsteps;
  }
}

__device__ __forceinline__ bool field_at(const Req& r, int stage) { return stage == 0 || r.field != 0; }

__device__ int unit_count(const Req& r, int ph, int k, int stage) {
  if (!active(r, ph, k)) return 0;
  switch (ph) {
    case PH_KICK_INIT:
    case PH_KICK_ADD:
    case PH_START:
    case PH_C:
      return row_units(r);
    case PH_KICK_F:
    case PH_OBS_F:
      return field_units(r) + 1;
    case PH_A:
      return (field_at(r, stage) ? field_units(r) + 1 : 0) + c1_units(r) + z_units(r);
    case PH_B:
      return c2_units(r) + main_units(r) + (stage == 0 ? 1 : 0);
    case PH_OBS:
      return 1;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Unit bodies
// ---------------------------------------------------------------------------
// Field product rows F_ia = sum_b X_ib mu_ab - sum_j mu_ji X_ja + m_ia X_0
// (both columns) for an 8 x 32 block of (i, a); TC = float (FP32 stages) or
// df32 (the step's start).  The same order of operations as k_field_small
// (b ascending, then j ascending, then the ground term); the operands come
// from shared-memory tiles: the block's 8 rows of X, mu_vv in 32 x 32 tiles
// and the X rows of 16 values of j at a time.
template <typename TM, typename TC>
__device__ void field_unit(const Req& r, int u, const double* X, const TM* moo, const TM* mvv, const TM* m0,
                           uint8_t* smem) {
  const int nab = (r.v + 31) / 32;
  const int i0 = (u / nab) * 8, a0 = (u % nab) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = i0 + ty, a = a0 + tx;
  const int v = r.v, o = r.o;
  TC* xs = reinterpret_cast<TC*>(smem);  // [2][8][v]
  TC* mt = xs + 2 * 8 * v;               // [32][32]: mu_vv[b0 + bb][a0 + aa]
  TC* xj = mt + 32 * 32;                 // [2][16][32]: X[(j0 + jj, a0 + aa)]
  TC* mo_s = xj + 2 * 16 * 32;           // [o][8]: mu_oo[j][i0 + ii]
  for (int e = threadIdx.x; e < o * 8; e += kThreads) {
    const int j = e >> 3, ii = e & 7;
    mo_s[e] = i0 + ii < o ? cvt<TC>(moo[(size_t)j * o + i0 + ii]) : TC(0);
  }
  for (int e = threadIdx.x; e < 8 * v; e += kThreads) {
    const int ii = e / v, b = e - ii * v;
    const bool ok = i0 + ii < o;
    const size_t row = 1 + (size_t)(i0 + ii) * v + b;
    xs[e] = ok ? (TC)ldx(X + row * 2) : TC(0);
    xs[8 * v + e] = ok ? (TC)ldx(X + row * 2 + 1) : TC(0);
  }
  TC fr = TC(0), fi = TC(0);
  for (int b0 = 0; b0 < v; b0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += kThreads) {
      const int bb = e >> 5, aa = e & 31;
      mt[e] = (b0 + bb < v && a0 + aa < v) ? cvt<TC>(mvv[(size_t)(b0 + bb) * v + a0 + aa]) : TC(0);
    }
    __syncthreads();
    const int nb = min(32, v - b0);
    for (int bb = 0; bb < nb; ++bb) {
      const TC mv = mt[bb * 32 + tx];
      fr = fma(xs[ty * v + b0 + bb], mv, fr);
      fi = fma(xs[8 * v + ty * v + b0 + bb], mv, fi);
    }
  }
  for (int j0 = 0; j0 < o; j0 += 16) {
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 32; e += kThreads) {
      const int jj = e >> 5, aa = e & 31;
      const bool ok = j0 + jj < o && a0 + aa < v;
      const size_t row = 1 + (size_t)(j0 + jj) * v + a0 + aa;
      xj[e] = ok ? (TC)ldx(X + row * 2) : TC(0);
      xj[512 + e] = ok ? (TC)ldx(X + row * 2 + 1) : TC(0);
    }
    __syncthreads();
    if (i < o) {
      const int nj = min(16, o - j0);
      for (int jj = 0; jj < nj; ++jj) {
        const TC mo = mo_s[(j0 + jj) * 8 + ty];
        fr = fma(-mo, xj[jj * 32 + tx], fr);
        fi = fma(-mo, xj[512 + jj * 32 + tx], fi);
      }
    }
  }
  if (a < v && i < o) {
    const TC mz = cvt<TC>(m0[(size_t)i * v + a]);
    fr = fma(mz, (TC)ldx(X), fr);
    fi = fma(mz, (TC)ldx(X + 1), fi);
    const size_t row = 1 + (size_t)i * v + a;
    r.F[row * 2] = (double)fr;
    r.F[row * 2 + 1] = (double)fi;
  }
  __syncthreads();
}

// Ground row F_0 = sum_ia m_ia X_ia in TC, fixed order.
template <typename TM, typename TC>
__device__ void field0_unit(const Req& r, const double* X, const TM* m0, uint8_t* smem) {
  TC s[2] = {TC(0), TC(0)};
  for (int ia = threadIdx.x; ia < r.ov; ia += kThreads) {
    const TC m = cvt<TC>(m0[ia]);
    s[0] = fma(m, (TC)ldx(X + (size_t)(1 + ia) * 2), s[0]);
    s[1] = fma(m, (TC)ldx(X + (size_t)(1 + ia) * 2 + 1), s[1]);
  }
  block_sums<TC, 2>(s, reinterpret_cast<TC*>(smem));
  if (threadIdx.x == 0) {
    r.F[0] = (double)s[0];
    r.F[1] = (double)s[1];
  }
}

// Coulomb pass 1: w[p][col] = sum_ia B^p_ia X_ia,col for 8 rows p (FP32).
__device__ void c1_unit(const Req& r, int u, const double* X, uint8_t* smem) {
  const int p0 = u * kC1Rows, np = min(kC1Rows, r.P - p0);
  float s[2 * kC1Rows];
#pragma unroll
  for (int k = 0; k < 2 * kC1Rows; ++k) s[k] = 0.f;
#pragma unroll 4
  for (int ia = threadIdx.x; ia < r.ov; ia += kThreads) {
    const float x0 = (float)ldx(X + (size_t)(1 + ia) * 2), x1 = (float)ldx(X + (size_t)(1 + ia) * 2 + 1);
#pragma unroll
    for (int p = 0; p < kC1Rows; ++p) {
      if (p < np) {
        const float b = __bfloat162float(r.Bov[(size_t)(p0 + p) * r.ov + ia]);
        s[2 * p] = fmaf(b, x0, s[2 * p]);
        s[2 * p + 1] = fmaf(b, x1, s[2 * p + 1]);
      }
    }
  }
  block_sums<float, 2 * kC1Rows>(s, reinterpret_cast<float*>(smem));
  if (threadIdx.x == 0)
    for (int p = 0; p < np; ++p) {
      r.w[(size_t)(p0 + p) * 2] = s[2 * p];
      r.w[(size_t)(p0 + p) * 2 + 1] = s[2 * p + 1];
    }
}

// Coulomb pass 2: J[ia][col] = 2 sum_p B^p_ia w[p][col] for 32 rows ia; eight
// threads per row sum the p of one residue mod 8 each, and the eight sums are
// added in a fixed tree ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7)).
__device__ void c2_unit(const Req& r, int u, uint8_t* smem) {
  float* ws = reinterpret_cast<float*>(smem);
  for (int e = threadIdx.x; e < 2 * r.P; e += kThreads) ws[e] = ldx(r.w + e);
  __syncthreads();
  const int lane8 = threadIdx.x & 7;
  const int ia = u * (kThreads / 8) + (threadIdx.x >> 3);
  float j0 = 0.f, j1 = 0.f;
  if (ia < r.ov) {
#pragma unroll 4
    for (int p = lane8; p < r.P; p += 8) {
      const float b = __bfloat162float(r.Bov[(size_t)p * r.ov + ia]);
      j0 = fmaf(b, ws[2 * p], j0);
      j1 = fmaf(b, ws[2 * p + 1], j1);
    }
  }
  // fixed tree within each group of eight lanes
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) {
    j0 += __shfl_down_sync(0xffffffffu, j0, off);
    j1 += __shfl_down_sync(0xffffffffu, j1, off);
  }
  if (ia < r.ov && lane8 == 0) {
    r.J[(size_t)ia * 2] = 2.f * j0;
    r.J[(size_t)ia * 2 + 1] = 2.f * j1;
  }
  __syncthreads();
}

// Exchange intermediate for kZP values of P (one per warp) and one column:
// Z^P[(col, i)][b] = sum_j B^P_ij X_(j,b),col  (M = i, N = b, K = j).  The
// column's X^T tile is staged in shared memory once per unit; each warp reads
// its P's B_oo fragments straight from L2 and runs its MMAs without CTA-wide
// synchronisation; BF16 operands, FP32 accumulate, stored as BF16.
__device__ void z_unit(const Req& r, int u, uint8_t* smem) {
  const int col = u & 1, pg = u >> 1;
  const int op = r.op, vp = r.vp, o = r.o, M = 2 * r.o;
  const int ld = op + 8;
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem);  // [vp][ld]: X^T of this column
  const int cpr = op / 8;                                      // 16-byte chunks per row
  for (int e = threadIdx.x; e < vp * cpr; e += kThreads) {
    const int b = e / cpr, c = e - b * cpr;
    cp16(xs + (size_t)b * ld + 8 * c, r.Xt + ((size_t)col * vp + b) * op + 8 * c, 16);
  }
  cp_commit();
  cp_wait0();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  const int P = pg * kZP + warp;
  if (P < r.P) {
    const int mt = op / 16, nt = vp / 8, ks = op / 16;
    for (int mi = 0; mi < mt; ++mi) {
      // A fragments of rows mi*16.. for every k step (zero past nocc)
      uint32_t af[4][4];
      const int i_lo = mi * 16 + g, i_hi = i_lo + 8;
      const uint32_t* rlo = reinterpret_cast<const uint32_t*>(r.Boo + ((size_t)P * o + min(i_lo, o - 1)) * op);
      const uint32_t* rhi = reinterpret_cast<const uint32_t*>(r.Boo + ((size_t)P * o + min(i_hi, o - 1)) * op);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k < ks) {
          const int w0 = (k * 16 + 2 * tg) / 2, w1 = w0 + 4;
          af[k][0] = i_lo < o ? rlo[w0] : 0u;
          af[k][1] = i_hi < o ? rhi[w0] : 0u;
          af[k][2] = i_lo < o ? rlo[w1] : 0u;
          af[k][3] = i_hi < o ? rhi[w1] : 0u;
        }
      }
      for (int ni = 0; ni < nt; ++ni) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const __nv_bfloat16* br = xs + (size_t)(ni * 8 + g) * ld + 2 * tg;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < ks) mma16816(d, af[k][0], af[k][1], af[k][2], af[k][3], lds32(br + k * 16), lds32(br + k * 16 + 8));
        const int b = ni * 8 + 2 * tg;
        if (i_lo < o)
          *reinterpret_cast<__nv_bfloat162*>(r.Z + ((size_t)P * M + col * o + i_lo) * vp + b) =
              __floats2bfloat162_rn(d[0], d[1]);
        if (i_hi < o)
          *reinterpret_cast<__nv_bfloat162*>(r.Z + ((size_t)P * M + col * o + i_hi) * vp + b) =
              __floats2bfloat162_rn(d[2], d[3]);
      }
    }
  }
  __syncthreads();
}

// Exchange main contraction, one 64 x 64 tile of K_(col,i),a over the K
// chunks of split s: K = (P, b) in chunks of 32 (never across two P), A = Z
// rows, B = B_vv rows (B^P_ab symmetric, stored [P][a][b]).  A four-stage
// cp.async ring of tiles; 8 warps as 2 (rows) x 4 (columns), each 32 x 16.
__device__ void main_unit(const Req& r, int u, uint8_t* smem) {
  const int M = 2 * r.o, vp = r.vp;
  const int ntn = (r.v + kMainBN - 1) / kMainBN, ntm = (M + kMainBM - 1) / kMainBM;
  const int nt = u % ntn, mt = (u / ntn) % ntm, s = u / (ntn * ntm);
  const int m0 = mt * kMainBM, n0 = nt * kMainBN;
  const int vt = vp / kKC;
  const int KT = r.P * vt;
  const int per = (KT + r.S - 1) / r.S;
  const int kc0 = s * per, kc1 = min(KT, kc0 + per);
  __nv_bfloat16* as = reinterpret_cast<__nv_bfloat16*>(smem);  // [kMainStages][64][kLd]
  __nv_bfloat16* bsh = as + kMainStages * kMainBM * kLd;        // [kMainStages][64][kLd]
  auto load = [&](int kc, int buf) {
    const int P = kc / vt, kb = (kc - P * vt) * kKC;
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // 64 rows x 8 chunks of 8 per operand
      const int e = threadIdx.x + h * kThreads, row = e >> 3, ch = e & 7;
      const int b0 = kb + 8 * ch;
      const bool okA = m0 + row < M, okB = n0 + row < r.v;
      cp16(as + ((size_t)buf * kMainBM + row) * kLd + 8 * ch,
           r.Z + ((size_t)P * M + (okA ? m0 + row : 0)) * vp + b0, okA ? 16 : 0);
      cp16(bsh + ((size_t)buf * kMainBN + row) * kLd + 8 * ch,
           r.Bvv + ((size_t)P * vp + (okB ? n0 + row : 0)) * vp + b0, okB ? 16 : 0);
    }
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tg = lane & 3;
  const int wm = warp >> 2, wn = warp & 3;
  float acc[2][2][4];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int z = 0; z < 4; ++z) acc[x][y][z] = 0.f;
  // pipeline: chunks kc0 .. kc0 + kMainStages - 2 in flight before the first
  // is consumed; one commit group per chunk (empty groups past the end keep
  // the group count uniform)
#pragma unroll
  for (int q = 0; q < kMainStages - 1; ++q) {
    if (kc0 + q < kc1) load(kc0 + q, q);
    cp_commit();
  }
  for (int kc = kc0; kc < kc1; ++kc) {
    const int buf = (kc - kc0) % kMainStages;
    cp_wait_stages();
    __syncthreads();
    {
      const int nk = kc + kMainStages - 1;
      if (nk < kc1) load(nk, (nk - kc0) % kMainStages);
      cp_commit();
    }
    const __nv_bfloat16* A = as + (size_t)buf * kMainBM * kLd;
    const __nv_bfloat16* B = bsh + (size_t)buf * kMainBN * kLd;
#pragma unroll
    for (int k0 = 0; k0 < kKC; k0 += 16) {
      uint32_t af[2][4], bf[2][2];
#pragma unroll
      for (int im = 0; im < 2; ++im) {
        const __nv_bfloat16* ap = A + (size_t)(wm * 32 + im * 16 + g) * kLd + k0 + 2 * tg;
        af[im][0] = lds32(ap);
        af[im][1] = lds32(ap + 8 * kLd);
        af[im][2] = lds32(ap + 8);
        af[im][3] = lds32(ap + 8 * kLd + 8);
      }
#pragma unroll
      for (int in = 0; in < 2; ++in) {
        const __nv_bfloat16* bp = B + (size_t)(wn * 16 + in * 8 + g) * kLd + k0 + 2 * tg;
        bf[in][0] = lds32(bp);
        bf[in][1] = lds32(bp + 8);
      }
#pragma unroll
      for (int im = 0; im < 2; ++im)
#pragma unroll
        for (int in = 0; in < 2; ++in)
          mma16816(acc[im][in], af[im][0], af[im][1], af[im][2], af[im][3], bf[in][0], bf[in][1]);
    }
  }
  cp_wait0();
  __syncthreads();
  float* out = r.Kp + (size_t)s * M * r.v;
#pragma unroll
  for (int im = 0; im < 2; ++im)
#pragma unroll
    for (int in = 0; in < 2; ++in) {
      const int rr = m0 + wm * 32 + im * 16 + g, cc = n0 + wn * 16 + in * 8 + 2 * tg;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = rr + 8 * h;
        if (m < M) {
          if (cc < r.v) out[(size_t)m * r.v + cc] = acc[im][in][2 * h];
          if (cc + 1 < r.v) out[(size_t)m * r.v + cc + 1] = acc[im][in][2 * h + 1];
        }
      }
    }
}

// Observables of the state Xn with the field product F = M_d Xn: the dipole
// Re Xn^dagger F and the norm, FP64, fixed order, written at trace index k.
__device__ void obs_unit(const Req& r, long long k, uint8_t* smem) {
  double s[2] = {0.0, 0.0};
  for (int n = threadIdx.x; n < r.N; n += kThreads) {
    const double xr = ldx(r.Xn + (size_t)n * 2), xi = ldx(r.Xn + (size_t)n * 2 + 1);
    s[0] = fma(xr, ldx(r.F + (size_t)n * 2), s[0]);
    s[0] = fma(xi, ldx(r.F + (size_t)n * 2 + 1), s[0]);
    s[1] = fma(xr, xr, s[1]);
    s[1] = fma(xi, xi, s[1]);
  }
  block_sums<double, 2>(s, reinterpret_cast<double*>(smem));
  if (threadIdx.x == 0) {
    r.dip[r.trace_off + k] = s[0];
    r.nrm[r.trace_off + k] = s[1];
  }
}

// BF16 copy of one element of a stage input: X^T[col][b][j] for row n = 1 + j v + b.
__device__ __forceinline__ void put_xt(const Req& r, int n, int col, double x) {
  if (n == 0) return;
  const int j = (n - 1) / r.v, b = (n - 1) - j * r.v;
  r.Xt[((size_t)col * r.vp + b) * r.op + j] = __float2bfloat16_rn((float)x);
}

// sigma assembly and RK4 stage update of 128 rows (k_combine's arithmetic,
// one split of the Coulomb term, S splits of the exchange).
__device__ void combine_unit(const Req& r, int u, int stage, long long step) {
  const int n = u * kRowsPerUnit + (threadIdx.x >> 1), q = threadIdx.x & 1;
  if (n >= r.N) return;
  const double* Xin = (stage % 2 == 0) ? r.Xs : r.Xs2;
  double* Xnext = (stage % 2 == 0) ? r.Xs2 : r.Xs;
  const size_t idx = (size_t)n * 2 + q;
  double sg = 0.0;
  if (n > 0) {
    const int i = (n - 1) / r.v, a = (n - 1) - i * r.v;
    const double jsum = sum_parts(r.J + (size_t)(n - 1) * 2 + q, (size_t)r.ov * 2, 1);
    const double ksum = sum_parts(r.Kp + ((size_t)q * r.o + i) * r.v + a, (size_t)2 * r.o * r.v, r.S);
    sg = (r.eps_v[a] - r.eps_o[i]) * ldx(Xin + idx) + jsum - r.cx * ksum;
  }
  if (r.field) {
    const double cs[4] = {0.0, 0.5, 0.5, 1.0};
    const double E = pulse_field(r.pulse, ((double)(r.step0 + step) + cs[stage]) * r.dt);
    sg -= E * ldx(r.F + idx);
  }
  const size_t kidx = (size_t)n * 2 + (1 - q);
  const double kv = q == 0 ? -sg : sg;
  const double dt = r.dt;
  double xn;
  switch (stage) {
    case 0:
      r.acc[kidx] = kv;
      xn = ldx(r.Xn + kidx) + 0.5 * dt * kv;
      break;
    case 1:
      r.acc[kidx] = ldx(r.acc + kidx) + 2.0 * kv;
      xn = ldx(r.Xn + kidx) + 0.5 * dt * kv;
      break;
    case 2:
      r.acc[kidx] = ldx(r.acc + kidx) + 2.0 * kv;
      xn = ldx(r.Xn + kidx) + dt * kv;
      break;
    default:
      xn = ldx(r.Xn + kidx) + (dt / 6.0) * (ldx(r.acc + kidx) + kv);
      r.Xn[kidx] = xn;
  }
  Xnext[kidx] = xn;
  put_xt(r, n, (int)(1 - q), xn);
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
__device__ void run_unit(const Req& r, int ph, int u, int k, int stage, uint8_t* smem) {
  switch (ph) {
    case PH_KICK_INIT: {
      const int n = u * kRowsPerUnit + (threadIdx.x >> 1), q = threadIdx.x & 1;
      if (n < r.N) r.term[(size_t)n * 2 + q] = ldx(r.Xn + (size_t)n * 2 + q);
      return;
    }
    case PH_KICK_F:
    case PH_OBS_F: {
      const double* X = ph == PH_KICK_F ? r.term : r.Xn;
      const int nf = field_units(r);
      if (u < nf)
        field_unit<double, df32>(r, u, X, r.moo64, r.mvv64, r.m064, smem);
      else
        field0_unit<double, double>(r, X, r.m064, smem);
      return;
    }
    case PH_KICK_ADD: {
      const int n = u * kRowsPerUnit + (threadIdx.x >> 1), q = threadIdx.x & 1;
      if (n >= r.N) return;
      // (i s) (fr + i fi) with s = kappa / k (k_kick_term's arithmetic)
      const double s = r.kappa * (1.0 / (double)(k + 1));
      const size_t ir = (size_t)n * 2;
      const double fr = ldx(r.F + ir), fi = ldx(r.F + ir + 1);
      const double t = q == 0 ? -s * fi : s * fr;
      r.term[ir + q] = t;
      r.Xn[ir + q] = ldx(r.Xn + ir + q) + t;
      return;
    }
    case PH_START: {
      const int n = u * kRowsPerUnit + (threadIdx.x >> 1), q = threadIdx.x & 1;
      if (n >= r.N) return;
      const double x = ldx(r.Xn + (size_t)n * 2 + q);
      r.Xs[(size_t)n * 2 + q] = x;
      put_xt(r, n, q, x);
      return;
    }
    case PH_A: {
      const double* X = (stage % 2 == 0) ? r.Xs : r.Xs2;
      if (field_at(r, stage)) {
        const int nf = field_units(r);
        if (u < nf) {
          if (stage == 0)
            field_unit<double, df32>(r, u, X, r.moo64, r.mvv64, r.m064, smem);
          else
            field_unit<float, float>(r, u, X, r.mooF, r.mvvF, r.m0F, smem);
          return;
        }
        u -= nf;
        if (u == 0) {
          if (stage == 0)
            field0_unit<double, double>(r, X, r.m064, smem);
          else
            field0_unit<float, float>(r, X, r.m0F, smem);
          return;
        }
        u -= 1;
      }
      const int n1 = c1_units(r);
      if (u < n1) {
        c1_unit(r, u, X, smem);
        return;
      }
      z_unit(r, u - n1, smem);
      return;
    }
    case PH_B: {
      const int n2 = c2_units(r), nm = main_units(r);
      if (u < n2) {
        c2_unit(r, u, smem);
        return;
      }
      u -= n2;
      if (u < nm) {
        main_unit(r, u, smem);
        return;
      }
      obs_unit(r, k, smem);  // stage 0 only
      return;
    }
    case PH_C:
      combine_unit(r, u, stage, k);
      return;
    case PH_OBS:
      obs_unit(r, r.nsteps, smem);
      return;
  }
}

// Run every unit of one phase over all requests; units are dealt to the
// CTAs round-robin in request order.
__device__ void run_phase(const Table& tb, int ph, int k, int stage, uint8_t* smem) {
  int total = 0;
  for (int q = 0; q < tb.nreq; ++q) total += unit_count(tb.req[q], ph, k, stage);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    int q = 0, rem = u;
    for (;; ++q) {
      const int c = unit_count(tb.req[q], ph, k, stage);
      if (rem < c) break;
      rem -= c;
    }
    run_unit(tb.req[q], ph, rem, k, stage, smem);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 3) k_group_chunk(const Table* __restrict__ tbp) {
  extern __shared__ __align__(16) uint8_t smem[];
  const Table& tb = *tbp;
  Barrier* bar = tb.bar;
  const unsigned nb = gridDim.x;
  // optional phase clock: CTA 0 records %globaltimer after every barrier
  int tick = 0;
  auto grid_barrier = [&](Barrier* b, unsigned n) {
    const bool ok = grp::grid_barrier(b, n);
    if (tb.phase_ns && blockIdx.x == 0 && threadIdx.x == 0 && tick < kMaxPhaseTicks) tb.phase_ns[tick++] = gtimer();
    return ok;
  };
  // kick of the requests starting in this chunk (exact exp(i kappa M_d)|0>
  // by its Taylor series, every term's field product in double-float)
  if (tb.kick_terms > 0) {
    run_phase(tb, PH_KICK_INIT, 0, 0, smem);
    if (!grid_barrier(bar, nb)) return;
    for (int k = 0; k < tb.kick_terms; ++k) {
      run_phase(tb, PH_KICK_F, k, 0, smem);
      if (!grid_barrier(bar, nb)) return;
      run_phase(tb, PH_KICK_ADD, k, 0, smem);
      if (!grid_barrier(bar, nb)) return;
    }
  }
  run_phase(tb, PH_START, 0, 0, smem);
  if (!grid_barrier(bar, nb)) return;
  for (int k = 0; k < tb.max_steps; ++k) {
    for (int st = 0; st < 4; ++st) {
      run_phase(tb, PH_A, k, st, smem);
      if (!grid_barrier(bar, nb)) return;
      run_phase(tb, PH_B, k, st, smem);
      if (!grid_barrier(bar, nb)) return;
      run_phase(tb, PH_C, k, st, smem);
      if (!grid_barrier(bar, nb)) return;
    }
  }
  run_phase(tb, PH_OBS_F, 0, 0, smem);
  if (!grid_barrier(bar, nb)) return;
  run_phase(tb, PH_OBS, 0, 0, smem);
}

// dst[e] = sum_x d_x src[x][e] (direction-combined dipole block, FP64) and
// its FP32 copy.
__global__ void k_dir_combine(long long n, double d0, double d1, double d2, const double* __restrict__ src,
                              double* __restrict__ dst, float* __restrict__ dstf) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double x = d0 * src[e] + d1 * src[n + e] + d2 * src[2 * n + e];
  dst[e] = x;
  dstf[e] = (float)x;
}

// BF16 copy of an FP64 array [lead][rows][cols] into [lead] slabs of pitch
// lds with rows of pitch ldr (padding left as it is: zero).
__global__ void k_bf16_pad(long long lead, int rows, int cols, int ldr, long long lds,
                           const double* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)rows * cols;
  if (e >= lead * per) return;
  const long long l = e / per;
  const long long rc = e - l * per;
  const int r = (int)(rc / cols), c = (int)(rc - (long long)r * cols);
  dst[l * lds + (long long)r * ldr + c] = __float2bfloat16_rn((float)src[e]);
}

}  // namespace grp

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

inline long long cdivl(long long a, long long b) { return (a + b - 1) / b; }
inline unsigned nblk(long long n) { return (unsigned)std::max<long long>(1, cdivl(n, 256)); }

double fro_host(const double* a, size_t n) {
  double s = 0.0;
  for (size_t k = 0; k < n; ++k) s += a[k] * a[k];
  return std::sqrt(s);
}

}  // namespace

double group_work(const rttda_request& q) { return (double)q.nocc * q.nvirt * q.nvirt * q.naux; }

bool group_eligible(const rttda_request& q) {
  // small BF16 requests whose step is launch-bound: exchange work
  // nocc nvirt^2 naux multiply-adds per column at most kMaxWork (measured:
  // grouped steps beat one handle per request up to about nocc 32, nvirt 128,
  // naux 512, and lose beyond)
  return q.prec == RTTDA_BF16 && q.nocc <= grp::kMaxO && q.nvirt <= grp::kMaxV && q.naux <= grp::kMaxP &&
         (double)q.nocc * q.nvirt * q.nvirt * q.naux <= grp::kMaxWork;
}

size_t group_estimate_bytes(const rttda_request& q) {
  const long long o = q.nocc, v = q.nvirt, P = q.naux;
  const long long op = cdivl(o, 16) * 16, vp = cdivl(v, grp::kKC) * grp::kKC, ov = o * v, N = 1 + ov;
  const long long KT = P * (vp / grp::kKC);
  const long long S = std::max<long long>(1, cdivl(KT * grp::kKC, grp::kMainK));
  size_t b = 0;
  b += 8 * (o + v);                                      // orbital energies
  b += 2 * (P * ov + P * o * op + P * vp * vp);          // BF16 factors
  b += 8 * (o * o + v * v + ov) + 4 * (o * o + v * v + ov);  // dipole blocks
  b += 8 * 2 * N * 6;                                    // Xn Xs Xs2 acc F term
  b += 2 * 2 * vp * op + 2 * P * 2 * o * vp;             // X^T, Z
  b += 4 * (2 * P + 2 * ov + S * 2 * o * v);             // w, J, K partials
  b += 8 * 2 * (q.nsteps + 1);                           // traces
  return b + (1 << 20);
}

rttda_status group_admit(const rttda_request& q, cudaStream_t s, GroupReq** out) {
  using namespace grp;
  *out = nullptr;
  auto g = std::make_unique<GroupReq>();
  Req& r = g->r;
  const int o = q.nocc, v = q.nvirt, P = q.naux;
  r.o = o;
  r.v = v;
  r.P = P;
  r.op = (int)cdivl(o, 16) * 16;
  r.vp = (int)cdivl(v, grp::kKC) * grp::kKC;
  r.ov = o * v;
  r.N = 1 + o * v;
  const long long KT = (long long)P * (r.vp / kKC);
  r.S = (int)std::max<long long>(1, cdivl(KT * kKC, kMainK));
  r.cx = q.c_x;
  r.dt = q.dt;
  // pulse (as rttda_set_field)
  const rttda_pulse& p = q.pulse;
  const double dn = std::sqrt(p.dir[0] * p.dir[0] + p.dir[1] * p.dir[1] + p.dir[2] * p.dir[2]);
  if (!(dn > 0.0) || !std::isfinite(dn)) return set_error(RTTDA_E_ARG, "grouped request: zero polarisation vector");
  if ((p.kind == RTTDA_GAUSS_TL || p.kind == RTTDA_CHIRP) && !(p.fwhm > 0.0))
    return set_error(RTTDA_E_ARG, "grouped request: fwhm must be > 0");
  if (p.kind == RTTDA_SIN2 && !(p.duration > 0.0))
    return set_error(RTTDA_E_ARG, "grouped request: duration must be > 0");
  double dir[3];
  for (int x = 0; x < 3; ++x) dir[x] = p.dir[x] / dn;
  r.pulse.kind = p.kind;
  r.pulse.E0 = p.E0;
  r.pulse.omega = p.omega;
  r.pulse.t0 = p.t0;
  r.pulse.sigma = p.fwhm / 2.35482;  // Sec. 2.2: sigma = FWHM / 2.35482
  r.pulse.beta = p.beta;
  r.pulse.duration = p.duration;
  r.field = p.kind != RTTDA_KICK;
  // Taylor length of the kick: x^K / K! < 1e-18 for the bound
  // x = kappa sum_x |d_x| (|m_x| + |mu_vv,x| + |mu_oo,x|) on |kappa M_d|
  if (p.kind == RTTDA_KICK) {
    r.kappa = p.E0;
    // host copies of the dipole blocks (the sources may be host or device)
    std::vector<double> hm0((size_t)3 * o * v), hmv((size_t)3 * v * v), hmo((size_t)3 * o * o);
    if (cudaMemcpy(hm0.data(), q.mu_0ov, 8 * hm0.size(), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(hmv.data(), q.mu_vv, 8 * hmv.size(), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(hmo.data(), q.mu_oo, 8 * hmo.size(), cudaMemcpyDefault) != cudaSuccess)
      return set_error(RTTDA_E_CUDA, "grouped request: reading the dipole blocks failed");
    double b = 0.0;
    for (int x = 0; x < 3; ++x)
      b += std::fabs(dir[x]) * (fro_host(hm0.data() + (size_t)x * o * v, (size_t)o * v) +
                                fro_host(hmv.data() + (size_t)x * v * v, (size_t)v * v) +
                                fro_host(hmo.data() + (size_t)x * o * o, (size_t)o * o));
    const double xmax = std::fabs(p.E0) * b;
    int K = 0;
    double term = 1.0;
    while (K < 400) {
      ++K;
      term *= xmax / K;
      if (term < 1e-18 && K > xmax) break;
    }
    if (K >= 400) return set_error(RTTDA_E_ARG, "grouped request: kick too strong for the Taylor series");
    g->kick_terms = K;
  }

  // device buffers (stream-ordered, freed in group_release)
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMallocAsync(ptr, bytes, s) != cudaSuccess) return false;
    g->allocs.push_back(*ptr);
    return cudaMemsetAsync(*ptr, 0, bytes, s) == cudaSuccess;
  };
  const size_t N = (size_t)r.N, ov = (size_t)r.ov;
  double *eo = nullptr, *ev = nullptr, *tmp = nullptr, *mu3 = nullptr;
  bool ok = alloc((void**)&eo, 8 * o) && alloc((void**)&ev, 8 * v);
  __nv_bfloat16 *bov = nullptr, *boo = nullptr, *bvv = nullptr, *xt = nullptr, *z = nullptr;
  ok = ok && alloc((void**)&bov, 2 * (size_t)P * ov) && alloc((void**)&boo, 2 * (size_t)P * o * r.op) &&
       alloc((void**)&bvv, 2 * (size_t)P * r.vp * r.vp);
  double *moo64 = nullptr, *mvv64 = nullptr, *m064 = nullptr;
  float *mooF = nullptr, *mvvF = nullptr, *m0F = nullptr;
  ok = ok && alloc((void**)&moo64, 8 * (size_t)o * o) && alloc((void**)&mvv64, 8 * (size_t)v * v) &&
       alloc((void**)&m064, 8 * ov) && alloc((void**)&mooF, 4 * (size_t)o * o) &&
       alloc((void**)&mvvF, 4 * (size_t)v * v) && alloc((void**)&m0F, 4 * ov);
  double* st[6] = {};
  for (int k = 0; k < 6 && ok; ++k) ok = alloc((void**)&st[k], 16 * N);
  float *w = nullptr, *J = nullptr, *Kp = nullptr;
  ok = ok && alloc((void**)&xt, 2 * 2 * (size_t)r.vp * r.op) && alloc((void**)&z, 2 * (size_t)P * 2 * o * r.vp) &&
       alloc((void**)&w, 4 * 2 * (size_t)P) && alloc((void**)&J, 4 * 2 * ov) &&
       alloc((void**)&Kp, 4 * (size_t)r.S * 2 * o * v);
  ok = ok && alloc((void**)&g->trace, 8 * 2 * (size_t)(q.nsteps + 1));
  // staging for the FP64 uploads (the largest factor)
  const size_t stage_n = std::max({(size_t)P * v * v, (size_t)P * ov, (size_t)P * o * o});
  ok = ok && cudaMallocAsync((void**)&tmp, 8 * stage_n, s) == cudaSuccess;
  ok = ok && cudaMallocAsync((void**)&mu3, 8 * (size_t)3 * v * v, s) == cudaSuccess;
  auto cleanup_tmp = [&]() {
    if (tmp) cudaFreeAsync(tmp, s);
    if (mu3) cudaFreeAsync(mu3, s);
  };
  if (!ok) {
    cleanup_tmp();
    group_release(g.release(), s);
    return set_error(RTTDA_E_OOM, "grouped request: device allocation failed");
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](double* dst, const double* src, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, 8 * n, cudaMemcpyDefault, s);  // host or device source
  };
  up(eo, q.eps_occ, o);
  up(ev, q.eps_virt, v);
  up(tmp, q.B_ov, (size_t)P * ov);
  if (e == cudaSuccess)
    grp::k_bf16_pad<<<nblk((long long)P * ov), 256, 0, s>>>(P, 1, (int)ov, (int)ov, (long long)ov, tmp, bov);
  up(tmp, q.B_oo, (size_t)P * o * o);
  if (e == cudaSuccess)
    grp::k_bf16_pad<<<nblk((long long)P * o * o), 256, 0, s>>>(P, o, o, r.op, (long long)o * r.op, tmp, boo);
  up(tmp, q.B_vv, (size_t)P * v * v);
  if (e == cudaSuccess)
    grp::k_bf16_pad<<<nblk((long long)P * v * v), 256, 0, s>>>(P, v, v, r.vp, (long long)r.vp * r.vp, tmp, bvv);
  up(mu3, q.mu_oo, (size_t)3 * o * o);
  if (e == cudaSuccess)
    grp::k_dir_combine<<<nblk((long long)o * o), 256, 0, s>>>((long long)o * o, dir[0], dir[1], dir[2], mu3, moo64,
                                                               mooF);
  up(mu3, q.mu_vv, (size_t)3 * v * v);
  if (e == cudaSuccess)
    grp::k_dir_combine<<<nblk((long long)v * v), 256, 0, s>>>((long long)v * v, dir[0], dir[1], dir[2], mu3, mvv64,
                                                               mvvF);
  up(mu3, q.mu_0ov, (size_t)3 * ov);
  if (e == cudaSuccess)
    grp::k_dir_combine<<<nblk((long long)ov), 256, 0, s>>>((long long)ov, dir[0], dir[1], dir[2], mu3, m064, m0F);
  if (e == cudaSuccess) {
    // ground state |0>
    const double one = 1.0;
    e = cudaMemcpyAsync(st[0], &one, 8, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host sources may be freed after return
  cleanup_tmp();
  if (e != cudaSuccess) {
    group_release(g.release(), s);
    return set_error(RTTDA_E_CUDA, std::string("grouped request: upload: ") + cudaGetErrorString(e));
  }
  r.eps_o = eo;
  r.eps_v = ev;
  r.Bov = bov;
  r.Boo = boo;
  r.Bvv = bvv;
  r.moo64 = moo64;
  r.mvv64 = mvv64;
  r.m064 = m064;
  r.mooF = mooF;
  r.mvvF = mvvF;
  r.m0F = m0F;
  r.Xn = st[0];
  r.Xs = st[1];
  r.Xs2 = st[2];
  r.acc = st[3];
  r.F = st[4];
  r.term = st[5];
  r.Xt = xt;
  r.Z = z;
  r.w = w;
  r.J = J;
  r.Kp = Kp;
  r.dip = g->trace;
  r.nrm = g->trace + (q.nsteps + 1);
  *out = g.release();
  return RTTDA_OK;
}

void group_release(GroupReq* g, cudaStream_t s) {
  if (!g) return;
  for (void* p : g->allocs)
    if (p) cudaFreeAsync(p, s);
  delete g;
}

rttda_status group_runner_init(GroupRunner* g) {
  using namespace grp;
  int dev = 0, coop = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_group_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_group_chunk, kThreads, kSmemBytes);
  if (e != cudaSuccess) return set_error(RTTDA_E_CUDA, std::string("grouped step: ") + cudaGetErrorString(e));
  if (!coop || occ < 1) return set_error(RTTDA_E_CUDA, "grouped step: cooperative launch unavailable");
  g->grid = nsm * occ;
  g->nsm = nsm;
  // diagnostics: RTTDA_GROUP_PHASE_CLOCK=<file> appends, after every chunk,
  // the device clock (ns) of each grid barrier relative to the first
  const char* pc = std::getenv("RTTDA_GROUP_PHASE_CLOCK");
  if (pc && *pc) {
    if ((e = cudaMalloc((void**)&g->phase_ns, 8 * kMaxPhaseTicks)) != cudaSuccess)
      return set_error(RTTDA_E_CUDA, std::string("grouped step: ") + cudaGetErrorString(e));
    g->phase_file = pc;
  }
  if ((e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&g->upload, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc((void**)&g->d_table, sizeof(Table))) != cudaSuccess ||
      (e = cudaMalloc((void**)&g->d_bar, sizeof(Barrier))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&g->h_table, sizeof(Table))) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming)) != cudaSuccess) {
    group_runner_free(g);
    return set_error(RTTDA_E_CUDA, std::string("grouped step: set-up: ") + cudaGetErrorString(e));
  }
  return RTTDA_OK;
}

void group_runner_free(GroupRunner* g) {
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->d_table) cudaFree(g->d_table);
  if (g->d_bar) cudaFree(g->d_bar);
  if (g->phase_ns) cudaFree(g->phase_ns);
  if (g->h_table) cudaFreeHost(g->h_table);
  if (g->upload) cudaStreamSynchronize(g->upload);
  if (g->ev) cudaEventDestroy(g->ev);
  if (g->stream) cudaStreamDestroy(g->stream);
  if (g->upload) cudaStreamDestroy(g->upload);
  *g = GroupRunner{};
}

rttda_status group_launch(GroupRunner* g, const std::vector<GroupReq*>& reqs, const std::vector<long>& nsteps,
                          const std::vector<long>& done, const std::vector<int>& fresh) {
  using namespace grp;
  if (reqs.empty()) return RTTDA_OK;
  if ((int)reqs.size() > kMaxGroup) return set_error(RTTDA_E_ARG, "grouped step: too many requests in a group");
  Table* t = g->h_table;
  t->nreq = (int)reqs.size();
  t->max_steps = 0;
  t->kick_terms = 0;
  t->bar = g->d_bar;
  for (size_t k = 0; k < reqs.size(); ++k) {
    Req r = reqs[k]->r;
    r.nsteps = (int)nsteps[k];
    r.step0 = done[k];
    r.trace_off = done[k];
    r.kick_terms = fresh[k] ? reqs[k]->kick_terms : 0;
    t->req[k] = r;
    t->max_steps = std::max(t->max_steps, r.nsteps);
    t->kick_terms = std::max(t->kick_terms, r.kick_terms);
  }
  t->phase_ns = g->phase_ns;
  // Grid sized by the group's work: a small group takes a share of the SMs
  // (at least 16) and leaves the rest to the requests stepped on their own
  // handles, which run concurrently on other streams; a group of half the
  // work cap or more takes all of them.  Results do not depend on the grid
  // (the CTAs only take work units in turn; every sum has a fixed order).
  double work = 0.0;
  for (int k = 0; k < t->nreq; ++k) work += (double)t->req[k].o * t->req[k].v * t->req[k].v * t->req[k].P;
  const int occ = std::max(1, g->grid / std::max(1, g->nsm));
  const int nsm = std::min(g->nsm, std::max(16, (int)std::ceil(2.0 * g->nsm * work / kMaxGroupWork)));
  const unsigned grid = (unsigned)std::min(g->grid, nsm * occ);
  cudaError_t e = cudaMemcpyAsync(g->d_table, t, sizeof(Table), cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_bar, 0, sizeof(Barrier), g->stream);
  if (e == cudaSuccess && g->phase_ns) e = cudaMemsetAsync(g->phase_ns, 0, 8 * kMaxPhaseTicks, g->stream);
  if (e == cudaSuccess) {
    const Table* arg = g->d_table;
    void* args[] = {(void*)&arg};
    e = cudaLaunchCooperativeKernel((void*)k_group_chunk, dim3(grid), dim3(kThreads), args, kSmemBytes, g->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(g->ev, g->stream);
  if (e != cudaSuccess) return set_error(RTTDA_E_CUDA, std::string("grouped step: launch: ") + cudaGetErrorString(e));
  return RTTDA_OK;
}

rttda_status group_status(GroupRunner* g) {
  grp::Barrier b{};
  cudaError_t e = cudaMemcpyAsync(&b, g->d_bar, sizeof(b), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return set_error(RTTDA_E_CUDA, std::string("grouped step: ") + cudaGetErrorString(e));
  if (b.err) return set_error(RTTDA_E_TIMEOUT, "grouped step: a grid barrier wait ran out");
  if (g->phase_ns) {
    std::vector<unsigned long long> t(grp::kMaxPhaseTicks);
    if (cudaMemcpy(t.data(), g->phase_ns, 8 * t.size(), cudaMemcpyDeviceToHost) == cudaSuccess) {
      if (FILE* f = std::fopen(g->phase_file, "a")) {
        for (size_t k = 1; k < t.size() && t[k]; ++k) std::fprintf(f, "%llu ", t[k] - t[k - 1]);
        std::fprintf(f, "\n");
        std::fclose(f);
      }
    }
  }
  return RTTDA_OK;
}

}  // namespace rttda
