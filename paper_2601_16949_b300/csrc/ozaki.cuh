// FP64-accurate contractions on the BF16 tensor cores by exponent-aligned
// slicing: the Ozaki scheme (K. Ozaki, T. Ogita, S. Oishi, S. M. Rump,
// "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012), here for the exchange term -c_x sum_P B^P_ij B^P_ab
// of the A matrix elements (Sec. 2.2) when sigma must match FP64.
//
// Digits.  A block of values (one row of an operand over at most 512
// consecutive K elements) with |x| < 2^e for all of its x is written as
//     x = 2^e sum_{s<S} d_s 2^(-7(s+1)) + r,      |r| <= 2^(e - 7S - 1),
// d_0 in [-128, 128] and d_s in [-64, 63] for s >= 1: small integers, exact
// in BF16.  They come from the fixed-point integer F = round(x 2^(7S - e))
// (|F| <= 2^(7S)) by centred base-128 division, in integer arithmetic only.
// A value is handled as a pair (I, E) with x = I 2^E: an FP64 number as its
// 53-bit significand and exponent, a product sum of this file as an int64
// and the exponent its operands' blocks imply.
//
// Products.  Over one block, sum_k A[m][k] B[n][k] equals
//     2^(ea + eb) sum_{s,t} 2^(-7(s+t+2)) sum_k d_s[m][k] g_t[n][k].
// Pairs with s + t = g carry one weight, so the tensor cores sum each group
// g < S in a TMEM accumulator of its own; pairs with s + t >= S are dropped
// (the scheme's triangular truncation, relative size 2^(-7S) of the block's
// scale).  A product of two digits is at most 2^14 in magnitude and group g
// collects at most 2^14 (g <= 1) or (g + 3) 2^12 (g >= 2) per K element, so
// for S = 6 and a block of at most 512 elements every partial sum is an
// integer of magnitude <= 2^24: exact in FP32 in any order of addition.
// The epilogue joins the groups exactly in int64,
//     I = sum_g acc_g 2^(7(S-1-g)),        block value = I 2^(ea + eb - 7(S+1)),
// and adds the block values of a K range in FP64 (or, for the Z build, a
// contraction of one block, stores I).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_gemm.cuh"

namespace rttda {
namespace oz {

constexpr int kS = 6;                        // digits per value
constexpr int kDigitBits = 7;
constexpr int kFixBits = kS * kDigitBits;    // 42: fixed-point bits of F
constexpr int kOutShift = kDigitBits * (kS + 1);  // 49: 2^(ea+eb-49) I
constexpr int kKB = 32;                      // K tile: 32 BF16 = 64-byte rows, 64-byte swizzle
constexpr int kBlkTiles = 16;                // K tiles per exactness block (512 elements)
constexpr int kBlk = kKB * kBlkTiles;
constexpr int kBN = 64;
constexpr int kStagesVV = 3;     // long K loops
constexpr int kStagesPlain = 2;  // Z build (K = nocc): room for the store staging
constexpr int kEpiWarps = 16;                    // four per TMEM lane quarter, 16 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;   // producer + MMA warp + epilogue
constexpr int kCW = kBN * 4 / kEpiWarps;        // columns per epilogue thread
constexpr int kEmptyExp = -400;              // block exponent of an all-zero block
constexpr int kASlice = tc::kBM * kKB * 2;   // one A digit plane of a K tile (8 KB)
constexpr int kBSlice = kBN * kKB * 2;       // one B digit plane (4 KB)
constexpr int kStageBytes = kS * (kASlice + kBSlice);
constexpr uint32_t kTmemCols = 512;
static_assert(kS * kBN <= (int)kTmemCols, "group accumulators exceed TMEM");
static_assert(kStageBytes % 1024 == 0, "stage must keep 1024-byte alignment");
static_assert(kBlk * 8 * 4096 <= (1 << 24), "a group sum of one block must stay exact in FP32");
// operand addressing and epilogue
enum : int {
  OZ_PLAIN = 0,    // A [digit][row][k], B [digit][row][k]: 3-D maps (k, row, digit); one block, out int64 I
  OZ_VV = 1,       // A = Z digits [digit][(P, b/64)][row][64]; B = B_vv digits [digit][P][a][b]; out FP64
  OZ_PLAIN64 = 2   // 3-D maps as OZ_PLAIN over many blocks (a "P" below is one block); out FP64
};

constexpr int kStgRow = kCW + 1;  // int64 words per staged row (+1 against bank conflicts)
constexpr int kStgWarpBytes = 32 * kStgRow * 8;

template <int MODE>
constexpr int stages() { return MODE == OZ_PLAIN ? kStagesPlain : kStagesVV; }
template <int MODE>
constexpr size_t smem_bytes() {
  return (size_t)stages<MODE>() * kStageBytes + (MODE == OZ_PLAIN ? (size_t)kEpiWarps * kStgWarpBytes : 0) + 1024 +
         256;
}


struct Params {
  int M, N;
  int vt;        // K tiles per P (OZ_VV, OZ_PLAIN64); all K tiles of the contraction (OZ_PLAIN)
  int pc;        // P in this chunk (OZ_VV); blocks (OZ_PLAIN64); 1 (OZ_PLAIN)
  int pps;       // P per split
  int nsplit;
  int nbp;       // exactness blocks per P: ceil(vt / kBlkTiles)
  void* out;     // OZ_VV, OZ_PLAIN64: double [split][M][ldo]; OZ_PLAIN: long long [M][ldo]
  long long ldo, split_stride;
  int accum;     // out += result (later chunks of P)
  const int* ea;    // A block exponents ea[block * lde_a + m] (OZ_VV, OZ_PLAIN64)
  long long lde_a;
  const short* eb;  // B block exponents eb[block * lde_b + n] (OZ_VV, OZ_PLAIN64; lde_b % 32 == 0)
  long long lde_b;
  int* err;
};

__device__ __forceinline__ void tmem_ld4_nowait(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// I 2^E as a double, assembled from the bits of I (rounding toward zero,
// relative error below 2^-52; zero below the normal range): no int-to-FP64
// conversion, which B300 runs on its narrow FP64 pipe.
__device__ __forceinline__ double scaled_i64(long long I, int E) {
  if (I == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)I & 0x8000000000000000ull;
  unsigned long long a = I < 0 ? 0ull - (unsigned long long)I : (unsigned long long)I;
  const int lz = __clzll((long long)a);
  a <<= lz;  // leading one at bit 63
  const int ex = 63 - lz + E + 1023;
  if (ex <= 0) return 0.0;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)min(ex, 2046) << 52) |
                                          ((a >> 11) & 0xFFFFFFFFFFFFFull)));
}

// ---------------------------------------------------------------------------
// Digits of a value x = I 2^E in a block of exponent e (|x| < 2^e):
// F = round(I 2^(E + 7S - e)), then d_{S-1}, ..., d_1 centred in [-64, 63]
// and d_0 = what remains (|d_0| <= 128).
// ---------------------------------------------------------------------------
// Rounding half up (arithmetic shift of I + half); |I 2^(E-e)| <= 1 keeps
// |F| <= 2^(7S).
__device__ __forceinline__ long long fixed_point(long long I, int E, int e) {
  const int sh = E + kFixBits - e;
  if (sh >= 0) return (long long)((unsigned long long)I << sh);
  if (sh <= -63) return 0;
  return (I + (1ll << (-sh - 1))) >> (-sh);
}

// Adding 64 at each of the five low base-128 positions turns every centred
// digit into a plain 7-bit field: with G = F + 64 (1 + 128 + ... + 128^4),
// d_s = bits [7(5-s), 7(5-s) + 7) of G minus 64 (s >= 1) and d_0 = G >> 35.
// The fields become floats without a conversion instruction: 2^23 + u has
// the bit pattern 0x4B000000 | u for 0 <= u < 2^23.
constexpr long long kDigitBias = 64LL * (1 + 128 + 16384 + 2097152 + 268435456);
static_assert(kS == 6, "digits() unpacks six base-128 digits");

__device__ __forceinline__ float field_digit(uint32_t u) {
  return __uint_as_float(0x4B000000u | (u & 127u)) - 8388672.0f;  // u - 64
}

__device__ __forceinline__ void digits(long long F, float (&d)[kS]) {
  const long long G = F + kDigitBias;
  const uint32_t lo = (uint32_t)G;
  const uint32_t hi = (uint32_t)((unsigned long long)G >> 32);
  d[5] = field_digit(lo);
  d[4] = field_digit(lo >> 7);
  d[3] = field_digit(lo >> 14);
  d[2] = field_digit(lo >> 21);
  d[1] = field_digit(__funnelshift_r(lo, hi, 28));
  d[0] = __int_as_float(0x4B400000 + ((int)hi >> 3)) - 12582912.0f;  // |d_0| <= 128
}

// Bits of |I| (of |I| - 1 for negative I) plus E: |x| = |I 2^E| <= 2^(that),
// with equality only for x = -2^(that), whose fixed-point form -2^(7S) still
// has a leading digit of -128 (-2^30 for I = 0).
__device__ __forceinline__ int top_exp(long long I, int E) {
  if (I == 0) return -0x40000000;
  return 64 - __clzll(I ^ (I >> 63)) + E;
}

__device__ __forceinline__ void f64_parts(double x, long long& I, int& E) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  long long m = b & 0xFFFFFFFFFFFFFll;
  if (ex != 0) m |= 1ll << 52;
  E = (ex != 0 ? ex : 1) - 1075;
  I = b < 0 ? -m : m;
}

// ---------------------------------------------------------------------------
// Slicing kernels.  One warp per block; lane l holds the block's elements
// l, l + 32, ... (up to kBlk / 32 = 16 of them).
// ---------------------------------------------------------------------------
constexpr int kPerLane = kBlk / 32;

__device__ __forceinline__ int warp_block_exp(int e) {
  e = __reduce_max_sync(0xffffffffu, e);
  return e < -0x20000000 ? kEmptyExp : e;
}

// Rows r of an FP64 matrix with element k of row r at src[r * lds + k * ldk]
// (k < klen, zero beyond): digits [digit][r][ldd] (BF16, zero padded up to
// kpad) and one exponent per (row, block of 512 along k), stored at
// exps[((r / rin) * nblk + blk) * lde + r % rin].  B_oo: rows (P, i), K = j,
// rin = all rows, nblk = 1.  B_vv: rows (P, a), K = b, rin = nvirt, lde =
// the padded nvirt (exponents [P][blk][a]).
template <typename TE>
__global__ void __launch_bounds__(256) k_slice_rows(long long rows, long long rin, int klen, int kpad,
                                                    const double* __restrict__ src, long long lds, long long ldk,
                                                    __nv_bfloat16* __restrict__ dst, long long ldd, long long plane,
                                                    TE* __restrict__ exps, long long lde, int nblk) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= rows * nblk) return;
  const long long r = wid / nblk;
  const int blk = (int)(wid - r * nblk);
  const int k0 = blk * kBlk;
  long long I[kPerLane];
  int E[kPerLane];
  int emax = -0x40000000;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const int k = k0 + lane + 32 * q;
    I[q] = 0;
    E[q] = 0;
    if (k < klen) f64_parts(src[r * lds + (long long)k * ldk], I[q], E[q]);
    emax = max(emax, top_exp(I[q], E[q]));
  }
  const int e = warp_block_exp(emax);
  if (lane == 0) exps[((r / rin) * nblk + blk) * lde + r % rin] = (TE)e;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const int k = k0 + lane + 32 * q;
    if (k >= kpad || k >= k0 + kBlk) continue;
    float d[kS];
    digits(fixed_point(I[q], E[q], e), d);
#pragma unroll
    for (int s = 0; s < kS; ++s) dst[(size_t)s * plane + r * ldd + k] = __float2bfloat16_rn(d[s]);
  }
}

// Stage amplitudes for Z = B_oo c: rows (col, b) (b < vp; rows b >= v are
// zero), K = j < o.  X[n * C + col] with n = 1 + j v + b.  Digits
// [digit][col * vp + b][op], exponents ex[col * vp + b] (o <= 512: one block).
__global__ void __launch_bounds__(256) k_slice_x(int o, int v, int vp, int op, int C, const double* __restrict__ X,
                                                 __nv_bfloat16* __restrict__ dst, long long plane,
                                                 int* __restrict__ ex) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)C * vp) return;
  const int col = (int)(wid / vp), b = (int)(wid - (long long)col * vp);
  long long I[kPerLane];
  int E[kPerLane];
  int emax = -0x40000000;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const int j = lane + 32 * q;
    I[q] = 0;
    E[q] = 0;
    if (j < o && b < v) f64_parts(X[(1 + (long long)j * v + b) * C + col], I[q], E[q]);
    emax = max(emax, top_exp(I[q], E[q]));
  }
  const int e = warp_block_exp(emax);
  if (lane == 0) ex[wid] = e;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const int j = lane + 32 * q;
    if (j >= op) continue;
    float d[kS];
    digits(fixed_point(I[q], E[q], e), d);
#pragma unroll
    for (int s = 0; s < kS; ++s) dst[(size_t)s * plane + wid * op + j] = __float2bfloat16_rn(d[s]);
  }
}

// Stage amplitudes for the Coulomb pass w_P = sum_ia B^P_ia c_ia: rows col
// (< cp; rows col >= C are zero), K = ia < ov in blocks of 512, element
// X[(1 + ia) * C + col].  Digits [digit][col][ovp], exponents
// ex[blk * cp + col]; one warp per (col, block).
__global__ void __launch_bounds__(256) k_slice_xc(long long ov, int ovp, int C, int cp, int nkb,
                                                  const double* __restrict__ X, __nv_bfloat16* __restrict__ dst,
                                                  long long plane, short* __restrict__ ex) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)cp * nkb) return;
  const int col = (int)(wid / nkb), blk = (int)(wid - (long long)col * nkb);
  long long I[kPerLane];
  int E[kPerLane];
  int emax = -0x40000000;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const long long ia = (long long)blk * kBlk + lane + 32 * q;
    I[q] = 0;
    E[q] = 0;
    if (ia < ov && col < C) f64_parts(X[(1 + ia) * C + col], I[q], E[q]);
    emax = max(emax, top_exp(I[q], E[q]));
  }
  const int e = warp_block_exp(emax);
  if (lane == 0) ex[(long long)blk * cp + col] = (short)e;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const long long ia = (long long)blk * kBlk + lane + 32 * q;
    if (ia >= ovp) continue;
    float d[kS];
    digits(fixed_point(I[q], E[q], e), d);
#pragma unroll
    for (int s = 0; s < kS; ++s) dst[(size_t)s * plane + (long long)col * ovp + ia] = __float2bfloat16_rn(d[s]);
  }
}

// The Coulomb intermediate 2 w: rows col (< cp), K = P in blocks of 512,
// 2 w[P][col] = 2 sum_s wpart[s][P][col] (the nsp split-K partials of the
// first pass, added in order).  Digits [digit][col][Pp], exponents
// ew[blk * cp + col].
__global__ void __launch_bounds__(256) k_slice_w(int P, int Pp, int C, int cp, int npb, int nsp,
                                                 const double* __restrict__ wpart, __nv_bfloat16* __restrict__ dst,
                                                 long long plane, short* __restrict__ ew) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)cp * npb) return;
  const int col = (int)(wid / npb), blk = (int)(wid - (long long)col * npb);
  long long I[kPerLane];
  int E[kPerLane];
  int emax = -0x40000000;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const int Pi = blk * kBlk + lane + 32 * q;
    I[q] = 0;
    E[q] = 0;
    if (Pi < P && col < C) {
      double a = 0.0;
      for (int sp = 0; sp < nsp; ++sp) a += wpart[((size_t)sp * P + Pi) * C + col];
      f64_parts(2.0 * a, I[q], E[q]);
    }
    emax = max(emax, top_exp(I[q], E[q]));
  }
  const int e = warp_block_exp(emax);
  if (lane == 0) ew[(long long)blk * cp + col] = (short)e;
#pragma unroll
  for (int q = 0; q < kPerLane; ++q) {
    const int Pi = blk * kBlk + lane + 32 * q;
    if (Pi >= Pp) continue;
    float d[kS];
    digits(fixed_point(I[q], E[q], e), d);
#pragma unroll
    for (int s = 0; s < kS; ++s) dst[(size_t)s * plane + (size_t)col * Pp + Pi] = __float2bfloat16_rn(d[s]);
  }
}

// Z digits for the main contraction.  Zi[(P, i)][(col, b)] = I from the
// Z build, with x = I 2^(eoo[P, i] + ex[col, b] - 49).  Rows (col, i), K =
// (P, b): one warp per (row, P, block of 512 along b); lane l handles the
// pairs b = 2l + 64q, 2l + 1 + 64q of the block.  Digits in the tile order
// of the main contraction, [digit][(P, b/64)][col * o + i][64]; exponents
// ez[(P * nbp + blk) * (C * o) + col * o + i].
__global__ void __launch_bounds__(256, 4) k_slice_z(int o, int vp, int C, int pc, int nbp, int p0,
                                                 const long long* __restrict__ Zi, const short* __restrict__ eoo,
                                                 const int* __restrict__ ex, __nv_bfloat16* __restrict__ dst,
                                                 long long plane, int* __restrict__ ez) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)C * o * pc * nbp;
  if (wid >= nw) return;
  // warp order: block fastest, then P, then row, so that neighbouring warps
  // read neighbouring stretches of Zi
  const int blk = (int)(wid % nbp);
  const int P = (int)((wid / nbp) % pc);
  const long long row = wid / ((long long)nbp * pc);
  const int col = (int)(row / o), i = (int)(row - (long long)col * o);
  const long long zrow = ((long long)P * o + i) * ((long long)C * vp) + (long long)col * vp;
  const int eo = eoo[(long long)(p0 + P) * o + i];
  constexpr int kPairs = kBlk / 64;  // pairs per lane
  long long I[2 * kPairs];
  int E[2 * kPairs];
  int emax = -0x40000000;
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const int b = blk * kBlk + 64 * q + 2 * lane;
    I[2 * q] = I[2 * q + 1] = 0;
    E[2 * q] = E[2 * q + 1] = 0;
    if (b < vp) {
      const longlong2 z = *reinterpret_cast<const longlong2*>(Zi + zrow + b);
      I[2 * q] = z.x;
      I[2 * q + 1] = z.y;
      E[2 * q] = eo + ex[(long long)col * vp + b] - kOutShift;
      E[2 * q + 1] = eo + ex[(long long)col * vp + b + 1] - kOutShift;
    }
    emax = max(emax, max(top_exp(I[2 * q], E[2 * q]), top_exp(I[2 * q + 1], E[2 * q + 1])));
  }
  const int e = warp_block_exp(emax);
  if (lane == 0) ez[((long long)P * nbp + blk) * ((long long)C * o) + row] = e;
  const int vt64 = vp / 64;
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    const int b = blk * kBlk + 64 * q + 2 * lane;
    if (b >= vp) continue;
    float d0[kS], d1[kS];
    digits(fixed_point(I[2 * q], E[2 * q], e), d0);
    digits(fixed_point(I[2 * q + 1], E[2 * q + 1], e), d1);
    const size_t off = (((size_t)P * vt64 + (b >> 6)) * ((size_t)C * o) + (size_t)row) * 64 + (b & 63);
#pragma unroll
    for (int s = 0; s < kS; ++s)
      *reinterpret_cast<__nv_bfloat162*>(dst + (size_t)s * plane + off) = __floats2bfloat162_rn(d0[s], d1[s]);
  }
}

// ---------------------------------------------------------------------------
// The contraction kernel: persistent over (split, m tile, n tile) tiles of
// 128 x 64; per K tile one pipeline stage (3 stages for OZ_VV and
// OZ_PLAIN64, 2 for OZ_PLAIN, whose epilogue stages its int64 rows in shared
// memory) holds the S digit planes of A and of B; the MMA warp issues the
// S(S+1)/2 digit pairs of the tile into the group accumulators g = s + t
// (TMEM columns g * 64 .. +63) and hands them to the epilogue at the end of
// each exactness block.  Warp roles as in the other tensor-core kernels:
// warp 0 TMA producer, warp 1 TMEM owner and MMA issuer, warps 2..17
// epilogue (TMEM lane quarter warp % 4, columns 16 ((warp - 2) / 4) .. +15;
// sixteen warps so that the integer work of the drain, which stalls the
// MMAs of the next block, has latency cover).  Every wait is bounded (error
// code in *err).
//
// K tiles of a split: P in [split * pps, min(pc, (split + 1) * pps)), each
// P with vt tiles; within a P a block ends every kBlkTiles tiles and at the
// P's last tile, so blocks never straddle two P.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params p) {
  using namespace tc;
  constexpr int ST = stages<MODE>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // [stages][store staging (OZ_PLAIN)][barriers]
  uint8_t* stg_base = smem + ST * kStageBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(stg_base + (MODE == OZ_PLAIN ? kEpiWarps * kStgWarpBytes : 0));
  uint64_t* empty = full + ST;
  uint64_t* accf = empty + ST;
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (p.N + kBN - 1) / kBN;
  const int tiles_m = (p.M + kBM - 1) / kBM;
  const int ntiles = tiles_n * tiles_m * p.nsplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, oz::kEpiWarps);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto coords = [&](int t, int& n0, int& m0, int& kr0, int& kr1) {
    n0 = (t % tiles_n) * kBN;
    m0 = ((t / tiles_n) % tiles_m) * kBM;
    const int split = t / (tiles_n * tiles_m);
    const int P0 = split * p.pps, P1 = min(p.pc, P0 + p.pps);
    kr0 = P0 * p.vt;
    kr1 = max(P0, P1) * p.vt;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0;
      bool alive = true;
      for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
        int n0, m0, kr0, kr1;
        coords(t, n0, m0, kr0, kr1);
        for (int kr = kr0; kr < kr1; ++kr, ++it) {
          const int s = it % ST;
          const uint32_t ph = (uint32_t)(it / ST) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, p.err, ERR_WAIT_EMPTY)) {
            alive = false;
            break;
          }
          uint8_t* st = smem + s * kStageBytes;
          mbar_expect_tx(&full[s], (uint32_t)kStageBytes);
          if (MODE != OZ_VV) {
#pragma unroll
            for (int q = 0; q < kS; ++q) tma_load_3d(st + q * kASlice, &tmA, &full[s], kr * kKB, m0, q);
#pragma unroll
            for (int q = 0; q < kS; ++q)
              tma_load_3d(st + kS * kASlice + q * kBSlice, &tmB, &full[s], kr * kKB, n0, q);
          } else {
            // Z digits in 64-wide tiles along (P, b): K tile kr is half kr & 1
            // of tile kr / 2 (vt is even); B_vv digits at (b, a, P)
            const int P = kr / p.vt, b0 = (kr - P * p.vt) * kKB;
#pragma unroll
            for (int q = 0; q < kS; ++q)
              tma_load_4d(st + q * kASlice, &tmA, &full[s], (kr & 1) * kKB, m0, kr >> 1, q);
#pragma unroll
            for (int q = 0; q < kS; ++q)
              tma_load_4d(st + kS * kASlice + q * kBSlice, &tmB, &full[s], b0, n0, P, q);
          }
        }
      }
      drain_loads(full, it, ST);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int it = 0, nb = 0;
      bool alive = true;
      for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
        int n0, m0, kr0, kr1;
        coords(t, n0, m0, kr0, kr1);
        for (int kr = kr0; kr < kr1; ++kr, ++it) {
          const int bt = kr % p.vt;
          const bool bstart = (bt % kBlkTiles) == 0;
          const bool bend = (bt % kBlkTiles) == kBlkTiles - 1 || bt == p.vt - 1;
          if (bstart) {
            // the epilogue has drained the group accumulators of the last block
            if (!mbar_wait(acce, ((uint32_t)nb & 1u) ^ 1u, p.err, ERR_WAIT_ACC)) {
              alive = false;
              break;
            }
            tc_fence_after();
          }
          const int s = it % ST;
          const uint32_t ph = (uint32_t)(it / ST) & 1u;
          if (!mbar_wait(&full[s], ph, p.err, ERR_WAIT_FULL)) {
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * kStageBytes);
          // A digit sa against the B digits sb = 0 .. S-1-sa, whose 64-row
          // planes lie back to back and so form one B operand of
          // (S - sa) * 64 rows: product (sa, sb) lands in accumulator
          // columns (sa + sb) * 64, the columns of its group.  At most 256
          // rows per MMA.  The MMA of sa = 0 writes every group first.
#pragma unroll
          for (int sa = 0; sa < kS; ++sa) {
            const uint64_t adesc = sdesc_sw64(base + sa * kASlice);
#pragma unroll
            for (int t0 = 0; t0 < kS - sa; t0 += 4) {
              const int nt = min(4, kS - sa - t0);
              const uint64_t bdesc = sdesc_sw64(base + kS * kASlice + t0 * kBSlice);
              const uint32_t d = tmem + (uint32_t)((sa + t0) * kBN);
              const uint32_t idesc = idesc_bf16(kBM, nt * kBN);
#pragma unroll
              for (int k = 0; k < kKB / 16; ++k)
                mma_bf16(d, adesc + 2 * k, bdesc + 2 * k, idesc, (!bstart || sa > 0 || k > 0) ? 1u : 0u);
            }
          }
          mma_commit(&empty[s]);
          if (bend) {
            mma_commit(accf);
            ++nb;
          }
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2..17) ----------------
    const int q = warp & 3;
    const int cg = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cg * kCW);
    int nb = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int n0, m0, kr0, kr1;
      coords(t, n0, m0, kr0, kr1);
      const int m = m0 + row;
      const int nbase = n0 + cg * kCW;
      if constexpr (MODE != OZ_PLAIN) {
        double acc[kCW];
#pragma unroll
        for (int j = 0; j < kCW; ++j) acc[j] = 0.0;
        for (int kr = kr0; kr < kr1; ++kr) {
          const int P = kr / p.vt, bt = kr - P * p.vt;
          if (!((bt % kBlkTiles) == kBlkTiles - 1 || bt == p.vt - 1)) continue;
          const int blk = P * p.nbp + bt / kBlkTiles;
          // the block's exponents, loaded while its MMAs still run
          const int ea = m < p.M ? __ldg(p.ea + (size_t)blk * p.lde_a + m) : kEmptyExp;
          uint4 eb4[kCW / 8];  // int16 exponents of the thread's columns
          const uint4* ebp = reinterpret_cast<const uint4*>(p.eb + (size_t)blk * p.lde_b + nbase);
#pragma unroll
          for (int u = 0; u < kCW / 8; ++u) eb4[u] = __ldg(ebp + u);
          ok = mbar_wait(accf, (uint32_t)nb & 1u, p.err, ERR_WAIT_ACC);
          ++nb;
          tc_fence_after();
          if (!ok) break;
          // join the groups into integers and release the accumulators;
          // the FP64 additions then overlap the next block's MMAs
          long long Iv[kCW];
#pragma unroll
          for (int c4 = 0; c4 < kCW / 4; ++c4) {
            uint32_t r[kS][4];
#pragma unroll
            for (int g = 0; g < kS; ++g) tmem_ld4_nowait(tl + (uint32_t)(g * kBN + c4 * 4), r[g]);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              // I = sum_g acc_g 2^(7(S-1-g)) (Horner from the leading group)
              long long I = __float2int_rn(__uint_as_float(r[0][j]));
#pragma unroll
              for (int g = 1; g < kS; ++g) I = I * 128 + __float2int_rn(__uint_as_float(r[g][j]));
              Iv[c4 * 4 + j] = I;
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce);
          const int eab = ea - kOutShift;
#pragma unroll
          for (int j = 0; j < kCW; ++j) {
            const uint32_t w = (j & 4) ? ((j & 2) ? eb4[j >> 3].w : eb4[j >> 3].z) : ((j & 2) ? eb4[j >> 3].y : eb4[j >> 3].x);
            const int ebj = (j & 1) ? (int)w >> 16 : (int)(short)(w & 0xFFFFu);
            acc[j] += scaled_i64(Iv[j], eab + ebj);
          }
        }
        if (!ok) break;
        if (m < p.M) {
          double* dst = reinterpret_cast<double*>(p.out) + (size_t)(t / (tiles_n * tiles_m)) * p.split_stride +
                        (size_t)m * p.ldo;
#pragma unroll
          for (int j = 0; j < kCW; ++j) {
            const int n = nbase + j;
            if (n < p.N) dst[n] = p.accum ? dst[n] + acc[j] : acc[j];
          }
        }
      } else {
        // one block (K = nocc <= 512): the integers I, staged per warp in
        // shared memory and stored two rows at a time (16 consecutive words
        // per row)
        long long* stg = reinterpret_cast<long long*>(stg_base + (warp - 2) * kStgWarpBytes);
        for (int kr = kr0; kr < kr1; ++kr) {
          const int bt = kr % p.vt;
          if (!((bt % kBlkTiles) == kBlkTiles - 1 || bt == p.vt - 1)) continue;
          ok = mbar_wait(accf, (uint32_t)nb & 1u, p.err, ERR_WAIT_ACC);
          ++nb;
          tc_fence_after();
          if (!ok) break;
#pragma unroll
          for (int c4 = 0; c4 < kCW / 4; ++c4) {
            uint32_t r[kS][4];
#pragma unroll
            for (int g = 0; g < kS; ++g) tmem_ld4_nowait(tl + (uint32_t)(g * kBN + c4 * 4), r[g]);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              long long I = __float2int_rn(__uint_as_float(r[0][j]));
#pragma unroll
              for (int g = 1; g < kS; ++g) I = I * 128 + __float2int_rn(__uint_as_float(r[g][j]));
              stg[lane * kStgRow + c4 * 4 + j] = I;
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce);
        }
        if (!ok) break;
        long long* out = reinterpret_cast<long long*>(p.out);
        const int n = nbase + (lane & (kCW - 1));
        const int mrow0 = m0 + q * 32;
        for (int rr = lane / kCW; rr < 32; rr += 32 / kCW) {
          if (mrow0 + rr < p.M && n < p.N)
            out[(size_t)(mrow0 + rr) * p.ldo + n] = stg[rr * kStgRow + (lane & (kCW - 1))];
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace oz
}  // namespace rttda
