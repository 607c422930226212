// tcgen05 tensor-core GEMM for sm_103a (inline PTX: TMA, mbarrier, tcgen05).
//
//   D[m][n] = sum_k A[m][k] * B[n][k]   (A, B K-major BF16, D FP32 in TMEM)
//
// One CTA computes a 128 x BN tile over a K range (split-K).  Warp roles:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..5  epilogue: tcgen05.ld of the accumulator, one TMEM lane
//               (tile row) per thread.
// Shared-memory tiles are 128-byte rows (64 BF16 along K) in the 128-byte
// swizzled K-major layout that TMA writes with CU_TENSOR_MAP_SWIZZLE_128B.
//
// Split precision ("virtual K"): each real K tile is visited nprod times
// with operand planes (hi,hi), (hi,lo), (lo,hi), so A*B is accumulated from
// BF16 hi/lo pairs (x = hi + lo) in one FP32 accumulator.
//
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the kernel
// records an error code in *err and leaves its loops.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rttda {
namespace tc {

constexpr int kThreads = 192;
constexpr int kBM = 128;
constexpr int kBK = 64;                  // BF16 elements per 128-byte row
constexpr int kABytes = kBM * 128;       // one A stage
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

// error codes written to *err
enum : int { ERR_NONE = 0, ERR_WAIT_EMPTY = 1, ERR_WAIT_FULL = 2, ERR_WAIT_ACC = 3 };

// B operand addressing
enum : int { BMODE_PLAIN = 0,  // B[plane][n][k], 3-D map (k, n, plane)
             BMODE_VV = 1 };   // B^P_ab: 4-D map (b, a, P, plane), k = (P, b)

// epilogue kinds
enum : int { EPI_PARTIAL = 0,  // out[split][m][n] FP32
             EPI_ZSPLIT = 1 }; // Z[plane][(col*o + i)][P*vp + b] BF16 hi/lo

struct Params {
  int M, N;              // logical output extents
  int kt_total;          // real K tiles
  int kt_per_split;      // real K tiles per split
  int nprod;             // 1 (single BF16) or 3 (hi/lo split)
  int vtiles;            // vp / 64 (BMODE_VV)
  // EPI_PARTIAL
  float* out;
  long long ldo, split_stride;
  int accum;             // 1: out += tile (later P chunks), 0: out = tile
  // EPI_ZSPLIT
  __nv_bfloat16* zhi;
  __nv_bfloat16* zlo;
  int o, vp;
  long long zld;         // row length of Z (= P * vp)
  int* err;
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on the given phase parity; false (and *err set) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > kWaitLimitNs) {
      if (err) atomicCAS(err, 0, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), fixed version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);      // start address
  d |= (uint64_t)1 << 16;                       // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;             // SBO
  d |= (uint64_t)1 << 46;                       // version
  d |= (uint64_t)2 << 61;                       // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D F32, A/B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 32 lanes x 32 columns of 32-bit: thread t of the warp gets lane (base + t).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
struct Cfg {
  static constexpr int kBBytes = BN * 128;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kTmemCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : BN <= 256 ? 256 : 512;
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M=128 must be a multiple of 16 in [16, 256]");
  static_assert(kStageBytes % 1024 == 0, "stage must keep 1024-byte alignment");
};

template <int BN, int STAGES>
constexpr size_t smem_bytes() {
  return (size_t)STAGES * Cfg<BN>::kStageBytes + 1024 /*alignment slack*/ + 256 /*barriers*/;
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <int BN, int STAGES, int BMODE, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params p) {
  using CF = Cfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * CF::kStageBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM, split = blockIdx.z;
  const int kr0 = split * p.kt_per_split;
  const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
  const int niter = max(0, kr1 - kr0) * p.nprod;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, CF::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      for (int it = 0; it < niter; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, p.err, ERR_WAIT_EMPTY)) break;
        const int kr = kr0 + it / p.nprod, pr = it % p.nprod;
        const int pa = (pr == 2) ? 1 : 0, pb = (pr == 1) ? 1 : 0;
        uint8_t* sA = smem + s * CF::kStageBytes;
        uint8_t* sB = sA + kABytes;
        mbar_expect_tx(&full[s], CF::kStageBytes);
        tma_load_3d(sA, &tmA, &full[s], kr * kBK, m0, pa);
        if (BMODE == BMODE_PLAIN) {
          tma_load_3d(sB, &tmB, &full[s], kr * kBK, n0, pb);
        } else {
          const int P = kr / p.vtiles, b0 = (kr % p.vtiles) * kBK;
          tma_load_4d(sB, &tmB, &full[s], b0, n0, P, pb);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      for (int it = 0; it < niter; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!mbar_wait(&full[s], ph, p.err, ERR_WAIT_FULL)) break;
        tc_fence_after();
        const uint32_t aaddr = smem_u32(smem + s * CF::kStageBytes);
        const uint64_t adesc = sdesc_sw128(aaddr);
        const uint64_t bdesc = sdesc_sw128(aaddr + kABytes);
#pragma unroll
        for (int k = 0; k < kBK / 16; ++k)  // 16 BF16 = 32 bytes per MMA along K
          mma_bf16(tmem, adesc + 2 * k, bdesc + 2 * k, idesc, (it > 0 || k > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      mma_commit(accf);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const int m = m0 + row;
    const bool ok = mbar_wait(accf, 0, p.err, ERR_WAIT_ACC);
    tc_fence_after();
    if (EPI == EPI_PARTIAL) {
      float* dst = p.out + (size_t)split * p.split_stride + (size_t)m * p.ldo;
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + c, r);
        if (m < p.M && ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = n0 + c + j;
            if (n < p.N) {
              const float x = niter > 0 ? __uint_as_float(r[j]) : 0.0f;
              dst[n] = p.accum ? dst[n] + x : x;
            }
          }
        }
      }
    } else {
      // rows m = (P, i); columns n = (col, b) with b inside one 32-aligned chunk
      const int P = m / p.o, i = m - P * p.o;
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + c, r);
        const int n = n0 + c;
        if (m < p.M && n < p.N && ok) {
          const int col = n / p.vp, b = n - col * p.vp;
          const size_t off = (size_t)(col * p.o + i) * p.zld + (size_t)P * p.vp + b;
          uint4 hi4[4], lo4[4];
          __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(hi4);
          __nv_bfloat16* lo = reinterpret_cast<__nv_bfloat16*>(lo4);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float x = niter > 0 ? __uint_as_float(r[j]) : 0.0f;
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            hi[j] = h;
            lo[j] = __float2bfloat16_rn(x - __bfloat162float(h));
          }
          uint4* dh = reinterpret_cast<uint4*>(p.zhi + off);
#pragma unroll
          for (int j = 0; j < 4; ++j) dh[j] = hi4[j];
          if (p.zlo) {
            uint4* dl = reinterpret_cast<uint4*>(p.zlo + off);
#pragma unroll
            for (int j = 0; j < 4; ++j) dl[j] = lo4[j];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, CF::kTmemCols);
  }
}

}  // namespace tc
}  // namespace rttda
