// tcgen05 tensor-core GEMM for sm_103a (inline PTX: TMA, mbarrier, tcgen05).
//
//   D[m][n] = sum_k A[m][k] * B[n][k]   (A, B K-major BF16, D FP32 in TMEM)
//
// Persistent: each CTA walks a strided list of 128 x BN output tiles (each
// over one K range of a split-K decomposition).  Warp roles:
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..9  epilogue: tcgen05.ld of the accumulator, one TMEM lane
//               (tile row) per thread, two warps per lane quarter.
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

constexpr int kEpiWarps = 8;                    // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer + MMA warp + epilogue
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
             EPI_ZSPLIT = 1,   // Z as BF16 hi/lo planes (see Params)
             EPI_ZONE = 2,     // Z as one BF16 plane
             EPI_ZRES = 3,     // EPI_ZONE with the B operand resident (K of at most kResKT tiles)
             EPI_ZRES1 = 4 };  // EPI_ZRES with one A plane per stage (one product: plain BF16)

// EPI_ZRES: the whole K extent of the B tile (at most kResKT K tiles) stays
// in shared memory while a CTA walks its tiles m-fastest, so a B tile is
// loaded once per run of tiles with the same n0 instead of once per tile.
constexpr int kResKT = 2;

struct Params {
  int M, N;              // logical output extents
  int kt_total;          // real K tiles
  int kt_per_split;      // real K tiles per split
  int nsplit;            // number of K splits
  int nprod;             // 1 (single BF16), 2 or 3 (hi/lo split)
  int alo;               // with nprod 2: products (hi,hi), (lo,hi) instead of (hi,hi), (hi,lo)
  int vtiles;            // vp / (K tile width) (BMODE_VV)
  // EPI_PARTIAL
  float* out;
  long long ldo, split_stride;
  int accum;             // 1: out += tile (later P chunks), 0: out = tile
  // EPI_ZSPLIT / EPI_ZONE: Z stored as [plane][(P, b/64)][(col, i)][64]
  // (the main contraction's TMA box order)
  __nv_bfloat16* zhi;
  __nv_bfloat16* zlo;
  int o, vp;
  int zrows;             // C * o rows per K tile
  int ztma;              // 1: store Z chunks with TMA (nocc % 32 == 0)
  int zhint;             // 1: Z stores under the L2 evict-first policy
  // EPI_ZRES tile order: slabs of gridDim.x * zrun row tiles; inside a slab
  // the columns advance slowest, so each CTA runs zrun tiles per resident B
  // tile and the slab's A rows stay in L2 across all column tiles
  // (0: one slab of all rows)
  int zrun;
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Before a CTA leaves its producer loop: wait (bounded) until every TMA load
// issued into the last `stages` pipeline slots has landed.  After a wait
// elsewhere in the CTA ran out, loads may still be in flight, and the CTA
// must not exit (and free its shared memory) while asynchronous writes into
// it are pending.  On the normal path every issued load was consumed, so
// each of these waits returns at once.
__device__ __forceinline__ void drain_loads(uint64_t* full, int issued, int stages) {
  for (int j = max(0, issued - stages); j < issued; ++j)
    mbar_wait(&full[j % stages], (uint32_t)(j / stages) & 1u, nullptr, 0);
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

// TMA tensor store from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                             int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
// The same store with an L2 cache policy (createpolicy).
__device__ __forceinline__ void tma_store_4d_hint(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                                  int c3, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3, %4, %5}], [%1], %6;" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "l"(policy)
      : "memory");
}
// L2 policy under which the lines a kernel writes are the first to be
// evicted: a write stream (Z) then leaves the operands it is computed from
// in L2.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// Same with 64-byte swizzle (rows of 32 BF16 along K): 8-row groups 512
// bytes apart, layout type 4.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;                       // SWIZZLE_64B
  return d;
}

template <int KB>
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr) {
  static_assert(KB == 64 || KB == 32, "K tile of 64 (128-byte rows) or 32 (64-byte rows) BF16");
  return KB == 64 ? sdesc_sw128(saddr) : sdesc_sw64(saddr);
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

// Cluster forms (thread-block clusters of the main contraction).
// The commit arrives on the barrier at the same shared-memory offset in every
// CTA of `mask` once this CTA's prior MMAs have completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
// A tile load delivered to the same shared-memory offset (and completing on
// the barrier at the same offset) in every CTA of `mask`.
__device__ __forceinline__ void tma_load_4d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                               int c2, int c3, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4, %5, %6}], [%2], %7;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
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
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Z epilogue staging, per epilogue warp.  TMA path: two buffers x ZPL
// planes of one 32-row x 64-column BF16 group (128-byte rows in the
// 128-byte swizzled layout that the store map reads, so the row writes are
// free of bank conflicts).  Manual path: hi and lo blocks of 32 rows x 64 B,
// rows padded to 80 B.
constexpr int kStageRowWords = 20;
constexpr int kZGroupBytes = 32 * 128;
template <int EPI>
constexpr int zstage_bytes_per_warp() {
  return EPI == 1 ? 4 * kZGroupBytes : (EPI == 2 || EPI == 3 || EPI == 4) ? 2 * kZGroupBytes : 0;
}
static_assert(2 * 32 * kStageRowWords * 4 <= 2 * kZGroupBytes, "manual staging must fit");

// BF16 hi/lo of two floats: hi = rn(x), lo = rn(x - hi), each packed (x0 in
// the low half).
__device__ __forceinline__ void split_pack(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16x2(x0, x1);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  lo = pack_bf16x2(x0 - h0, x1 - h1);
}

template <int BN, int NA = 1>
struct Cfg {
  static constexpr int kBBytes = BN * 128;
  static constexpr int kStageBytes = NA * kABytes + kBBytes;  // NA A planes + one B plane
  static constexpr uint32_t kAccCols = 256;   // column offset of accumulator buffer 1
  static constexpr uint32_t kTmemCols = 512;  // two accumulator buffers
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M=128 must be a multiple of 16 in [16, 256]");
  static_assert(kStageBytes % 1024 == 0, "stage must keep 1024-byte alignment");
};

// EPI_ZONE stages hold both A planes and the B plane of one K tile (all
// products of the tile from one stage); the other kinds one plane each.
template <int EPI>
constexpr int stage_a_planes() {
  return (EPI == 2 || EPI == 3) ? 2 : 1;  // EPI_ZRES1: one
}

// bytes of one pipeline stage: with EPI_ZRES the A planes only
template <int BN, int EPI>
constexpr int stage_bytes() {
  return EPI == 3 ? 2 * kABytes : EPI == 4 ? kABytes : Cfg<BN, stage_a_planes<EPI>()>::kStageBytes;
}

template <int BN, int STAGES, int EPI = 0>
constexpr size_t smem_bytes() {
  return (size_t)STAGES * stage_bytes<BN, EPI>() + ((EPI == 3 || EPI == 4) ? (size_t)kResKT * BN * 128 : 0) +
         1024 /*alignment slack*/ + 256 /*barriers*/ + (size_t)kEpiWarps * zstage_bytes_per_warp<EPI>();
}

// Tile t -> (split, m tile, n tile), n fastest so that consecutive tiles of a
// CTA reuse the same A rows from L2.
struct TileCoord {
  int n0, m0, split;
};
__device__ __forceinline__ TileCoord tile_coord(int t, int tiles_n, int tiles_m, int BN) {
  TileCoord c;
  c.n0 = (t % tiles_n) * BN;
  c.m0 = ((t / tiles_n) % tiles_m) * kBM;
  c.split = t / (tiles_n * tiles_m);
  return c;
}

// ---------------------------------------------------------------------------
// The kernel: persistent, one CTA per SM; CTA b handles tiles b, b + grid, ...
// Two TMEM accumulators (columns [0, BN) and [256, 256 + BN)) let the
// epilogue of one tile overlap the loads and MMAs of the next.
// ---------------------------------------------------------------------------
template <int BN, int STAGES, int BMODE, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmZ, const Params p) {
  // MERGED: a stage holds A hi, A lo and B hi of one K tile and the MMA warp
  // issues every product of the tile from it (products (hi,hi), (lo,hi),
  // i.e. nprod <= 2 with alo); otherwise one stage per product.  BRES: the
  // B tile (all K tiles) is resident and stages hold the A planes only.
  constexpr bool BRES = EPI == EPI_ZRES || EPI == EPI_ZRES1;
  constexpr bool MERGED = EPI == EPI_ZONE || BRES;
  using CF = Cfg<BN, stage_a_planes<EPI>()>;
  constexpr int kStage = stage_bytes<BN, EPI>();
  constexpr int kStgWarp = zstage_bytes_per_warp<EPI>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // [stages][resident B (BRES)][Z staging (1024-aligned)][barriers]
  uint8_t* bres = smem + STAGES * kStage;
  uint8_t* zstage = bres + (BRES ? kResKT * CF::kBBytes : 0);
  uint64_t* full = reinterpret_cast<uint64_t*>(zstage + kEpiWarps * kStgWarp);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2] accumulator ready (MMA -> epilogue)
  uint64_t* acce = accf + 2;        // [2] accumulator drained (epilogue -> MMA)
  uint64_t* bfull = acce + 2;       // resident B loaded (BRES)
  uint64_t* bempty = bfull + 1;     // resident B no longer read by MMAs (BRES)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bempty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (p.N + BN - 1) / BN;
  const int tiles_m = (p.M + kBM - 1) / kBM;
  const int ntiles = tiles_n * tiles_m * p.nsplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], kEpiWarps);  // one arrive per epilogue warp
    }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, CF::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // tile t -> coordinates: n fastest, or (BRES, one split) m fastest, so that
  // a CTA's consecutive tiles (t, t + grid, ...) share n0 for long runs
  const int slab_w = (BRES && p.zrun > 0) ? min(tiles_m, (int)gridDim.x * p.zrun) : tiles_m;
  const int slab_full = (tiles_m / slab_w) * slab_w * tiles_n;  // tiles in full slabs
  auto coord = [&](int t) {
    if constexpr (BRES) {
      TileCoord c;
      int m, n;
      if (t < slab_full) {
        const int s = t / (slab_w * tiles_n), rem = t - s * slab_w * tiles_n;
        n = rem / slab_w;
        m = s * slab_w + rem % slab_w;
      } else {  // the last, narrower slab
        const int rem = t - slab_full, w = tiles_m - (tiles_m / slab_w) * slab_w;
        n = rem / w;
        m = (tiles_m / slab_w) * slab_w + rem % w;
      }
      c.m0 = m * kBM;
      c.n0 = n * BN;
      c.split = 0;
      return c;
    } else {
      return tile_coord(t, tiles_n, tiles_m, BN);
    }
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0, bl = 0, cur_n = -1;
      bool alive = true;
      for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
        const TileCoord tc = coord(t);
        const int kr0 = tc.split * p.kt_per_split;
        const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
        const int niter = max(0, kr1 - kr0) * (MERGED ? 1 : p.nprod);
        if (BRES && tc.n0 != cur_n) {
          // a new B tile: once the MMAs reading the previous one are done
          if (bl > 0 && !mbar_wait(bempty, (uint32_t)(bl - 1) & 1u, p.err, ERR_WAIT_EMPTY)) {
            alive = false;
            break;
          }
          mbar_expect_tx(bfull, (uint32_t)(p.kt_total * CF::kBBytes));
          for (int k = 0; k < p.kt_total; ++k) tma_load_3d(bres + k * CF::kBBytes, &tmB, bfull, k * kBK, tc.n0, 0);
          cur_n = tc.n0;
          ++bl;
        }
        for (int j = 0; j < niter; ++j, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, p.err, ERR_WAIT_EMPTY)) {
            alive = false;
            break;
          }
          if (MERGED) {
            const int kr = kr0 + j, na = p.nprod >= 2 ? 2 : 1;
            uint8_t* st = smem + s * kStage;
            if (BRES) {
              mbar_expect_tx(&full[s], (uint32_t)(na * kABytes));
              for (int a = 0; a < na; ++a) tma_load_3d(st + a * kABytes, &tmA, &full[s], kr * kBK, tc.m0, a);
              continue;
            }
            mbar_expect_tx(&full[s], (uint32_t)(na * kABytes + CF::kBBytes));
            for (int a = 0; a < na; ++a) tma_load_3d(st + a * kABytes, &tmA, &full[s], kr * kBK, tc.m0, a);
            tma_load_3d(st + 2 * kABytes, &tmB, &full[s], kr * kBK, tc.n0, 0);
            continue;
          }
          const int kr = kr0 + j / p.nprod, pr = j % p.nprod;
          // operand planes of product pr: (hi,hi), (hi,lo), (lo,hi); with
          // alo the second product is (lo,hi)
          const int pa = (pr == 2 || (pr == 1 && p.alo)) ? 1 : 0;
          const int pb = (pr == 1 && !p.alo) ? 1 : 0;
          uint8_t* sA = smem + s * kStage;
          uint8_t* sB = sA + kABytes;
          mbar_expect_tx(&full[s], CF::kStageBytes);
          if (BMODE == BMODE_PLAIN)
            tma_load_3d(sA, &tmA, &full[s], kr * kBK, tc.m0, pa);
          else  // A pre-tiled: (k in tile, row, K tile, plane)
            tma_load_4d(sA, &tmA, &full[s], 0, tc.m0, kr, pa);
          if (BMODE == BMODE_PLAIN) {
            tma_load_3d(sB, &tmB, &full[s], kr * kBK, tc.n0, pb);
          } else {
            const int P = kr / p.vtiles, b0 = (kr % p.vtiles) * kBK;
            tma_load_4d(sB, &tmB, &full[s], b0, tc.n0, P, pb);
          }
        }
      }
      drain_loads(full, it, STAGES);
      if (BRES && bl > 0) mbar_wait(bfull, (uint32_t)(bl - 1) & 1u, nullptr, 0);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      int it = 0, tcount = 0, bl = 0, cur_n = -1;
      bool alive = true;
      for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x, ++tcount) {
        const TileCoord tc = coord(t);
        const int kr0 = tc.split * p.kt_per_split;
        const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
        const int niter = max(0, kr1 - kr0) * (MERGED ? 1 : p.nprod);
        const int buf = tcount & 1;
        const uint32_t aph = (uint32_t)(tcount >> 1) & 1u;
        if (!mbar_wait(&acce[buf], aph ^ 1u, p.err, ERR_WAIT_ACC)) break;
        tc_fence_after();
        if (BRES && tc.n0 != cur_n) {
          if (!mbar_wait(bfull, (uint32_t)bl & 1u, p.err, ERR_WAIT_FULL)) break;
          tc_fence_after();
          cur_n = tc.n0;
          ++bl;
        }
        const uint32_t dcol = tmem + (buf ? CF::kAccCols : 0u);
        for (int j = 0; j < niter; ++j, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph, p.err, ERR_WAIT_FULL)) {
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t aaddr = smem_u32(smem + s * kStage);
          if (MERGED) {
            const uint64_t bdesc =
                sdesc_sw128(BRES ? smem_u32(bres + (kr0 + j) * CF::kBBytes) : aaddr + 2 * kABytes);
            for (int pr = 0; pr < p.nprod; ++pr) {
              const uint64_t adesc = sdesc_sw128(aaddr + pr * kABytes);
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k)
                mma_bf16(dcol, adesc + 2 * k, bdesc + 2 * k, idesc, (j > 0 || pr > 0 || k > 0) ? 1u : 0u);
            }
          } else {
            const uint64_t adesc = sdesc_sw128(aaddr);
            const uint64_t bdesc = sdesc_sw128(aaddr + kABytes);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)  // 16 BF16 = 32 bytes per MMA along K
              mma_bf16(dcol, adesc + 2 * k, bdesc + 2 * k, idesc, (j > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&accf[buf]);
        if (BRES) {
          // the resident B is released after the last tile that reads it
          const int tn = t + (int)gridDim.x;
          if (tn >= ntiles || coord(tn).n0 != cur_n) mma_commit(bempty);
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    // warp w may read TMEM lanes 32*(w % 4) .. +31; the two warps of a lane
    // quarter take alternate 32-column chunks.
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int nchunks = (BN + 31) / 32;
    const int row = q * 32 + lane;
    int tcount = 0;
    int zcount = 0;  // TMA-stored Z chunks of this warp (staging double buffer)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tcount) {
      const TileCoord tc = coord(t);
      const int kr0 = tc.split * p.kt_per_split;
      const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
      const bool has_k = kr1 > kr0;
      const int buf = tcount & 1;
      const uint32_t aph = (uint32_t)(tcount >> 1) & 1u;
      const bool ok = mbar_wait(&accf[buf], aph, p.err, ERR_WAIT_ACC);
      tc_fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (buf ? CF::kAccCols : 0u);
      const int m = tc.m0 + row;
      if (EPI == EPI_PARTIAL) {
        float* dst = p.out + (size_t)tc.split * p.split_stride + (size_t)m * p.ldo;
        for (int ci = half; ci < nchunks; ci += 2) {
          const int c = ci * 32;
          uint32_t r[32];
          tmem_ld32(tbase + c, r);
          if (m < p.M && ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = tc.n0 + c + j;
              if (n < p.N) {
                const float x = has_k ? __uint_as_float(r[j]) : 0.0f;
                dst[n] = p.accum ? dst[n] + x : x;
              }
            }
          }
        }
      } else {
        // rows m = (P, i); columns n = (col, b).  Each warp converts its 32
        // rows of the tile to BF16 (hi, and lo with EPI_ZSPLIT), stages them
        // in shared memory and writes them out in the Z tile order.
        constexpr int ZPL = EPI == EPI_ZSPLIT ? 2 : 1;
        uint8_t* wst = zstage + (size_t)(warp - 2) * kStgWarp;
        const bool two = ZPL == 2 && p.zlo != nullptr;
        // (P, i) of this warp's first row; later rows step i and wrap into P
        const int mb = tc.m0 + q * 32;
        const int Pb = mb / p.o, ib = mb - Pb * p.o;
        const int vt = p.vp >> 6;
        if (p.ztma) {
          // 32 rows of one P (nocc % 32 == 0) by 64 columns of one col (vp and
          // the tile start are multiples of 64): one TMA box per plane.  The
          // two warps of a lane quarter take alternate 64-column groups;
          // staging is double-buffered per warp.
          for (int gi = half; gi < BN / 64; gi += 2, ++zcount) {
            const int c = gi * 64;
            uint32_t r0[32], r1[32];
            tmem_ld32_nowait(tbase + c, r0);
            tmem_ld32_nowait(tbase + c + 32, r1);
            tmem_wait_ld();
            if (!has_k) {
#pragma unroll
              for (int j = 0; j < 32; ++j) r0[j] = r1[j] = 0u;
            }
            const int zb = zcount & 1;
            if (zcount >= 2) {
              if (lane == 0) bulk_wait_read1();
              __syncwarp();
            }
            uint8_t* gh = wst + (zb * ZPL) * kZGroupBytes + lane * 128;
            uint8_t* gl = gh + kZGroupBytes;
            // 16-byte chunk j of row `lane` lives at chunk j ^ (lane & 7)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const uint32_t* r = j < 4 ? r0 : r1;
              const int o8 = (j & 3) * 8;
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                if (two)
                  split_pack(__uint_as_float(r[o8 + 2 * e]), __uint_as_float(r[o8 + 2 * e + 1]), hw[e], lw[e]);
                else
                  hw[e] = pack_bf16x2(__uint_as_float(r[o8 + 2 * e]), __uint_as_float(r[o8 + 2 * e + 1]));
              }
              const int sw = (j ^ (lane & 7)) * 16;
              *reinterpret_cast<uint4*>(gh + sw) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              if (two) *reinterpret_cast<uint4*>(gl + sw) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            fence_proxy_async_smem();
            __syncwarp();
            const int n = tc.n0 + c;
            if (lane == 0 && n < p.N && mb < p.M && ok) {
              const int col = n / p.vp, b = n - col * p.vp;
              const int kt = Pb * vt + (b >> 6);
              if (p.zhint) {
                const uint64_t pol = l2_policy_evict_first();
                tma_store_4d_hint(&tmZ, wst + (zb * ZPL) * kZGroupBytes, 0, col * p.o + ib, kt, 0, pol);
                if (two) tma_store_4d_hint(&tmZ, wst + (zb * ZPL + 1) * kZGroupBytes, 0, col * p.o + ib, kt, 1, pol);
              } else {
                tma_store_4d(&tmZ, wst + (zb * ZPL) * kZGroupBytes, 0, col * p.o + ib, kt, 0);
                if (two) tma_store_4d(&tmZ, wst + (zb * ZPL + 1) * kZGroupBytes, 0, col * p.o + ib, kt, 1);
              }
            }
            if (lane == 0) bulk_commit();
          }
        } else {
          uint32_t* stg = reinterpret_cast<uint32_t*>(wst);
          uint32_t* stg_lo = stg + 32 * kStageRowWords;
          for (int ci = half; ci < nchunks; ci += 2) {
            const int c = ci * 32;
            uint32_t r[32];
            tmem_ld32(tbase + c, r);
            if (!has_k) {
#pragma unroll
              for (int j = 0; j < 32; ++j) r[j] = 0u;
            }
            uint4* sh = reinterpret_cast<uint4*>(stg + lane * kStageRowWords);
            if (two) {
              uint32_t hw[16], lw[16];
#pragma unroll
              for (int j = 0; j < 16; ++j)
                split_pack(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]), hw[j], lw[j]);
              uint4* sl = reinterpret_cast<uint4*>(stg_lo + lane * kStageRowWords);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                sh[j] = make_uint4(hw[4 * j], hw[4 * j + 1], hw[4 * j + 2], hw[4 * j + 3]);
                sl[j] = make_uint4(lw[4 * j], lw[4 * j + 1], lw[4 * j + 2], lw[4 * j + 3]);
              }
            } else {
              uint32_t hw[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) hw[j] = pack_bf16x2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
#pragma unroll
              for (int j = 0; j < 4; ++j) sh[j] = make_uint4(hw[4 * j], hw[4 * j + 1], hw[4 * j + 2], hw[4 * j + 3]);
            }
            __syncwarp();
            const int n = tc.n0 + c;
            if (n < p.N && ok) {
              const int col = n / p.vp, b = n - col * p.vp;
              const size_t cbase = (size_t)(b >> 6) * p.zrows + (size_t)col * p.o;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const int rr = (lane >> 2) + 8 * k, cc = lane & 3;
                if (mb + rr < p.M) {
                  int ir = ib + rr, Pr = Pb;
                  while (ir >= p.o) {
                    ir -= p.o;
                    ++Pr;
                  }
                  const size_t off = ((size_t)Pr * vt * p.zrows + cbase + (size_t)ir) * 64 + (b & 63) + 8 * cc;
                  *reinterpret_cast<uint4*>(p.zhi + off) =
                      *reinterpret_cast<const uint4*>(stg + rr * kStageRowWords + 4 * cc);
                  if (two)
                    *reinterpret_cast<uint4*>(p.zlo + off) =
                        *reinterpret_cast<const uint4*>(stg_lo + rr * kStageRowWords + 4 * cc);
                }
              }
            }
            __syncwarp();
          }
        }
      }
      // hand the accumulator buffer back to the MMA warp
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
      if (!ok) break;
    }
    // every TMA store of this warp must have completed before the CTA exits
    if (EPI != EPI_PARTIAL && lane == 0) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, CF::kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Wide-M variant for the main exchange contraction (A = Z, one BF16 plane):
// a CTA tile is MB x 128 rows by BN columns, i.e. MB TMEM accumulators that
// share every B tile, and one pipeline stage holds the MB A tiles together
// with all NBP planes of the B tile (B_hi, B_lo).  Per K tile the MMA warp
// issues NBP x MB x KB/16 MMAs.  Fewer bytes move from L2 per multiply-add
// than with 128-row tiles.  KB = 32 halves the stage (64-byte swizzled rows)
// so that twice as many stages, and twice the bytes in flight, fit in
// shared memory.  Persistent over (split, m tile, n tile); the accumulators
// are drained by the epilogue before the next tile starts.
//
// K tiles are numbered in units of KB along (P, b): tile kr covers
// b = (kr % (vp/KB)) * KB .. +KB of P = kr / (vp/KB).  Z is stored in
// 64-wide b tiles, so a 32-wide K tile is the half (kr & 1) of Z tile kr/2.
//
// TR (transposed): the same contraction with the operands swapped, for
// batches whose C*o rows fill 128-row tiles poorly (one trajectory): rows
// are a (A = the NBP B_vv planes, MB 128-row blocks each), columns are
// (col, i) (B = one Z plane of BN rows), and the epilogue writes the
// partials transposed, out[split][(col, i)][a], the layout the combine
// reads; a warp then stores 32 consecutive a of one (col, i).
// ---------------------------------------------------------------------------
template <int BN, int MB, int NBP, int KB, bool TR = false>
struct WideCfg {
  static constexpr int kRowBytes = KB * 2;
  static constexpr int kABlock = kBM * kRowBytes;   // one 128-row A tile
  static constexpr int kBBytes = BN * kRowBytes;    // one B plane
  static constexpr int kATiles = TR ? MB * NBP : MB;
  static constexpr int kBTiles = TR ? 1 : NBP;
  static constexpr int kStageBytes = kATiles * kABlock + kBTiles * kBBytes;
  static constexpr int kCols = MB * BN;
  static constexpr uint32_t kTmemCols = kCols <= 32 ? 32 : kCols <= 64 ? 64 : kCols <= 128 ? 128
                                        : kCols <= 256 ? 256 : 512;
  static_assert(kCols <= 512, "accumulators exceed TMEM");
  static_assert(kStageBytes % 1024 == 0, "stage must keep 1024-byte alignment");
  static_assert(BN % 32 == 0 && BN <= 256, "BN must be a multiple of 32 and <= 256");
  static_assert(KB == 64 || KB == 32, "K tile of 64 or 32 BF16");
};

template <int BN, int MB, int NBP, int STAGES, int KB, bool TR = false>
constexpr size_t wide_smem_bytes() {
  return (size_t)STAGES * WideCfg<BN, MB, NBP, KB, TR>::kStageBytes + 1024 + 256;
}

// CL > 1 (not TR): the kernel runs in clusters of CL CTAs that take CL
// consecutive column tiles of the same rows and K range (launch with a grid
// that is a multiple of CL, and tiles_n a multiple of CL).  Each CTA loads
// 128/CL rows of every A (Z) block and multicasts them to the whole cluster,
// so a Z tile leaves L2 once per cluster instead of once per CTA and the
// cluster's CTAs advance through K together.  tmA is then the map of
// 128/CL-row boxes.  A stage is refilled only when every CTA of the
// cluster has released it: each CTA's MMA commit arrives on the stage's
// empty barrier in all CL CTAs.
template <int BN, int MB, int NBP, int STAGES, int KB, bool TR = false, int CL = 1>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_wide(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Params p) {
  static_assert(CL == 1 || (!TR && (CL == 2 || CL == 4)), "clusters of 2 or 4, not transposed");
  using CF = WideCfg<BN, MB, NBP, KB, TR>;
  constexpr int TM = kBM * MB;  // rows per tile
  constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * CF::kStageBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (p.N + BN - 1) / BN;
  const int tiles_m = (p.M + TM - 1) / TM;
  const int ntiles = tiles_n * tiles_m * p.nsplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CL);  // one commit per CTA of the cluster
    }
    mbar_init(accf, 1);
    mbar_init(acce, kEpiWarps);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, CF::kTmemCols);
  tc_fence_before();
  __syncthreads();
  // the cluster's barriers are initialised before any CTA multicasts into them
  if constexpr (CL > 1) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto coords = [&](int t, int& n0, int& m0, int& split) {
    n0 = (t % tiles_n) * BN;
    m0 = ((t / tiles_n) % tiles_m) * TM;
    split = t / (tiles_n * tiles_m);
  };

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool alive = true;
      for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
        int n0, m0, split;
        coords(t, n0, m0, split);
        const int kr0 = split * p.kt_per_split;
        const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
        for (int kr = kr0; kr < kr1; ++kr, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, p.err, ERR_WAIT_EMPTY)) {
            alive = false;
            break;
          }
          uint8_t* st = smem + s * CF::kStageBytes;
          mbar_expect_tx(&full[s], CF::kStageBytes);
          const int zt = KB == 64 ? kr : kr >> 1, zx = KB == 64 ? 0 : (kr & 1) * KB;
          const int P = kr / p.vtiles, b0 = (kr % p.vtiles) * KB;
          if (TR) {
            // A: plane q, row block b of B_vv at (b0, a, P); B: the Z tile
#pragma unroll
            for (int q = 0; q < NBP; ++q)
#pragma unroll
              for (int b = 0; b < MB; ++b)
                tma_load_4d(st + (q * MB + b) * CF::kABlock, &tmA, &full[s], b0, m0 + b * kBM, P, q);
            tma_load_4d(st + MB * NBP * CF::kABlock, &tmB, &full[s], zx, n0, zt, 0);
          } else {
            if constexpr (CL > 1) {
              // this CTA's 128/CL rows of every A block, to the whole cluster
              constexpr int RS = kBM / CL;
              const int rk = (int)cluster_rank();
#pragma unroll
              for (int b = 0; b < MB; ++b)
                tma_load_4d_mc(st + b * CF::kABlock + rk * RS * CF::kRowBytes, &tmA, &full[s], zx,
                               m0 + b * kBM + rk * RS, zt, 0, kMask);
            } else {
#pragma unroll
              for (int b = 0; b < MB; ++b)
                tma_load_4d(st + b * CF::kABlock, &tmA, &full[s], zx, m0 + b * kBM, zt, 0);
            }
#pragma unroll
            for (int q = 0; q < NBP; ++q)
              tma_load_4d(st + MB * CF::kABlock + q * CF::kBBytes, &tmB, &full[s], b0, n0, P, q);
          }
        }
      }
      drain_loads(full, it, STAGES);
      if constexpr (CL > 1) {
        // every CTA of the cluster has released the last stages, so no
        // commit of another CTA is still on its way to this CTA's barriers
        for (int j = max(0, it - STAGES); j < it; ++j)
          mbar_wait(&empty[j % STAGES], (uint32_t)(j / STAGES) & 1u, nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      int it = 0, tcount = 0;
      bool alive = true;
      for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x, ++tcount) {
        int n0, m0, split;
        coords(t, n0, m0, split);
        const int kr0 = split * p.kt_per_split;
        const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
        if (!mbar_wait(acce, ((uint32_t)tcount & 1u) ^ 1u, p.err, ERR_WAIT_ACC)) break;
        tc_fence_after();
        for (int kr = kr0; kr < kr1; ++kr, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph, p.err, ERR_WAIT_FULL)) {
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * CF::kStageBytes);
#pragma unroll
          for (int q = 0; q < NBP; ++q) {
            const uint64_t bdesc = sdesc_k<KB>(base + CF::kATiles * CF::kABlock + (TR ? 0 : q) * CF::kBBytes);
#pragma unroll
            for (int b = 0; b < MB; ++b) {
              const uint64_t adesc = sdesc_k<KB>(base + (TR ? q * MB + b : b) * CF::kABlock);
#pragma unroll
              for (int k = 0; k < KB / 16; ++k)
                mma_bf16(tmem + b * BN, adesc + 2 * k, bdesc + 2 * k, idesc,
                         (kr > kr0 || q > 0 || k > 0) ? 1u : 0u);
            }
          }
          if constexpr (CL > 1)
            mma_commit_mc(&empty[s], kMask);
          else
            mma_commit(&empty[s]);
        }
        mma_commit(accf);
      }
    }
  } else {
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    int tcount = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tcount) {
      int n0, m0, split;
      coords(t, n0, m0, split);
      const int kr0 = split * p.kt_per_split;
      const int kr1 = min(p.kt_total, kr0 + p.kt_per_split);
      const bool has_k = kr1 > kr0;
      const bool ok = mbar_wait(accf, (uint32_t)tcount & 1u, p.err, ERR_WAIT_ACC);
      tc_fence_after();
      for (int b = 0; b < MB; ++b) {
        const int m = m0 + b * kBM + row;
        // TR: element (m = a, n = (col, i)) goes to out[n][a] (ldo = nvirt)
        float* dst = p.out + (size_t)split * p.split_stride + (TR ? (size_t)m : (size_t)m * p.ldo);
        const size_t nstride = TR ? (size_t)p.ldo : 1;
        for (int ci = half; ci < BN / 32; ci += 2) {
          const int c = ci * 32;
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + b * BN + c, r);
          if (m < p.M && ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = n0 + c + j;
              if (n < p.N) {
                const float x = has_k ? __uint_as_float(r[j]) : 0.0f;
                float* d = dst + (size_t)n * nstride;
                *d = p.accum ? *d + x : x;
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce);
      if (!ok) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  // no CTA leaves while another CTA of its cluster may still write to it
  if constexpr (CL > 1) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, CF::kTmemCols);
  }
}

}  // namespace tc
}  // namespace rttda
