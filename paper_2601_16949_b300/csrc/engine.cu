// RT-TDA engine: device buffers, precision plan, RK4 schedule, CUDA graphs,
// and the C ABI declared in include/rttda.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/rttda.h"
#include "engine_internal.h"
#include "kernels_simt.cuh"
#include "tc_gemm.cuh"
#include "ozaki.cuh"
#include "coul_stream.cuh"

using namespace rttda;

namespace rttda {
thread_local std::string g_last_error;

rttda_status set_error(rttda_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
}  // namespace rttda

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      return set_error(e_ == cudaErrorMemoryAllocation ? RTTDA_E_OOM : RTTDA_E_CUDA,               \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                              \
  } while (0)

#define CKS(expr)                         \
  do {                                    \
    rttda_status s_ = (expr);             \
    if (s_ != RTTDA_OK) return s_;        \
  } while (0)

namespace {

constexpr int kNumSM = 148;

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

inline unsigned blocks_for(long long n, int threads) { return (unsigned)std::max(1LL, cdiv(n, threads)); }

// SIMT GEMM tile shapes per compute type.
template <typename TC> struct Tile;
template <> struct Tile<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <> struct Tile<float> { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };

// A handle's device buffers are allocated and freed in stream order on the
// handle's stream (CUDA's memory pool) while a function of that handle runs:
// creating, re-batching or destroying one handle then never waits for the
// work of other handles on the device, as cudaMalloc / cudaFree can.
thread_local cudaStream_t g_alloc_stream = nullptr;

struct AllocStream {
  cudaStream_t prev;
  explicit AllocStream(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocStream() { g_alloc_stream = prev; }
};

rttda_status dalloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  if (g_alloc_stream)
    CK(cudaMallocAsync(p, bytes, g_alloc_stream));
  else
    CK(cudaMalloc(p, bytes));
  return RTTDA_OK;
}

template <typename T>
rttda_status dalloc(T** p, size_t count) {
  return dalloc_bytes((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

void dfree(void* p) {
  if (!p) return;
  if (g_alloc_stream)
    cudaFreeAsync(p, g_alloc_stream);
  else
    cudaFree(p);
}

double fro(const double* a, size_t n) {
  double s = 0.0;
  for (size_t k = 0; k < n; ++k) s += a[k] * a[k];
  return std::sqrt(s);
}

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct rttda_ctx {
  int o = 0, v = 0, P = 0, prec = 0;
  long long ov = 0, N = 0;
  double cx = 0.0;
  size_t fbytes = 8, cbytes = 8;
  cudaStream_t stream = nullptr;

  // factors (working precision)
  void* Bov = nullptr;
  void* Boo = nullptr;
  void* Bvv = nullptr;
  double* eps_o = nullptr;
  double* eps_v = nullptr;
  double* mu_oo = nullptr;  // [3][o][o]
  double* mu_vv = nullptr;  // [3][v][v]
  double* mu_0 = nullptr;   // [3][o][v]
  double mu_bound[3] = {0, 0, 0};

  // batch
  int T = 0;
  std::vector<rttda_pulse> pulses;
  PulseDev* d_pulses = nullptr;
  double* d_kappa = nullptr;
  double* d_dirs = nullptr;
  double* moo64 = nullptr;
  double* mvv64 = nullptr;
  double* m064 = nullptr;
  void* mooC = nullptr;
  void* mvvC = nullptr;
  // one-polarisation batches in the FP32 modes: the field GEMMs' operands
  // in their arithmetic types (the stage input cast per call into Xfc; the
  // first trajectory's FP64 dipole blocks as double-float pairs)
  void* Xfc = nullptr;     // [N][C] float or df32
  void* moo_df = nullptr;  // [o][o] df32
  void* mvv_df = nullptr;  // [v][v] df32
  void* m0C = nullptr;
  bool any_field = false, any_kick = false;
  bool same_dir = false;  // every trajectory of the batch has the same polarisation
  int kick_terms = 0;

  // state and scratch
  double* Xn = nullptr;
  double* Xs = nullptr;
  double* Xs2 = nullptr;  // second stage-input buffer
  double* acc = nullptr;
  double* F = nullptr;
  double* E = nullptr;
  double* term = nullptr;
  double* obs_part = nullptr;
  double* Xq = nullptr;  // sigma entry input
  long long* d_step = nullptr;
  cudaGraphExec_t step_exec = nullptr;  // the step graph kept between calls
  void* w = nullptr;
  void* Jpart = nullptr;
  void* Zt = nullptr;
  void* Kpart = nullptr;
  int SJ = 1, pchunkJ = 1, SK = 1, zchunk = 1, obsG = 1, SW = 1, wslice = 1;
  bool coul_vec = false;
  bool coul_stream = false;  // Coulomb on the FP32 streaming kernels (FP32 / BF16 factors, 2T <= 12)
  float* Xf = nullptr;       // [ov][C] FP32 amplitudes of the stage (streaming Coulomb)
  double* f0_part = nullptr; // [T][chunks][2] ground-row field partial sums
  long long obs_rows = 1;
  size_t dev_bytes = 0;

  bool have_state = false;
  double t_now = 0.0;

  // tensor-core exchange (BF16 / BF16X3): padded BF16 planes and TMA maps
  bool tc = false;
  int nplanes = 1, nprod = 1, vp = 0, op = 0, tc_bn = 256;
  int zplanes = 1, nprod_main = 1;  // Z planes kept; products in the main contraction
  int wide_mb = 0;                   // >0: main contraction on the wide-M kernel with this many 128-row blocks
  int wide_kb = 32;                  // K tile width of the wide-M kernel (32 or 64 BF16)
  bool wide_tr = false;              // wide kernel with the contraction transposed (rows a)
  int wide_cl = 1;                   // >1: clustered wide kernel, CL CTAs share Z tiles by multicast
  int wide_grid = 0;                 // its grid (co-resident clusters x CL)
  long capture_fallbacks = 0;        // propagation calls whose step-graph capture was invalidated
  bool break_capture = false;        // test hook (RTTDA_TEST_BREAK_CAPTURE): invalidate every capture
  int z_hint = 1;                    // Z stores evict-first in L2 (RTTDA_ZHINT)
  int z_res1 = 1;                    // one-plane stages for the one-product Z build (RTTDA_ZRES1)
  int z_run = 4;                     // Z-build tiles per CTA and column run in a slab, 0: no slabs (RTTDA_ZRUN)
  int integrator = RTTDA_INT_RK4;    // rttda_integrator
  // projectors (Eq. (22)) and the overlaps of the last propagation
  int nproj = 0;
  double* d_proj = nullptr;   // [nproj][N]
  double* d_ovl = nullptr;    // [T][ovl_ld][nproj][2]
  double* d_proj_part = nullptr;
  long long ovl_ld = 0, ovl_cap = 0, proj_rows = 1, part_cap = 0;
  int proj_G = 1;
  // autocorrelation R(t) = X(eps)^dagger X(eps + t) (Eq. (20))
  bool acf_on = false;
  double* d_xeps = nullptr;   // [N][2T] state right after the kick of the last fresh propagation
  double* d_acf = nullptr;    // [T][acf_ld][2]
  double* d_acf_part = nullptr;
  long long acf_ld = 0, acf_cap = 0, acf_eps_cap = 0, acf_part_cap = 0;
  bool have_eps = false;
  rttda_plan_info plan{};            // the exchange plan in use (rttda_plan)
  __nv_bfloat16* Bvv_tc = nullptr;  // [plane][P][vp][vp]
  __nv_bfloat16* Boo_tc = nullptr;  // [plane][P*o][op]
  __nv_bfloat16* Xt = nullptr;      // [plane][C*vp][op]
  __nv_bfloat16* Zk = nullptr;      // [plane][C*o][zchunk*vp]
  size_t zplane = 0;
  std::vector<CUtensorMap> tmZA, tmMA, tmMB, tmZS;
  std::vector<CUtensorMap> tmMAc;  // Z in 128/wide_cl-row boxes (clustered main contraction)
  CUtensorMap tmZB;
  std::vector<int> tc_kper;
  int* d_err = nullptr;
  // tensor-core Coulomb (batches with 2T >= 16 columns)
  __nv_bfloat16* Bov_tc = nullptr;   // [plane][P][ov]
  __nv_bfloat16* BovT_tc = nullptr;  // [plane][ov][P]
  __nv_bfloat16* Xc = nullptr;       // [plane][C][ov]
  __nv_bfloat16* Wt = nullptr;       // [plane][C][P]
  float* wpart_tc = nullptr;         // [SKc1][P][C]
  bool coul_tc = false;
  int SKc1 = 1, SKc2 = 1;
  CUtensorMap tmC1A, tmC1B, tmC2A, tmC2B;
  // FP64-accurate exchange by BF16 digits (FP64_OZ): factor digits (set up
  // at create), per-batch digits of the amplitudes and of Z, and the maps
  bool oz = false;
  __nv_bfloat16* oz_boo = nullptr;  // [digit][P*o][op]
  short* oz_eoo = nullptr;          // [P*o] block exponents
  __nv_bfloat16* oz_bvv = nullptr;  // [digit][P][v][vp]
  short* oz_evv = nullptr;          // [P*nbp][vp] (columns a < v used)
  int oz_nbp = 1;                   // exactness blocks per P along b
  __nv_bfloat16* oz_x = nullptr;    // [digit][C*vp][op]
  int* oz_ex = nullptr;             // [C*vp]
  long long* oz_zi = nullptr;       // [zchunk*o][C*vp] integer Z of the Z build
  __nv_bfloat16* oz_z = nullptr;    // [digit][(zchunk, vp/64)][C*o][64]
  int* oz_ez = nullptr;             // [zchunk*nbp][C*o] block exponents of Z
  size_t oz_zplane = 0;
  int oz_pps = 1;                   // P per split of the main contraction
  // Coulomb on digits: B_ov (rows P, K = ia) and its transpose (rows ia,
  // K = P) set up at create; per batch the amplitudes (rows col, K = ia),
  // the first pass's FP64 partials and the digits of 2w (rows col, K = P)
  __nv_bfloat16* oz_bov = nullptr;   // [digit][P][ovp]
  int* oz_ebov = nullptr;            // [nkb][P]
  __nv_bfloat16* oz_bovt = nullptr;  // [digit][ov][Pp]
  int* oz_ebovt = nullptr;           // [npb][ov]
  int oz_ovp = 8, oz_Pp = 8, oz_nkb = 1, oz_npb = 1;
  __nv_bfloat16* oz_xc = nullptr;    // [digit][cp][ovp]
  short* oz_exc = nullptr;           // [nkb][cp]
  double* oz_wpart = nullptr;        // [SW][P][C]
  __nv_bfloat16* oz_w = nullptr;     // [digit][cp][Pp]
  short* oz_ew = nullptr;            // [npb][cp]
  int oz_cp = 64, oz_pps1 = 1, oz_pps2 = 1;
  CUtensorMap tmOzBov, tmOzBovT, tmOzXc, tmOzW;
  CUtensorMap tmOzX;
  std::vector<CUtensorMap> tmOzBoo, tmOzZ, tmOzBvv;

  // host staging for the host-buffer entry points
  double* h_io = nullptr;  // device staging [T][N][2] + traces
  size_t h_io_count = 0;

  // profiling: CUDA events around every kernel class (no graphs while on)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev[RTTDA_NUM_KERNEL_CLASSES];
  size_t prof_used[RTTDA_NUM_KERNEL_CLASSES] = {};
  long long launches = 0;        // kernels enqueued (running count)
  long long launches_per_step = 0;

  ~rttda_ctx();
  rttda_status alloc_batch();
  rttda_status alloc_tc(int C);
  void free_batch();
};

rttda_ctx::~rttda_ctx() {
  if (stream) cudaStreamSynchronize(stream);
  if (step_exec) cudaGraphExecDestroy(step_exec);
  AllocStream as(stream);
  for (auto& v : prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  free_batch();
  dfree(Bov);
  dfree(Boo);
  dfree(Bvv);
  dfree(eps_o);
  dfree(eps_v);
  dfree(mu_oo);
  dfree(mu_vv);
  dfree(mu_0);
  dfree(Bvv_tc);
  dfree(Boo_tc);
  dfree(oz_boo);
  dfree(oz_eoo);
  dfree(oz_bvv);
  dfree(oz_evv);
  dfree(oz_bov);
  dfree(oz_ebov);
  dfree(oz_bovt);
  dfree(oz_ebovt);
  dfree(Bov_tc);
  dfree(BovT_tc);
  dfree(d_err);
  dfree(d_proj);
  dfree(d_ovl);
  dfree(d_proj_part);
  dfree(d_xeps);
  dfree(d_acf);
  dfree(d_acf_part);
  if (stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
}

void rttda_ctx::free_batch() {
  void* ps[] = {d_pulses, d_kappa, d_dirs, moo64, mvv64, m064, mooC, mvvC, m0C, Xfc, moo_df, mvv_df,
                Xn, Xs, Xs2, acc, F, E, term,
                obs_part, Xq, d_step, w, Jpart, Zt, Kpart, h_io, Xt, Zk, Xc, Wt, wpart_tc, Xf, f0_part,
                oz_x, oz_ex, oz_zi, oz_z, oz_ez, oz_xc, oz_exc, oz_wpart, oz_w, oz_ew};
  for (void* p : ps) dfree(p);
  d_pulses = nullptr;
  d_kappa = d_dirs = moo64 = mvv64 = m064 = nullptr;
  mooC = mvvC = m0C = nullptr;
  Xfc = moo_df = mvv_df = nullptr;
  Xn = Xs = Xs2 = acc = F = E = term = obs_part = Xq = nullptr;
  d_step = nullptr;
  w = Jpart = Zt = Kpart = nullptr;
  Xt = Zk = nullptr;
  Xc = Wt = nullptr;
  wpart_tc = nullptr;
  Xf = nullptr;
  f0_part = nullptr;
  oz_x = nullptr;
  oz_ex = nullptr;
  oz_zi = nullptr;
  oz_z = nullptr;
  oz_ez = nullptr;
  oz_xc = nullptr;
  oz_exc = nullptr;
  oz_wpart = nullptr;
  oz_w = nullptr;
  oz_ew = nullptr;
  tmOzBoo.clear();
  tmOzZ.clear();
  tmOzBvv.clear();
  coul_tc = false;
  coul_stream = false;
  tmZA.clear();
  tmZS.clear();
  tmMA.clear();
  tmMAc.clear();
  tmMB.clear();
  tc_kper.clear();
  h_io = nullptr;
  h_io_count = 0;
  T = 0;
  have_state = false;
  have_eps = false;
  acf_ld = 0;
}

// ---------------------------------------------------------------------------
// Profiling hooks: an event pair around each launch of a kernel class.
// ---------------------------------------------------------------------------
namespace {

struct Prof {
  rttda_ctx* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t stop = nullptr;
  Prof(rttda_ctx* h_, int cls_, cudaStream_t s_) : h(h_), cls(cls_), s(s_) {
    if (!h->prof_on) return;
    auto& v = h->prof_ev[cls];
    size_t& u = h->prof_used[cls];
    while (v.size() < u + 2) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      v.push_back(e);
    }
    cudaEventRecord(v[u], s);
    stop = v[u + 1];
    u += 2;
  }
  ~Prof() {
    if (stop) cudaEventRecord(stop, s);
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// Precision-dispatched launches
// ---------------------------------------------------------------------------
namespace {

// --- tensor-core exchange -------------------------------------------------
// Z = B_oo c (K = nocc, short): pipeline stages with hi/lo Z staging (two
// planes) or one-plane staging
constexpr int kZBN = 256, kZStages2 = 2, kZStages1 = 2, kZStagesR = 3, kZStagesR1 = 6;

// Persistent launch: one CTA per SM (or per tile if fewer tiles).
template <int BN, int ST, int BM, int EP>
void tc_launch(const CUtensorMap& a, const CUtensorMap& b, const tc::Params& prm, cudaStream_t s,
               const CUtensorMap* z = nullptr) {
  const long long tiles = cdiv(prm.N, BN) * cdiv(prm.M, tc::kBM) * prm.nsplit;
  const unsigned grid = (unsigned)std::max(1LL, std::min<long long>(tiles, kNumSM));
  tc::k_tc_gemm<BN, ST, BM, EP><<<grid, tc::kThreads, tc::smem_bytes<BN, ST, EP>(), s>>>(a, b, z ? *z : a, prm);
}

template <int BN, int MB, int NBP, int ST, int KB, bool TR = false>
void wide_launch(const CUtensorMap& a, const CUtensorMap& b, const tc::Params& prm, cudaStream_t s) {
  const long long tiles = cdiv(prm.N, BN) * cdiv(prm.M, (long long)tc::kBM * MB) * prm.nsplit;
  const unsigned grid = (unsigned)std::max(1LL, std::min<long long>(tiles, kNumSM));
  tc::k_tc_wide<BN, MB, NBP, ST, KB, TR>
      <<<grid, tc::kThreads, tc::wide_smem_bytes<BN, MB, NBP, ST, KB, TR>(), s>>>(a, b, prm);
}

template <int BN, int MB, int NBP, int ST, int KB, bool TR = false>
void wide_attr() {
  static_assert(tc::wide_smem_bytes<BN, MB, NBP, ST, KB, TR>() <= 232448, "shared memory per block exceeds 227 KB");
  cudaFuncSetAttribute(tc::k_tc_wide<BN, MB, NBP, ST, KB, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::wide_smem_bytes<BN, MB, NBP, ST, KB, TR>());
}

// Clustered wide-M main contraction (BN 192, two 128-row blocks, K tile KB
// of 64 or 32): clusters of CL CTAs over CL consecutive column tiles share
// every Z tile by TMA multicast.  `a` is the map of 128/CL-row Z boxes;
// `grid` a multiple of CL that is co-resident (wide_cluster_capacity).
// Stages as in the plain plans: K tile 64 holds 4 (one B_vv plane) or 2
// (two planes), K tile 32 holds 8 or 5.
template <int NBP, int KB>
constexpr int wide_cluster_stages() {
  return KB == 64 ? (NBP == 2 ? 2 : 4) : (NBP == 2 ? 5 : 8);
}

template <int NBP, int KB, int CL>
cudaLaunchConfig_t wide_cluster_config(cudaLaunchAttribute* at, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(tc::kThreads);
  cfg.dynamicSmemBytes = tc::wide_smem_bytes<192, 2, NBP, wide_cluster_stages<NBP, KB>(), KB>();
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <int NBP, int KB, int CL>
void wide_cluster_launch(const CUtensorMap& a, const CUtensorMap& b, const tc::Params& prm, cudaStream_t s,
                         int grid) {
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = wide_cluster_config<NBP, KB, CL>(at, grid, s);
  cudaLaunchKernelEx(&cfg, tc::k_tc_wide<192, 2, NBP, wide_cluster_stages<NBP, KB>(), KB, false, CL>, a, b, prm);
}

// CTAs of the clustered kernel that can be resident at once (a multiple of
// CL; clusters must fit inside one GPC), 0 if none.
template <int NBP, int KB, int CL>
int wide_cluster_capacity() {
  constexpr int ST = wide_cluster_stages<NBP, KB>();
  auto kern = tc::k_tc_wide<192, 2, NBP, ST, KB, false, CL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::wide_smem_bytes<192, 2, NBP, ST, KB>());
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = wide_cluster_config<NBP, KB, CL>(at, CL * 64, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n * CL;
}

template <int KB>
int wide_cluster_capacity_kb(int nbp, int cl) {
  if (nbp == 2) return cl == 4 ? wide_cluster_capacity<2, KB, 4>() : wide_cluster_capacity<2, KB, 2>();
  return cl == 4 ? wide_cluster_capacity<1, KB, 4>() : wide_cluster_capacity<1, KB, 2>();
}

int wide_cluster_capacity(int nbp, int kb, int cl) {
  return kb == 32 ? wide_cluster_capacity_kb<32>(nbp, cl) : wide_cluster_capacity_kb<64>(nbp, cl);
}

template <int KB>
void wide_cluster_dispatch_kb(int nbp, int cl, const CUtensorMap& a, const CUtensorMap& b, const tc::Params& prm,
                              cudaStream_t s, int grid) {
  if (nbp == 2) {
    if (cl == 4) wide_cluster_launch<2, KB, 4>(a, b, prm, s, grid);
    else wide_cluster_launch<2, KB, 2>(a, b, prm, s, grid);
  } else {
    if (cl == 4) wide_cluster_launch<1, KB, 4>(a, b, prm, s, grid);
    else wide_cluster_launch<1, KB, 2>(a, b, prm, s, grid);
  }
}

void wide_cluster_dispatch(int nbp, int kb, int cl, const CUtensorMap& a, const CUtensorMap& b,
                           const tc::Params& prm, cudaStream_t s, int grid) {
  if (kb == 32)
    wide_cluster_dispatch_kb<32>(nbp, cl, a, b, prm, s, grid);
  else
    wide_cluster_dispatch_kb<64>(nbp, cl, a, b, prm, s, grid);
}

// Transposed wide configurations (rows a in two 128-row blocks, columns
// (col, i) in tiles of BN, K tiles of 32): BN in {64, 96, 128, 160, 192,
// 256}; 4 stages with both B_vv planes, 6 with one.
constexpr int kTrBN[6] = {64, 96, 128, 160, 192, 256};

template <int NBP>
void wide_tr_launch(int bn, const CUtensorMap& a, const CUtensorMap& b, const tc::Params& prm, cudaStream_t s) {
  constexpr int ST = NBP == 2 ? 4 : 6;
  switch (bn) {
    case 64: wide_launch<64, 2, NBP, ST, 32, true>(a, b, prm, s); break;
    case 96: wide_launch<96, 2, NBP, ST, 32, true>(a, b, prm, s); break;
    case 128: wide_launch<128, 2, NBP, ST, 32, true>(a, b, prm, s); break;
    case 160: wide_launch<160, 2, NBP, ST, 32, true>(a, b, prm, s); break;
    case 192: wide_launch<192, 2, NBP, ST, 32, true>(a, b, prm, s); break;
    default: wide_launch<256, 2, NBP, ST, 32, true>(a, b, prm, s); break;
  }
}

template <int NBP>
void wide_tr_attr() {
  constexpr int ST = NBP == 2 ? 4 : 6;
  wide_attr<64, 2, NBP, ST, 32, true>();
  wide_attr<96, 2, NBP, ST, 32, true>();
  wide_attr<128, 2, NBP, ST, 32, true>();
  wide_attr<160, 2, NBP, ST, 32, true>();
  wide_attr<192, 2, NBP, ST, 32, true>();
  wide_attr<256, 2, NBP, ST, 32, true>();
}

// The wide-M configurations: (BN, MB) in {(160, 3), (192, 2)}, one or two B
// planes, K tiles of 64 (128-byte rows) or 32 (64-byte rows, twice the
// stages).  Stage counts fill the 227 KB of shared memory.
void wide_dispatch(int bn, int mb, int nbp, int kb, const CUtensorMap& a, const CUtensorMap& b,
                   const tc::Params& prm, cudaStream_t s, bool tr = false) {
  if (tr) {
    if (nbp == 2)
      wide_tr_launch<2>(bn, a, b, prm, s);
    else
      wide_tr_launch<1>(bn, a, b, prm, s);
    return;
  }
  const bool w3 = bn == 160 && mb == 3;
  if (kb == 32) {
    if (nbp == 2) {
      if (w3) wide_launch<160, 3, 2, 5, 32>(a, b, prm, s);
      else wide_launch<192, 2, 2, 5, 32>(a, b, prm, s);
    } else {
      if (w3) wide_launch<160, 3, 1, 6, 32>(a, b, prm, s);
      else wide_launch<192, 2, 1, 8, 32>(a, b, prm, s);
    }
  } else {
    if (nbp == 2) {
      if (w3) wide_launch<160, 3, 2, 2, 64>(a, b, prm, s);
      else wide_launch<192, 2, 2, 2, 64>(a, b, prm, s);
    } else {
      if (w3) wide_launch<160, 3, 1, 3, 64>(a, b, prm, s);
      else wide_launch<192, 2, 1, 4, 64>(a, b, prm, s);
    }
  }
}

template <int BN, int ST, int BM, int EP>
void tc_attr() {
  static_assert(tc::smem_bytes<BN, ST, EP>() <= 232448, "shared memory per block exceeds 227 KB");
  cudaFuncSetAttribute(tc::k_tc_gemm<BN, ST, BM, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::smem_bytes<BN, ST, EP>());
}

void set_tc_smem_limits() {
  tc_attr<kZBN, kZStages2, tc::BMODE_PLAIN, tc::EPI_ZSPLIT>();
  tc_attr<kZBN, kZStages1, tc::BMODE_PLAIN, tc::EPI_ZONE>();
  tc_attr<kZBN, kZStagesR, tc::BMODE_PLAIN, tc::EPI_ZRES>();
  tc_attr<kZBN, kZStagesR1, tc::BMODE_PLAIN, tc::EPI_ZRES1>();
  tc_attr<128, 7, tc::BMODE_VV, tc::EPI_PARTIAL>();
  tc_attr<224, 5, tc::BMODE_VV, tc::EPI_PARTIAL>();
  tc_attr<256, 4, tc::BMODE_VV, tc::EPI_PARTIAL>();
  tc_attr<64, 8, tc::BMODE_PLAIN, tc::EPI_PARTIAL>();
  wide_attr<160, 3, 2, 5, 32>();
  wide_attr<192, 2, 2, 5, 32>();
  wide_attr<160, 3, 1, 6, 32>();
  wide_attr<192, 2, 1, 8, 32>();
  wide_attr<160, 3, 2, 2, 64>();
  wide_attr<192, 2, 2, 2, 64>();
  wide_attr<160, 3, 1, 3, 64>();
  wide_attr<192, 2, 1, 4, 64>();
  wide_tr_attr<2>();
  wide_tr_attr<1>();
}

// Batched Coulomb on tensor cores: w = B_ov c (split-K over ia), then
// J = B_ov^T (2w) with B_ov^T stored transposed; BF16 planes as in the
// exchange, J as FP32 split-K partials for the combine.
void coulomb_tc(rttda_ctx* h, const double* X, cudaStream_t s) {
  Prof pr(h, RTTDA_KC_COULOMB, s);
  h->launches += 4;
  const int C = 2 * h->T, P = h->P;
  const long long ov = h->ov;
  k_prep_xc<<<blocks_for(ov, 32), 256, (size_t)32 * (C + 1) * sizeof(double), s>>>(
      ov, C, X, h->Xc, h->nplanes > 1 ? h->Xc + (size_t)C * ov : nullptr);
  {
    tc::Params prm{};
    prm.M = P;
    prm.N = C;
    prm.kt_total = (int)cdiv(ov, tc::kBK);
    prm.nsplit = h->SKc1;
    prm.kt_per_split = (int)cdiv(prm.kt_total, h->SKc1);
    prm.nprod = h->nprod;
    prm.out = h->wpart_tc;
    prm.ldo = C;
    prm.split_stride = (long long)P * C;
    prm.err = h->d_err;
    tc_launch<64, 8, tc::BMODE_PLAIN, tc::EPI_PARTIAL>(h->tmC1A, h->tmC1B, prm, s);
  }
  k_prep_wt<<<blocks_for((long long)P * C, 256), 256, 0, s>>>(P, C, h->SKc1, h->wpart_tc, h->Wt,
                                                               h->nplanes > 1 ? h->Wt + (size_t)C * P : nullptr);
  {
    tc::Params prm{};
    prm.M = (int)ov;
    prm.N = C;
    prm.kt_total = (int)cdiv(P, tc::kBK);
    prm.nsplit = h->SKc2;
    prm.kt_per_split = (int)cdiv(prm.kt_total, h->SKc2);
    prm.nprod = h->nprod;
    prm.out = (float*)h->Jpart;
    prm.ldo = C;
    prm.split_stride = ov * C;
    prm.err = h->d_err;
    tc_launch<64, 8, tc::BMODE_PLAIN, tc::EPI_PARTIAL>(h->tmC2A, h->tmC2B, prm, s);
  }
}

// BF16 planes of the stage's amplitudes for the Z build; with_xf: the same
// launch writes the FP32 copy the streaming Coulomb reads (ov x C <= the
// plane grid, since vp >= v and op >= o).
void prep_xt(rttda_ctx* h, const double* X, bool with_xf, cudaStream_t s) {
  const int C = 2 * h->T;
  const long long tot = (long long)C * h->vp * h->op;
  k_prep_xt<<<blocks_for(tot, 256), 256, 0, s>>>(h->o, h->v, h->vp, h->op, C, X, h->Xt,
                                                h->nplanes > 1 ? h->Xt + tot : nullptr,
                                                with_xf ? h->ov * C : 0, with_xf ? h->Xf : nullptr);
}

// xt_done: the planes of X are already in Xt (written with the Coulomb's
// FP32 copy by one launch).
void exchange_tc(rttda_ctx* h, const double* X, cudaStream_t s, bool xt_done = false) {
  const int C = 2 * h->T, o = h->o, v = h->v, vp = h->vp, op = h->op;
  if (!xt_done) {
    Prof pr(h, RTTDA_KC_EXCHANGE_Z, s);
    h->launches += 1;
    prep_xt(h, X, false, s);
  }
  for (int c = 0, p0 = 0; p0 < h->P; p0 += h->zchunk, ++c) {
    const int pc = std::min(h->zchunk, h->P - p0);
    {
      // Z^P_(col,i),b = sum_j B^P_ij c_(j,b),col for P in the chunk (BF16 planes out)
      Prof pr(h, RTTDA_KC_EXCHANGE_Z, s);
      h->launches += 1;
      tc::Params prm{};
      prm.M = pc * o;
      prm.N = C * vp;
      prm.kt_total = (int)cdiv(op, tc::kBK);
      prm.kt_per_split = prm.kt_total;
      prm.nsplit = 1;
      // Z enters the main contraction as one BF16 plane in BF16X2: its
      // activation part needs no lo plane, B_oo keeps hi + lo
      prm.nprod = h->zplanes == 1 && h->nplanes > 1 ? 2 : h->nprod;
      prm.alo = prm.nprod == 2 ? 1 : 0;
      prm.zhi = h->Zk;
      prm.zlo = h->zplanes > 1 ? h->Zk + h->zplane : nullptr;
      prm.o = o;
      prm.vp = vp;
      prm.zrows = C * o;
      prm.ztma = (o % 32 == 0) ? 1 : 0;
      prm.zhint = h->z_hint;
      prm.zrun = h->z_run;
      prm.err = h->d_err;
      if (h->zplanes > 1)
        tc_launch<kZBN, kZStages2, tc::BMODE_PLAIN, tc::EPI_ZSPLIT>(h->tmZA[c], h->tmZB, prm, s, &h->tmZS[c]);
      else if (prm.kt_total <= tc::kResKT) {
        // the amplitude tile (all of K = nocc) stays resident across a
        // CTA's run of tiles with the same columns (m-fastest order); one
        // product (plain BF16) needs one A plane per stage, so twice the
        // stages fit
        if (prm.nprod == 1 && h->z_res1)
          tc_launch<kZBN, kZStagesR1, tc::BMODE_PLAIN, tc::EPI_ZRES1>(h->tmZA[c], h->tmZB, prm, s, &h->tmZS[c]);
        else
          tc_launch<kZBN, kZStagesR, tc::BMODE_PLAIN, tc::EPI_ZRES>(h->tmZA[c], h->tmZB, prm, s, &h->tmZS[c]);
      } else {
        tc_launch<kZBN, kZStages1, tc::BMODE_PLAIN, tc::EPI_ZONE>(h->tmZA[c], h->tmZB, prm, s, &h->tmZS[c]);
      }
    }
    {
      // K_(col,i),a (+)= sum_{P in chunk, b} Z^P_(col,i),b B^P_ab   (split-K)
      Prof pr(h, RTTDA_KC_EXCHANGE_MAIN, s);
      h->launches += 1;
      tc::Params prm{};
      const int kb = h->wide_mb ? h->wide_kb : tc::kBK;
      // wide_tr: rows a, columns (col, i), partials written transposed
      prm.M = h->wide_tr ? v : C * o;
      prm.N = h->wide_tr ? C * o : v;
      prm.kt_total = pc * (vp / kb);
      prm.kt_per_split = h->tc_kper[c];
      prm.nsplit = h->SK;
      prm.nprod = h->nprod_main;
      prm.vtiles = vp / kb;
      prm.out = (float*)h->Kpart;
      prm.ldo = v;
      prm.split_stride = (long long)C * o * v;
      prm.accum = c > 0 ? 1 : 0;
      prm.err = h->d_err;
      if (h->wide_mb) {
        // wide-M tiles: MB accumulators share each B tile; both B planes per stage
        if (h->wide_cl > 1)
          wide_cluster_dispatch(h->nprod_main, h->wide_kb, h->wide_cl, h->tmMAc[c], h->tmMB[c], prm, s, h->wide_grid);
        else
          wide_dispatch(h->tc_bn, h->wide_mb, h->nprod_main, h->wide_kb, h->tmMA[c], h->tmMB[c], prm, s,
                        h->wide_tr);
      } else switch (h->tc_bn) {
        case 128: tc_launch<128, 7, tc::BMODE_VV, tc::EPI_PARTIAL>(h->tmMA[c], h->tmMB[c], prm, s); break;
        case 224: tc_launch<224, 5, tc::BMODE_VV, tc::EPI_PARTIAL>(h->tmMA[c], h->tmMB[c], prm, s); break;
        default: tc_launch<256, 4, tc::BMODE_VV, tc::EPI_PARTIAL>(h->tmMA[c], h->tmMB[c], prm, s); break;
      }
    }
  }
}

// --- FP64-accurate exchange: Ozaki digits on the tensor cores ------------
void oz_attr() {
  static_assert(oz::smem_bytes<oz::OZ_PLAIN>() <= 232448, "shared memory per block exceeds 227 KB");
  static_assert(oz::smem_bytes<oz::OZ_VV>() <= 232448, "shared memory per block exceeds 227 KB");
  cudaFuncSetAttribute(oz::k_oz_gemm<oz::OZ_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)oz::smem_bytes<oz::OZ_PLAIN>());
  cudaFuncSetAttribute(oz::k_oz_gemm<oz::OZ_VV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)oz::smem_bytes<oz::OZ_VV>());
  cudaFuncSetAttribute(oz::k_oz_gemm<oz::OZ_PLAIN64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)oz::smem_bytes<oz::OZ_PLAIN64>());
}

template <int MODE>
void oz_launch(const CUtensorMap& a, const CUtensorMap& b, const oz::Params& prm, cudaStream_t s) {
  const long long tiles = cdiv(prm.N, oz::kBN) * cdiv(prm.M, tc::kBM) * prm.nsplit;
  const unsigned grid = (unsigned)std::max(1LL, std::min<long long>(tiles, kNumSM));
  oz::k_oz_gemm<MODE><<<grid, oz::kThreads, oz::smem_bytes<MODE>(), s>>>(a, b, prm);
}

// K_(col,i),a = sum_{P,b} Z^P_(col,i),b B^P_ab to FP64 accuracy: digits of
// the stage amplitudes, then per chunk of P the Z build (Z^P = B^P_oo c as
// exact integers, one exactness block since nocc <= 512), the digits of Z per
// block of (row, P, b / 512) and the main contraction into FP64 split-K
// partials.
void exchange_oz(rttda_ctx* h, const double* X, cudaStream_t s) {
  const int C = 2 * h->T, o = h->o, v = h->v, vp = h->vp, op = h->op;
  {
    Prof pr(h, RTTDA_KC_EXCHANGE_Z, s);
    h->launches += 1;
    oz::k_slice_x<<<blocks_for((long long)C * vp * 32, 256), 256, 0, s>>>(o, v, vp, op, C, X, h->oz_x,
                                                                         (long long)C * vp * op, h->oz_ex);
  }
  for (int c = 0, p0 = 0; p0 < h->P; p0 += h->zchunk, ++c) {
    const int pc = std::min(h->zchunk, h->P - p0);
    {
      Prof pr(h, RTTDA_KC_EXCHANGE_Z, s);
      h->launches += 2;
      oz::Params prm{};
      prm.M = pc * o;
      prm.N = C * vp;
      prm.vt = (int)cdiv(op, oz::kKB);
      prm.pc = 1;
      prm.pps = 1;
      prm.nsplit = 1;
      prm.nbp = 1;
      prm.out = h->oz_zi;
      prm.ldo = (long long)C * vp;
      prm.err = h->d_err;
      oz_launch<oz::OZ_PLAIN>(h->tmOzBoo[c], h->tmOzX, prm, s);
      const long long warps = (long long)C * o * pc * h->oz_nbp;
      oz::k_slice_z<<<blocks_for(warps * 32, 256), 256, 0, s>>>(o, vp, C, pc, h->oz_nbp, p0, h->oz_zi, h->oz_eoo,
                                                                h->oz_ex, h->oz_z, (long long)h->oz_zplane, h->oz_ez);
    }
    {
      Prof pr(h, RTTDA_KC_EXCHANGE_MAIN, s);
      h->launches += 1;
      oz::Params prm{};
      prm.M = C * o;
      prm.N = v;
      prm.vt = vp / oz::kKB;
      prm.pc = pc;
      prm.pps = h->oz_pps;
      prm.nsplit = h->SK;
      prm.nbp = h->oz_nbp;
      prm.out = h->Kpart;
      prm.ldo = v;
      prm.split_stride = (long long)C * o * v;
      prm.accum = c > 0 ? 1 : 0;
      prm.ea = h->oz_ez;
      prm.lde_a = (long long)C * o;
      prm.eb = h->oz_evv + (size_t)p0 * h->oz_nbp * vp;
      prm.lde_b = vp;
      prm.err = h->d_err;
      oz_launch<oz::OZ_VV>(h->tmOzZ[c], h->tmOzBvv[c], prm, s);
    }
  }
}

// Coulomb 2 sum_jb (ia|jb) c_jb to FP64 accuracy on digits: w = B_ov c
// (M = naux, K = nocc*nvirt, split-K partials), then J = B_ov^T (2w)
// (M = nocc*nvirt, K = naux) into the FP64 partials the combine reads.
void coulomb_oz(rttda_ctx* h, const double* X, cudaStream_t s) {
  Prof pr(h, RTTDA_KC_COULOMB, s);
  h->launches += 4;
  const int C = 2 * h->T, P = h->P, cp = h->oz_cp;
  const long long ov = h->ov;
  oz::k_slice_xc<<<blocks_for((long long)cp * h->oz_nkb * 32, 256), 256, 0, s>>>(
      ov, h->oz_ovp, C, cp, h->oz_nkb, X, h->oz_xc, (long long)cp * h->oz_ovp, h->oz_exc);
  oz::Params prm{};
  prm.M = P;
  prm.N = C;
  prm.vt = oz::kBlkTiles;
  prm.pc = h->oz_nkb;
  prm.pps = h->oz_pps1;
  prm.nsplit = h->SW;
  prm.nbp = 1;
  prm.out = h->oz_wpart;
  prm.ldo = C;
  prm.split_stride = (long long)P * C;
  prm.ea = h->oz_ebov;
  prm.lde_a = P;
  prm.eb = h->oz_exc;
  prm.lde_b = cp;
  prm.err = h->d_err;
  oz_launch<oz::OZ_PLAIN64>(h->tmOzBov, h->tmOzXc, prm, s);
  oz::k_slice_w<<<blocks_for((long long)cp * h->oz_npb * 32, 256), 256, 0, s>>>(
      P, h->oz_Pp, C, cp, h->oz_npb, h->SW, h->oz_wpart, h->oz_w, (long long)cp * h->oz_Pp, h->oz_ew);
  prm.M = (int)ov;
  prm.pc = h->oz_npb;
  prm.pps = h->oz_pps2;
  prm.nsplit = h->SJ;
  prm.out = h->Jpart;
  prm.split_stride = ov * C;
  prm.ea = h->oz_ebovt;
  prm.lde_a = ov;
  prm.eb = h->oz_ew;
  oz_launch<oz::OZ_PLAIN64>(h->tmOzBovT, h->tmOzW, prm, s);
}

// Coulomb on the FP32 streaming kernels: FP32 copy of the stage's amplitudes,
// then both passes; column count as a template argument (2T in {2, ..., 12}).
template <typename TF, int C>
void coul_stream_launch_c(rttda_ctx* h, const double* X, bool xf_done, cudaStream_t s) {
  const long long nx = h->ov * C;
  if (!xf_done)
    stream::k_prep_xf<<<(unsigned)std::min<long long>(cdiv(nx, 256), 8 * kNumSM), 256, 0, s>>>(nx, C, X, h->Xf);
  stream::k_coul_w_stream<TF, C><<<dim3((unsigned)cdiv(h->P, stream::kW1Rows), h->SW), stream::kThreads,
                                   (size_t)h->wslice * C * sizeof(float), s>>>((const TF*)h->Bov, h->Xf, h->P, h->ov,
                                                                               h->wslice, (float*)h->w);
  constexpr int V = 16 / sizeof(TF);
  stream::k_coul_J_stream<TF, C><<<dim3((unsigned)cdiv(h->ov, 256 * V), h->SJ), stream::kThreads,
                                   (size_t)h->pchunkJ * C * sizeof(float), s>>>(
      (const TF*)h->Bov, (const float*)h->w, h->SW, h->P, h->ov, h->pchunkJ, (float*)h->Jpart);
}

template <typename TF>
void coul_stream_launch(rttda_ctx* h, int C, const double* X, bool xf_done, cudaStream_t s) {
  switch (C) {
    case 2: coul_stream_launch_c<TF, 2>(h, X, xf_done, s); break;
    case 4: coul_stream_launch_c<TF, 4>(h, X, xf_done, s); break;
    case 6: coul_stream_launch_c<TF, 6>(h, X, xf_done, s); break;
    case 8: coul_stream_launch_c<TF, 8>(h, X, xf_done, s); break;
    case 10: coul_stream_launch_c<TF, 10>(h, X, xf_done, s); break;
    default: coul_stream_launch_c<TF, 12>(h, X, xf_done, s); break;
  }
}

template <typename TF, int C>
void coul_stream_attr_c() {
  cudaFuncSetAttribute(stream::k_coul_w_stream<TF, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       stream::kW1SmemBytes);
  cudaFuncSetAttribute(stream::k_coul_J_stream<TF, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
}

// CTAs per SM of the two passes for C columns (register and shared-memory
// limits as compiled).
template <typename TF, int C>
void coul_stream_occ_c(size_t smem_w, size_t smem_j, int* ow, int* oj) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(ow, stream::k_coul_w_stream<TF, C>, stream::kThreads, smem_w);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(oj, stream::k_coul_J_stream<TF, C>, stream::kThreads, smem_j);
}

template <typename TF>
void coul_stream_occ(int C, size_t smem_w, size_t smem_j, int* ow, int* oj) {
  switch (C) {
    case 2: coul_stream_occ_c<TF, 2>(smem_w, smem_j, ow, oj); break;
    case 4: coul_stream_occ_c<TF, 4>(smem_w, smem_j, ow, oj); break;
    case 6: coul_stream_occ_c<TF, 6>(smem_w, smem_j, ow, oj); break;
    case 8: coul_stream_occ_c<TF, 8>(smem_w, smem_j, ow, oj); break;
    case 10: coul_stream_occ_c<TF, 10>(smem_w, smem_j, ow, oj); break;
    default: coul_stream_occ_c<TF, 12>(smem_w, smem_j, ow, oj); break;
  }
  *ow = std::max(1, *ow);
  *oj = std::max(1, *oj);
}

template <typename TF>
void coul_stream_attr() {
  coul_stream_attr_c<TF, 2>();
  coul_stream_attr_c<TF, 4>();
  coul_stream_attr_c<TF, 6>();
  coul_stream_attr_c<TF, 8>();
  coul_stream_attr_c<TF, 10>();
  coul_stream_attr_c<TF, 12>();
}

constexpr int kF0Chunks = 64;  // most chunks of the ground-row field sum

// kernels of one field product: the rows (one kernel, or two GEMMs for a
// batch with one polarisation), the ground row's chunks and their sum
// launches of one field product: M_d X rows (two GEMMs, after the cast of
// the stage input when its operands are pre-converted), ground-row chunks,
// their sum
inline int field_launches(const rttda_ctx* h) {
  return (h->same_dir && 2 * h->T >= 8) ? (h->Xfc ? 5 : 4) : 3;
}

// F = M_d X (singles rows): the register-tiled kernel when its 32 x 64
// tiles give at least one block per SM, else one output per thread.
template <typename TM_, typename TC>
void launch_field(rttda_ctx* h, const double* X, const TM_* moo, const TM_* mvv, const TM_* m0, cudaStream_t s) {
  const int C = 2 * h->T;
  if (h->same_dir && C >= 8) {
    // one polarisation for the whole batch: two GEMMs over the C columns
    // (the first trajectory's dipole blocks stand for all)
    const dim3 gvv((unsigned)cdiv(C, 64), (unsigned)cdiv(h->v, 64), h->o);
    const dim3 goo((unsigned)cdiv(C, 64), (unsigned)cdiv(h->o, 64), h->v);
    if constexpr (!std::is_same<TC, double>::value) {
      if (h->Xfc) {
        // operands in the arithmetic's type: the stage input cast once here,
        // the dipole blocks (float, or df32 pairs of the FP64 blocks) at
        // rttda_set_field
        const long long n = h->N * C;
        k_to_type<TC><<<blocks_for(n, 256), 256, 0, s>>>(n, X, (TC*)h->Xfc);
        const TC* xf = (const TC*)h->Xfc;
        const TC* mv = std::is_same<TC, df32>::value ? (const TC*)h->mvv_df : (const TC*)(const void*)mvv;
        const TC* mo = std::is_same<TC, df32>::value ? (const TC*)h->moo_df : (const TC*)(const void*)moo;
        k_field_gemm<TC, TC, false, TC, TM_><<<gvv, 256, 0, s>>>(h->o, h->v, C, xf, mv, m0, h->F);
        k_field_gemm<TC, TC, true, TC, TM_><<<goo, 256, 0, s>>>(h->o, h->v, C, xf, mo, m0, h->F);
        return;
      }
    }
    k_field_gemm<TM_, TC, false><<<gvv, 256, 0, s>>>(h->o, h->v, C, X, mvv, m0, h->F);
    k_field_gemm<TM_, TC, true><<<goo, 256, 0, s>>>(h->o, h->v, C, X, moo, m0, h->F);
    return;
  }
  const long long tiled = cdiv(h->v, 64) * cdiv(h->o, 32) * (long long)h->T;
  if (tiled >= kNumSM) {
    dim3 g((unsigned)cdiv(h->v, 64), (unsigned)cdiv(h->o, 32), h->T);
    k_field<TM_, TC><<<g, dim3(16, 16), 0, s>>>(h->o, h->v, h->T, X, moo, mvv, m0, h->F);
  } else {
    dim3 g((unsigned)cdiv(h->v, 32), (unsigned)cdiv(h->o, 8), h->T);
    k_field_small<TM_, TC><<<g, dim3(32, 8), 0, s>>>(h->o, h->v, h->T, X, moo, mvv, m0, h->F);
  }
}

// F_0 = sum_ia m_ia X_ia per trajectory: chunk sums, then their ordered sum.
template <typename TM_, typename TC>
void launch_field0(rttda_ctx* h, const double* X, const TM_* m0, cudaStream_t s) {
  const long long rows = std::max<long long>(2048, cdiv(h->ov, kF0Chunks));
  const int G = (int)cdiv(h->ov, rows);
  k_field0<TM_, TC><<<dim3(G, h->T), 256, 0, s>>>(h->ov, h->T, rows, X, m0, h->f0_part);
  k_field0_final<<<1, 64, 0, s>>>(G, h->T, h->f0_part, h->F);
}

template <typename TF, typename TC, bool XTC>
struct Ops {
  using TL = Tile<TC>;

  // Returns whether it also wrote the exchange's BF16 planes of X (only when
  // asked with prep_xt, on the tensor-core exchange with the streaming
  // Coulomb: one launch writes them and the FP32 copy); the caller then
  // passes that to exchange() on the same X.
  static bool coulomb(rttda_ctx* h, const double* X, cudaStream_t s, bool prep_xt_too = false) {
    if (XTC && h->coul_tc) {
      coulomb_tc(h, X, s);
      return false;
    }
    Prof pr(h, RTTDA_KC_COULOMB, s);
    h->launches += 2;
    const int C = 2 * h->T;
    if constexpr (!std::is_same<TF, double>::value) {
      if (h->coul_stream) {
        h->launches += 1;  // the FP32 amplitude copy
        const bool fused = XTC && prep_xt_too;
        if (fused) prep_xt(h, X, true, s);
        coul_stream_launch<TF>(h, C, X, fused, s);
        return fused;
      }
    }
    if (h->coul_vec) {
      // 16-byte vector loads of B_ov rows (ov a multiple of the vector width)
      constexpr int V = Vec16<TF>::V;
      k_coul_w_vec<TF, TC, 6><<<dim3(blocks_for(h->P, 32), h->SW), 256, (size_t)h->wslice * C * sizeof(TC), s>>>(
          (const TF*)h->Bov, X, h->P, h->ov, C, h->wslice, (TC*)h->w);
      dim3 g(blocks_for(cdiv(h->ov, V), 256), h->SJ);
      const size_t smem = (size_t)h->pchunkJ * C * sizeof(TC);
      k_coul_J_vec<TF, TC, 6><<<g, 256, smem, s>>>((const TF*)h->Bov, (const TC*)h->w, h->SW, h->P, h->ov, C,
                                                  h->pchunkJ, (TC*)h->Jpart);
      return false;
    }
    constexpr int PB = 8;
    k_coul_w<TF, TC, 8, PB><<<dim3(blocks_for(h->P, PB), h->SW), 256, 0, s>>>((const TF*)h->Bov, X, h->P, h->ov, C,
                                                                             (TC*)h->w);
    dim3 g(blocks_for(h->ov, 256), h->SJ);
    const size_t smem = (size_t)h->pchunkJ * C * sizeof(TC);
    k_coul_J<TF, TC, 8><<<g, 256, smem, s>>>((const TF*)h->Bov, (const TC*)h->w, h->SW, h->P, h->ov, C,
                                            h->pchunkJ, (TC*)h->Jpart);
    return false;
  }

  static void exchange(rttda_ctx* h, const double* X, cudaStream_t s, bool xt_done = false) {
    if (XTC) {
      exchange_tc(h, X, s, xt_done);
      return;
    }
    const int C = 2 * h->T, o = h->o, v = h->v;
    const int M = C * o;
    for (int p0 = 0, c = 0; p0 < h->P; p0 += h->zchunk, ++c) {
      const int pc = std::min(h->zchunk, h->P - p0);
      // Z^P_(b,col),i = sum_j X_(j,b),col B^P_ji  for P in the chunk
      {
        Prof pr(h, RTTDA_KC_EXCHANGE_Z, s);
        h->launches += 1;
        dim3 g(blocks_for(o, TL::BN), blocks_for((long long)v * C, TL::BM), pc);
        k_gemm_tn<double, TF, TC, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN>
            <<<g, (TL::BM / TL::TM) * (TL::BN / TL::TN), 0, s>>>(
                v * C, o, o, X + C, (long long)v * C, 0, (const TF*)h->Boo + (size_t)p0 * o * o, o,
                (long long)o * o, (TC*)h->Zt, o, (long long)v * C * o, 0, 1, o, 0);
      }
      // K_(col,i),a += sum_{P in chunk, b} Z^P_(col,i),b B^P_ba   (split-K)
      {
        Prof pr(h, RTTDA_KC_EXCHANGE_MAIN, s);
        h->launches += 1;
        const long long Kc = (long long)pc * v;
        const long long kper = cdiv(cdiv(Kc, h->SK), TL::BK) * TL::BK;
        dim3 g(blocks_for(v, TL::BN), blocks_for(M, TL::BM), h->SK);
        k_gemm_tn<TC, TF, TC, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN>
            <<<g, (TL::BM / TL::TM) * (TL::BN / TL::TN), 0, s>>>(
                M, v, Kc, (const TC*)h->Zt, M, 0, (const TF*)h->Bvv + (size_t)p0 * v * v, v, 0,
                (TC*)h->Kpart, v, 0, (long long)M * v, h->SK, kper, c > 0 ? 1 : 0);
      }
    }
  }

  static void field(rttda_ctx* h, const double* X, cudaStream_t s) {
    Prof pr(h, RTTDA_KC_FIELD, s);
    h->launches += field_launches(h);  // M_d X rows, ground-row chunks, their sum
    if (std::is_same<TC, double>::value) {
      launch_field<double, double>(h, X, h->moo64, h->mvv64, h->m064, s);
      launch_field0<double, double>(h, X, h->m064, s);
    } else {
      launch_field<TC, TC>(h, X, (const TC*)h->mooC, (const TC*)h->mvvC, (const TC*)h->m0C, s);
      launch_field0<TC, TC>(h, X, (const TC*)h->m0C, s);
    }
  }

  // The field product of the step's start, which also feeds the dipole
  // expectation: FP64-accurate in every precision.  The modes whose field
  // products are FP32 take it in double-float arithmetic from the FP64
  // dipole blocks (ground row in FP64); the FP64 modes take their own.
  static void field_obs(rttda_ctx* h, const double* X, cudaStream_t s) {
    if (std::is_same<TC, double>::value) {
      field(h, X, s);
      return;
    }
    Prof pr(h, RTTDA_KC_FIELD, s);
    h->launches += field_launches(h);
    launch_field<double, df32>(h, X, h->moo64, h->mvv64, h->m064, s);
    launch_field0<double, double>(h, X, h->m064, s);
  }

  static void combine(rttda_ctx* h, int mode, int stage, bool use_field, double dt, const double* Xin,
                      double* Xnext, double* sig_out, cudaStream_t s, long long* step_ctr = nullptr) {
    Prof pr(h, RTTDA_KC_COMBINE, s);
    h->launches += 1;
    const int C = 2 * h->T;
    // column tile: all C columns when C <= 32 (C is even), else 32
    const int cc = C >= 32 ? 32 : C > 8 ? 16 : C > 4 ? 8 : C > 2 ? 4 : 2;
    const dim3 grid((unsigned)cdiv(h->N, kCombineTile / cc), (unsigned)cdiv(C, cc));
    auto go = [&](auto kern) {
      kern<<<grid, 256, 0, s>>>(mode, stage, h->N, h->o, h->v, h->T, h->eps_o, h->eps_v, h->cx,
                                (const TC*)h->Jpart, h->SJ, (const TC*)h->Kpart, h->SK,
                                (long long)C * h->o * h->v, h->F, h->E, use_field ? 1 : 0, dt, h->Xn, Xin, Xnext,
                                h->acc, sig_out, step_ctr);
    };
    switch (cc) {
      case 2: go(k_combine<TC, 2>); break;
      case 4: go(k_combine<TC, 4>); break;
      case 8: go(k_combine<TC, 8>); break;
      case 16: go(k_combine<TC, 16>); break;
      default: go(k_combine<TC, 32>); break;
    }
  }

  // split-operator sub-step on the stage input X (in place); see k_sso_update
  static void sso_update(rttda_ctx* h, int mode, int stage, bool use_field, double dt, double* X, cudaStream_t s,
                         long long* step_ctr = nullptr) {
    Prof pr(h, RTTDA_KC_COMBINE, s);
    h->launches += 1;
    const int C = 2 * h->T;
    // trajectory tile: all T when T <= 32, else 32
    const int ct = h->T >= 32 ? 32 : h->T > 8 ? 16 : h->T > 4 ? 8 : h->T > 2 ? 4 : h->T > 1 ? 2 : 1;
    const dim3 grid((unsigned)cdiv(h->N, kCombineTile / ct), (unsigned)cdiv(h->T, ct));
    auto go = [&](auto kern) {
      kern<<<grid, 256, 0, s>>>(mode, stage, h->N, h->o, h->v, h->T, h->eps_o, h->eps_v, h->cx,
                                (const TC*)h->Jpart, h->SJ, (const TC*)h->Kpart, h->SK,
                                (long long)C * h->o * h->v, h->F, h->E, use_field ? 1 : 0, dt, h->Xn, X, step_ctr);
    };
    switch (ct) {
      case 1: go(k_sso_update<TC, 1>); break;
      case 2: go(k_sso_update<TC, 2>); break;
      case 4: go(k_sso_update<TC, 4>); break;
      case 8: go(k_sso_update<TC, 8>); break;
      case 16: go(k_sso_update<TC, 16>); break;
      default: go(k_sso_update<TC, 32>); break;
    }
  }

  static void set_smem_limits() {
    cudaFuncSetAttribute(k_coul_J<TF, TC, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_coul_J_vec<TF, TC, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_coul_w_vec<TF, TC, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if constexpr (!std::is_same<TF, double>::value) coul_stream_attr<TF>();
    if (XTC) set_tc_smem_limits();
  }
};

// FP64_OZ: the FP64 paths with the exchange on Ozaki digits
struct OpsOz : Ops<double, double, false> {
  static bool coulomb(rttda_ctx* h, const double* X, cudaStream_t s, bool = false) {
    coulomb_oz(h, X, s);
    return false;
  }
  static void exchange(rttda_ctx* h, const double* X, cudaStream_t s, bool = false) { exchange_oz(h, X, s); }
  static void set_smem_limits() {
    Ops<double, double, false>::set_smem_limits();
    oz_attr();
  }
};

template <typename F>
void dispatch(int prec, F&& f) {
  switch (prec) {
    case RTTDA_FP64: f(Ops<double, double, false>{}); break;
    case RTTDA_FP64_OZ: f(OpsOz{}); break;
    case RTTDA_FP32: f(Ops<float, float, false>{}); break;
    case RTTDA_BF16: f(Ops<__nv_bfloat16, float, true>{}); break;
    default: f(Ops<float, float, true>{}); break;  // RTTDA_BF16X3, RTTDA_BF16X2
  }
}

// Exact kick exp(+i kappa M_d) on h->Xn: Taylor terms accumulated in FP64.
// The first-order term, which carries the whole linear response, always
// takes FP64 field products.  The higher terms (each at most x^k / k! of
// the state for x the bound on |kappa M_d|) take the field products of the
// precision's sigma build when that is FP32, where B300's FP64 pipe would
// make them cost as much as a few time steps.
void enqueue_kick(rttda_ctx* h, cudaStream_t s) {
  Prof pr(h, RTTDA_KC_KICK, s);
  h->launches += (field_launches(h) + 1) * h->kick_terms;
  const long long NT = h->N * h->T;
  cudaMemcpyAsync(h->term, h->Xn, sizeof(double) * NT * 2, cudaMemcpyDeviceToDevice, s);
  for (int k = 1; k <= h->kick_terms; ++k) {
    if (k == 1 || h->cbytes == 8) {
      launch_field<double, double>(h, h->term, h->moo64, h->mvv64, h->m064, s);
      launch_field0<double, double>(h, h->term, h->m064, s);
    } else {
      launch_field<float, float>(h, h->term, (const float*)h->mooC, (const float*)h->mvvC, (const float*)h->m0C, s);
      launch_field0<float, float>(h, h->term, (const float*)h->m0C, s);
    }
    k_kick_term<<<blocks_for(NT, 256), 256, 0, s>>>(h->N, h->T, h->d_kappa, 1.0 / k, h->F, h->term, h->Xn);
  }
}

void enqueue_observe(rttda_ctx* h, const double* X, double* dip, double* nrm, long long ld, long long step_offset,
                     cudaStream_t s) {
  Prof pr(h, RTTDA_KC_OBSERVE, s);
  h->launches += 2;
  k_obs_partial<<<h->obsG, 256, 0, s>>>(h->N, h->T, h->obs_rows, X, h->F, h->obs_part);
  k_obs_final<<<1, 128, 0, s>>>(h->obsG, h->T, h->obs_part, h->d_step, step_offset, ld, dip, nrm);
}

// Overlaps of the state X with the projectors, recorded at the step index.
void enqueue_project(rttda_ctx* h, const double* X, long long ld, long long step_offset, cudaStream_t s) {
  if (h->nproj < 1 || !h->d_ovl) return;
  Prof pr(h, RTTDA_KC_OBSERVE, s);
  h->launches += 2;
  const int C = 2 * h->T;
  k_proj_partial<<<dim3(h->proj_G, h->nproj), 256, 0, s>>>(h->N, C, h->nproj, h->proj_rows, h->d_proj, X,
                                                          h->d_proj_part);
  k_proj_final<<<1, 256, 0, s>>>(h->proj_G, C, h->nproj, h->d_proj_part, h->d_step, step_offset, ld, h->d_ovl);
}

// Autocorrelation of the state X with the stored X(eps), recorded at the step index.
void enqueue_acf(rttda_ctx* h, const double* X, long long ld, long long step_offset, cudaStream_t s) {
  if (!h->acf_on || !h->have_eps || !h->d_acf) return;
  Prof pr(h, RTTDA_KC_OBSERVE, s);
  h->launches += 2;
  k_acf_partial<<<dim3(h->proj_G, h->T), 256, 0, s>>>(h->N, h->T, h->proj_rows, h->d_xeps, X, h->d_acf_part);
  k_acf_final<<<1, 128, 0, s>>>(h->proj_G, h->T, h->d_acf_part, h->d_step, step_offset, ld, h->d_acf);
}

// One RK4 step (four sigma builds) plus the observables of the step's start.
template <typename O>
void enqueue_step(rttda_ctx* h, O, long long base, double t_off, double dt, double* dip, double* nrm, long long ld,
                  long long offset, cudaStream_t s) {
  // the step counter advances in the last stage's combine
  h->launches += 1;
  k_efield<<<1, 128, 0, s>>>(h->T, h->d_pulses, h->d_step, base, t_off, dt, h->E);
  for (int st = 0; st < 4; ++st) {
    // stage inputs alternate between two buffers (the combine reads one and
    // writes the other); stage 3 writes back into Xs, so every step starts there
    double* xin = (st % 2 == 0) ? h->Xs : h->Xs2;
    double* xnext = (st % 2 == 0) ? h->Xs2 : h->Xs;
    const bool fld = h->any_field;
    if (st == 0)
      O::field_obs(h, xin, s);  // xin holds c_n: also the observables' M_d c_n
    else if (fld)
      O::field(h, xin, s);
    if (st == 0 && dip) enqueue_observe(h, h->Xn, dip, nrm, ld, offset, s);
    if (st == 0) {
      enqueue_project(h, h->Xn, ld, offset, s);
      enqueue_acf(h, h->Xn, ld, offset, s);
    }
    const bool xt = O::coulomb(h, xin, s, true);
    O::exchange(h, xin, s, xt);
    O::combine(h, 0, st, fld, dt, xin, xnext, nullptr, s, st == 3 ? h->d_step : nullptr);
  }
}

// One symplectic split-operator step (Sec. 2.2): two sigma builds, each on one
// component of the stage input Xs, which holds (q_n, p_{n+1/2}) at the start
// of a step; Xn holds (q_n, p_n) for the observables and the state.
//   sigma build at t_n + dt/2 (stage 1) -> drift  q_{n+1} = q_n + dt H p_{n+1/2}
//   sigma build at t_n + dt   (stage 3) -> p_{n+1}, then p_{n+3/2}
template <typename O>
void enqueue_step_sso(rttda_ctx* h, O, long long base, double t_off, double dt, double* dip, double* nrm,
                      long long ld, long long offset, cudaStream_t s) {
  // the step counter advances in the second half's update
  h->launches += 1;
  k_efield<<<1, 128, 0, s>>>(h->T, h->d_pulses, h->d_step, base, t_off, dt, h->E);
  const bool fld = h->any_field;
  if (dip) {
    O::field_obs(h, h->Xn, s);
    enqueue_observe(h, h->Xn, dip, nrm, ld, offset, s);
  }
  enqueue_project(h, h->Xn, ld, offset, s);
  enqueue_acf(h, h->Xn, ld, offset, s);
  for (int half = 0; half < 2; ++half) {
    if (fld) O::field(h, h->Xs, s);
    const bool xt = O::coulomb(h, h->Xs, s, true);
    O::exchange(h, h->Xs, s, xt);
    O::sso_update(h, half == 0 ? 1 : 2, half == 0 ? 1 : 3, fld, dt, h->Xs, s, half == 1 ? h->d_step : nullptr);
  }
}

// First half step of the split operator at the start of a propagation:
// Xs = (q_0, p_0) -> (q_0, p_0 - dt/2 H(t_0) q_0).
template <typename O>
void enqueue_sso_prologue(rttda_ctx* h, O, long long base, double t_off, double dt, cudaStream_t s) {
  h->launches += 1;
  k_efield<<<1, 128, 0, s>>>(h->T, h->d_pulses, h->d_step, base, t_off, dt, h->E);
  const bool fld = h->any_field;
  if (fld) O::field(h, h->Xs, s);
  const bool xt = O::coulomb(h, h->Xs, s, true);
  O::exchange(h, h->Xs, s, xt);
  O::sso_update(h, 0, 0, fld, dt, h->Xs, s);
}

rttda_status run_steps(rttda_ctx* h, double t_call, double dt, long nsteps, double* dip, double* nrm,
                       long long ld, long long offset, cudaStream_t s) {
  // stage times are t_off + (base + k + c_s) dt with an integer base when the
  // start time is a whole number of steps
  long long base = 0;
  double t_off = t_call;
  const double nb = std::nearbyint(t_call / dt);
  if (std::fabs(nb * dt - t_call) <= 1e-12 * std::max(1.0, std::fabs(t_call))) {
    base = (long long)nb;
    t_off = 0.0;
  }
  CK(cudaMemsetAsync(h->d_step, 0, sizeof(long long), s));
  CK(cudaMemcpyAsync(h->Xs, h->Xn, sizeof(double) * h->N * 2 * h->T, cudaMemcpyDeviceToDevice, s));
  const bool sso = h->integrator == RTTDA_INT_SSO;
  auto step = [&](auto ops) {
    if (sso)
      enqueue_step_sso(h, ops, base, t_off, dt, dip, nrm, ld, offset, s);
    else
      enqueue_step(h, ops, base, t_off, dt, dip, nrm, ld, offset, s);
  };
  if (nsteps > 0 && sso) dispatch(h->prec, [&](auto ops) { enqueue_sso_prologue(h, ops, base, t_off, dt, s); });
  if (nsteps > 0 && h->prof_on) {
    // profiling: direct launches so that every kernel class gets its events
    const long long l0 = h->launches;
    for (long k = 0; k < nsteps; ++k) dispatch(h->prec, step);
    h->launches_per_step = (h->launches - l0) / nsteps;
  } else if (nsteps > 0) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const long long l0 = h->launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    dispatch(h->prec, step);
    h->launches_per_step = h->launches - l0;
    if (h->break_capture) cudaStreamSynchronize(s);  // test hook: invalidates the capture
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess) {
      // The capture was invalidated, e.g. by a device-wide synchronisation
      // that another thread of the process issued meanwhile.  None of the
      // captured work ran: enqueue the same steps as direct launches.
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      h->launches = l0;
      for (long k = 0; k < nsteps; ++k) dispatch(h->prec, step);
      ++h->capture_fallbacks;
    } else {
      h->launches = l0 + h->launches_per_step * nsteps;
      // Keep the executable step graph of the handle and give it this call's
      // parameters with cudaGraphExecUpdate (launches in flight keep theirs);
      // a new one is instantiated only when the update is refused (a different
      // topology).  With an instantiation per call, the steps of concurrent
      // handles (the server's requests) were measured not to overlap at all;
      // instantiation allocates device memory, which keeps commands of
      // different streams from running concurrently.  RTTDA_GRAPH_CACHE=0
      // instantiates per call.
      const char* gc = std::getenv("RTTDA_GRAPH_CACHE");
      const bool keep = !(gc && std::atoi(gc) == 0);
      if (keep && h->step_exec) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(h->step_exec, graph, &info) == cudaSuccess) {
          exec = h->step_exec;
        } else {
          cudaGetLastError();
          cudaGraphExecDestroy(h->step_exec);
        }
        h->step_exec = nullptr;
      }
      if (!exec) {
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) {
          cudaGraphDestroy(graph);
          return set_error(RTTDA_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
      }
      for (long k = 0; k < nsteps; ++k) {
        ce = cudaGraphLaunch(exec, s);
        if (ce != cudaSuccess) break;
      }
      if (keep && ce == cudaSuccess)
        h->step_exec = exec;
      else
        cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return set_error(RTTDA_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
    }
  }
  if (dip) {
    dispatch(h->prec, [&](auto ops) { decltype(ops)::field_obs(h, h->Xn, s); });
    enqueue_observe(h, h->Xn, dip, nrm, ld, offset, s);
  }
  enqueue_project(h, h->Xn, ld, offset, s);
  enqueue_acf(h, h->Xn, ld, offset, s);
  CK(cudaGetLastError());
  h->t_now = t_off + (double)(base + nsteps) * dt;
  h->have_state = true;
  return RTTDA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Batch set-up
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// TMA tensor maps (driver entry point; no link-time dependency on libcuda)
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  // looked up once (function-local static: thread-safe initialisation, so
  // handles created on several threads, as the server does, share it)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// BF16 tile map with 128-byte swizzle; dims/box innermost first, strides in
// bytes for dims 1..rank-1.
static rttda_status bf16_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims,
                             const uint64_t* strides, const uint32_t* box,
                             CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  auto enc = tmap_encoder();
  if (!enc) return set_error(RTTDA_E_CUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base),
                   reinterpret_cast<const cuuint64_t*>(dims), reinterpret_cast<const cuuint64_t*>(strides),
                   reinterpret_cast<const cuuint32_t*>(box), es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(RTTDA_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return RTTDA_OK;
}

// Bytes allowed for one chunk of Z (all of P when it fits): at most 40 GiB
// and at most a third of the device memory free now.
static size_t zbudget_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = (size_t)6 << 30;
  return std::max<size_t>((size_t)256 << 20, std::min<size_t>((size_t)40 << 30, fr / 3));
}

// P per Z chunk: what the byte budget allows, at most RTTDA_ZCHUNK when that
// environment variable holds a positive count (tests and experiments).
static int zchunk_for(int P, size_t budget, size_t per_p) {
  size_t zc = std::max<size_t>(1, std::min<size_t>(P, budget / std::max<size_t>(per_p, 1)));
  const char* e = std::getenv("RTTDA_ZCHUNK");
  if (e && *e) {
    const long cap = std::atol(e);
    if (cap > 0) zc = std::min<size_t>(zc, (size_t)cap);
  }
  return (int)zc;
}

// Split-K count for a persistent launch over `tiles` output tiles: the split
// whose tile count best fills whole waves of the SMs (ties and near-ties go
// to fewer splits), keeping at least 16 K tiles per split.
static int choose_splits(long long tiles, long long kt, int grid = kNumSM) {
  int best = 1;
  double best_score = -1.0;
  for (int sk = 1; sk <= grid; ++sk) {
    if (sk > 1 && kt / sk < 16) break;
    const double x = (double)(tiles * sk) / grid;
    const double score = x / std::ceil(x) - 0.002 * sk;
    if (score > best_score) {
      best = sk;
      best_score = score;
    }
  }
  return best;
}

// Buffers, split-K plans and TMA maps of the tensor-core Coulomb.
static rttda_status alloc_coul_tc(rttda_ctx* h, int C) {
  const int P = h->P;
  const long long ov = h->ov;
  const size_t np = (size_t)h->nplanes;
  CKS(dalloc(&h->Xc, (size_t)C * ov * np));
  CKS(dalloc(&h->Wt, (size_t)C * P * np));
  h->SKc1 = choose_splits(cdiv(P, tc::kBM) * cdiv(C, 64), cdiv(ov, tc::kBK));
  h->SKc2 = choose_splits(cdiv(ov, tc::kBM) * cdiv(C, 64), cdiv(P, tc::kBK));
  CKS(dalloc(&h->wpart_tc, (size_t)h->SKc1 * P * C));
  char* p = nullptr;
  CKS(dalloc_bytes((void**)&p, (size_t)h->SKc2 * ov * C * sizeof(float)));
  h->Jpart = p;
  h->SJ = h->SKc2;
  h->SW = 1;
  CKS(dalloc_bytes((void**)&p, sizeof(float)));  // pass-1 SIMT scratch is unused here
  h->w = p;
  {
    const uint64_t dims[3] = {(uint64_t)ov, (uint64_t)P, np};
    const uint64_t str[2] = {(uint64_t)ov * 2, (uint64_t)P * ov * 2};
    const uint32_t box[3] = {64, 128, 1};
    CKS(bf16_map(&h->tmC1A, h->Bov_tc, 3, dims, str, box));
  }
  {
    const uint64_t dims[3] = {(uint64_t)ov, (uint64_t)C, np};
    const uint64_t str[2] = {(uint64_t)ov * 2, (uint64_t)C * ov * 2};
    const uint32_t box[3] = {64, 64, 1};
    CKS(bf16_map(&h->tmC1B, h->Xc, 3, dims, str, box));
  }
  {
    const uint64_t dims[3] = {(uint64_t)P, (uint64_t)ov, np};
    const uint64_t str[2] = {(uint64_t)P * 2, (uint64_t)ov * P * 2};
    const uint32_t box[3] = {64, 128, 1};
    CKS(bf16_map(&h->tmC2A, h->BovT_tc, 3, dims, str, box));
  }
  {
    const uint64_t dims[3] = {(uint64_t)P, (uint64_t)C, np};
    const uint64_t str[2] = {(uint64_t)P * 2, (uint64_t)C * P * 2};
    const uint32_t box[3] = {64, 64, 1};
    CKS(bf16_map(&h->tmC2B, h->Wt, 3, dims, str, box));
  }
  return RTTDA_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the main exchange contraction (wide-M kernel).  Candidates:
// (BN, MB) in {(160, 3), (192, 2)} x K tile {32, 64}, plus the transposed
// kernel (rows a, MB = 2, K tile 32) with the column tile of least padding
// for the C*o columns, each with the split-K count of choose_splits.  Each candidate runs the contraction over the
// first Z chunk (filled with hashed values, so that the tensor cores see
// data-like operands and power) once to warm up and then five times,
// interleaved with the others, timed with CUDA events on the handle's
// stream; the candidate with the fastest launch wins.  Results are cached per shape for the process
// and, when RTTDA_TUNE_CACHE names a file, in that file (one JSON object per
// line).  RTTDA_TUNE=0 skips the timing and takes the first candidate with
// the least padded work and K tile 32; RTTDA_WIDE_PLAN="BN,MB,KB" names the
// candidate to use, "BN,2,32,t" a transposed plan with column tile BN (for
// tests and experiments).
// ---------------------------------------------------------------------------
struct WidePlan {
  int bn = 160, mb = 3, kb = 32, sk = 1;
  int tr = 0;  // 1: transposed (rows a, MB = 2, K tile 32)
};

static bool tr_bn_ok(int bn) {
  for (int x : kTrBN)
    if (x == bn) return true;
  return false;
}

static std::mutex g_tune_mu;
static std::map<std::string, WidePlan> g_tune_cache;
static bool g_tune_file_loaded = false;

static std::string tune_key(int o, int v, int vp, int pc, int C, int nprod, int zplanes) {
  std::ostringstream k;
  k << "wide:o=" << o << ",v=" << v << ",vp=" << vp << ",pc=" << pc << ",C=" << C << ",nprod=" << nprod
    << ",zplanes=" << zplanes;
  return k.str();
}

// {"key": "...", "bn": B, "mb": M, "kb": K, "sk": S, "tr": T}
static void tune_file_load() {
  const char* f = std::getenv("RTTDA_TUNE_CACHE");
  if (g_tune_file_loaded || !f || !*f) return;
  g_tune_file_loaded = true;
  std::ifstream in(f);
  std::string line;
  while (std::getline(in, line)) {
    const size_t k0 = line.find("\"key\": \"");
    if (k0 == std::string::npos) continue;
    const size_t ks = k0 + 8, ke = line.find('"', ks);
    if (ke == std::string::npos) continue;
    WidePlan w;
    auto num = [&](const char* name, int& dst) {
      const size_t q = line.find(std::string("\"") + name + "\": ");
      if (q != std::string::npos) dst = std::atoi(line.c_str() + q + std::strlen(name) + 4);
    };
    num("bn", w.bn);
    num("mb", w.mb);
    num("kb", w.kb);
    num("sk", w.sk);
    num("tr", w.tr);
    const bool valid = w.tr ? (tr_bn_ok(w.bn) && w.mb == 2 && w.kb == 32 && w.sk >= 1 && w.sk <= kNumSM)
                            : (((w.bn == 160 && w.mb == 3) || (w.bn == 192 && w.mb == 2)) && (w.kb == 32 || w.kb == 64) &&
                               w.sk >= 1 && w.sk <= kNumSM);
    if (valid) g_tune_cache[line.substr(ks, ke - ks)] = w;
  }
}

static void tune_file_append(const std::string& key, const WidePlan& w) {
  const char* f = std::getenv("RTTDA_TUNE_CACHE");
  if (!f || !*f) return;
  std::ofstream out(f, std::ios::app);
  out << "{\"key\": \"" << key << "\", \"bn\": " << w.bn << ", \"mb\": " << w.mb << ", \"kb\": " << w.kb
      << ", \"sk\": " << w.sk << ", \"tr\": " << w.tr << "}\n";
}

// Operand maps of the main contraction: Z tiles (rows (col, i)) and B^P_vv
// planes (rows a).  Normal: A = Z with 128-row boxes, B = B_vv with bn-row
// boxes; transposed (tr): A = B_vv with 128-row boxes, B = Z with bn-row boxes.
static rttda_status wide_maps(rttda_ctx* h, int C, int pc, int p0, int bn, int kb, CUtensorMap* ma, CUtensorMap* mb,
                              bool tr = false, int arows = 128) {
  const int o = h->o, vp = h->vp, P = h->P;
  const CUtensorMapSwizzle sw = kb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  {
    const uint64_t dims[4] = {64, (uint64_t)C * o, (uint64_t)pc * (vp / 64), (uint64_t)h->zplanes};
    const uint64_t str[3] = {128, (uint64_t)C * o * 128, (uint64_t)h->zplane * 2};
    const uint32_t box[4] = {(uint32_t)kb, tr ? (uint32_t)bn : (uint32_t)arows, 1, 1};
    CKS(bf16_map(tr ? mb : ma, h->Zk, 4, dims, str, box, sw));
  }
  {
    const uint64_t dims[4] = {(uint64_t)vp, (uint64_t)vp, (uint64_t)pc, (uint64_t)h->nplanes};
    const uint64_t str[3] = {(uint64_t)vp * 2, (uint64_t)vp * vp * 2, (uint64_t)P * vp * vp * 2};
    const uint32_t box[4] = {(uint32_t)kb, tr ? 128u : (uint32_t)bn, 1, 1};
    CKS(bf16_map(tr ? ma : mb, h->Bvv_tc + (size_t)p0 * vp * vp, 4, dims, str, box, sw));
  }
  return RTTDA_OK;
}

static rttda_status tune_wide(rttda_ctx* h, int C, WidePlan& out) {
  const int o = h->o, v = h->v, vp = h->vp;
  const long long M = (long long)C * o;
  const int pc = std::min(h->zchunk, h->P);
  struct Cand {
    WidePlan w;
    float ms = 0.0f;
  };
  std::vector<Cand> cands;
  const int shapes[2][2] = {{160, 3}, {192, 2}};
  long long bestw = -1;
  int first = 0;
  for (int si = 0; si < 2; ++si) {
    const long long tm = (long long)tc::kBM * shapes[si][1];
    const long long work = cdiv(M, tm) * tm * cdiv(v, shapes[si][0]) * shapes[si][0];
    if (bestw < 0 || work < bestw) {
      bestw = work;
      first = si;
    }
  }
  for (int si = 0; si < 2; ++si)
    for (int kb : {32, 64}) {
      Cand c;
      c.w.bn = shapes[si][0];
      c.w.mb = shapes[si][1];
      c.w.kb = kb;
      const long long tiles = cdiv(M, (long long)tc::kBM * c.w.mb) * cdiv(v, c.w.bn);
      c.w.sk = choose_splits(tiles, (long long)h->zchunk * (vp / kb));
      cands.push_back(c);
    }
  auto tr_plan = [&](int bn) {
    WidePlan w;
    w.tr = 1;
    w.bn = bn;
    w.mb = 2;
    w.kb = 32;
    w.sk = choose_splits(cdiv((long long)v, 2LL * tc::kBM) * cdiv(M, (long long)bn), (long long)h->zchunk * (vp / 32));
    return w;
  };
  {
    // transposed candidate: the column tile that pads C*o least (ties to the wider)
    int best_bn = kTrBN[0];
    long long bestp = -1;
    for (int bn : kTrBN) {
      const long long padded = cdiv(M, (long long)bn) * bn;
      if (bestp < 0 || padded <= bestp) {
        bestp = padded;
        best_bn = bn;
      }
    }
    Cand c;
    c.w = tr_plan(best_bn);
    cands.push_back(c);
  }
  const char* force = std::getenv("RTTDA_WIDE_PLAN");
  if (force && *force) {
    int fb = 0, fm = 0, fk = 0;
    char ft = 0;
    const int nf = std::sscanf(force, "%d,%d,%d,%c", &fb, &fm, &fk, &ft);
    if (nf == 4 && ft == 't' && fm == 2 && fk == 32 && tr_bn_ok(fb)) {
      out = tr_plan(fb);
      h->plan.tuned = 3;
      return RTTDA_OK;
    }
    if (nf == 3)
      for (const Cand& c : cands)
        if (!c.w.tr && c.w.bn == fb && c.w.mb == fm && c.w.kb == fk) {
          out = c.w;
          h->plan.tuned = 3;
          return RTTDA_OK;
        }
    return set_error(RTTDA_E_ARG, std::string("RTTDA_WIDE_PLAN names no candidate: ") + force);
  }
  // default: least padded work, K tile 32 (index 2*first)
  const char* env = std::getenv("RTTDA_TUNE");
  const bool timed = !(env && env[0] == '0');
  const std::string key = tune_key(o, v, vp, pc, C, h->nprod_main, h->zplanes);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_file_load();
    auto it = g_tune_cache.find(key);
    if (timed && it != g_tune_cache.end()) {
      out = it->second;
      h->plan.tuned = 2;
      return RTTDA_OK;
    }
  }
  out = cands[2 * first].w;
  h->plan.ncand = (int)cands.size();
  if (!timed) return RTTDA_OK;

  int maxsk = 1;
  for (auto& c : cands) maxsk = std::max(maxsk, c.w.sk);
  float* part = nullptr;
  CKS(dalloc_bytes((void**)&part, (size_t)maxsk * M * v * sizeof(float)));
  struct Free {
    float* p;
    ~Free() { dfree(p); }
  } fr{part};
  k_fill_hash_bf16<<<4 * kNumSM, 256, 0, h->stream>>>((long long)(h->zplane * h->zplanes), 0.05f, h->Zk);
  std::vector<CUtensorMap> ma(cands.size()), mb(cands.size());
  for (size_t i = 0; i < cands.size(); ++i)
    CKS(wide_maps(h, C, pc, 0, cands[i].w.bn, cands[i].w.kb, &ma[i], &mb[i], cands[i].w.tr != 0));
  auto launch = [&](size_t i) {
    const WidePlan& w = cands[i].w;
    tc::Params prm{};
    prm.M = w.tr ? v : (int)M;
    prm.N = w.tr ? (int)M : v;
    prm.kt_total = pc * (vp / w.kb);
    prm.kt_per_split = (int)cdiv(prm.kt_total, w.sk);
    prm.nsplit = w.sk;
    prm.nprod = h->nprod_main;
    prm.vtiles = vp / w.kb;
    prm.out = part;
    prm.ldo = v;
    prm.split_stride = M * v;
    prm.accum = 0;
    prm.err = h->d_err;
    wide_dispatch(w.bn, w.mb, h->nprod_main, w.kb, ma[i], mb[i], prm, h->stream, w.tr != 0);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (size_t i = 0; i < cands.size(); ++i) launch(i);
  for (auto& c : cands) c.ms = 1e30f;
  for (int r = 0; r < 5; ++r)
    for (size_t i = 0; i < cands.size(); ++i) {
      cudaEventRecord(e0, h->stream);
      launch(i);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      cands[i].ms = std::min(cands[i].ms, ms);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  int herr = 0;
  CK(cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) return set_error(RTTDA_E_TIMEOUT, "exchange autotuner: a device wait ran out (code " + std::to_string(herr) + ")");
  size_t bi = 0;
  for (size_t i = 0; i < cands.size(); ++i) {
    if (i < 8) h->plan.tune_ms[i] = cands[i].ms;
    if (cands[i].ms < cands[bi].ms) bi = i;
  }
  out = cands[bi].w;
  h->plan.tuned = 1;
  std::lock_guard<std::mutex> g(g_tune_mu);
  if (g_tune_cache.emplace(key, out).second) tune_file_append(key, out);
  return RTTDA_OK;
}

// Buffers, split-K plan and TMA maps of the tensor-core exchange for C columns.
static rttda_status alloc_tc(rttda_ctx* h, int C) {
  const int o = h->o, v = h->v, P = h->P, vp = h->vp, op = h->op;
  const size_t xt = (size_t)C * vp * op;
  CKS(dalloc(&h->Xt, xt * h->nplanes));
  // Z chunk: C*o rows of zchunk*vp BF16 per plane, at most ~2 GiB in total
  const size_t zper = (size_t)C * o * vp * 2 * h->zplanes;
  h->zchunk = zchunk_for(P, zbudget_bytes(), zper);
  h->zplane = (size_t)C * o * h->zchunk * vp;
  CKS(dalloc(&h->Zk, h->zplane * h->zplanes));
  // main contraction tiles.  BF16 and BF16X2 (Z is one plane): wide-M tiles
  // (MB 128-row accumulators per CTA), plan chosen by timing the candidates
  // (tune_wide); BF16X3: 128-row tiles with the N width that wastes least.
  const long long M = (long long)C * o;
  int kb = tc::kBK;  // main K tile width
  h->wide_mb = 0;
  h->wide_tr = false;
  h->plan = rttda_plan_info{};
  if (h->nprod_main <= 2) {
    WidePlan wp;
    CKS(tune_wide(h, C, wp));
    h->tc_bn = wp.bn;
    h->wide_mb = wp.mb;
    h->wide_kb = kb = wp.kb;
    h->wide_tr = wp.tr != 0;
    h->SK = wp.sk;
  } else {
    int best = 256;
    long long bestw = -1;
    for (int bn : {128, 224, 256}) {
      const long long wasted = cdiv(v, bn) * bn;
      if (bestw < 0 || wasted < bestw || (wasted == bestw && bn > best)) {
        best = bn;
        bestw = wasted;
      }
    }
    h->tc_bn = best;
    h->SK = choose_splits(cdiv(M, tc::kBM) * cdiv(v, best), (long long)h->zchunk * (vp / kb));
  }
  const int best = h->tc_bn;
  // Clustered main contraction: clusters of 4 CTAs over 4 column tiles share
  // every Z tile by TMA multicast when the plan is the wide-M tile with BN
  // 192 (K tile 64 or 32) and a multiple of 4 column tiles, and Z dominates the
  // operand bytes (Z is C o / v times B_vv; here at least twice).  Measured
  // under the power cap: on the batched field scan (Z 10.7 x B_vv) the
  // kernel's DRAM reads drop from 68 to 55 GB per launch, the SM clock
  // rises by about 10 % and the step runs 4-6 % faster, although only 33
  // clusters of 4 (132 CTAs) are co-resident; on the large system (Z 0.33 x
  // B_vv) the fewer CTAs cost 1.5 %.  Clusters of 2 read more, not less.
  // RTTDA_WIDE_CLUSTER = 1 (off), 2 or 4 overrides the choice.
  h->wide_cl = 1;
  h->wide_grid = 0;
  {
    int cl = M >= 2LL * v ? 4 : 1;
    if (const char* e = std::getenv("RTTDA_WIDE_CLUSTER")) cl = std::atoi(e);
    if ((cl == 2 || cl == 4) && h->wide_mb == 2 && !h->wide_tr && best == 192 && (kb == 64 || kb == 32) &&
        cdiv(v, best) % cl == 0 && (h->nprod_main == 1 || h->nprod_main == 2)) {
      const long long tmn = cdiv(v, best) * cdiv(M, 2LL * tc::kBM);
      const int cap = wide_cluster_capacity(h->nprod_main, kb, cl);
      if (cap >= cl) {
        // fewer CTAs than SMs: keep the plan's split count unless its last
        // wave leaves more than a tenth of the launch idle, then choose the
        // split count for the cluster grid (units are multiples of CL)
        auto eff = [&](long long units) {
          const long long g = std::min<long long>(cap, units);
          return (double)units / (double)(cdiv(units, g) * g);
        };
        if (eff(tmn * h->SK) < 0.9) h->SK = choose_splits(tmn, (long long)h->zchunk * (vp / kb), cap);
        h->wide_cl = cl;
        h->wide_grid = (int)std::min<long long>(cap, tmn * h->SK);
      }
    }
  }
  h->plan.main_kernel = h->wide_tr ? 4 : h->wide_mb ? 2 : 1;
  h->plan.main_bn = best;
  h->plan.main_mb = h->wide_mb ? h->wide_mb : 1;
  h->plan.main_kb = kb;
  h->plan.main_splits = h->SK;
  h->plan.main_cluster = h->wide_cl;
  h->plan.main_grid = h->wide_cl > 1 ? h->wide_grid
                      : h->wide_mb ? (int)std::min<long long>(kNumSM, cdiv(h->wide_tr ? v : M, (long long)tc::kBM * h->wide_mb) *
                                                                         cdiv(h->wide_tr ? M : v, best) * h->SK)
                                   : 0;
  h->plan.z_chunk = h->zchunk;
  char* p = nullptr;
  CKS(dalloc_bytes((void**)&p, (size_t)h->SK * C * o * v * sizeof(float)));
  h->Kpart = p;
  // maps
  {
    const uint64_t dims[3] = {(uint64_t)op, (uint64_t)C * vp, (uint64_t)h->nplanes};
    const uint64_t str[2] = {(uint64_t)op * 2, (uint64_t)xt * 2};
    const uint32_t box[3] = {64, (uint32_t)kZBN, 1};
    CKS(bf16_map(&h->tmZB, h->Xt, 3, dims, str, box));
  }
  for (int p0 = 0; p0 < P; p0 += h->zchunk) {
    const int pc = std::min(h->zchunk, P - p0);
    CUtensorMap za, ma, mb, zs;
    {
      const uint64_t dims[3] = {(uint64_t)op, (uint64_t)pc * o, (uint64_t)h->nplanes};
      const uint64_t str[2] = {(uint64_t)op * 2, (uint64_t)P * o * op * 2};
      const uint32_t box[3] = {64, 128, 1};
      CKS(bf16_map(&za, h->Boo_tc + (size_t)p0 * o * op, 3, dims, str, box));
    }
    {
      // Z as [plane][(P, b/64)][(col, i)][64]; the Z build stores 32-row x
      // 64-column boxes from 128-byte swizzled staging
      const uint64_t dims[4] = {64, (uint64_t)C * o, (uint64_t)pc * (vp / 64), (uint64_t)h->zplanes};
      const uint64_t str[3] = {128, (uint64_t)C * o * 128, (uint64_t)h->zplane * 2};
      const uint32_t sbox[4] = {64, 32, 1, 1};
      CKS(bf16_map(&zs, h->Zk, 4, dims, str, sbox, CU_TENSOR_MAP_SWIZZLE_128B));
    }
    // main contraction operands: Z tiles and B^P_vv tiles of K-tile width kb
    CKS(wide_maps(h, C, pc, p0, best, kb, &ma, &mb, h->wide_tr));
    if (h->wide_cl > 1) {
      CUtensorMap mac, mbc;
      CKS(wide_maps(h, C, pc, p0, best, kb, &mac, &mbc, false, tc::kBM / h->wide_cl));
      h->tmMAc.push_back(mac);
    }
    h->tmZA.push_back(za);
    h->tmMA.push_back(ma);
    h->tmZS.push_back(zs);
    h->tmMB.push_back(mb);
    const long long kt = (long long)pc * (vp / kb);
    h->tc_kper.push_back((int)cdiv(kt, h->SK));
  }
  return RTTDA_OK;
}

rttda_status rttda_ctx::alloc_tc(int C) { return ::alloc_tc(this, C); }

// Buffers, split-K plan and TMA maps of the FP64-accurate exchange (FP64_OZ)
// for C columns.  Main contraction: split-K over whole P, enough splits that
// the (m, n) tiles times the splits fill the SMs once.
static rttda_status alloc_oz(rttda_ctx* h, int C) {
  const int o = h->o, v = h->v, P = h->P, vp = h->vp, op = h->op;
  constexpr int S = oz::kS;
  const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_64B;
  CKS(dalloc(&h->oz_x, (size_t)S * C * vp * op));
  CKS(dalloc(&h->oz_ex, (size_t)C * vp));
  // Z chunk: the integer Z (8 bytes) and its digits (2 bytes each) per element
  const size_t zper = (size_t)C * o * vp * (8 + 2 * S);
  h->zchunk = zchunk_for(P, zbudget_bytes(), zper);
  const int zc = h->zchunk;
  CKS(dalloc(&h->oz_zi, (size_t)zc * o * C * vp));
  h->oz_zplane = (size_t)C * o * zc * vp;
  CKS(dalloc(&h->oz_z, h->oz_zplane * S));
  CKS(dalloc(&h->oz_ez, (size_t)C * o * zc * h->oz_nbp));
  const long long tiles = cdiv((long long)C * o, tc::kBM) * cdiv(v, oz::kBN);
  const int sk = (int)std::max(1LL, std::min<long long>(zc, kNumSM / tiles));
  h->oz_pps = (int)cdiv(zc, sk);
  h->SK = (int)cdiv(zc, h->oz_pps);
  char* p = nullptr;
  CKS(dalloc_bytes((void**)&p, (size_t)h->SK * C * o * v * sizeof(double)));
  h->Kpart = p;
  h->plan = rttda_plan_info{};
  h->plan.main_kernel = 3;
  h->plan.main_bn = oz::kBN;
  h->plan.main_mb = 1;
  h->plan.main_kb = oz::kKB;
  h->plan.main_splits = h->SK;
  h->plan.z_chunk = zc;
  {
    // amplitude digits: B operand of the Z build, rows (col, b), K = j
    const uint64_t dims[3] = {(uint64_t)op, (uint64_t)C * vp, (uint64_t)S};
    const uint64_t str[2] = {(uint64_t)op * 2, (uint64_t)C * vp * op * 2};
    const uint32_t box[3] = {(uint32_t)oz::kKB, (uint32_t)oz::kBN, 1};
    CKS(bf16_map(&h->tmOzX, h->oz_x, 3, dims, str, box, sw));
  }
  for (int p0 = 0; p0 < P; p0 += zc) {
    const int pc = std::min(zc, P - p0);
    CUtensorMap mo, mz, mv;
    {
      // B_oo digits of the chunk: A of the Z build, rows (P, i), K = j
      const uint64_t dims[3] = {(uint64_t)op, (uint64_t)pc * o, (uint64_t)S};
      const uint64_t str[2] = {(uint64_t)op * 2, (uint64_t)P * o * op * 2};
      const uint32_t box[3] = {(uint32_t)oz::kKB, (uint32_t)tc::kBM, 1};
      CKS(bf16_map(&mo, h->oz_boo + (size_t)p0 * o * op, 3, dims, str, box, sw));
    }
    {
      // Z digits: A of the main contraction, [digit][(P, b/64)][(col, i)][64]
      const uint64_t dims[4] = {64, (uint64_t)C * o, (uint64_t)pc * (vp / 64), (uint64_t)S};
      const uint64_t str[3] = {128, (uint64_t)C * o * 128, (uint64_t)h->oz_zplane * 2};
      const uint32_t box[4] = {(uint32_t)oz::kKB, (uint32_t)tc::kBM, 1, 1};
      CKS(bf16_map(&mz, h->oz_z, 4, dims, str, box, sw));
    }
    {
      // B_vv digits of the chunk: B of the main contraction, (b, a, P, digit)
      const uint64_t dims[4] = {(uint64_t)vp, (uint64_t)v, (uint64_t)pc, (uint64_t)S};
      const uint64_t str[3] = {(uint64_t)vp * 2, (uint64_t)v * vp * 2, (uint64_t)P * v * vp * 2};
      const uint32_t box[4] = {(uint32_t)oz::kKB, (uint32_t)oz::kBN, 1, 1};
      CKS(bf16_map(&mv, h->oz_bvv + (size_t)p0 * v * vp, 4, dims, str, box, sw));
    }
    h->tmOzBoo.push_back(mo);
    h->tmOzZ.push_back(mz);
    h->tmOzBvv.push_back(mv);
  }
  return RTTDA_OK;
}

// Coulomb on digits for C columns: split-K counts of both passes (whole
// blocks of 512 per split, enough splits to fill the SMs once), buffers and
// maps.
static rttda_status alloc_oz_coul(rttda_ctx* h, int C) {
  constexpr int S = oz::kS;
  const int P = h->P;
  const long long ov = h->ov;
  const int cp = (int)cdiv(C, oz::kBN) * oz::kBN;
  h->oz_cp = cp;
  auto splits = [](long long tiles, int nblk, int& pps) {
    const int sk = (int)std::max(1LL, std::min<long long>(nblk, kNumSM / std::max(1LL, tiles)));
    pps = (int)cdiv(nblk, sk);
    return (int)cdiv(nblk, pps);
  };
  h->SW = splits(cdiv(P, tc::kBM) * (cp / oz::kBN), h->oz_nkb, h->oz_pps1);
  h->SJ = splits(cdiv(ov, tc::kBM) * (cp / oz::kBN), h->oz_npb, h->oz_pps2);
  CKS(dalloc(&h->oz_xc, (size_t)S * cp * h->oz_ovp));
  CKS(dalloc(&h->oz_exc, (size_t)h->oz_nkb * cp));
  CKS(dalloc(&h->oz_wpart, (size_t)h->SW * P * C));
  CKS(dalloc(&h->oz_w, (size_t)S * cp * h->oz_Pp));
  CKS(dalloc(&h->oz_ew, (size_t)h->oz_npb * cp));
  char* p = nullptr;
  CKS(dalloc_bytes((void**)&p, (size_t)h->SJ * ov * C * sizeof(double)));
  h->Jpart = p;
  CKS(dalloc_bytes((void**)&p, sizeof(double)));  // SIMT pass-1 scratch is unused here
  h->w = p;
  const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_64B;
  auto map3 = [&](CUtensorMap* m, const void* base, uint64_t k, uint64_t rows, uint32_t boxr) {
    const uint64_t dims[3] = {k, rows, (uint64_t)S};
    const uint64_t str[2] = {k * 2, rows * k * 2};
    const uint32_t box[3] = {(uint32_t)oz::kKB, boxr, 1};
    return bf16_map(m, base, 3, dims, str, box, sw);
  };
  CKS(map3(&h->tmOzBov, h->oz_bov, (uint64_t)h->oz_ovp, (uint64_t)P, tc::kBM));
  CKS(map3(&h->tmOzXc, h->oz_xc, (uint64_t)h->oz_ovp, (uint64_t)cp, oz::kBN));
  CKS(map3(&h->tmOzBovT, h->oz_bovt, (uint64_t)h->oz_Pp, (uint64_t)ov, tc::kBM));
  CKS(map3(&h->tmOzW, h->oz_w, (uint64_t)h->oz_Pp, (uint64_t)cp, oz::kBN));
  return RTTDA_OK;
}

rttda_status rttda_ctx::alloc_batch() {
  const int C = 2 * T;
  const long long NC = N * C;
  CKS(dalloc(&Xn, NC));
  CKS(dalloc(&Xs, NC));
  CKS(dalloc(&Xs2, NC));
  CKS(dalloc(&acc, NC));
  CKS(dalloc(&F, NC));
  CKS(dalloc(&term, NC));
  CKS(dalloc(&Xq, NC));
  CKS(dalloc(&E, 4 * (size_t)T));
  CKS(dalloc(&d_step, 1));
  // Coulomb scratch
  coul_tc = tc && Bov_tc != nullptr && C >= 16;
  if (oz) {
    CKS(::alloc_oz_coul(this, C));
  } else if (coul_tc) {
    CKS(alloc_coul_tc(this, C));
  } else {
    const int V = (int)(16 / fbytes);
    coul_vec = (ov % V) == 0 && C <= 12;
    coul_stream = coul_vec && cbytes != 8;
    const size_t max_smem = 96 * 1024;
    if (coul_stream) {
      // pass 1 over (32-row blocks) x SW slices (a slice's FP32 amplitudes
      // fit the 48 KB of shared memory), pass 2 over (256 V-wide ia blocks) x
      // SJ chunks of P; each count chosen for whole waves of the CTAs that
      // fit on the SMs (ties to fewer partials)
      const long long smax = std::max<long long>(V, (stream::kW1SmemBytes / (C * 4)) / V * V);
      int occ_w = 1, occ_j = 1;
      if (prec == RTTDA_BF16)
        coul_stream_occ<__nv_bfloat16>(C, (size_t)smax * C * 4, (size_t)cdiv(P, 8) * C * 4, &occ_w, &occ_j);
      else
        coul_stream_occ<float>(C, (size_t)smax * C * 4, (size_t)cdiv(P, 8) * C * 4, &occ_w, &occ_j);
      auto waves = [](long long blocks, int occ) {
        const double x = (double)blocks / ((double)kNumSM * occ);
        return x / std::ceil(x);
      };
      const long long nrb = cdiv(P, stream::kW1Rows);
      double best = -1.0;
      for (int sw = (int)cdiv(ov, smax); sw <= std::max<long long>(64, cdiv(ov, smax)); ++sw) {
        const long long sl = cdiv(cdiv(ov, sw), V) * V;
        if (cdiv(ov, sl) != sw || sl > smax) continue;
        const double sc = waves(nrb * sw, occ_w) - 0.002 * sw;
        if (sc > best) {
          best = sc;
          SW = sw;
          wslice = (int)sl;
        }
      }
      const long long nib = cdiv(ov, 256LL * V);
      best = -1.0;
      for (int sj = 1; sj <= 64; ++sj) {
        const long long pc = cdiv(P, sj);
        if (cdiv(P, pc) != sj || (sj > 1 && pc < 8) || pc * C * 4 > 48 * 1024) continue;
        const double sc = waves(nib * sj, occ_j) - 0.002 * sj;
        if (sc > best) {
          best = sc;
          SJ = sj;
          pchunkJ = (int)pc;
        }
      }
    } else if (coul_vec) {
      // pass 1: amplitude slices of wslice rows staged in shared memory
      wslice = (int)std::min<long long>(ov, std::max<long long>(V * 32, (long long)(max_smem / (C * cbytes)) / (V * 32) * (V * 32)));
      wslice = (int)std::min<long long>(wslice, std::max<long long>(V * 32, cdiv(cdiv(ov, cdiv(4 * kNumSM, cdiv(P, 32))), V * 32) * V * 32));
      SW = (int)cdiv(ov, wslice);
      // pass 2: each thread owns V rows; split P so that ~4 blocks per SM run
      const long long xblocks = cdiv(cdiv(ov, V), 256);
      SJ = (int)std::max(1LL, std::min<long long>(std::min(P, 16), cdiv(4 * kNumSM, xblocks)));
    } else {
      SW = (int)std::max(1LL, std::min(cdiv(4 * kNumSM, cdiv(P, 8)), cdiv(ov, 2048)));
      const long long xblocks = cdiv(ov, 256);
      SJ = (int)std::max(1LL, std::min<long long>(P, cdiv(4 * kNumSM, xblocks)));
    }
    if (!coul_stream) {
      pchunkJ = (int)cdiv(P, SJ);
      while ((size_t)pchunkJ * C * cbytes > max_smem && pchunkJ > 1) pchunkJ = (pchunkJ + 1) / 2;
      SJ = (int)cdiv(P, pchunkJ);
    }
    if (coul_stream) CKS(dalloc(&Xf, (size_t)ov * C));
    char* p = nullptr;
    CKS(dalloc_bytes((void**)&p, (size_t)SW * P * C * cbytes));
    w = p;
    CKS(dalloc_bytes((void**)&p, (size_t)SJ * ov * C * cbytes));
    Jpart = p;
  }
  // exchange scratch: Z for a chunk of P (bounded size), split-K partials
  if (oz) {
    CKS(::alloc_oz(this, C));
  } else if (!tc) {
    const size_t zper = (size_t)v * C * o * cbytes;
    const size_t zbudget = (size_t)1 << 30;
    zchunk = zchunk_for(P, zbudget, zper);
    char* p = nullptr;
    CKS(dalloc_bytes((void**)&p, (size_t)zchunk * zper));
    Zt = p;
    const int BM = prec == RTTDA_FP64 ? Tile<double>::BM : Tile<float>::BM;
    const int BN = prec == RTTDA_FP64 ? Tile<double>::BN : Tile<float>::BN;
    const int BK = prec == RTTDA_FP64 ? Tile<double>::BK : Tile<float>::BK;
    const long long tiles = cdiv((long long)C * o, BM) * cdiv(v, BN);
    const long long kchunks = cdiv((long long)zchunk * v, BK);
    SK = (int)std::max(1LL, std::min(kchunks, cdiv(4 * kNumSM, tiles)));
    CKS(dalloc_bytes((void**)&p, (size_t)SK * C * o * v * cbytes));
    Kpart = p;
  } else {
    CKS(alloc_tc(C));
  }
  obsG = (int)std::max(1LL, std::min(1024LL, cdiv(N, 2048)));
  obs_rows = cdiv(N, obsG);
  obsG = (int)cdiv(N, obs_rows);
  CKS(dalloc(&obs_part, (size_t)obsG * T * 2));
  CKS(dalloc(&f0_part, (size_t)kF0Chunks * T * 2));
  return RTTDA_OK;
}

// Upload the molecule: factors cast on the device to the working type.
static rttda_status create_impl(rttda_ctx* h, const double* eps_occ, const double* eps_virt, const double* B_ov,
                                const double* B_oo, const double* B_vv, const double* mu_oo, const double* mu_vv,
                                const double* mu_0ov) {
  CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
  AllocStream as(h->stream);
  dispatch(h->prec, [&](auto ops) { decltype(ops)::set_smem_limits(); });
  if (const char* e = std::getenv("RTTDA_ZHINT")) h->z_hint = std::atoi(e) != 0;
  if (const char* e = std::getenv("RTTDA_ZRES1")) h->z_res1 = std::atoi(e) != 0;
  if (const char* e = std::getenv("RTTDA_TEST_BREAK_CAPTURE")) h->break_capture = std::atoi(e) != 0;
  if (const char* e = std::getenv("RTTDA_ZRUN")) h->z_run = std::max(0, std::atoi(e));
  const size_t o = h->o, v = h->v, P = h->P;
  const size_t chunk = (size_t)1 << 26;  // elements per staging pass
  const size_t stage_n = std::min(chunk, std::max({P * o * v, P * o * o, P * v * v}));
  double* stage = nullptr;
  struct Guard {
    double*& p;
    ~Guard() { dfree(p); }
  } guard{stage};
  if (h->prec != RTTDA_FP64)
    CKS(dalloc(&stage, std::max(stage_n, h->tc || h->oz ? std::max(v * v, o * o) : (size_t)1)));
  CKS(dalloc(&h->d_err, 1));
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  auto upload = [&](const double* src, size_t n, void** dst) -> rttda_status {
    CKS(dalloc_bytes((void**)dst, std::max<size_t>(n, 1) * h->fbytes));
    for (size_t off = 0; off < n; off += chunk) {
      const size_t m = std::min(chunk, n - off);
      if (h->fbytes == 8) {
        CK(cudaMemcpyAsync((double*)*dst + off, src + off, m * 8, cudaMemcpyDefault, h->stream));
      } else {
        CK(cudaMemcpyAsync(stage, src + off, m * 8, cudaMemcpyDefault, h->stream));
        if (h->fbytes == 4)
          k_cast<float><<<blocks_for(m, 256), 256, 0, h->stream>>>(m, stage, (float*)*dst + off);
        else
          k_cast<__nv_bfloat16><<<blocks_for(m, 256), 256, 0, h->stream>>>(m, stage, (__nv_bfloat16*)*dst + off);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->stream));
      }
    }
    return RTTDA_OK;
  };
  // tensor-core operands: BF16 hi (and lo) planes with zero padding, packed
  // slab by slab of whole P
  auto pack = [&](const double* src, size_t slab, size_t out_slab, bool vv, __nv_bfloat16** dst) -> rttda_status {
    const size_t plane = P * out_slab;
    CKS(dalloc_bytes((void**)dst, plane * h->nplanes * 2));
    const size_t per = std::max<size_t>(1, chunk / std::max<size_t>(slab, 1));
    for (size_t p0 = 0; p0 < P; p0 += per) {
      const size_t pc = std::min(per, P - p0);
      CK(cudaMemcpyAsync(stage, src + p0 * slab, pc * slab * 8, cudaMemcpyDefault, h->stream));
      __nv_bfloat16* hi = *dst + p0 * out_slab;
      __nv_bfloat16* lo = h->nplanes > 1 ? hi + plane : nullptr;
      const long long tot = (long long)(pc * out_slab);
      if (vv)
        k_pack_vv<<<blocks_for(tot, 256), 256, 0, h->stream>>>((int)pc, h->v, h->vp, stage, hi, lo);
      else
        k_pack_oo<<<blocks_for(tot, 256), 256, 0, h->stream>>>((int)pc, h->o, h->op, stage, hi, lo);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(h->stream));
    }
    return RTTDA_OK;
  };
  auto upload64 = [&](const double* src, size_t n, double** dst) -> rttda_status {
    CKS(dalloc_bytes((void**)dst, std::max<size_t>(n, 1) * 8));
    CK(cudaMemcpyAsync(*dst, src, n * 8, cudaMemcpyDefault, h->stream));
    return RTTDA_OK;
  };
  CKS(upload(B_ov, P * o * v, &h->Bov));
  if (h->oz) {
    // Ozaki digits of B_ov (rows P, K = ia) and of its transpose (rows ia,
    // K = P) for the Coulomb passes; the FP64 copy goes afterwards
    constexpr int S = oz::kS;
    const long long ovl = (long long)(o * v);
    h->oz_ovp = (int)(cdiv(ovl, 8) * 8);
    h->oz_Pp = (int)(cdiv((long long)P, 8) * 8);
    h->oz_nkb = (int)cdiv(ovl, oz::kBlk);
    h->oz_npb = (int)cdiv((long long)P, oz::kBlk);
    CKS(dalloc(&h->oz_bov, S * P * (size_t)h->oz_ovp));
    CKS(dalloc(&h->oz_ebov, (size_t)h->oz_nkb * P));
    CKS(dalloc(&h->oz_bovt, S * (size_t)ovl * h->oz_Pp));
    CKS(dalloc(&h->oz_ebovt, (size_t)h->oz_npb * ovl));
    const double* B = (const double*)h->Bov;
    oz::k_slice_rows<int><<<blocks_for((long long)P * h->oz_nkb * 32, 256), 256, 0, h->stream>>>(
        (long long)P, (long long)P, (int)ovl, h->oz_ovp, B, ovl, 1, h->oz_bov, (long long)h->oz_ovp,
        (long long)P * h->oz_ovp, h->oz_ebov, (long long)P, h->oz_nkb);
    oz::k_slice_rows<int><<<blocks_for(ovl * h->oz_npb * 32, 256), 256, 0, h->stream>>>(
        ovl, ovl, (int)P, h->oz_Pp, B, 1, ovl, h->oz_bovt, (long long)h->oz_Pp, ovl * h->oz_Pp, h->oz_ebovt, ovl,
        h->oz_npb);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    dfree(h->Bov);
    h->Bov = nullptr;
  }
  if (h->tc) {
    CKS(pack(B_oo, o * o, o * (size_t)h->op, false, &h->Boo_tc));
    CKS(pack(B_vv, v * v, (size_t)h->vp * h->vp, true, &h->Bvv_tc));
    if ((o * v) % 8 == 0 && P % 8 == 0) {
      // B_ov and its transpose as BF16 planes for batched Coulomb passes
      const size_t ov = o * v, plane = P * ov;
      CKS(dalloc_bytes((void**)&h->Bov_tc, plane * h->nplanes * 2));
      CKS(dalloc_bytes((void**)&h->BovT_tc, plane * h->nplanes * 2));
      const size_t per = std::max<size_t>(1, chunk / ov);
      for (size_t p0 = 0; p0 < P; p0 += per) {
        const size_t pc = std::min(per, P - p0);
        CK(cudaMemcpyAsync(stage, B_ov + p0 * ov, pc * ov * 8, cudaMemcpyDefault, h->stream));
        dim3 g((unsigned)cdiv(ov, 32), (unsigned)cdiv(pc, 32));
        k_pack_ov<<<g, dim3(32, 8), 0, h->stream>>>((int)pc, (int)p0, (int)P, (long long)ov, stage, h->Bov_tc,
                                                   h->nplanes > 1 ? h->Bov_tc + plane : nullptr, h->BovT_tc,
                                                   h->nplanes > 1 ? h->BovT_tc + plane : nullptr, (long long)plane);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->stream));
      }
    }
  } else if (h->oz) {
    // Ozaki digits of B_oo (rows (P, i), K = j: one block, nocc <= 512) and
    // of B_vv (rows (P, a), K = b in blocks of 512), sliced slab by slab of
    // whole P from a staging copy; no FP64 copy of these factors is kept
    constexpr int S = oz::kS;
    const size_t op = h->op, vp = h->vp, nbp = (size_t)cdiv(vp, oz::kBlk);
    h->oz_nbp = (int)nbp;
    CKS(dalloc(&h->oz_boo, S * P * o * op));
    CKS(dalloc(&h->oz_eoo, P * o));
    CKS(dalloc(&h->oz_bvv, S * P * v * vp));
    CKS(dalloc(&h->oz_evv, vp * P * nbp));
    auto slice = [&](const double* src, size_t slab, bool vv) -> rttda_status {
      const size_t per = std::max<size_t>(1, chunk / slab);
      for (size_t p0 = 0; p0 < P; p0 += per) {
        const size_t pc = std::min(per, P - p0);
        CK(cudaMemcpyAsync(stage, src + p0 * slab, pc * slab * 8, cudaMemcpyDefault, h->stream));
        if (vv) {
          const long long rows = (long long)(pc * v);
          oz::k_slice_rows<short><<<blocks_for(rows * (long long)nbp * 32, 256), 256, 0, h->stream>>>(
              rows, (long long)v, (int)v, (int)vp, stage, (long long)v, 1, h->oz_bvv + p0 * v * vp, (long long)vp,
              (long long)(P * v * vp), h->oz_evv + p0 * nbp * vp, (long long)vp, (int)nbp);
        } else {
          const long long rows = (long long)(pc * o);
          oz::k_slice_rows<short><<<blocks_for(rows * 32, 256), 256, 0, h->stream>>>(
              rows, rows, (int)o, (int)op, stage, (long long)o, 1, h->oz_boo + p0 * o * op, (long long)op,
              (long long)(P * o * op), h->oz_eoo + p0 * o, rows, 1);
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->stream));
      }
      return RTTDA_OK;
    };
    CKS(slice(B_oo, o * o, false));
    CKS(slice(B_vv, v * v, true));
  } else {
    CKS(upload(B_oo, P * o * o, &h->Boo));
    CKS(upload(B_vv, P * v * v, &h->Bvv));
  }
  CKS(upload64(eps_occ, o, &h->eps_o));
  CKS(upload64(eps_virt, v, &h->eps_v));
  CKS(upload64(mu_oo, 3 * o * o, &h->mu_oo));
  CKS(upload64(mu_vv, 3 * v * v, &h->mu_vv));
  CKS(upload64(mu_0ov, 3 * o * v, &h->mu_0));
  CK(cudaStreamSynchronize(h->stream));
  // spectral-norm bound of M_x: |m_x| + |mu_vv,x|_F + |mu_oo,x|_F (from host
  // copies, so the inputs may live in host or device memory)
  std::vector<double> hm0(3 * o * v), hmv(3 * v * v), hmo(3 * o * o);
  CK(cudaMemcpy(hm0.data(), mu_0ov, hm0.size() * 8, cudaMemcpyDefault));
  CK(cudaMemcpy(hmv.data(), mu_vv, hmv.size() * 8, cudaMemcpyDefault));
  CK(cudaMemcpy(hmo.data(), mu_oo, hmo.size() * 8, cudaMemcpyDefault));
  for (int x = 0; x < 3; ++x)
    h->mu_bound[x] = fro(hm0.data() + x * o * v, o * v) + fro(hmv.data() + x * v * v, v * v) +
                     fro(hmo.data() + x * o * o, o * o);
  return RTTDA_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int rttda_abi_version(void) { return RTTDA_ABI_VERSION; }

const char* rttda_last_error(void) { return g_last_error.c_str(); }

rttda_status rttda_create(int nocc, int nvirt, int naux, const double* eps_occ, const double* eps_virt,
                          const double* B_ov, const double* B_oo, const double* B_vv, const double* mu_oo,
                          const double* mu_vv, const double* mu_0ov, double c_x, int prec, rttda_t* out) {
  g_last_error.clear();
  if (!out) return set_error(RTTDA_E_ARG, "rttda_create: out is NULL");
  *out = nullptr;
  if (nocc < 1 || nvirt < 1 || naux < 1) return set_error(RTTDA_E_ARG, "rttda_create: nocc, nvirt, naux must be >= 1");
  if (!eps_occ || !eps_virt || !B_ov || !B_oo || !B_vv || !mu_oo || !mu_vv || !mu_0ov)
    return set_error(RTTDA_E_ARG, "rttda_create: NULL input array");
  if (prec == RTTDA_TF32)
    return set_error(RTTDA_E_ARG, "rttda_create: TF32 is not provided (BF16X2 is faster and more accurate on B300)");
  if (prec != RTTDA_FP64 && prec != RTTDA_FP32 && prec != RTTDA_BF16 && prec != RTTDA_BF16X3 &&
      prec != RTTDA_BF16X2 && prec != RTTDA_FP64_OZ)
    return set_error(RTTDA_E_ARG, "rttda_create: unsupported precision");
  if (prec == RTTDA_FP64_OZ && nocc > oz::kBlk)
    return set_error(RTTDA_E_ARG, "rttda_create: FP64_OZ needs nocc <= 512");
  if (!std::isfinite(c_x)) return set_error(RTTDA_E_ARG, "rttda_create: c_x not finite");

  rttda_ctx* h = new rttda_ctx();
  h->o = nocc;
  h->v = nvirt;
  h->P = naux;
  h->ov = (long long)nocc * nvirt;
  h->N = 1 + h->ov;
  h->cx = c_x;
  h->prec = prec;
  const bool f64 = prec == RTTDA_FP64 || prec == RTTDA_FP64_OZ;
  h->fbytes = f64 ? 8 : prec == RTTDA_BF16 ? 2 : 4;
  h->cbytes = f64 ? 8 : 4;
  h->tc = prec == RTTDA_BF16 || prec == RTTDA_BF16X3 || prec == RTTDA_BF16X2;
  h->oz = prec == RTTDA_FP64_OZ;
  h->nplanes = prec == RTTDA_BF16 ? 1 : 2;          // factor / amplitude planes
  h->nprod = prec == RTTDA_BF16 ? 1 : 3;            // Z = B_oo c products
  h->zplanes = prec == RTTDA_BF16X3 ? 2 : 1;        // Z planes kept
  h->nprod_main = prec == RTTDA_BF16X3 ? 3 : prec == RTTDA_BF16X2 ? 2 : 1;
  h->vp = (int)cdiv(nvirt, 64) * 64;
  h->op = (int)cdiv(nocc, 8) * 8;

  rttda_status st = create_impl(h, eps_occ, eps_virt, B_ov, B_oo, B_vv, mu_oo, mu_vv, mu_0ov);
  if (st != RTTDA_OK) {
    delete h;
    return st;
  }
  *out = h;
  return RTTDA_OK;
}

rttda_status rttda_create_device(int nocc, int nvirt, int naux, const double* eps_occ, const double* eps_virt,
                                 const double* B_ov, const double* B_oo, const double* B_vv, const double* mu_oo,
                                 const double* mu_vv, const double* mu_0ov, double c_x, int prec, rttda_t* out) {
  // the upload path copies with cudaMemcpyDefault, so device sources work as is
  return rttda_create(nocc, nvirt, naux, eps_occ, eps_virt, B_ov, B_oo, B_vv, mu_oo, mu_vv, mu_0ov, c_x, prec, out);
}

rttda_status rttda_memory_bytes(rttda_t h, size_t* bytes) {
  if (!h || !bytes) return set_error(RTTDA_E_ARG, "rttda_memory_bytes: NULL argument");
  const size_t o = h->o, v = h->v, P = h->P;
  size_t b = (h->oz ? 0 : P * o * v * h->fbytes) + (o + v + 3 * (o * o + v * v + o * v)) * 8;
  if (h->tc)
    b += (P * o * (size_t)h->op + P * (size_t)h->vp * h->vp) * 2 * h->nplanes;
  else if (h->oz)
    b += (P * o * (size_t)h->op + P * v * (size_t)h->vp + P * (size_t)h->oz_ovp + (size_t)h->ov * h->oz_Pp) * 2 * oz::kS +
         (P * o + (size_t)h->vp * P * h->oz_nbp + (size_t)h->oz_nkb * P + (size_t)h->oz_npb * h->ov) * 2;
  else
    b += (P * o * o + P * v * v) * h->fbytes;
  if (h->T > 0) {
    const size_t C = 2 * h->T, NC = h->N * C;
    const size_t zb = h->oz ? (size_t)h->zchunk * C * o * h->vp * (8 + 2 * oz::kS) + C * (size_t)h->vp * h->op * 2 * oz::kS
                            : (size_t)h->zchunk * v * C * o * h->cbytes;
    b += NC * 8 * 6 + (size_t)P * C * h->cbytes + (size_t)h->SJ * h->ov * C * h->cbytes + zb +
         (size_t)h->SK * C * o * v * h->cbytes +
         (size_t)h->T * (o * o + v * v + o * v) * (8 + (h->cbytes == 8 ? 0 : h->cbytes));
  }
  *bytes = b;
  return RTTDA_OK;
}

rttda_status rttda_set_field(rttda_t h, const rttda_pulse* pulses, int ntraj) {
  g_last_error.clear();
  if (!h || !pulses) return set_error(RTTDA_E_ARG, "rttda_set_field: NULL argument");
  if (ntraj < 1) return set_error(RTTDA_E_ARG, "rttda_set_field: ntraj must be >= 1");
  if ((long long)h->N * 2 * ntraj >= (1LL << 31))
    return set_error(RTTDA_E_ARG, "rttda_set_field: (1 + nocc*nvirt) * 2 * ntraj must be below 2^31");
  std::vector<PulseDev> pd(ntraj);
  std::vector<double> kappa(ntraj, 0.0), dirs(3 * ntraj);
  bool any_field = false, any_kick = false;
  double xmax = 0.0;
  for (int t = 0; t < ntraj; ++t) {
    const rttda_pulse& p = pulses[t];
    if (p.kind < RTTDA_KICK || p.kind > RTTDA_SIN2) return set_error(RTTDA_E_ARG, "rttda_set_field: unknown pulse kind");
    const double dn = std::sqrt(p.dir[0] * p.dir[0] + p.dir[1] * p.dir[1] + p.dir[2] * p.dir[2]);
    if (!(dn > 0.0) || !std::isfinite(dn)) return set_error(RTTDA_E_ARG, "rttda_set_field: zero polarisation vector");
    if (!std::isfinite(p.E0) || !std::isfinite(p.omega)) return set_error(RTTDA_E_ARG, "rttda_set_field: non-finite E0/omega");
    if ((p.kind == RTTDA_GAUSS_TL || p.kind == RTTDA_CHIRP) && !(p.fwhm > 0.0))
      return set_error(RTTDA_E_ARG, "rttda_set_field: fwhm must be > 0");
    if (p.kind == RTTDA_SIN2 && !(p.duration > 0.0)) return set_error(RTTDA_E_ARG, "rttda_set_field: duration must be > 0");
    for (int x = 0; x < 3; ++x) dirs[3 * t + x] = p.dir[x] / dn;
    pd[t].kind = p.kind;
    pd[t].E0 = p.E0;
    pd[t].omega = p.omega;
    pd[t].t0 = p.t0;
    pd[t].sigma = p.fwhm / 2.35482;  // Sec. 2.2: sigma = FWHM / 2.35482
    pd[t].beta = p.beta;
    pd[t].duration = p.duration;
    if (p.kind == RTTDA_KICK) {
      any_kick = true;
      kappa[t] = p.E0;
      double b = 0.0;
      for (int x = 0; x < 3; ++x) b += std::fabs(dirs[3 * t + x]) * h->mu_bound[x];
      xmax = std::max(xmax, std::fabs(p.E0) * b);
    } else {
      any_field = true;
    }
  }
  // Taylor terms: x^K / K! below 1e-18 with x a bound on |kappa M_d|.
  int K = 0;
  if (any_kick) {
    double term = 1.0;
    K = 0;
    while (K < 400) {
      ++K;
      term *= xmax / K;
      if (term < 1e-18 && K > xmax) break;
    }
    if (K >= 400) return set_error(RTTDA_E_ARG, "rttda_set_field: kick too strong for the Taylor series");
  }

  AllocStream as(h->stream);
  h->free_batch();
  h->T = ntraj;
  h->pulses.assign(pulses, pulses + ntraj);
  h->any_field = any_field;
  h->any_kick = any_kick;
  h->kick_terms = K;
  h->same_dir = true;
  for (int t = 1; t < ntraj; ++t)
    for (int x = 0; x < 3; ++x) h->same_dir = h->same_dir && dirs[3 * t + x] == dirs[x];
  CKS(dalloc(&h->d_pulses, ntraj));
  CKS(dalloc(&h->d_kappa, ntraj));
  CKS(dalloc(&h->d_dirs, 3 * ntraj));
  CK(cudaMemcpyAsync(h->d_pulses, pd.data(), sizeof(PulseDev) * ntraj, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_kappa, kappa.data(), sizeof(double) * ntraj, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_dirs, dirs.data(), sizeof(double) * 3 * ntraj, cudaMemcpyHostToDevice, h->stream));
  const long long loo = (long long)h->o * h->o, lvv = (long long)h->v * h->v, lov = h->ov;
  CKS(dalloc(&h->moo64, loo * ntraj));
  CKS(dalloc(&h->mvv64, lvv * ntraj));
  CKS(dalloc(&h->m064, lov * ntraj));
  cudaStream_t s = h->stream;
  k_dipole_dir<double><<<blocks_for(loo * ntraj, 256), 256, 0, s>>>(loo, ntraj, h->d_dirs, h->mu_oo, h->moo64);
  k_dipole_dir<double><<<blocks_for(lvv * ntraj, 256), 256, 0, s>>>(lvv, ntraj, h->d_dirs, h->mu_vv, h->mvv64);
  k_dipole_dir<double><<<blocks_for(lov * ntraj, 256), 256, 0, s>>>(lov, ntraj, h->d_dirs, h->mu_0, h->m064);
  if (h->cbytes != 8) {
    float* p = nullptr;
    CKS(dalloc(&p, loo * ntraj));
    h->mooC = p;
    CKS(dalloc(&p, lvv * ntraj));
    h->mvvC = p;
    CKS(dalloc(&p, lov * ntraj));
    h->m0C = p;
    k_dipole_dir<float><<<blocks_for(loo * ntraj, 256), 256, 0, s>>>(loo, ntraj, h->d_dirs, h->mu_oo, (float*)h->mooC);
    k_dipole_dir<float><<<blocks_for(lvv * ntraj, 256), 256, 0, s>>>(lvv, ntraj, h->d_dirs, h->mu_vv, (float*)h->mvvC);
    k_dipole_dir<float><<<blocks_for(lov * ntraj, 256), 256, 0, s>>>(lov, ntraj, h->d_dirs, h->mu_0, (float*)h->m0C);
    if (h->same_dir && 2 * ntraj >= 8) {
      // the field GEMMs' operands in their arithmetic types (launch_field)
      CKS(dalloc_bytes(&h->Xfc, (size_t)h->N * 2 * ntraj * sizeof(df32)));
      CKS(dalloc_bytes(&h->moo_df, (size_t)loo * sizeof(df32)));
      CKS(dalloc_bytes(&h->mvv_df, (size_t)lvv * sizeof(df32)));
      k_to_type<df32><<<blocks_for(loo, 256), 256, 0, s>>>(loo, h->moo64, (df32*)h->moo_df);
      k_to_type<df32><<<blocks_for(lvv, 256), 256, 0, s>>>(lvv, h->mvv64, (df32*)h->mvv_df);
    }
  }
  CKS(h->alloc_batch());
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return RTTDA_OK;
}

static rttda_status propagate_impl(rttda_t h, bool fresh, const double* c0_dev, double dt, long nsteps,
                                   double* c_out_dev, double* dip_dev, double* nrm_dev, cudaStream_t s,
                                   long long ld = -1, long long offset = 0) {
  if (h->T < 1) return set_error(RTTDA_E_STATE, "rttda_propagate: call rttda_set_field first");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(RTTDA_E_ARG, "rttda_propagate: dt must be > 0");
  if (nsteps < 0) return set_error(RTTDA_E_ARG, "rttda_propagate: nsteps must be >= 0");
  const long long NT = h->N * h->T;
  double t_call = 0.0;
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  if (fresh) {
    if (c0_dev)
      k_abi_to_dev<<<blocks_for(NT, 256), 256, 0, s>>>(h->N, h->T, c0_dev, h->Xn);
    else
      k_ground<<<blocks_for(NT * 2, 256), 256, 0, s>>>(h->N, h->T, h->Xn);
    if (h->any_kick) enqueue_kick(h, s);
    if (h->acf_on) {
      const long long ne = h->N * 2 * h->T;
      if (ne > h->acf_eps_cap) {
        dfree(h->d_xeps);
        h->d_xeps = nullptr;
        h->acf_eps_cap = 0;
        CKS(dalloc(&h->d_xeps, (size_t)ne));
        h->acf_eps_cap = ne;
      }
      CK(cudaMemcpyAsync(h->d_xeps, h->Xn, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
      h->have_eps = true;
    }
  } else {
    if (!h->have_state) return set_error(RTTDA_E_STATE, "rttda_resume: no state to resume from");
    t_call = h->t_now;
  }
  // traces: both or neither are needed by the kernels; use scratch for a missing one
  double* dip = dip_dev;
  double* nrm = nrm_dev;
  double* tmp = nullptr;
  if ((dip == nullptr) != (nrm == nullptr)) {
    CKS(dalloc(&tmp, (size_t)h->T * (nsteps + 1)));
    if (!dip) dip = tmp;
    if (!nrm) nrm = tmp;
  }
  if (ld < 0) ld = nsteps + 1;
  if (h->nproj > 0) {
    const long long need = (long long)h->T * ld * h->nproj * 2;
    if (need > h->ovl_cap) {
      dfree(h->d_ovl);
      h->d_ovl = nullptr;
      h->ovl_cap = 0;
      CKS(dalloc(&h->d_ovl, (size_t)need));
      h->ovl_cap = need;
    }
    const long long pneed = (long long)h->proj_G * h->nproj * 2 * h->T;
    if (pneed > h->part_cap) {
      dfree(h->d_proj_part);
      h->d_proj_part = nullptr;
      h->part_cap = 0;
      CKS(dalloc(&h->d_proj_part, (size_t)pneed));
      h->part_cap = pneed;
    }
    h->ovl_ld = ld;
  }
  if (h->acf_on && h->have_eps) {
    const long long need = (long long)h->T * ld * 2, pneed = (long long)h->proj_G * h->T * 2;
    if (need > h->acf_cap) {
      dfree(h->d_acf);
      h->d_acf = nullptr;
      h->acf_cap = 0;
      CKS(dalloc(&h->d_acf, (size_t)need));
      h->acf_cap = need;
    }
    if (pneed > h->acf_part_cap) {
      dfree(h->d_acf_part);
      h->d_acf_part = nullptr;
      h->acf_part_cap = 0;
      CKS(dalloc(&h->d_acf_part, (size_t)pneed));
      h->acf_part_cap = pneed;
    }
    h->acf_ld = ld;
  }
  rttda_status st = run_steps(h, t_call, dt, nsteps, dip, nrm, ld, offset, s);
  if (st == RTTDA_OK && c_out_dev) k_dev_to_abi<<<blocks_for(NT, 256), 256, 0, s>>>(h->N, h->T, h->Xn, c_out_dev);
  if (tmp) {
    cudaStreamSynchronize(s);
    cudaFree(tmp);
  }
  if (st != RTTDA_OK) return st;
  CK(cudaGetLastError());
  return RTTDA_OK;
}

}  // extern "C"
namespace rttda {
rttda_status advance(rttda_t h, bool fresh, double dt, long nsteps, double* dip, double* nrm, long long ld,
                     long long offset, cudaStream_t s) {
  return propagate_impl(h, fresh, nullptr, dt, nsteps, nullptr, dip, nrm, s ? s : h->stream, ld, offset);
}
cudaStream_t handle_stream(rttda_t h) { return h->stream; }

rttda_status batch_view(rttda_t h, BatchView* bv) {
  if (h->T < 1) return set_error(RTTDA_E_STATE, "no batch: call rttda_set_field first");
  bv->N = h->N;
  bv->T = h->T;
  bv->nocc = h->o;
  bv->nvirt = h->v;
  bv->eps_o = h->eps_o;
  bv->eps_v = h->eps_v;
  bv->X = h->Xq;
  bv->out = h->term;
  bv->stream = h->stream;
  return RTTDA_OK;
}

rttda_status sigma_A(rttda_t h, cudaStream_t s) {
  dispatch(h->prec, [&](auto ops) {
    using O = decltype(ops);
    O::coulomb(h, h->Xq, s);
    O::exchange(h, h->Xq, s);
    O::combine(h, 1, 0, false, 0.0, h->Xq, nullptr, h->term, s);
  });
  CK(cudaGetLastError());
  return RTTDA_OK;
}
}  // namespace rttda
extern "C" {

rttda_status rttda_propagate_device(rttda_t h, const double* c0_dev, double dt, long nsteps, double* c_out_dev,
                                    double* dipole_dev, double* norm_dev, void* stream) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_propagate_device: NULL handle");
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  return propagate_impl(h, true, c0_dev, dt, nsteps, c_out_dev, dipole_dev, norm_dev, s);
}

// A bounded device wait that ran out leaves a code in d_err.
static rttda_status check_device_error(rttda_t h);
}  // extern "C"
namespace rttda {
rttda_status device_error(rttda_t h) { return check_device_error(h); }
}  // namespace rttda
extern "C" {
static rttda_status check_device_error(rttda_t h) {
  int e = 0;
  CK(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0)
    return set_error(RTTDA_E_TIMEOUT, "a tensor-core pipeline wait exceeded its time limit (code " +
                                          std::to_string(e) + ")");
  return RTTDA_OK;
}

static rttda_status host_call(rttda_t h, bool fresh, const double* c0, double dt, long nsteps, double* c_out,
                              double* dip, double* nrm) {
  if (h->T < 1) return set_error(RTTDA_E_STATE, "rttda_propagate: call rttda_set_field first");
  if (nsteps < 0) return set_error(RTTDA_E_ARG, "rttda_propagate: nsteps must be >= 0");
  const size_t NT2 = (size_t)h->N * h->T * 2, TR = (size_t)h->T * (nsteps + 1);
  const size_t need = 2 * NT2 + 2 * TR;
  if (h->h_io_count < need) {
    dfree(h->h_io);
    h->h_io = nullptr;
    h->h_io_count = 0;
    CKS(dalloc(&h->h_io, need));
    h->h_io_count = need;
  }
  double* d_c0 = h->h_io;
  double* d_cout = d_c0 + NT2;
  double* d_dip = d_cout + NT2;
  double* d_nrm = d_dip + TR;
  cudaStream_t s = h->stream;
  if (c0) CK(cudaMemcpyAsync(d_c0, c0, NT2 * 8, cudaMemcpyHostToDevice, s));
  const bool want_tr = dip || nrm;
  CKS(propagate_impl(h, fresh, c0 ? d_c0 : nullptr, dt, nsteps, c_out ? d_cout : nullptr, want_tr ? d_dip : nullptr,
                     want_tr ? d_nrm : nullptr, s));
  if (c_out) CK(cudaMemcpyAsync(c_out, d_cout, NT2 * 8, cudaMemcpyDeviceToHost, s));
  if (dip) CK(cudaMemcpyAsync(dip, d_dip, TR * 8, cudaMemcpyDeviceToHost, s));
  if (nrm) CK(cudaMemcpyAsync(nrm, d_nrm, TR * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_device_error(h);
}

rttda_status rttda_propagate(rttda_t h, const double* c0, double dt, long nsteps, double* c_out,
                             double* dipole_trace, double* norm_trace) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_propagate: NULL handle");
  return host_call(h, true, c0, dt, nsteps, c_out, dipole_trace, norm_trace);
}

rttda_status rttda_resume(rttda_t h, double dt, long nsteps, double* c_out, double* dipole_trace,
                          double* norm_trace) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_resume: NULL handle");
  if (!h->have_state) return set_error(RTTDA_E_STATE, "rttda_resume: no state to resume from");
  return host_call(h, false, nullptr, dt, nsteps, c_out, dipole_trace, norm_trace);
}

rttda_status rttda_get_state(rttda_t h, double* c, double* t) {
  g_last_error.clear();
  if (!h || !c) return set_error(RTTDA_E_ARG, "rttda_get_state: NULL argument");
  if (!h->have_state) return set_error(RTTDA_E_STATE, "rttda_get_state: no state");
  const long long NT = h->N * h->T;
  k_dev_to_abi<<<blocks_for(NT, 256), 256, 0, h->stream>>>(h->N, h->T, h->Xn, h->term);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c, h->term, NT * 2 * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (t) *t = h->t_now;
  return RTTDA_OK;
}

rttda_status rttda_set_state(rttda_t h, const double* c, double t) {
  g_last_error.clear();
  if (!h || !c) return set_error(RTTDA_E_ARG, "rttda_set_state: NULL argument");
  if (h->T < 1) return set_error(RTTDA_E_STATE, "rttda_set_state: call rttda_set_field first");
  if (!std::isfinite(t)) return set_error(RTTDA_E_ARG, "rttda_set_state: t not finite");
  const long long NT = h->N * h->T;
  CK(cudaMemcpyAsync(h->term, c, NT * 2 * 8, cudaMemcpyHostToDevice, h->stream));
  k_abi_to_dev<<<blocks_for(NT, 256), 256, 0, h->stream>>>(h->N, h->T, h->term, h->Xn);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  h->t_now = t;
  h->have_state = true;
  return RTTDA_OK;
}

rttda_status rttda_sigma(rttda_t h, const double* c_dev, double t, double* sigma_dev, void* stream) {
  g_last_error.clear();
  if (!h || !c_dev || !sigma_dev) return set_error(RTTDA_E_ARG, "rttda_sigma: NULL argument");
  if (h->T < 1) return set_error(RTTDA_E_STATE, "rttda_sigma: call rttda_set_field first");
  if (!std::isfinite(t)) return set_error(RTTDA_E_ARG, "rttda_sigma: t not finite");
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  const long long NT = h->N * h->T;
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  k_abi_to_dev<<<blocks_for(NT, 256), 256, 0, s>>>(h->N, h->T, c_dev, h->Xq);
  // E at time t goes to slot 0 of the stage table (step counter 0, stage 0)
  CK(cudaMemsetAsync(h->d_step, 0, sizeof(long long), s));
  k_efield<<<1, 128, 0, s>>>(h->T, h->d_pulses, h->d_step, 0, t, 0.0, h->E);
  dispatch(h->prec, [&](auto ops) {
    using O = decltype(ops);
    if (h->any_field) O::field(h, h->Xq, s);
    O::coulomb(h, h->Xq, s);
    O::exchange(h, h->Xq, s);
    O::combine(h, 1, 0, h->any_field, 0.0, h->Xq, nullptr, h->term, s);
  });
  k_dev_to_abi<<<blocks_for(NT, 256), 256, 0, s>>>(h->N, h->T, h->term, sigma_dev);
  CK(cudaGetLastError());
  return RTTDA_OK;
}

}  // extern "C"
namespace rttda {
rttda_status spectrum_device(const double* trace_dev, long long ntr, long long npts, double dt, double kappa,
                             double gamma, double wmin, double wmax, long long nfreq, double* om_dev, double* S_dev,
                             cudaStream_t s) {
  if (ntr < 1 || npts < 2 || nfreq < 1 || !(dt > 0.0) || kappa == 0.0 || !(gamma >= 0.0))
    return set_error(RTTDA_E_ARG, "spectrum: bad arguments");
  const double dw = nfreq > 1 ? (wmax - wmin) / (double)(nfreq - 1) : 0.0;
  k_spectrum<<<(unsigned)nfreq, 256, 0, s>>>(trace_dev, ntr, npts, dt, kappa, gamma, wmin, dw, om_dev, S_dev);
  CK(cudaGetLastError());
  return RTTDA_OK;
}

// Device bytes a handle needs for a batch (upper estimate, used for admission).
size_t estimate_bytes(int nocc, int nvirt, int naux, int ntraj, int prec, long nsteps) {
  const size_t o = nocc, v = nvirt, P = naux, T = ntraj, C = 2 * T, ov = o * v, N = 1 + ov;
  const bool tc = prec == RTTDA_BF16 || prec == RTTDA_BF16X3 || prec == RTTDA_BF16X2;
  const bool ozk = prec == RTTDA_FP64_OZ, f64 = prec == RTTDA_FP64 || ozk;
  const size_t fb = f64 ? 8 : prec == RTTDA_BF16 ? 2 : 4, cb = f64 ? 8 : 4;
  const size_t vp = (v + 63) / 64 * 64, op = (o + 7) / 8 * 8;
  const size_t planes = prec == RTTDA_BF16 ? 1 : 2, zplanes = prec == RTTDA_BF16X3 ? 2 : 1;
  size_t b = P * ov * fb + (o + v + 3 * (o * o + v * v + ov)) * 8;
  if (ozk)  // digits of B_oo and B_vv
    b += (P * o * op + P * v * vp) * 2 * oz::kS + (P * o + vp * P * ((vp + 511) / 512)) * 2;
  else
    b += tc ? (P * o * op + P * vp * vp + 2 * P * ov) * 2 * planes : (P * o * o + P * v * v) * fb;
  b += N * C * 8 * 6 + T * (o * o + v * v + ov) * (8 + cb);               // state, dipole blocks
  b += (size_t)32 * P * C * cb + (size_t)16 * ov * C * cb;                 // Coulomb partials
  const size_t zcap = (size_t)40 << 30;
  if (tc)
    b += std::min(zcap, C * o * vp * 2 * zplanes * P) + C * vp * op * 2 * planes + (size_t)kNumSM * C * o * v * 4;
  else if (ozk)
    b += std::min(zcap, C * o * vp * (8 + 2 * oz::kS) * P) + C * vp * op * 2 * oz::kS + (size_t)kNumSM * C * o * v * 8;
  else
    b += std::min((size_t)1 << 30, v * C * o * cb * P) + (size_t)4 * kNumSM * C * o * v * cb;
  b += (2 * N * T * 2 + 2 * T * (size_t)(nsteps + 1)) * 8;                 // host-call staging
  return b + b / 10 + ((size_t)64 << 20);
}
}  // namespace rttda
extern "C" {

rttda_status rttda_estimate_bytes(int nocc, int nvirt, int naux, int ntraj, int prec, long nsteps, size_t* bytes) {
  g_last_error.clear();
  if (!bytes || nocc < 1 || nvirt < 1 || naux < 1 || ntraj < 1 || nsteps < 0)
    return set_error(RTTDA_E_ARG, "rttda_estimate_bytes: bad arguments");
  *bytes = estimate_bytes(nocc, nvirt, naux, ntraj, prec, nsteps);
  return RTTDA_OK;
}

rttda_status rttda_spectrum(const double* trace, long ntraces, long npts, double dt, double kappa, double gamma,
                            double wmin, double wmax, long nfreq, double* omega_out, double* S_out) {
  g_last_error.clear();
  if (!trace || !S_out) return set_error(RTTDA_E_ARG, "rttda_spectrum: NULL argument");
  if (ntraces < 1 || npts < 2 || nfreq < 1) return set_error(RTTDA_E_ARG, "rttda_spectrum: bad sizes");
  if (!(dt > 0.0) || kappa == 0.0 || !(gamma >= 0.0) || !std::isfinite(kappa))
    return set_error(RTTDA_E_ARG, "rttda_spectrum: bad dt/kappa/gamma");
  if (nfreq > (1L << 30)) return set_error(RTTDA_E_ARG, "rttda_spectrum: nfreq too large");
  double *d_tr = nullptr, *d_S = nullptr, *d_w = nullptr;
  const size_t ntr = (size_t)ntraces * npts;
  auto cleanup = [&]() {
    dfree(d_tr);
    dfree(d_S);
    dfree(d_w);
  };
  rttda_status st = RTTDA_OK;
  if ((st = dalloc(&d_tr, ntr)) != RTTDA_OK || (st = dalloc(&d_S, nfreq)) != RTTDA_OK ||
      (st = dalloc(&d_w, nfreq)) != RTTDA_OK) {
    cleanup();
    return st;
  }
  cudaError_t e = cudaMemcpy(d_tr, trace, ntr * 8, cudaMemcpyHostToDevice);
  const double dw = nfreq > 1 ? (wmax - wmin) / (double)(nfreq - 1) : 0.0;
  if (e == cudaSuccess) {
    k_spectrum<<<(unsigned)nfreq, 256>>>(d_tr, ntraces, npts, dt, kappa, gamma, wmin, dw, d_w, d_S);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(S_out, d_S, nfreq * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && omega_out) e = cudaMemcpy(omega_out, d_w, nfreq * 8, cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) return set_error(RTTDA_E_CUDA, std::string("rttda_spectrum: ") + cudaGetErrorString(e));
  return RTTDA_OK;
}

rttda_status rttda_sync(rttda_t h, void* stream) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_sync: NULL handle");
  CK(cudaStreamSynchronize(stream ? (cudaStream_t)stream : h->stream));
  return check_device_error(h);
}

rttda_status rttda_profile(rttda_t h, int enable) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_profile: NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  h->prof_on = enable != 0;
  for (size_t& u : h->prof_used) u = 0;
  return RTTDA_OK;
}

rttda_status rttda_profile_read(rttda_t h, double* ms, long long* launches) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_profile_read: NULL handle");
  for (int c = 0; c < RTTDA_NUM_KERNEL_CLASSES; ++c) {
    double tot = 0.0;
    for (size_t k = 0; k + 1 < h->prof_used[c]; k += 2) {
      CK(cudaEventSynchronize(h->prof_ev[c][k + 1]));
      float x = 0.f;
      CK(cudaEventElapsedTime(&x, h->prof_ev[c][k], h->prof_ev[c][k + 1]));
      tot += x;
    }
    if (ms) ms[c] = tot;
    if (launches) launches[c] = (long long)(h->prof_used[c] / 2);
    h->prof_used[c] = 0;
  }
  return RTTDA_OK;
}

rttda_status rttda_launch_stats(rttda_t h, long long* total, long long* per_step) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_launch_stats: NULL handle");
  if (total) *total = h->launches;
  if (per_step) *per_step = h->launches_per_step;
  return RTTDA_OK;
}

rttda_status rttda_set_projectors(rttda_t h, int k, const double* X) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_set_projectors: NULL handle");
  if (k < 0 || k > 4096 || (k > 0 && !X)) return set_error(RTTDA_E_ARG, "rttda_set_projectors: need 0 <= k <= 4096 and X");
  dfree(h->d_proj);
  dfree(h->d_proj_part);
  dfree(h->d_ovl);
  h->d_proj = h->d_proj_part = h->d_ovl = nullptr;
  h->nproj = 0;
  h->ovl_cap = h->ovl_ld = h->part_cap = 0;
  if (k == 0) return RTTDA_OK;
  CKS(dalloc(&h->d_proj, (size_t)k * h->N));
  CK(cudaMemcpy(h->d_proj, X, sizeof(double) * (size_t)k * h->N, cudaMemcpyDefault));
  h->proj_rows = std::max<long long>(2048, cdiv(h->N, 2 * kNumSM));
  h->proj_G = (int)cdiv(h->N, h->proj_rows);
  h->nproj = k;
  return RTTDA_OK;
}

rttda_status rttda_get_overlaps(rttda_t h, double* out, long npts) {
  g_last_error.clear();
  if (!h || !out) return set_error(RTTDA_E_ARG, "rttda_get_overlaps: NULL argument");
  if (h->nproj < 1 || !h->d_ovl || h->ovl_ld < 1)
    return set_error(RTTDA_E_STATE, "rttda_get_overlaps: no projectors or no propagation since they were set");
  if (npts != h->ovl_ld) return set_error(RTTDA_E_ARG, "rttda_get_overlaps: npts must be nsteps + 1 of the last call");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out, h->d_ovl, sizeof(double) * (size_t)h->T * npts * h->nproj * 2, cudaMemcpyDefault));
  return RTTDA_OK;
}

rttda_status rttda_set_autocorrelation(rttda_t h, int enable) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_set_autocorrelation: NULL handle");
  h->acf_on = enable != 0;
  if (h->acf_on && h->nproj == 0) {
    h->proj_rows = std::max<long long>(2048, cdiv(h->N, 2 * kNumSM));
    h->proj_G = (int)cdiv(h->N, h->proj_rows);
  }
  h->acf_ld = 0;
  return RTTDA_OK;
}

rttda_status rttda_get_autocorrelation(rttda_t h, double* out, long npts) {
  g_last_error.clear();
  if (!h || !out) return set_error(RTTDA_E_ARG, "rttda_get_autocorrelation: NULL argument");
  if (!h->acf_on || !h->d_acf || h->acf_ld < 1)
    return set_error(RTTDA_E_STATE, "rttda_get_autocorrelation: not enabled, or no fresh propagation since");
  if (npts != h->acf_ld)
    return set_error(RTTDA_E_ARG, "rttda_get_autocorrelation: npts must be nsteps + 1 of the last call");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out, h->d_acf, sizeof(double) * (size_t)h->T * npts * 2, cudaMemcpyDefault));
  return RTTDA_OK;
}

rttda_status rttda_spectrum_autocorr(const double* R, long ntraces, long npts, double dt, long npad, long nfreq,
                                     int normalize, double* omega_out, double* S_out) {
  g_last_error.clear();
  if (!R || !S_out || ntraces < 1 || npts < 2 || nfreq < 1 || npad < 0 || !(dt > 0.0))
    return set_error(RTTDA_E_ARG, "rttda_spectrum_autocorr: bad arguments");
  double *d_R = nullptr, *d_w = nullptr, *d_S = nullptr;
  struct Free {
    double** p[3];
    ~Free() {
      for (auto q : p)
        if (*q) cudaFree(*q);
    }
  } fr{{&d_R, &d_w, &d_S}};
  CKS(dalloc(&d_R, (size_t)ntraces * npts * 2));
  CKS(dalloc(&d_w, (size_t)nfreq));
  CKS(dalloc(&d_S, (size_t)nfreq));
  CK(cudaMemcpy(d_R, R, sizeof(double) * (size_t)ntraces * npts * 2, cudaMemcpyDefault));
  k_spectrum_acf<<<(unsigned)nfreq, 256>>>(d_R, ntraces, npts, dt, npad, d_w, d_S);
  CK(cudaGetLastError());
  std::vector<double> S(nfreq);
  CK(cudaMemcpy(S.data(), d_S, sizeof(double) * nfreq, cudaMemcpyDeviceToHost));
  if (omega_out) CK(cudaMemcpy(omega_out, d_w, sizeof(double) * nfreq, cudaMemcpyDeviceToHost));
  if (normalize) {
    const double mx = *std::max_element(S.begin(), S.end());
    if (mx > 0.0)
      for (double& x : S) x /= mx;
  }
  std::memcpy(S_out, S.data(), sizeof(double) * nfreq);
  return RTTDA_OK;
}

rttda_status rttda_set_integrator(rttda_t h, int integrator) {
  g_last_error.clear();
  if (!h) return set_error(RTTDA_E_ARG, "rttda_set_integrator: NULL handle");
  if (integrator != RTTDA_INT_RK4 && integrator != RTTDA_INT_SSO)
    return set_error(RTTDA_E_ARG, "rttda_set_integrator: unknown integrator");
  h->integrator = integrator;
  return RTTDA_OK;
}

rttda_status rttda_plan(rttda_t h, rttda_plan_info* out) {
  g_last_error.clear();
  if (!h || !out) return set_error(RTTDA_E_ARG, "rttda_plan: NULL argument");
  if (h->T == 0) return set_error(RTTDA_E_STATE, "rttda_plan: no batch (call rttda_set_field first)");
  rttda_plan_info p = h->tc || h->oz ? h->plan : rttda_plan_info{};
  if (!h->tc && !h->oz) {
    p.main_bn = h->prec == RTTDA_FP64 ? Tile<double>::BN : Tile<float>::BN;
    p.main_mb = 1;
    p.main_kb = h->prec == RTTDA_FP64 ? Tile<double>::BK : Tile<float>::BK;
    p.main_splits = h->SK;
    p.z_chunk = h->zchunk;
  }
  p.prec = (int)h->prec;
  p.ntraj = h->T;
  p.coulomb_kernel = h->oz ? 2 : h->coul_tc ? 1 : 0;
  *out = p;
  return RTTDA_OK;
}

void rttda_destroy(rttda_t h) { delete h; }

}  // extern "C"
