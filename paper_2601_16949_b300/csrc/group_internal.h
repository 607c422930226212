// The grouped serving step (group.cu) as seen by the server (server.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/rttda_server.h"
#include "device_common.cuh"

namespace rttda {
namespace grp {

// size limits of the grouped path (small molecules, launch-bound otherwise)
constexpr int kMaxO = 64, kMaxV = 256, kMaxP = 2048;
constexpr double kMaxWork = 3e8;  // nocc nvirt^2 naux of one request the grouped step takes at all
// routed to the grouped step by default (rttda_server_set_grouping mode 1):
// one request's nocc nvirt^2 naux at most this (measured: the grouped step
// wins for many requests of (16, 64, 256), 1.7e7 each, and on a trace of
// molecules up to (48, 192, 768) grouping requests up to 3e8 lost 5 % of
// the throughput to one handle per request)
constexpr double kAutoWork = 6e7;
// summed nocc nvirt^2 naux of the requests in the grouped step at once: the
// grouped kernel wins while the group's step is launch- or latency-bound
// (measured: 16 requests of (16, 64, 256), 2.7e8 in total, and one of
// (32, 128, 512), 2.7e8) and loses to one tcgen05 handle per request
// beyond (16 of (32, 128, 512), 4.3e9 in total)
constexpr double kMaxGroupWork = 4e8;

// one request of a group, as the kernel reads it (device pointers)
struct Req {
  int o, v, P, op, vp;  // op = o rounded up to 16, vp = v rounded up to 32
  int ov, N;            // nocc*nvirt, 1 + nocc*nvirt
  int S;                // split-K count of the exchange main contraction
  int field;            // 1: the pulse acts after t = 0 (every stage needs M_d X)
  int kick_terms;       // Taylor terms of the kick in this chunk (0: no kick now)
  int nsteps;           // RK4 steps in this chunk
  double kappa, cx, dt;
  PulseDev pulse;
  long long step0;      // global index of this chunk's first step
  long long trace_off;  // trace index of step0
  const double *eps_o, *eps_v;
  const __nv_bfloat16* Bov;  // [P][ov]
  const __nv_bfloat16* Boo;  // [P][o][op]
  const __nv_bfloat16* Bvv;  // [P][vp][vp] (symmetric; padding zero)
  const double *moo64, *mvv64, *m064;  // direction-combined dipole blocks
  const float *mooF, *mvvF, *m0F;
  double *Xn, *Xs, *Xs2, *acc, *F, *term;  // [N][2] FP64
  __nv_bfloat16* Xt;  // [2][vp][op]: BF16 copy of the stage input, X^T per column
  __nv_bfloat16* Z;   // [P][2 o][vp]: exchange intermediate, rows (col, i)
  float* w;           // [P][2]
  float* J;           // [ov][2]
  float* Kp;          // [S][2 o][v]
  double *dip, *nrm;  // traces of the whole request
};

struct Barrier {
  unsigned count, gen;
  int err;  // 1: a barrier wait ran out
};

constexpr int kMaxGroup = 64;

struct Table {
  int nreq, max_steps, kick_terms;
  Barrier* bar;
  unsigned long long* phase_ns;  // optional: %globaltimer after every barrier (CTA 0), else NULL
  Req req[kMaxGroup];
};

}  // namespace grp

// Host-side state of one grouped request.
struct GroupReq {
  grp::Req r{};
  int kick_terms = 0;     // Taylor terms of its kick (applied in its first chunk)
  double* trace = nullptr;
  std::vector<void*> allocs;
};

// Group state of a server: table buffers, barrier, stream.
struct GroupRunner {
  cudaStream_t stream = nullptr;
  cudaStream_t upload = nullptr;  // admissions: never waits for a running chunk
  grp::Table* d_table = nullptr;
  grp::Table* h_table = nullptr;  // pinned
  grp::Barrier* d_bar = nullptr;
  int grid = 0;  // largest co-resident grid (SMs x CTAs per SM)
  int nsm = 0;
  cudaEvent_t ev = nullptr;
  unsigned long long* phase_ns = nullptr;  // device clock of every barrier of the last chunk, or NULL
  const char* phase_file = nullptr;        // diagnostics: where group_status appends those clocks
};

bool group_eligible(const rttda_request& q);  // within the grouped kernel's limits
double group_work(const rttda_request& q);  // nocc nvirt^2 naux
size_t group_estimate_bytes(const rttda_request& q);
// Allocate a grouped request's device state and upload its molecule (the
// arrays of q, host or device memory, are copied before return).
rttda_status group_admit(const rttda_request& q, cudaStream_t s, GroupReq** out);
void group_release(GroupReq* g, cudaStream_t s);
rttda_status group_runner_init(GroupRunner* g);
void group_runner_free(GroupRunner* g);
// Enqueue one chunk for the given requests: nsteps[k] steps each (>= 0),
// starting at step done[k]; fresh[k] applies the request's kick first.
rttda_status group_launch(GroupRunner* g, const std::vector<GroupReq*>& reqs, const std::vector<long>& nsteps,
                          const std::vector<long>& done, const std::vector<int>& fresh);
// After the chunk's event: RTTDA_E_TIMEOUT when a barrier wait ran out.
rttda_status group_status(GroupRunner* g);

}  // namespace rttda
