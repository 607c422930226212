/*
 * rttda_server.h - continuous-batching RT-TDA propagation server.
 *
 * Serving pattern for the RT-TDA hot path (real-time TDA propagation,
 * arXiv 2601.16949, Sec. 2.2 "Propagation Algorithm", followed by the
 * spectrum of Eq. (21) on the dipole trace): many independent
 * propagation requests, each with its own molecule (nocc, nvirt, naux), pulse
 * and length, arrive over time.  A scheduler thread admits a request when
 * its device-memory footprint fits the budget and an active slot is free,
 * keeps its factors and amplitudes resident on the GPU, and advances every
 * active request in chunks of RK4 steps on its own CUDA stream, so the work
 * of different requests overlaps on the device.  Small requests in the BF16
 * precision (see rttda_server_set_grouping) are instead stepped together:
 * one persistent kernel per chunk advances every such active request at
 * once.  A finished request's
 * dipole trace is turned into a spectrum on the GPU; its memory is then
 * released and the next request is admitted.
 *
 * Handles of admitted requests are created on a second server thread, so
 * the scheduler keeps stepping the other requests meanwhile.
 *
 * Conventions are those of rttda.h.  All functions are thread-safe.  The
 * server captures CUDA graphs on its own threads: while it runs, other
 * threads of the process should synchronise their own streams, not the
 * whole device.  A device-wide synchronisation during a capture fails in the
 * calling thread (cudaErrorStreamCaptureUnsupported); the server runs the
 * chunk whose capture it invalidated as direct launches, with the same
 * results.
 */
#ifndef RTTDA_SERVER_H
#define RTTDA_SERVER_H

#include <stddef.h>

#include "rttda.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One propagation request: molecule (as in rttda_create), one pulse, the
 * time grid and the spectrum wanted.  Host arrays are copied by
 * rttda_server_submit and may be freed when it returns.  The spectrum is
 *   S(w_j) = (w_j / E0) sum_k wt_k (mu_k - mu_0) exp(-gamma t_k) sin(w_j t_k) dt
 * over the request's dipole trace (rttda_spectrum with kappa = pulse.E0). */
typedef struct {
  int nocc, nvirt, naux;
  const double *eps_occ, *eps_virt, *B_ov, *B_oo, *B_vv, *mu_oo, *mu_vv, *mu_0ov;
  double c_x;
  int prec;            /* rttda_prec */
  rttda_pulse pulse;
  double dt;           /* > 0 */
  long nsteps;         /* >= 1 */
  double gamma, wmin, wmax;
  long nfreq;          /* >= 1 */
  int factors_on_device;  /* 0: the eight arrays are host memory, copied by
                             rttda_server_submit.  1: they are device memory of
                             the server's GPU (e.g. factors drawn there), not
                             copied; they must stay valid until the request
                             leaves RTTDA_REQ_PENDING (rttda_server_poll
                             reports any other state), and may be freed then. */
} rttda_request;

typedef enum {
  RTTDA_REQ_PENDING = 0,
  RTTDA_REQ_ACTIVE = 1,
  RTTDA_REQ_DONE = 2,
  RTTDA_REQ_FAILED = 3,
  RTTDA_REQ_CANCELLED = 4
} rttda_request_state;

typedef struct {
  long submitted, completed, failed, cancelled, pending, active;
  int max_concurrent;          /* largest number of requests active at once */
  double trajectory_steps;     /* RK4 steps completed, summed over requests  */
  double p50_latency_s;        /* time to spectrum: submit -> spectrum ready */
  double p99_latency_s;
  double mean_latency_s;
  double busy_seconds;         /* first submit -> last completion            */
  size_t bytes_in_use, bytes_budget;
  long grouped;                /* requests admitted to the grouped step      */
} rttda_server_stats;

/* Start a server on the current CUDA device.
 *   hbm_budget   device bytes the server may hold for admitted requests
 *                (their estimated footprints, rttda_estimate_bytes);
 *   max_active   most requests on the GPU at once (>= 1);
 *   chunk_steps  RK4 steps per scheduling chunk (>= 1).
 * Errors: RTTDA_E_ARG, RTTDA_E_CUDA (no usable device). */
rttda_status rttda_server_create(size_t hbm_budget, int max_active, long chunk_steps, rttda_server_t* out);

/* Queue a request; *id receives its identifier.
 * Errors: RTTDA_E_ARG (NULL argument; invalid fields: sizes, NULL arrays,
 * pulse kind, dt, nsteps, nfreq, the spectrum window, E0 = 0). */
rttda_status rttda_server_submit(rttda_server_t s, const rttda_request* req, long* id);

/* Non-blocking status.  *state gets an rttda_request_state.  When the
 * request is DONE and the pointers are not NULL: spectrum[nfreq],
 * omega[nfreq], dipole[nsteps+1] receive its results and *latency_s its
 * time to spectrum.  A FAILED request's reason is in rttda_last_error().
 * Errors: RTTDA_E_ARG (NULL s or state, unknown id). */
rttda_status rttda_server_poll(rttda_server_t s, long id, int* state, double* spectrum, double* omega,
                               double* dipole, double* latency_s);

/* Block until the request leaves PENDING/ACTIVE or timeout_s elapses
 * (RTTDA_E_TIMEOUT; the request keeps running).
 * Errors: RTTDA_E_ARG (NULL s, timeout_s < 0, unknown id), RTTDA_E_TIMEOUT. */
rttda_status rttda_server_wait(rttda_server_t s, long id, double timeout_s);

/* Cancel a pending or active request (an active one stops after its chunk
 * in flight and releases its memory).
 * Errors: RTTDA_E_ARG (NULL s, unknown id). */
rttda_status rttda_server_cancel(rttda_server_t s, long id);

/* Grouped stepping of small BF16 requests.  A grouped request is advanced,
 * chunk by chunk, by one persistent cooperative kernel that steps all such
 * active requests together (about forty launches per RK4 step of each
 * request become one launch per chunk of the group); its grid takes a share
 * of the SMs in proportion to the group's work, so requests on their own
 * handles keep running beside it.  The kernel takes requests with prec =
 * RTTDA_BF16, nocc <= 64, nvirt <= 256, naux <= 2048 and nocc * nvirt^2 *
 * naux <= 3e8.  Modes (`enable`):
 *   0  no grouping: every request gets its own handle;
 *   1  (default) by work: such a request is grouped when its nocc nvirt^2
 *      naux is at most 6e7 and the summed nocc nvirt^2 naux of the grouped
 *      requests stays at most 4e8 (the regime where the grouped step was
 *      measured faster than one handle per request); the others get handles;
 *   2  every request within the kernel's limits is grouped.
 * Numerics are those of the BF16 path (BF16 factors and contraction inputs,
 * FP32 accumulation on the warp-level tensor-core instructions, FP64 state,
 * FP64-accurate dipole expectation); a request's results are bitwise the
 * same whichever requests share its group and whatever the grid, but not
 * bitwise equal to a plain rttda_propagate in the BF16 precision, whose
 * contractions sum in another order.  Applies to requests admitted
 * afterwards.  The serving pattern of the workload (Sec. 2.2 propagation
 * served as continuous batching) has no counterpart in the paper.
 * Errors: RTTDA_E_ARG (NULL s, mode not 0, 1 or 2). */
rttda_status rttda_server_set_grouping(rttda_server_t s, int enable);

/* Counters and latency percentiles of the requests so far (the serving
 * metrics: p50/p99 time to spectrum, trajectory-steps).
 * Errors: RTTDA_E_ARG (NULL argument). */
rttda_status rttda_server_stats_get(rttda_server_t s, rttda_server_stats* st);

/* Device bytes a handle with this shape and precision needs for ntraj
 * trajectories and nsteps-long host traces (upper estimate; host arithmetic,
 * no GPU work).  Errors: RTTDA_E_ARG (NULL bytes, a size < 1, nsteps < 0). */
rttda_status rttda_estimate_bytes(int nocc, int nvirt, int naux, int ntraj, int prec, long nsteps, size_t* bytes);

/* Stop the scheduler (active requests are cancelled) and free everything
 * (NULL is ignored).  Cannot fail. */
void rttda_server_destroy(rttda_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* RTTDA_SERVER_H */
