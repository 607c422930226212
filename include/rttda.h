/*
 * rttda.h - C ABI of the B300-native RT-TDA propagation library.
 *
 * Real-time Tamm-Dancoff (RT-TDA) electron dynamics after Knoll & Levine,
 * "Simulating Electron Dynamics with GPU-Accelerated Real-Time Tamm-Dancoff
 * Approximation" (arXiv 2601.16949).  The library propagates complex
 * amplitudes c in the ground-plus-singles basis {|0>, |ia>} under
 *
 *     i dc/dt = H(t) c,   H(t) = A - E(t) M_d            (Eqs. (11), (16))
 *
 * with A_00 = 0, A_0,ia = 0 (Sec. 2.1, last paragraph) and, on the singles
 * block (structure of Eq. (3), two-electron part written in
 * three-index factorised form for this library),
 *
 *     A_ia,jb = d_ij d_ab (e_a - e_i) + 2 sum_P B^P_ia B^P_jb
 *                                     - c_x sum_P B^P_ij B^P_ab.
 *
 * M_d is the CSF-basis dipole matrix along the unit polarisation d, built
 * from MO-basis blocks by the Slater-Condon rules (Eqs. (19a)-(19f)):
 * M_0,ia = <0|mu_d|ia>, M_ia,ia = mu_aa - mu_ii, M_ia,ib = mu_ab,
 * M_ia,ja = -mu_ji, zero otherwise (the constant <Phi0|mu|Phi0> is dropped).
 *
 * Conventions for every entry point:
 *  - Atomic units throughout.
 *  - Amplitude vectors have n = 1 + nocc*nvirt complex entries; entry 0 is
 *    |0>, entry 1 + i*nvirt + a is |ia> ("virtuals run fastest", Sec. 2.1).
 *    Complex numbers are stored as interleaved (re, im) doubles.
 *    A batch of ntraj trajectories is stored trajectory-major:
 *    c[(t*n + k)*2 + {0,1}].
 *  - Host pointers are owned by the caller and only read/written during the
 *    call.  Device pointers (functions with _device in their name or
 *    documented as such) must be CUDA device memory of the current device.
 *  - Every function returns an rttda_status; no C++ exception crosses the
 *    ABI.  On failure rttda_last_error() returns a message for the calling
 *    thread.  RTTDA_E_CUDA means a CUDA call failed; the handle must then be
 *    destroyed.
 *  - A handle is not thread-safe: use one handle per host thread.
 *  - All computation runs in this library's CUDA kernels on the GPU; there
 *    is no CPU fallback.  Calls fail with RTTDA_E_CUDA if no device is usable.
 */
#ifndef RTTDA_H
#define RTTDA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTTDA_ABI_VERSION 2

typedef struct rttda_ctx* rttda_t;
typedef struct rttda_server* rttda_server_t;

typedef enum {
  RTTDA_OK = 0,
  RTTDA_E_ARG = 1,      /* invalid argument (checked before any GPU work) */
  RTTDA_E_OOM = 2,      /* device allocation failed / budget exceeded     */
  RTTDA_E_CUDA = 3,     /* a CUDA runtime or driver call failed           */
  RTTDA_E_TIMEOUT = 4,  /* a bounded device or host wait ran out          */
  RTTDA_E_STATE = 5,    /* call not valid in the handle's current state   */
  RTTDA_E_BUSY = 6      /* resource in use (server queue full, etc.)      */
} rttda_status;

/* Arithmetic used for the factor contractions (Coulomb, exchange, field).
 * The RK4 amplitude state, the norm and the dipole expectation are FP64 in
 * every mode.
 *   FP64:   all contractions in FP64 (CUDA cores).
 *   FP32:   factors and contractions in FP32 (CUDA cores).
 *   TF32:   not provided (RTTDA_E_ARG): on B300 TF32 runs at half the BF16
 *           tensor rate with 4-byte operands; BF16X2 is faster and more
 *           accurate.
 *   BF16:   exchange on tcgen05 tensor cores with BF16 factors and BF16
 *           activations, FP32 accumulation; Coulomb with BF16 factors and
 *           FP32 arithmetic; field in FP32.
 *   BF16X3: exchange on tcgen05 tensor cores with every operand split into
 *           BF16 hi + lo parts (x = hi + lo) and the products hi*hi + hi*lo +
 *           lo*hi accumulated in FP32 (about 16 significant bits per
 *           operand); Coulomb and field in FP32 on CUDA cores.
 *   BF16X2: as BF16X3 for the factors and for Z = B_oo c, but Z enters the
 *           main contraction as one BF16 plane: products Z*B_hi + Z*B_lo.
 *   FP64_OZ: FP64-accurate exchange on tcgen05 tensor cores by the Ozaki
 *           scheme (exponent-aligned slicing, Ozaki, Ogita, Oishi and Rump,
 *           Numer. Algorithms 59, 2012): in blocks of at most 512 K
 *           elements every operand row is written as 6 BF16 digits of 7
 *           bits under a common power of two, digit products are summed per
 *           weight without rounding in FP32 and joined in int64, and blocks
 *           are added in FP64.  Z = B_oo c is exact up to the digits' 42
 *           bits; relative error of the exchange about 2^-42 of the block
 *           scales.  The Coulomb passes w = B_ov c and B_ov^T (2w) run on
 *           the same digits; field in FP64 (CUDA cores).  Requires
 *           nocc <= 512 (RTTDA_E_ARG otherwise). */
typedef enum {
  RTTDA_FP64 = 0, RTTDA_FP32 = 1, RTTDA_TF32 = 2, RTTDA_BF16 = 3, RTTDA_BF16X3 = 4, RTTDA_BF16X2 = 5,
  RTTDA_FP64_OZ = 6
} rttda_prec;

/* Pulse shapes E(t) (Sec. 2.2, Eqs. (18a), (18b),
 * (18c), (18d)) plus a sin^2 envelope:
 *   KICK     : E0 delta(t); applied exactly as c(0+) = exp(+i E0 M_d) c(0)
 *              at the start of rttda_propagate, E = 0 afterwards.  Taylor
 *              series accumulated in FP64; its first-order term from FP64
 *              products in every precision, the higher terms from the field
 *              products of the precision (FP32 in FP32, BF16, BF16X2,
 *              BF16X3: about n 2^-24 x^2 / 2 for x = E0 ||M_d||_2, n = nocc
 *              + nvirt + 1).
 *   CW       : E0 sin(omega t)
 *   GAUSS_TL : E0 exp(-(t-t0)^2 / (2 s^2)) sin(omega (t-t0)), s = fwhm/2.35482
 *   CHIRP    : E0 exp(-(t-t0)^2 / (2 s^2)) sin((omega + beta (t-t0)/2)(t-t0))
 *   SIN2     : E0 sin^2(pi t / duration) sin(omega t) for 0 <= t <= duration,
 *              0 otherwise. */
typedef enum {
  RTTDA_KICK = 0, RTTDA_CW = 1, RTTDA_GAUSS_TL = 2, RTTDA_CHIRP = 3, RTTDA_SIN2 = 4
} rttda_pulse_kind;

typedef struct {
  int kind;          /* rttda_pulse_kind                                   */
  double E0;         /* field amplitude (kick strength kappa for KICK)     */
  double omega;      /* carrier frequency (Ha)                             */
  double t0;         /* pulse centre (GAUSS_TL, CHIRP)                     */
  double fwhm;       /* full width at half maximum of the envelope         */
  double beta;       /* chirp rate (CHIRP)                                 */
  double duration;   /* sin^2 window length (SIN2)                         */
  double dir[3];     /* polarisation d (normalised by the library)         */
} rttda_pulse;

/* ABI version of the loaded library (RTTDA_ABI_VERSION it was built with).
 * Library utility, no counterpart in the paper; cannot fail. */
int rttda_abi_version(void);

/* Message describing the last failure on the calling thread ("" if none).
 * Library utility, no counterpart in the paper; cannot fail.  The string is
 * owned by the library and valid until the thread's next call. */
const char* rttda_last_error(void);

/* Create a handle for one molecule and upload its factors.
 * Defines A (Eq. (3), factorised as above) and the dipole
 * blocks of the Slater-Condon rules (Eqs. (19b)-(19e)).
 *   nocc, nvirt, naux >= 1.
 *   eps_occ[nocc], eps_virt[nvirt]       orbital energies (Ha).
 *   B_ov[naux][nocc][nvirt]               B^P_ia.
 *   B_oo[naux][nocc][nocc]                B^P_ij, symmetric in ij.
 *   B_vv[naux][nvirt][nvirt]              B^P_ab, symmetric in ab.
 *   mu_oo[3][nocc][nocc], mu_vv[3][nvirt][nvirt]  MO dipole blocks (x,y,z),
 *                                         symmetric.
 *   mu_0ov[3][nocc][nvirt]                <0|mu_x|ia> (pass sqrt(2) <i|mu|a>
 *                                         for MO-basis input, Eq. (19b)).
 *   c_x                                   exchange scaling.
 *   prec                                  rttda_prec.
 * All arrays are host FP64 and are copied (and cast to the working
 * precision) before the call returns; symmetry is assumed, not checked.
 * Errors: RTTDA_E_ARG (null pointer, non-positive size, bad prec),
 * RTTDA_E_OOM, RTTDA_E_CUDA.  *out is NULL on failure. */
rttda_status rttda_create(int nocc, int nvirt, int naux,
                          const double* eps_occ, const double* eps_virt,
                          const double* B_ov, const double* B_oo, const double* B_vv,
                          const double* mu_oo, const double* mu_vv, const double* mu_0ov,
                          double c_x, int prec, rttda_t* out);

/* As rttda_create, but every array argument is device memory of the current
 * device (FP64, same layouts), e.g. factors produced on the GPU; they are
 * read during the call and may be freed when it returns.  Needed for
 * molecules whose FP64 factors do not fit in host memory.
 * Errors: as rttda_create. */
rttda_status rttda_create_device(int nocc, int nvirt, int naux,
                                 const double* eps_occ, const double* eps_virt,
                                 const double* B_ov, const double* B_oo, const double* B_vv,
                                 const double* mu_oo, const double* mu_vv, const double* mu_0ov,
                                 double c_x, int prec, rttda_t* out);

/* Device memory the handle holds right now, in bytes (library utility, no
 * counterpart in the paper).  Errors: RTTDA_E_ARG (NULL argument). */
rttda_status rttda_memory_bytes(rttda_t h, size_t* bytes);

/* Set the batch: one pulse per trajectory (Eq. (16), Eqs. (18)).
 * ntraj >= 1; pulses[ntraj] (host).  Builds mu_d = sum_x d_x mu_x per
 * trajectory on the device.  Discards any propagated state.
 * Errors: RTTDA_E_ARG (ntraj < 1, (1 + nocc*nvirt) * 2 * ntraj >= 2^31,
 * unknown kind, zero polarisation, non-positive fwhm/duration where used),
 * RTTDA_E_OOM, RTTDA_E_CUDA. */
rttda_status rttda_set_field(rttda_t h, const rttda_pulse* pulses, int ntraj);

/* Propagate every trajectory of the batch from t = 0.
 *   c0        host [ntraj][n][2] initial amplitudes, or NULL for |0> (the
 *             Kohn-Sham ground state, Sec. 2.2 "initial conditions").
 *   dt > 0, nsteps >= 0.
 *   Kick pulses are applied at t = 0+ first.  Then nsteps RK4 steps of
 *   dc/dt = -i H(t) c (stages at t, t+dt/2, t+dt/2, t+dt).
 *   c_out        host [ntraj][n][2] final amplitudes, or NULL.
 *   dipole_trace host [ntraj][nsteps+1]: Re c^dagger M_d c at t_k = k dt
 *                (k = 0 is after the kick), or NULL.
 *   norm_trace   host [ntraj][nsteps+1]: |c|^2 at t_k, or NULL.
 * The handle keeps the final state and time for rttda_resume/get_state.
 * Errors: RTTDA_E_STATE (no rttda_set_field yet), RTTDA_E_ARG, RTTDA_E_OOM,
 * RTTDA_E_CUDA.  Blocks until the results are in the host buffers. */
rttda_status rttda_propagate(rttda_t h, const double* c0, double dt, long nsteps,
                             double* c_out, double* dipole_trace, double* norm_trace);

/* As rttda_propagate, but every buffer is device memory and the work is
 * enqueued on `stream` (a cudaStream_t; NULL = the handle's own stream).
 * Returns after enqueueing; results are valid once the stream reaches them.
 * The buffers must stay allocated until then.  The steps run as one CUDA
 * graph per step, replayed; the handle keeps the executable graph between
 * calls and updates its parameters, so that calls on handles with their
 * own streams run concurrently (instantiating a graph allocates device
 * memory, which would order the call against every stream's work;
 * RTTDA_GRAPH_CACHE=0 instantiates per call). */
rttda_status rttda_propagate_device(rttda_t h, const double* c0_dev, double dt, long nsteps,
                                    double* c_out_dev, double* dipole_dev, double* norm_dev,
                                    void* stream);

/* Wait for the work enqueued on `stream` (NULL = the handle's stream) and
 * report device-side failures: RTTDA_E_TIMEOUT if a bounded wait inside a
 * tensor-core kernel ran out (the results of that call are invalid).
 * Library utility, no counterpart in the paper.
 * Errors: RTTDA_E_ARG (NULL handle), RTTDA_E_CUDA, RTTDA_E_TIMEOUT. */
rttda_status rttda_sync(rttda_t h, void* stream);

/* Continue from the handle's current state and time (no kick): the same
 * integration of Eq. (11) as rttda_propagate, from t_now.  Buffers as
 * in rttda_propagate; entry 0 of each trace is the current state.
 * Errors: those of rttda_propagate, and RTTDA_E_STATE if there is no state
 * (nothing propagated or set). */
rttda_status rttda_resume(rttda_t h, double dt, long nsteps,
                          double* c_out, double* dipole_trace, double* norm_trace);

/* Checkpoint: copy the current state [ntraj][n][2] and time to the host
 * (c host, written; t may be NULL).  Library feature, no counterpart in the
 * paper.  Errors: RTTDA_E_ARG (NULL h or c), RTTDA_E_STATE (no state),
 * RTTDA_E_CUDA. */
rttda_status rttda_get_state(rttda_t h, double* c, double* t);

/* Restore: set the current state [ntraj][n][2] (host, copied) and time t.
 * Library feature, no counterpart in the paper.  Errors: RTTDA_E_ARG (NULL,
 * t not finite), RTTDA_E_STATE (no rttda_set_field yet), RTTDA_E_CUDA. */
rttda_status rttda_set_state(rttda_t h, const double* c, double t);

/* One evaluation of sigma = H(t) c for the whole batch (Eq. (16) with
 * Eq. (17); the field term uses each trajectory's pulse at time t; a kick
 * contributes nothing for t > 0).  c_dev and sigma_dev are device
 * [ntraj][n][2]; enqueued on `stream` (NULL = handle stream).  The handle's
 * propagation state is not touched.
 * Errors: RTTDA_E_ARG (NULL, t not finite), RTTDA_E_STATE (no
 * rttda_set_field yet), RTTDA_E_CUDA. */
rttda_status rttda_sigma(rttda_t h, const double* c_dev, double t, double* sigma_dev, void* stream);

/* Absorption spectrum from dipole traces (dipole-trace analogue of
 * Eq. (21), averaged over traces as in Eq. (23)):
 *   S(w) = (1/ntraces) sum_tr (w/kappa) sum_k w_k (mu_k - mu_0)
 *          exp(-gamma t_k) sin(w t_k) dt,
 * trapezoid weights w_k (1/2 at both ends), t_k = k dt.
 *   trace     host [ntraces][npts]; npts >= 2; kappa != 0; gamma >= 0.
 *   omega_out host [nfreq] (may be NULL): w_j = wmin + j (wmax-wmin)/(nfreq-1).
 *   S_out     host [nfreq].
 * Computed on the GPU (FP64).  No handle needed.
 * Errors: RTTDA_E_ARG (NULL trace or S_out, ntraces < 1, npts < 2, nfreq < 1
 * or > 2^30, dt <= 0, kappa 0 or not finite, gamma < 0), RTTDA_E_OOM,
 * RTTDA_E_CUDA. */
rttda_status rttda_spectrum(const double* trace, long ntraces, long npts, double dt,
                            double kappa, double gamma, double wmin, double wmax,
                            long nfreq, double* omega_out, double* S_out);

/* Kernel classes reported by rttda_profile_read (one event pair per launch
 * group of the class).  EXCHANGE_MAIN is the long-K contraction
 * sum_{P,b} Z^P_ib B^P_ab; EXCHANGE_Z builds Z^P = B^P_oo c. */
enum {
  RTTDA_KC_FIELD = 0,          /* M_d c (Slater-Condon rules, Eqs. (19b)-(19e))   */
  RTTDA_KC_COULOMB = 1,        /* both Coulomb passes                         */
  RTTDA_KC_EXCHANGE_Z = 2,     /* Z^P = B^P_oo c                              */
  RTTDA_KC_EXCHANGE_MAIN = 3,  /* sum_{P,b} Z^P_ib B^P_ab                     */
  RTTDA_KC_COMBINE = 4,        /* sigma assembly + RK4 stage update           */
  RTTDA_KC_OBSERVE = 5,        /* dipole and norm reductions                  */
  RTTDA_KC_KICK = 6,           /* exp(+i kappa M_d) Taylor series             */
  RTTDA_NUM_KERNEL_CLASSES = 7
};

/* Tracing.  enable != 0: later propagations launch kernels directly (no CUDA
 * graph) with a CUDA event pair around every kernel-class launch; the
 * counters restart.  rttda_profile_read waits for the recorded events, writes
 * the summed milliseconds ms[RTTDA_NUM_KERNEL_CLASSES] and the number of
 * timed launches per class launches[...] (either may be NULL) and resets.
 * The per-class analogue of the paper's per-task wall-clock totals (Table
 * timings).  Errors: RTTDA_E_ARG (NULL handle), RTTDA_E_CUDA. */
rttda_status rttda_profile(rttda_t h, int enable);
rttda_status rttda_profile_read(rttda_t h, double* ms, long long* launches);

/* Kernels this handle has enqueued so far (*total) and in one RK4 step of
 * the last propagation (*per_step).  Either pointer may be NULL.  Library
 * utility, no counterpart in the paper.  Errors: RTTDA_E_ARG (NULL handle). */
rttda_status rttda_launch_stats(rttda_t h, long long* total, long long* per_step);

/* Lowest excited states of the TI-TDA problem A X_i = w_i X_i (Sec. 2.1,
 * Eq. (2); A without the field, in the handle's precision), for the
 * population projections of Eq. (22).  Davidson iteration on the
 * library's sigma build (up to 2*ntraj vectors per build, so a batch must be
 * set with rttda_set_field first), diagonal preconditioner e_a - e_i, stop
 * when every residual norm |A X_i - w_i X_i| < tol.
 *   k        number of states, 1 <= k <= nocc*nvirt;
 *   evals    host [k], ascending;
 *   evecs    host or device [k][1 + nocc*nvirt] FP64, unit norm, component 0
 *            (the ground state) = 0; may be NULL;
 *   iters    iterations used (may be NULL).
 * Errors: RTTDA_E_ARG, RTTDA_E_STATE (no batch; or not converged within
 * max_iter -- evals/evecs then hold the last estimates), RTTDA_E_OOM,
 * RTTDA_E_CUDA. */
rttda_status rttda_eigenstates(rttda_t h, int k, double tol, int max_iter, double* evals, double* evecs, int* iters);

/* Projectors for overlap and population recording (Eq. (22),
 * P_i(t) = |X_i^T c(t)|^2 with real state vectors X_i).  X: host or device
 * [k][1 + nocc*nvirt] FP64, copied.  Later propagations record, for every
 * trajectory t, step n = 0..nsteps and projector i, the complex overlap
 * o[t][n][i] = sum_m X_i[m] c_t[m](t_n).  k = 0 removes the projectors.
 * Errors: RTTDA_E_ARG (k < 0, k > 4096, NULL X), RTTDA_E_OOM. */
rttda_status rttda_set_projectors(rttda_t h, int k, const double* X);

/* Overlaps (Eq. (22)) of the last rttda_propagate / rttda_resume call:
 * out[ntraj][npts][k][2] (host or device; re, im), npts = nsteps + 1 of
 * that call.  Synchronises the handle.
 * Errors: RTTDA_E_ARG (NULL, npts mismatch), RTTDA_E_STATE (no projectors,
 * or no propagation since they were set). */
rttda_status rttda_get_overlaps(rttda_t h, double* out, long npts);

/* Autocorrelation recording (Eq. (20)):
 * R_t(t_n) = X_t^dagger(eps) X_t(eps + t_n), with eps right after the kick
 * (the state a fresh propagation starts from, kick applied).  enable != 0:
 * every fresh propagation stores its X(eps) and every propagation or resume
 * records R for its steps n = 0..nsteps; 0 turns it off.
 * Errors: RTTDA_E_ARG (NULL handle). */
rttda_status rttda_set_autocorrelation(rttda_t h, int enable);

/* R (Eq. (20)) of the last call: out[ntraj][npts][2] (host or device; re, im),
 * npts = nsteps + 1 of that call.  Synchronises the handle.
 * Errors: RTTDA_E_ARG (NULL, npts mismatch), RTTDA_E_STATE (off, or no
 * fresh propagation since it was enabled). */
rttda_status rttda_get_autocorrelation(rttda_t h, double* out, long npts);

/* The paper's spectrum from autocorrelation records (Sec. 3.1 with Eqs.
 * (20), (21), (23)): each
 * record R(t_j), t_j = j dt, j < npts, is mirrored (R(-t) = conj R(t), 2
 * npts - 1 points), multiplied by a Hann window peaked at t = 0, padded with
 * npad zeros, and transformed, F(w) = sum_m win_m R(t_m) e^{+i w t_m} dt; the
 * spectrum w Re F(w) is averaged over the ntraces records and evaluated on
 * the padded FFT grid w_k = 2 pi k / ((2 npts - 1 + npad) dt), k < nfreq
 * (by a direct sum on the GPU, which equals the FFT there).  normalize != 0
 * divides by the largest value of the nfreq outputs.
 *   R host or device [ntraces][npts][2]; omega_out host [nfreq] (may be
 *   NULL); S_out host [nfreq].  No handle needed.
 * Errors: RTTDA_E_ARG, RTTDA_E_OOM, RTTDA_E_CUDA. */
rttda_status rttda_spectrum_autocorr(const double* R, long ntraces, long npts, double dt, long npad, long nfreq,
                                     int normalize, double* omega_out, double* S_out);

/* Time integrator of later propagations (the state and time are kept).
 *   RTTDA_INT_RK4  classical 4-stage Runge-Kutta on dc/dt = -i H(t) c,
 *                  stages at t, t+dt/2, t+dt/2, t+dt (default; 4 sigma
 *                  builds per step);
 *   RTTDA_INT_SSO  second-order symplectic split operator on
 *                  dq/dt = H p, dp/dt = -H q with c = q + i p (Sec. 2.2,
 *                  Eq. (12); convergence Sec. 3.4):
 *                    p_{n+1/2} = p_n - dt/2 H(t_n) q_n,
 *                    q_{n+1} = q_n + dt H(t_n + dt/2) p_{n+1/2},
 *                    p_{n+1} = p_{n+1/2} - dt/2 H(t_n + dt) q_{n+1};
 *                  two sigma builds per step plus one per propagation call.
 * A kick is applied exactly before either integrator.  Stopping after n
 * steps and resuming reproduces an uninterrupted run bit for bit with both.
 * Errors: RTTDA_E_ARG (NULL handle, unknown integrator). */
typedef enum { RTTDA_INT_RK4 = 0, RTTDA_INT_SSO = 1 } rttda_integrator;
rttda_status rttda_set_integrator(rttda_t h, int integrator);

/* Execution plan of the sigma build chosen for the current batch (after
 * rttda_set_field; library introspection, no counterpart in the paper).  The exchange main contraction sum_{P,b} Z^P_ib B^P_ab
 * (Sec. 2.2, exchange part of the A matrix elements) runs on
 *   main_kernel 0: SIMT (FP64 / FP32),
 *               1: tcgen05, 128-row tiles (BF16X3),
 *               2: tcgen05, wide-M tiles of main_mb x 128 rows (BF16, BF16X2),
 *               3: tcgen05, Ozaki digit pairs on 128 x 64 tiles (FP64_OZ),
 *               4: tcgen05, wide tiles with the contraction transposed: rows a
 *                  (main_mb x 128), columns (trajectory column, i) (BF16,
 *                  BF16X2; the tuner's choice when faster),
 * with main_bn output columns per tile, K tiles of main_kb BF16 and
 * main_splits split-K partials; Z^P = B^P_oo c is built for z_chunk values
 * of P at a time.  coulomb_kernel 0: SIMT, 1: tcgen05, 2: tcgen05 Ozaki digits
 * (FP64_OZ).
 * tuned 0: heuristic plan (or RTTDA_TUNE=0), 1: timed now (tune_ms[k] is the
 * fastest of five launches of candidate k in milliseconds, ncand
 * candidates), 2: taken
 * from the tuning cache of this process or of the RTTDA_TUNE_CACHE file,
 * 3: named by the environment variable RTTDA_WIDE_PLAN="BN,MB,KB" or, for
 * main_kernel 4, "BN,2,32,t" (an unknown candidate there makes
 * rttda_set_field fail with RTTDA_E_ARG).
 * RTTDA_ZCHUNK=n caps z_chunk at n values of P (all precisions).
 * RTTDA_WIDE_CLUSTER=2 or 4 runs main_kernel 2 (BN 192, MB 2, KB 64) in
 * clusters of that many CTAs (main_cluster) when the columns allow it.
 * Errors: RTTDA_E_ARG (NULL), RTTDA_E_STATE (no batch yet). */
typedef struct {
  int prec, ntraj;
  int main_kernel, main_bn, main_mb, main_kb, main_splits;
  int z_chunk;
  int coulomb_kernel;
  int tuned, ncand;
  double tune_ms[8];
  int main_cluster;  /* main_kernel 2: CTAs per thread-block cluster that share each Z tile (TMA multicast), 1: none */
  int main_grid;     /* main_kernel 2: CTAs of the main contraction's launch */
} rttda_plan_info;
rttda_status rttda_plan(rttda_t h, rttda_plan_info* out);

/* Coulomb term of sigma without allocating any device memory.
 * The paper has no counterpart; this entry point exists for callers that
 * may not allocate GPU memory while they run (an application whose device
 * memory is owned by its own pool or arena, an allocator-free real-time
 * loop, a process with a fixed device-memory budget).
 *   sigma[t][0] = 0,
 *   sigma[t][1+ia] = 2 sum_jb (ia|jb) c[t][1+jb],  (ia|jb) = sum_P B^P_ia B^P_jb,
 * in FP64 for every trajectory t (complex, [ntraj][1+nocc*nvirt][2]).
 *   B_ov_dev  device [naux][nocc*nvirt] FP64, read only.
 *   c_dev     device [ntraj][n][2] FP64, read only.
 *   sigma_dev device [ntraj][n][2] FP64, written.
 *   stream    cudaStream_t to enqueue on (NULL = the legacy default stream).
 * Its only scratch is a fixed array of 2^20 doubles (8 MiB) inside the
 * library, held on every device that loads the library until the process
 * exits; naux*2*ntraj must not exceed 2^20, otherwise RTTDA_E_ARG is
 * returned before any GPU work.  The call makes no cudaMalloc/cudaFree and
 * uses no allocating library routine.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress), so make that first
 * call outside any stream capture.  All calls share the one array and each
 * call overwrites the part it reads before reading it; calls whose work may
 * overlap on the GPU (different streams, or several host threads) race on
 * it and must be serialised by the caller.  Returns after enqueueing.
 * The paper has no counterpart for this entry point.  Errors: RTTDA_E_ARG (a size < 1, NULL pointer,
 * naux*2*ntraj > 2^20, ntraj > 65535, device index above the library's
 * limit), RTTDA_E_CUDA. */
rttda_status rttda_coulomb_noalloc(int nocc, int nvirt, int naux, const double* B_ov_dev, const double* c_dev,
                                   int ntraj, double* sigma_dev, void* stream);

/* Failure-detection self-test.  Launches one kernel whose single thread
 * waits, with a wall-clock limit of limit_s seconds (1e-3 .. 2), for a device
 * flag that nothing sets; the kernel then records the expiry and returns, as
 * the tensor-core kernels do when one of their pipeline waits runs out.
 * Returns RTTDA_E_TIMEOUT when the wait ran out (the expected outcome); the
 * CUDA context stays usable.  The paper has no counterpart.
 * Errors: RTTDA_E_ARG (limit_s outside [1e-3, 2]), RTTDA_E_CUDA; and
 * RTTDA_E_TIMEOUT as above. */
rttda_status rttda_selftest_wait(double limit_s);

/* Free every resource of the handle (NULL is ignored); waits for the
 * handle's own stream first.  Work the caller enqueued on other streams
 * must be finished before.  Cannot fail. */
void rttda_destroy(rttda_t h);

#ifdef __cplusplus
}
#endif

#endif /* RTTDA_H */
