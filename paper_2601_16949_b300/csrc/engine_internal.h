// Shared declarations between the translation units of the library.
#pragma once
#include <string>

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/rttda.h"

namespace rttda {
// Per-thread message returned by rttda_last_error().
extern thread_local std::string g_last_error;
// Record msg as the calling thread's last error and return s.
rttda_status set_error(rttda_status s, const std::string& msg);

// Used by the serving scheduler.
// Advance a handle by nsteps on stream s: fresh = start from |0> (+ kick) at
// t = 0, otherwise continue from its state.  Observables go to
// dip/nrm[t * ld + offset + k], k = 0..nsteps.
rttda_status advance(rttda_t h, bool fresh, double dt, long nsteps, double* dip, double* nrm, long long ld,
                     long long offset, cudaStream_t s);
cudaStream_t handle_stream(rttda_t h);
// RTTDA_E_TIMEOUT if a bounded device wait of the handle ran out (synchronous).
rttda_status device_error(rttda_t h);
// Damped spectrum of device traces into device buffers, on stream s.
rttda_status spectrum_device(const double* trace_dev, long long ntr, long long npts, double dt, double kappa,
                             double gamma, double wmin, double wmax, long long nfreq, double* om_dev, double* S_dev,
                             cudaStream_t s);
size_t estimate_bytes(int nocc, int nvirt, int naux, int ntraj, int prec, long nsteps);

// The handle's batch as seen by the eigensolver: N rows, C = 2T real
// columns, orbital energies (device), the sigma input X and output buffers
// (device, [N][C] row-major).
struct BatchView {
  long long N = 0;
  int T = 0, nocc = 0, nvirt = 0;
  const double* eps_o = nullptr;
  const double* eps_v = nullptr;
  double* X = nullptr;
  double* out = nullptr;
  cudaStream_t stream = nullptr;
};
// RTTDA_E_STATE when no batch is set.
rttda_status batch_view(rttda_t h, BatchView* bv);
// out = A X for the batch buffers of batch_view (the field term excluded), on stream s.
rttda_status sigma_A(rttda_t h, cudaStream_t s);
}  // namespace rttda
