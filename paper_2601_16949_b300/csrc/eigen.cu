// Lowest eigenpairs of A (TI-TDA states, Sec. 2.1 Eq. (2)) by the
// Davidson method on the library's own sigma build, for population
// projections (Eq. (22)).
//
// A is real symmetric; its ground row and column are zero (A_00 = 0,
// A_0,ia = 0), so the excited states live in the singles block and every
// vector here keeps component 0 at zero.  One sigma build multiplies up to
// C = 2T vectors at once (the batch's real columns: A is real, so the real
// and imaginary columns of a trajectory are two independent vectors).
//
// Davidson (E. R. Davidson, J. Comput. Phys. 17, 87 (1975)): keep a basis V
// (orthonormal) and W = A V; diagonalise S = V^T W; for the k lowest Ritz
// pairs (theta_j, y_j) form residuals r_j = W y_j - theta_j V y_j; stop when
// every |r_j| < tol; otherwise add the preconditioned corrections
// t_j = r_j / (theta_j - D) with D the orbital-energy differences
// e_a - e_i, orthogonalised against V (classical Gram-Schmidt, twice) and
// normalised.  When the basis is full it is collapsed to the current Ritz
// vectors.  The small dense eigenproblem is solved on the host by the cyclic
// Jacobi method; the long vectors stay on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/rttda.h"
#include "engine_internal.h"

using rttda::set_error;

namespace {

#define EG_CK(x)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess) return set_error(RTTDA_E_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

#define EG_CKS(x)                   \
  do {                              \
    rttda_status s_ = (x);          \
    if (s_ != RTTDA_OK) return s_;  \
  } while (0)

inline unsigned nblk(long long n, int b) { return (unsigned)std::max<long long>(1, (n + b - 1) / b); }

// out[a * nb + b] = A_a . B_b (A_a = A + a * N), fixed-order block reduction
__global__ void __launch_bounds__(256) k_dots(long long N, const double* __restrict__ A, const double* __restrict__ B,
                                              int nb, double* __restrict__ out) {
  __shared__ double red[8];
  const int a = blockIdx.x, b = blockIdx.y;
  const double* x = A + (size_t)a * N;
  const double* y = B + (size_t)b * N;
  double s = 0.0;
  for (long long n = threadIdx.x; n < N; n += blockDim.x) s = fma(x[n], y[n], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[(size_t)a * nb + b] = t;
  }
}

// out_j = beta * out_j + sum_a cx[a * nout + j] X_a + sum_a cy[a * nout + j] Y_a
__global__ void __launch_bounds__(256) k_lincomb(long long N, int m, int nout, const double* __restrict__ X,
                                                 const double* __restrict__ cx, const double* __restrict__ Y,
                                                 const double* __restrict__ cy, double beta, double* __restrict__ out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (n >= N) return;
  double s = beta == 0.0 ? 0.0 : beta * out[(size_t)j * N + n];
  for (int a = 0; a < m; ++a) {
    s = fma(cx[(size_t)a * nout + j], X[(size_t)a * N + n], s);
    if (Y) s = fma(cy[(size_t)a * nout + j], Y[(size_t)a * N + n], s);
  }
  out[(size_t)j * N + n] = s;
}

// t_j[n] = r_j[n] / (theta_j - D[n]) (n >= 1), 0 for n = 0; a denominator
// smaller than 1e-6 in magnitude is replaced by +-1e-6
__global__ void __launch_bounds__(256) k_precond(long long N, const double* __restrict__ R,
                                                 const double* __restrict__ theta, const double* __restrict__ D,
                                                 double* __restrict__ Tv) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (n >= N) return;
  double d = theta[j] - D[n];
  if (fabs(d) < 1e-6) d = d < 0.0 ? -1e-6 : 1e-6;
  Tv[(size_t)j * N + n] = n == 0 ? 0.0 : R[(size_t)j * N + n] / d;
}

__global__ void __launch_bounds__(256) k_scale(long long N, const double* __restrict__ s, double* __restrict__ V) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (n < N) V[(size_t)j * N + n] *= s[j];
}

// X[n * C + c] = V_c[n] for c < nb, 0 otherwise
__global__ void __launch_bounds__(256) k_pack_cols(long long N, int C, int nb, const double* __restrict__ V,
                                                   double* __restrict__ X) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * C) return;
  const long long n = e / C;
  const int c = (int)(e % C);
  X[e] = c < nb ? V[(size_t)c * N + n] : 0.0;
}

__global__ void __launch_bounds__(256) k_unpack_cols(long long N, int C, int nb, const double* __restrict__ X,
                                                     double* __restrict__ W) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nb) return;
  const int c = (int)(e / N);
  const long long n = e % N;
  W[e] = X[(size_t)n * C + c];
}

// Cyclic Jacobi eigen-decomposition of a symmetric m x m matrix (row-major
// a, destroyed): eigenvalues ascending in w, eigenvectors as columns of z.
void jacobi_eigen(int m, std::vector<double>& a, std::vector<double>& w, std::vector<double>& z) {
  z.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) z[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double x = a[(size_t)i * m + j] * a[(size_t)i * m + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
          a[(size_t)k * m + p] = c * akp - s * akq;
          a[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
          a[(size_t)p * m + k] = c * apk - s * aqk;
          a[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double zkp = z[(size_t)k * m + p], zkq = z[(size_t)k * m + q];
          z[(size_t)k * m + p] = c * zkp - s * zkq;
          z[(size_t)k * m + q] = s * zkp + c * zkq;
        }
      }
  }
  std::vector<int> ord(m);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return a[(size_t)x * m + x] < a[(size_t)y * m + y]; });
  w.resize(m);
  std::vector<double> zs((size_t)m * m);
  for (int c = 0; c < m; ++c) {
    w[c] = a[(size_t)ord[c] * m + ord[c]];
    for (int r = 0; r < m; ++r) zs[(size_t)r * m + c] = z[(size_t)r * m + ord[c]];
  }
  z.swap(zs);
}

struct DevBuf {
  double* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" rttda_status rttda_eigenstates(rttda_t h, int k, double tol, int max_iter, double* evals,
                                          double* evecs, int* iters) {
  rttda::g_last_error.clear();
  if (!h || !evals) return set_error(RTTDA_E_ARG, "rttda_eigenstates: NULL argument");
  rttda::BatchView bv;
  EG_CKS(rttda::batch_view(h, &bv));
  const long long N = bv.N;
  const int C = 2 * bv.T;
  if (k < 1 || k > N - 1) return set_error(RTTDA_E_ARG, "rttda_eigenstates: need 1 <= k <= nocc*nvirt");
  if (!(tol > 0.0) || max_iter < 1) return set_error(RTTDA_E_ARG, "rttda_eigenstates: need tol > 0, max_iter >= 1");
  cudaStream_t s = bv.stream;
  const int mmax = (int)std::min<long long>(N - 1, std::max(3 * k, k + 2 * C + 8));

  // D = e_a - e_i (preconditioner and initial guesses)
  std::vector<double> eo(bv.nocc), ev(bv.nvirt);
  EG_CK(cudaMemcpy(eo.data(), bv.eps_o, sizeof(double) * bv.nocc, cudaMemcpyDeviceToHost));
  EG_CK(cudaMemcpy(ev.data(), bv.eps_v, sizeof(double) * bv.nvirt, cudaMemcpyDeviceToHost));
  std::vector<double> D((size_t)N, 0.0);
  for (int i = 0; i < bv.nocc; ++i)
    for (int a = 0; a < bv.nvirt; ++a) D[1 + (size_t)i * bv.nvirt + a] = ev[a] - eo[i];
  std::vector<long long> idx(N - 1);
  std::iota(idx.begin(), idx.end(), 1LL);
  std::stable_sort(idx.begin(), idx.end(), [&](long long x, long long y) { return D[x] < D[y]; });

  DevBuf dV, dW, dT, dR, dD, dc1, dc2, dS;
  EG_CK(cudaMalloc(&dV.p, sizeof(double) * (size_t)mmax * N));
  EG_CK(cudaMalloc(&dW.p, sizeof(double) * (size_t)mmax * N));
  EG_CK(cudaMalloc(&dT.p, sizeof(double) * (size_t)std::max(k, mmax) * N));
  EG_CK(cudaMalloc(&dR.p, sizeof(double) * (size_t)k * N));
  EG_CK(cudaMalloc(&dD.p, sizeof(double) * (size_t)N));
  EG_CK(cudaMalloc(&dc1.p, sizeof(double) * (size_t)mmax * std::max(k, mmax)));
  EG_CK(cudaMalloc(&dc2.p, sizeof(double) * (size_t)mmax * std::max(k, mmax)));
  EG_CK(cudaMalloc(&dS.p, sizeof(double) * (size_t)mmax * mmax));
  EG_CK(cudaMemcpyAsync(dD.p, D.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));

  // initial basis: unit vectors on the k smallest orbital-energy gaps
  EG_CK(cudaMemsetAsync(dV.p, 0, sizeof(double) * (size_t)k * N, s));
  const double one = 1.0;
  for (int j = 0; j < k; ++j)
    EG_CK(cudaMemcpyAsync(dV.p + (size_t)j * N + idx[j], &one, sizeof(double), cudaMemcpyHostToDevice, s));
  EG_CK(cudaStreamSynchronize(s));

  int m = 0, nnew = k, it = 0;
  std::vector<double> S((size_t)mmax * mmax, 0.0), theta, Y, Sw;
  std::vector<double> h1, h2;
  bool converged = false;
  for (it = 1; it <= max_iter; ++it) {
    // W = A V for the new vectors, C at a time
    for (int b0 = 0; b0 < nnew; b0 += C) {
      const int nb = std::min(C, nnew - b0);
      k_pack_cols<<<nblk(N * C, 256), 256, 0, s>>>(N, C, nb, dV.p + (size_t)(m + b0) * N, bv.X);
      EG_CKS(rttda::sigma_A(h, s));
      k_unpack_cols<<<nblk(N * nb, 256), 256, 0, s>>>(N, C, nb, bv.out, dW.p + (size_t)(m + b0) * N);
    }
    // S[:, new] = V^T W_new (and its transpose)
    const int mt = m + nnew;
    k_dots<<<dim3(mt, nnew), 256, 0, s>>>(N, dV.p, dW.p + (size_t)m * N, nnew, dS.p);
    h1.resize((size_t)mt * nnew);
    EG_CK(cudaMemcpyAsync(h1.data(), dS.p, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, s));
    EG_CK(cudaStreamSynchronize(s));
    for (int a = 0; a < mt; ++a)
      for (int b = 0; b < nnew; ++b) {
        S[(size_t)a * mmax + m + b] = h1[(size_t)a * nnew + b];
        S[(size_t)(m + b) * mmax + a] = h1[(size_t)a * nnew + b];
      }
    m = mt;
    // symmetrised copy of the m x m block, diagonalised on the host
    Sw.assign((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b)
        Sw[(size_t)a * m + b] = 0.5 * (S[(size_t)a * mmax + b] + S[(size_t)b * mmax + a]);
    jacobi_eigen(m, Sw, theta, Y);
    // residuals of the k lowest Ritz pairs: R_j = W y_j - theta_j V y_j
    h1.assign((size_t)m * k, 0.0);
    h2.assign((size_t)m * k, 0.0);
    for (int a = 0; a < m; ++a)
      for (int j = 0; j < k; ++j) {
        h1[(size_t)a * k + j] = Y[(size_t)a * m + j];
        h2[(size_t)a * k + j] = -theta[j] * Y[(size_t)a * m + j];
      }
    EG_CK(cudaMemcpyAsync(dc1.p, h1.data(), sizeof(double) * h1.size(), cudaMemcpyHostToDevice, s));
    EG_CK(cudaMemcpyAsync(dc2.p, h2.data(), sizeof(double) * h2.size(), cudaMemcpyHostToDevice, s));
    k_lincomb<<<dim3(nblk(N, 256), k), 256, 0, s>>>(N, m, k, dW.p, dc1.p, dV.p, dc2.p, 0.0, dR.p);
    k_dots<<<dim3(k, k), 256, 0, s>>>(N, dR.p, dR.p, k, dS.p);
    std::vector<double> rr((size_t)k * k);
    EG_CK(cudaMemcpyAsync(rr.data(), dS.p, sizeof(double) * rr.size(), cudaMemcpyDeviceToHost, s));
    EG_CK(cudaStreamSynchronize(s));
    std::vector<int> open;
    for (int j = 0; j < k; ++j)
      if (std::sqrt(std::max(0.0, rr[(size_t)j * k + j])) >= tol) open.push_back(j);
    if (open.empty()) {
      converged = true;
      break;
    }
    if (it == max_iter) break;
    // corrections for the unconverged pairs (compacted to the front of dR)
    const int nu = (int)open.size();
    std::vector<double> th(nu);
    for (int q = 0; q < nu; ++q) {
      th[q] = theta[open[q]];
      if (open[q] != q)
        EG_CK(cudaMemcpyAsync(dR.p + (size_t)q * N, dR.p + (size_t)open[q] * N, sizeof(double) * N,
                              cudaMemcpyDeviceToDevice, s));
    }
    EG_CK(cudaMemcpyAsync(dc1.p, th.data(), sizeof(double) * nu, cudaMemcpyHostToDevice, s));
    k_precond<<<dim3(nblk(N, 256), nu), 256, 0, s>>>(N, dR.p, dc1.p, dD.p, dT.p);
    // collapse when the new vectors do not fit
    if (m + nu > mmax) {
      const int keep = std::max(k, mmax - 2 * nu - C);
      h1.assign((size_t)m * keep, 0.0);
      for (int a = 0; a < m; ++a)
        for (int j = 0; j < keep; ++j) h1[(size_t)a * keep + j] = Y[(size_t)a * m + j];
      EG_CK(cudaMemcpyAsync(dc2.p, h1.data(), sizeof(double) * h1.size(), cudaMemcpyHostToDevice, s));
      // new V, W built in dR-independent scratch: reuse dT's tail is unsafe, so go through dW/dV in two steps
      DevBuf tmp;
      EG_CK(cudaMalloc(&tmp.p, sizeof(double) * (size_t)keep * N));
      k_lincomb<<<dim3(nblk(N, 256), keep), 256, 0, s>>>(N, m, keep, dV.p, dc2.p, nullptr, nullptr, 0.0, tmp.p);
      EG_CK(cudaMemcpyAsync(dV.p, tmp.p, sizeof(double) * (size_t)keep * N, cudaMemcpyDeviceToDevice, s));
      k_lincomb<<<dim3(nblk(N, 256), keep), 256, 0, s>>>(N, m, keep, dW.p, dc2.p, nullptr, nullptr, 0.0, tmp.p);
      EG_CK(cudaMemcpyAsync(dW.p, tmp.p, sizeof(double) * (size_t)keep * N, cudaMemcpyDeviceToDevice, s));
      EG_CK(cudaStreamSynchronize(s));
      std::fill(S.begin(), S.end(), 0.0);
      for (int j = 0; j < keep; ++j) S[(size_t)j * mmax + j] = theta[j];
      m = keep;
    }
    // orthogonalise the corrections against V (twice) and among themselves
    for (int pass = 0; pass < 2; ++pass) {
      k_dots<<<dim3(m, nu), 256, 0, s>>>(N, dV.p, dT.p, nu, dc1.p);
      h1.resize((size_t)m * nu);
      EG_CK(cudaMemcpyAsync(h1.data(), dc1.p, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, s));
      EG_CK(cudaStreamSynchronize(s));
      for (double& x : h1) x = -x;
      EG_CK(cudaMemcpyAsync(dc1.p, h1.data(), sizeof(double) * h1.size(), cudaMemcpyHostToDevice, s));
      k_lincomb<<<dim3(nblk(N, 256), nu), 256, 0, s>>>(N, m, nu, dV.p, dc1.p, nullptr, nullptr, 1.0, dT.p);
    }
    int added = 0;
    for (int q = 0; q < nu; ++q) {
      double* tq = dT.p + (size_t)q * N;
      // against the vectors added in this iteration, then normalise
      for (int pass = 0; pass < 2; ++pass) {
        if (added > 0) {
          k_dots<<<dim3(added, 1), 256, 0, s>>>(N, dV.p + (size_t)m * N, tq, 1, dc1.p);
          h1.resize(added);
          EG_CK(cudaMemcpyAsync(h1.data(), dc1.p, sizeof(double) * added, cudaMemcpyDeviceToHost, s));
          EG_CK(cudaStreamSynchronize(s));
          for (double& x : h1) x = -x;
          EG_CK(cudaMemcpyAsync(dc1.p, h1.data(), sizeof(double) * added, cudaMemcpyHostToDevice, s));
          k_lincomb<<<dim3(nblk(N, 256), 1), 256, 0, s>>>(N, added, 1, dV.p + (size_t)m * N, dc1.p, nullptr,
                                                          nullptr, 1.0, tq);
        }
      }
      k_dots<<<dim3(1, 1), 256, 0, s>>>(N, tq, tq, 1, dc1.p);
      double nn = 0.0;
      EG_CK(cudaMemcpyAsync(&nn, dc1.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      EG_CK(cudaStreamSynchronize(s));
      if (!(nn > 1e-20)) continue;
      const double sc = 1.0 / std::sqrt(nn);
      EG_CK(cudaMemcpyAsync(dc2.p, &sc, sizeof(double), cudaMemcpyHostToDevice, s));
      k_scale<<<dim3(nblk(N, 256), 1), 256, 0, s>>>(N, dc2.p, tq);
      EG_CK(cudaMemcpyAsync(dV.p + (size_t)(m + added) * N, tq, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      ++added;
    }
    if (added == 0) break;  // no new direction: the subspace is invariant
    nnew = added;
  }
  if (iters) *iters = std::min(it, max_iter);
  for (int j = 0; j < k; ++j) evals[j] = theta[j];
  if (evecs) {
    h1.assign((size_t)m * k, 0.0);
    for (int a = 0; a < m; ++a)
      for (int j = 0; j < k; ++j) h1[(size_t)a * k + j] = Y[(size_t)a * m + j];
    EG_CK(cudaMemcpyAsync(dc1.p, h1.data(), sizeof(double) * h1.size(), cudaMemcpyHostToDevice, s));
    k_lincomb<<<dim3(nblk(N, 256), k), 256, 0, s>>>(N, m, k, dV.p, dc1.p, nullptr, nullptr, 0.0, dR.p);
    EG_CK(cudaMemcpyAsync(evecs, dR.p, sizeof(double) * (size_t)k * N, cudaMemcpyDefault, s));
  }
  EG_CK(cudaStreamSynchronize(s));
  EG_CK(cudaGetLastError());
  if (!converged) return set_error(RTTDA_E_STATE, "rttda_eigenstates: not converged within max_iter");
  return RTTDA_OK;
}
