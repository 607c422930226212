"""Plain FP64 CPU oracle for RT-TDA propagation (test infrastructure only).

This file is a slow, explicit reference used by the tests, by the smoke check
and by the CPU-baseline leg of the benchmark.  Nothing on the product path
imports it.  It shares no code with the CUDA library: the two only take the
same inputs from the seeded generator.

What it computes (Knoll & Levine, "Simulating Electron Dynamics with
GPU-Accelerated Real-Time Tamm-Dancoff Approximation", arXiv 2601.16949):

* Basis {|0>, |ia>}; the singles index is 1 + i*nvirt + a ("virtuals run
  fastest", Sec. 2.1 after Eq. (3)).  |0> is the Kohn-Sham
  ground state added to the basis (Sec. 2.1, last paragraph).
* A is built explicitly as a dense real symmetric matrix:
      A_00 = 0, A_0,ia = 0                                (Sec. 2.1, Brillouin)
      A_ia,jb = d_ij d_ab (e_a - e_i) + 2 (ia|jb) - c_x (ij|ab)
  with (pq|rs) = sum_P B^P_pq B^P_rs.  The structure follows
  Eq. (3); the RI-factorised Coulomb/exchange pair in place of
  (ia|jb) + (ia|f_xc|jb) is this project's synthetic workload.
* The dipole matrix in the CSF basis follows the Slater-Condon rules
  (Eqs. (19a)-(19f)), with the constant <Phi0|mu|Phi0> dropped from the diagonal
  (it is a multiple of the identity):
      M_00 = 0, M_0,ia = <0|mu|ia> (input; sqrt(2) mu_ia for MO input, Eq. (19b))
      M_ia,ia = mu_aa - mu_ii (Eq. (19c)), M_ia,ib = mu_ab (Eq. (19d)),
      M_ia,ja = -mu_ji (Eq. (19e)), every other element 0 (Eq. (19f)).
* H(t) = A - E(t) M_d with M_d = sum_x d_x M_x (Eq. (16)) and
  i dc/dt = H(t) c (Eq. (11)).
* Pulses: Eqs. (18a), (18b), (18c),
  (18d) (sigma = FWHM / 2.35482), plus a sin^2 envelope
  E0 sin^2(pi t / tau) sin(omega t) on [0, tau].
* The delta kick E0 delta(t) is applied exactly, c(0+) = exp(+i kappa M_d) c(0),
  by a Taylor series; E(t) = 0 afterwards.
* Time stepping: classical 4-stage Runge-Kutta on dc/dt = -i H(t) c, stages
  at t, t + dt/2, t + dt/2, t + dt (the integrator this project specifies),
  and the paper's own second-order symplectic split operator (Sec. 2.2,
  Sec. 3.4) on dq/dt = H p, dp/dt = -H q (sso_step).
* Observables after every step: mu_d(t_n) = Re c^dagger M_d c and |c|^2;
  populations P_i(t) = |X_i^T c(t)|^2 of the TI-TDA states X_i (eigenvectors
  of A's singles block, Eq. (22)).
* Spectrum: S(w) = (w / kappa) Im sum_n w_n (mu_n - mu_0) exp((i w - g) t_n) dt
  with trapezoid weights, the dipole-trace analogue of Eq. (21);
  several polarisations are averaged as in Eq. (23).  The
  paper's own mode (spectrum_autocorr): autocorrelation R(t) (Eq.
  (20)), mirrored, Hann window, zero padding, FFT,
  w Re F[R] (Eq. (21)), averaged and normalised to the highest
  peak (Sec. 3.1).

Pins: every function here is checked against the paper or against
mathematics that does not reuse it (closed forms, brute-force Slater
determinants, eigendecomposition, the Rabi table of Sec. 3); see
tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np

# Pulse kinds (Eqs. (18a)-(18d), plus sin^2).
KICK, CW, GAUSS_TL, CHIRP, SIN2 = 0, 1, 2, 3, 4

# sigma = FWHM / 2.35482 (Sec. 2.2, after Eq. (18d)).
FWHM_TO_SIGMA = 2.35482


@dataclass
class Pulse:
    """One trajectory's field: kind, amplitude E0 (kappa for a kick), carrier
    omega, centre t0, FWHM, chirp beta, sin^2 duration tau and the unit
    polarisation vector d."""
    kind: int = KICK
    E0: float = 1e-3
    omega: float = 0.0
    t0: float = 0.0
    fwhm: float = 1.0
    beta: float = 0.0
    duration: float = 0.0
    direction: tuple = (0.0, 0.0, 1.0)


# ---------------------------------------------------------------------------
# Index map (Sec. 2.1)
# ---------------------------------------------------------------------------

def csf_index(i: int, a: int, nvirt: int) -> int:
    """Position of |ia> in the amplitude vector; 0 is |0>."""
    return 1 + i * nvirt + a


def dim(nocc: int, nvirt: int) -> int:
    """N_CSF + 1 (Eq. (13) plus the ground state)."""
    return 1 + nocc * nvirt


# ---------------------------------------------------------------------------
# A matrix (Eq. (3) with the RI-factorised two-electron part)
# ---------------------------------------------------------------------------

def eri_ovov(B_ov: np.ndarray) -> np.ndarray:
    """(ia|jb) = sum_P B^P_ia B^P_jb as an [ov, ov] matrix."""
    P = B_ov.shape[0]
    Bf = B_ov.reshape(P, -1)
    return Bf.T @ Bf


def eri_oovv(B_oo: np.ndarray, B_vv: np.ndarray) -> np.ndarray:
    """(ij|ab) = sum_P B^P_ij B^P_ab, returned as [i, j, a, b]."""
    return np.einsum("pij,pab->ijab", B_oo, B_vv, optimize=True)


def build_A(mol: dict, c_x: float) -> np.ndarray:
    """Dense A in the extended basis {|0>, |ia>}."""
    o, v = mol["nocc"], mol["nvirt"]
    n = dim(o, v)
    ov = o * v
    A = np.zeros((n, n))
    # two-electron part on the singles block
    coul = eri_ovov(mol["B_ov"])                       # [(i,a), (j,b)]
    exch = eri_oovv(mol["B_oo"], mol["B_vv"])          # [i, j, a, b]
    exch = exch.transpose(0, 2, 1, 3).reshape(ov, ov)  # [(i,a), (j,b)]
    A[1:, 1:] = 2.0 * coul - c_x * exch
    # orbital-energy diagonal e_a - e_i
    for i in range(o):
        for a in range(v):
            k = csf_index(i, a, v)
            A[k, k] += mol["eps_virt"][a] - mol["eps_occ"][i]
    # A_00 = 0 and A_0,ia = 0 are already in place.
    return A


def A_rows(mol: dict, c_x: float, rows) -> np.ndarray:
    """Selected rows of A, each built from the definition without forming A.

    Used for sampled checks at sizes where the dense A does not fit."""
    o, v, P = mol["nocc"], mol["nvirt"], mol["naux"]
    n = dim(o, v)
    out = np.zeros((len(rows), n))
    B_ov = mol["B_ov"]
    for r, k in enumerate(rows):
        if k == 0:
            continue
        i, a = divmod(k - 1, v)
        coul = np.einsum("p,pjb->jb", B_ov[:, i, a], B_ov)
        exch = np.einsum("pj,pb->jb", mol["B_oo"][:, i, :], mol["B_vv"][:, a, :])
        row = 2.0 * coul - c_x * exch
        row[i, a] += mol["eps_virt"][a] - mol["eps_occ"][i]
        out[r, 1:] = row.reshape(-1)
    return out


def A_block(mol: dict, c_x: float, i0: int, i1: int) -> np.ndarray:
    """Rows of A for the occupied range i0 <= i < i1 (all a), as one block.

    Same definition as build_A restricted to those rows."""
    o, v, P = mol["nocc"], mol["nvirt"], mol["naux"]
    n = dim(o, v)
    ni = i1 - i0
    out = np.zeros((ni * v, n))
    Bf = mol["B_ov"].reshape(P, -1)
    coul = Bf[:, i0 * v:i1 * v].T @ Bf
    exch = np.einsum("pij,pab->iajb", mol["B_oo"][:, i0:i1, :], mol["B_vv"], optimize=True)
    out[:, 1:] = 2.0 * coul - c_x * exch.reshape(ni * v, o * v)
    for i in range(i0, i1):
        for a in range(v):
            r = (i - i0) * v + a
            out[r, csf_index(i, a, v)] += mol["eps_virt"][a] - mol["eps_occ"][i]
    return out


# ---------------------------------------------------------------------------
# Dipole matrix (Eqs. (19a)-(19f))
# ---------------------------------------------------------------------------

def dipole_along(mol: dict, direction) -> tuple:
    """mu_d = sum_x d_x mu_x for the three MO blocks (Eq. (16): mu . d)."""
    d = np.asarray(direction, dtype=np.float64)
    mu_oo = np.einsum("x,xij->ij", d, mol["mu_oo"])
    mu_vv = np.einsum("x,xab->ab", d, mol["mu_vv"])
    m0 = np.einsum("x,xia->ia", d, mol["mu_0ov"])
    return mu_oo, mu_vv, m0


def build_M(mu_oo: np.ndarray, mu_vv: np.ndarray, m0: np.ndarray) -> np.ndarray:
    """Dense CSF-basis dipole matrix from MO blocks (Slater-Condon rules)."""
    o, v = m0.shape
    n = dim(o, v)
    M = np.zeros((n, n))
    for i in range(o):
        for a in range(v):
            k = csf_index(i, a, v)
            M[0, k] = M[k, 0] = m0[i, a]                          # Eq. (19b)
            M[k, k] = mu_vv[a, a] - mu_oo[i, i]                   # Eq. (19c) minus (19a)
            for b in range(v):
                if b != a:
                    M[k, csf_index(i, b, v)] = mu_vv[a, b]        # Eq. (19d)
            for j in range(o):
                if j != i:
                    M[k, csf_index(j, a, v)] = -mu_oo[j, i]       # Eq. (19e)
    return M                                                       # Eq. (19f): rest 0


def M_rows(mu_oo, mu_vv, m0, rows) -> np.ndarray:
    """Selected rows of the dipole matrix, built element by element."""
    o, v = m0.shape
    n = dim(o, v)
    out = np.zeros((len(rows), n))
    for r, k in enumerate(rows):
        if k == 0:
            out[r, 1:] = m0.reshape(-1)
            continue
        i, a = divmod(k - 1, v)
        out[r, 0] = m0[i, a]
        for b in range(v):
            out[r, csf_index(i, b, v)] += mu_vv[a, b]
        for j in range(o):
            out[r, csf_index(j, a, v)] -= mu_oo[j, i]
    return out


# ---------------------------------------------------------------------------
# Pulses (Eqs. (18a), (18b), (18c), (18d))
# ---------------------------------------------------------------------------

def field(p: Pulse, t: float) -> float:
    """E(t) for t > 0.  A kick has already been applied at t = 0+."""
    if p.kind == KICK:
        return 0.0
    if p.kind == CW:
        return p.E0 * math.sin(p.omega * t)
    if p.kind in (GAUSS_TL, CHIRP):
        s = p.fwhm / FWHM_TO_SIGMA
        tau = t - p.t0
        env = math.exp(-tau * tau / (2.0 * s * s))
        w = p.omega + (0.5 * p.beta * tau if p.kind == CHIRP else 0.0)
        return p.E0 * env * math.sin(w * tau)
    if p.kind == SIN2:
        if t < 0.0 or t > p.duration:
            return 0.0
        return p.E0 * math.sin(math.pi * t / p.duration) ** 2 * math.sin(p.omega * t)
    raise ValueError(f"unknown pulse kind {p.kind}")


# ---------------------------------------------------------------------------
# Kick, sigma, RK4
# ---------------------------------------------------------------------------

def kick(M: np.ndarray, kappa: float, c: np.ndarray, tol: float = 1e-18) -> np.ndarray:
    """exp(+i kappa M) c by its Taylor series, stopped when a term's norm < tol."""
    out = c.astype(np.complex128).copy()
    term = out.copy()
    k = 0
    while True:
        k += 1
        term = (1j * kappa / k) * (M @ term)
        out += term
        if np.linalg.norm(term) < tol or k > 200:
            return out


def sigma(A: np.ndarray, M: np.ndarray, E: float, c: np.ndarray) -> np.ndarray:
    """sigma = H(t) c = (A - E(t) M) c (Eq. (16) with Eq. (17)).

    A and M are real, so the real and imaginary parts of c are multiplied
    separately (numpy would otherwise copy A to complex for every product)."""
    c = np.asarray(c)
    if np.iscomplexobj(c):
        return (A @ c.real - E * (M @ c.real)) + 1j * (A @ c.imag - E * (M @ c.imag))
    return A @ c - E * (M @ c)


def rk4_step(A, M, p: Pulse, t: float, dt: float, c: np.ndarray) -> np.ndarray:
    """One classical RK4 step of dc/dt = -i H(t) c."""
    f = lambda tt, cc: -1j * sigma(A, M, field(p, tt), cc)
    k1 = f(t, c)
    k2 = f(t + 0.5 * dt, c + 0.5 * dt * k1)
    k3 = f(t + 0.5 * dt, c + 0.5 * dt * k2)
    k4 = f(t + dt, c + dt * k3)
    return c + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def observables(M: np.ndarray, c: np.ndarray) -> tuple:
    """(mu_d = Re c^dagger M c, |c|^2)."""
    return float(np.real(np.vdot(c, M @ c))), float(np.real(np.vdot(c, c)))


@dataclass
class Trajectory:
    c: np.ndarray
    dipole: np.ndarray
    norm: np.ndarray
    c_history: list = dc_field(default_factory=list)


def propagate(A, M, p: Pulse, c0, dt: float, nsteps: int, keep_every: int = 0) -> Trajectory:
    """Kick (if the pulse is a kick), then nsteps RK4 steps from t = 0.

    dipole[n], norm[n] are taken at t_n = n dt for n = 0..nsteps (n = 0 is
    after the kick)."""
    n = A.shape[0]
    if c0 is None:
        c = np.zeros(n, dtype=np.complex128)
        c[0] = 1.0
    else:
        c = np.asarray(c0, dtype=np.complex128).copy()
    if p.kind == KICK:
        c = kick(M, p.E0, c)
    dip = np.zeros(nsteps + 1)
    nrm = np.zeros(nsteps + 1)
    dip[0], nrm[0] = observables(M, c)
    hist = [c.copy()] if keep_every else []
    for s in range(nsteps):
        c = rk4_step(A, M, p, s * dt, dt, c)
        dip[s + 1], nrm[s + 1] = observables(M, c)
        if keep_every and (s + 1) % keep_every == 0:
            hist.append(c.copy())
    return Trajectory(c=c, dipole=dip, norm=nrm, c_history=hist)


# ---------------------------------------------------------------------------
# Symplectic split-operator integrator (Sec. 2.2; convergence study Sec. 3.4)
# ---------------------------------------------------------------------------
# With c = q + i p (Eq. (12)) and a real symmetric H(t), the
# equation of motion i dc/dt = H(t) c is the pair dq/dt = H p, dp/dt = -H q
# (Sec. 2.2).  The second-order symmetric splitting takes half a step of the
# p-flow, a whole step of the q-flow and again half a step of the p-flow;
# with t treated as a coordinate, the p half steps use H at the two ends of
# the step and the q step uses H at its middle:
#     p_{n+1/2} = p_n       - (dt/2) H(t_n)       q_n
#     q_{n+1}   = q_n       +  dt    H(t_n + dt/2) p_{n+1/2}
#     p_{n+1}   = p_{n+1/2} - (dt/2) H(t_n + dt)  q_{n+1}
# Each sub-step multiplies one real vector by H: two sigma products per step
# (H q_{n+1} is reused by the next step's first half step).

def sso_step(A, M, p: Pulse, t: float, dt: float, c: np.ndarray) -> np.ndarray:
    """One symplectic split-operator step of i dc/dt = H(t) c (c complex)."""
    q = np.array(c.real, dtype=np.float64)
    pp = np.array(c.imag, dtype=np.float64)
    pp = pp - 0.5 * dt * sigma(A, M, field(p, t), q)
    q = q + dt * sigma(A, M, field(p, t + 0.5 * dt), pp)
    pp = pp - 0.5 * dt * sigma(A, M, field(p, t + dt), q)
    return q + 1j * pp


def propagate_sso(A, M, p: Pulse, c0, dt: float, nsteps: int) -> Trajectory:
    """As propagate(), with the symplectic split-operator step in place of RK4."""
    n = A.shape[0]
    if c0 is None:
        c = np.zeros(n, dtype=np.complex128)
        c[0] = 1.0
    else:
        c = np.asarray(c0, dtype=np.complex128).copy()
    if p.kind == KICK:
        c = kick(M, p.E0, c)
    dip = np.zeros(nsteps + 1)
    nrm = np.zeros(nsteps + 1)
    dip[0], nrm[0] = observables(M, c)
    for s in range(nsteps):
        c = sso_step(A, M, p, s * dt, dt, c)
        dip[s + 1], nrm[s + 1] = observables(M, c)
    return Trajectory(c=c, dipole=dip, norm=nrm)


# ---------------------------------------------------------------------------
# Stationary states and populations (Sec. 2.2, Eq. (22))
# ---------------------------------------------------------------------------

def ti_states(A: np.ndarray, k: int) -> tuple:
    """The k lowest excited TI-TDA states (Sec. 2.1, Eq. (2)): the
    eigenpairs of A's singles block, as full-length vectors with a zero
    ground component.  (The ground row and column of A are zero, so |0> is
    an eigenvector with eigenvalue 0 that is left out.)"""
    w, U = np.linalg.eigh(A[1:, 1:])
    X = np.zeros((k, A.shape[0]))
    X[:, 1:] = U[:, :k].T
    return w[:k], X


def overlaps(X: np.ndarray, c: np.ndarray) -> np.ndarray:
    """o_i = X_i^T c for real states X_i (rows of X)."""
    return np.asarray(X, dtype=np.float64) @ np.asarray(c)


def populations(X: np.ndarray, c: np.ndarray) -> np.ndarray:
    """P_i = |X_i^T c|^2 (Eq. (22))."""
    return np.abs(overlaps(X, c)) ** 2


# ---------------------------------------------------------------------------
# Spectrum (Eq. (21) on the dipole trace; Eq. (23))
# ---------------------------------------------------------------------------

def autocorrelation(c_eps: np.ndarray, states) -> np.ndarray:
    """R(t_n) = X^dagger(eps) X(eps + t_n) (Eq. (20)) for
    the states of a run started right after the kick (c_eps = its first)."""
    return np.array([np.vdot(c_eps, c) for c in states])


def autocorr_grid(npts: int, dt: float, npad: int, nfreq: int) -> np.ndarray:
    """Frequencies of the zero-padded FFT of the mirrored record: the record
    has 2 npts - 1 points, plus npad zeros; w_k = 2 pi k / (Ntot dt)."""
    ntot = 2 * npts - 1 + npad
    return 2.0 * np.pi * np.arange(nfreq) / (ntot * dt)


def spectrum_autocorr(R, dt: float, npad: int, nfreq: int, normalize: bool = True) -> np.ndarray:
    """Absorption spectrum from autocorrelation functions, the paper's way
    (Sec. 3.1 with Eqs. (20), (21) and
    (23)): each R(t) (t >= 0) is mirrored to negative times with
    R(-t) = conj(R(t)), multiplied by a Hann window over the mirrored record
    (peak at t = 0), padded with npad zeros and Fourier transformed,
    F(w) = sum_m w_m R(t_m) exp(+i w t_m) dt; the spectrum is w Re F(w) on the
    FFT grid (autocorr_grid), averaged over the records, and (normalize)
    divided by its largest value on the first nfreq grid points."""
    R = np.atleast_2d(np.asarray(R, dtype=np.complex128))
    npts = R.shape[1]
    ntot = 2 * npts - 1 + npad
    win = np.hanning(2 * npts - 1)
    w = autocorr_grid(npts, dt, npad, nfreq)
    k = np.arange(nfreq)
    S = np.zeros(nfreq)
    for r in R:
        rec = np.concatenate([np.conj(r[:0:-1]), r]) * win   # t_m = (m - npts + 1) dt
        x = np.zeros(ntot, dtype=np.complex128)
        x[: rec.size] = rec
        F = dt * ntot * np.fft.ifft(x)[:nfreq] * np.exp(-2j * np.pi * k * (npts - 1) / ntot)
        S += w * F.real
    S /= R.shape[0]
    if normalize:
        S = S / np.max(S)
    return S


def frequency_grid(wmin: float, wmax: float, nfreq: int) -> np.ndarray:
    if nfreq == 1:
        return np.array([wmin])
    return wmin + (wmax - wmin) * np.arange(nfreq) / (nfreq - 1)


def spectrum(traces, dt: float, kappa: float, gamma: float, omegas) -> np.ndarray:
    """Average over traces of S(w) = (w/kappa) Im sum_n w_n (mu_n - mu_0) e^{(iw-g)t_n} dt."""
    traces = np.atleast_2d(np.asarray(traces, dtype=np.float64))
    omegas = np.asarray(omegas, dtype=np.float64)
    npts = traces.shape[1]
    t = dt * np.arange(npts)
    wts = np.ones(npts)
    wts[0] = wts[-1] = 0.5
    S = np.zeros(len(omegas))
    for tr in traces:
        d = (tr - tr[0]) * wts * np.exp(-gamma * t)
        for k, w in enumerate(omegas):
            S[k] += (w / kappa) * np.sum(d * np.sin(w * t)) * dt
    return S / traces.shape[0]
