"""Pins for the FP64 CPU oracle.

Each test checks the oracle against something that does not reuse it: a
closed form, a brute-force Slater-determinant calculation, an
eigendecomposition (numpy eigh), or numbers printed in the paper
(tests/golden/).  A dropped term, a wrong sign, a swapped index or a wrong
RK4 coefficient in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
HARTREE_EV = 27.211386245988          # CODATA 2018
AU_TIME_FS = 2.4188843265857e-2       # CODATA 2018
AU_INTENSITY_W_CM2 = 3.50944758e16    # atomic unit of intensity


def small_mol(o=3, v=5, P=7, seed=11):
    return synth.molecule(o, v, P, seed=seed)


def zero_mol(o, v, P=1):
    z = lambda *s: np.zeros(s)
    return dict(nocc=o, nvirt=v, naux=P, eps_occ=z(o), eps_virt=z(v),
                B_ov=z(P, o, v), B_oo=z(P, o, o), B_vv=z(P, v, v),
                mu_oo=z(3, o, o), mu_vv=z(3, v, v), mu_0ov=z(3, o, v))


def rk4_R(z):
    """Stability polynomial of classical RK4 (a textbook fact)."""
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


# ---------------------------------------------------------------------------
# A matrix
# ---------------------------------------------------------------------------

def test_A_is_symmetric_and_ground_row_zero():
    mol = small_mol()
    A = orc.build_A(mol, 0.2)
    assert np.array_equal(A, A.T)
    assert np.all(A[0] == 0.0) and np.all(A[:, 0] == 0.0)


def test_A_rank_one_coulomb_secular_equation():
    """c_x = 0, P = 1: A_singles = D + 2 b b^T.  Its eigenvalues solve the
    secular equation 1 + 2 sum_k b_k^2 / (d_k - lam) = 0 (closed form)."""
    o, v = 2, 3
    rng = np.random.default_rng(5)
    mol = zero_mol(o, v, 1)
    mol["eps_occ"] = np.array([-0.9, -0.4])
    mol["eps_virt"] = np.array([0.1, 0.55, 1.3])
    b = rng.standard_normal((o, v)) * 0.2
    mol["B_ov"][0] = b
    A = orc.build_A(mol, c_x=0.7)   # exchange factors are zero, so c_x is inert
    lam = np.linalg.eigvalsh(A[1:, 1:])
    d = (mol["eps_virt"][None, :] - mol["eps_occ"][:, None]).reshape(-1)
    bf = b.reshape(-1)
    f = 1.0 + 2.0 * np.sum(bf[None, :] ** 2 / (d[None, :] - lam[:, None]), axis=1)
    assert np.max(np.abs(f)) < 1e-9
    # the largest eigenvalue is pushed above every d (positive rank-one update)
    assert lam[-1] > d.max()


def test_A_exchange_couples_ij_ab_not_ia_jb():
    """B_ov = 0, c_x = 1, P = 1 with B_oo = [[0,1],[1,0]], B_vv = e0 e0^T:
    (ij|ab) is nonzero only for i != j, a = b = 0, so A couples |0 0> with
    |1 0> by -1 and leaves the rest diagonal.  Closed-form 2x2 eigenvalues."""
    mol = zero_mol(2, 2, 1)
    mol["eps_occ"] = np.array([-0.8, -0.5])
    mol["eps_virt"] = np.array([0.3, 0.9])
    mol["B_oo"][0] = [[0.0, 1.0], [1.0, 0.0]]
    mol["B_vv"][0] = [[1.0, 0.0], [0.0, 0.0]]
    A = orc.build_A(mol, c_x=1.0)
    k00, k10 = orc.csf_index(0, 0, 2), orc.csf_index(1, 0, 2)
    d00, d10 = 0.3 + 0.8, 0.3 + 0.5
    assert A[k00, k10] == -1.0 and A[k10, k00] == -1.0
    off = A.copy()
    off[k00, k10] = off[k10, k00] = 0.0
    assert np.count_nonzero(off - np.diag(np.diag(off))) == 0
    lam = np.sort(np.linalg.eigvalsh(A[np.ix_([k00, k10], [k00, k10])]))
    mean, half = 0.5 * (d00 + d10), 0.5 * (d00 - d10)
    ref = np.array([mean - math.hypot(half, 1.0), mean + math.hypot(half, 1.0)])
    assert np.allclose(lam, ref, atol=1e-15)


def test_A_diagonal_only_when_two_electron_part_vanishes():
    mol = zero_mol(3, 4, 2)
    mol["eps_occ"] = np.array([-1.0, -0.7, -0.3])
    mol["eps_virt"] = np.array([0.1, 0.2, 0.4, 1.9])
    A = orc.build_A(mol, 0.3)
    d = (mol["eps_virt"][None, :] - mol["eps_occ"][:, None]).reshape(-1)
    assert np.array_equal(A, np.diag(np.concatenate([[0.0], d])))


def test_A_rows_equal_dense_rows():
    mol = small_mol(4, 6, 9, seed=3)
    A = orc.build_A(mol, 0.25)
    rows = [0, 1, 7, 13, 24]
    assert np.allclose(orc.A_rows(mol, 0.25, rows), A[rows], rtol=0, atol=1e-15)
    blk = orc.A_block(mol, 0.25, 1, 3)
    assert np.allclose(blk, A[1 + 6:1 + 18], rtol=0, atol=1e-15)


def test_sigma_complex_split_equals_complex_product():
    mol = small_mol(2, 3, 4, seed=1)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (1, 0, 0)))
    c = synth.random_state(A.shape[0], 1, seed=5)[0]
    ref = (A.astype(complex) - 0.3 * M.astype(complex)) @ c
    assert np.allclose(orc.sigma(A, M, 0.3, c), ref, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# Dipole matrix: brute-force Slater determinants
# ---------------------------------------------------------------------------

def _apply_excitation(det, p, q):
    """a^dagger_p a_q on a determinant bitmask; returns (sign, det) or None."""
    if not (det >> q) & 1:
        return None
    sign = -1 if bin(det & ((1 << q) - 1)).count("1") % 2 else 1
    det ^= 1 << q
    if (det >> p) & 1:
        return None
    if bin(det & ((1 << p) - 1)).count("1") % 2:
        sign = -sign
    return sign, det | (1 << p)


def _apply_one_body(state, h):
    """sum_{pq sigma} h_pq a^dagger_{p sigma} a_{q sigma} on {det: coeff}."""
    nmo = h.shape[0]
    out = {}
    for det, cf in state.items():
        for p, q in itertools.product(range(nmo), repeat=2):
            if h[p, q] == 0.0:
                continue
            for s in (0, 1):
                r = _apply_excitation(det, 2 * p + s, 2 * q + s)
                if r is not None:
                    out[r[1]] = out.get(r[1], 0.0) + r[0] * cf * h[p, q]
    return out


def _dot(x, y):
    return sum(c * y.get(d, 0.0) for d, c in x.items())


def test_M_matches_brute_force_slater_determinants():
    """Singlet CSFs from determinants; <I|mu|J> by second quantisation.
    Checks Eqs. (19b) (sqrt 2), (19c), (19d), (19e) (sign) and (19f) (zeros) at once."""
    o, v = 2, 3
    nmo = o + v
    rng = np.random.default_rng(7)
    mu = rng.standard_normal((nmo, nmo))
    mu = 0.5 * (mu + mu.T)
    ground = 0
    for i in range(o):
        ground |= (1 << (2 * i)) | (1 << (2 * i + 1))
    csfs = [{ground: 1.0}]
    for i in range(o):
        for a in range(v):
            e = np.zeros((nmo, nmo))
            e[o + a, i] = 1.0
            st = _apply_one_body({ground: 1.0}, e)   # spin-summed E_ai
            csfs.append({d: c / math.sqrt(2.0) for d, c in st.items()})
    n = len(csfs)
    for x in range(n):
        for y in range(n):
            assert abs(_dot(csfs[x], csfs[y]) - (x == y)) < 1e-14
    Mb = np.array([[_dot(csfs[x], _apply_one_body(csfs[y], mu)) for y in range(n)]
                   for x in range(n)])
    e0 = Mb[0, 0]
    assert abs(e0 - 2.0 * np.trace(mu[:o, :o])) < 1e-13
    Mo = orc.build_M(mu[:o, :o], mu[o:, o:], math.sqrt(2.0) * mu[:o, o:])
    assert np.allclose(Mo, Mb - e0 * np.eye(n), atol=1e-13)


def test_dipole_along_matches_brute_force_for_a_mixed_direction():
    """Eq. (16)'s mu . d for a polarisation mixing all three axes: the CSF
    dipole matrix built by second quantisation from the combined MO operator
    sum_x d_x mu_x equals build_M of dipole_along's blocks (a dropped or
    transposed component, or a wrong block, fails)."""
    o, v = 2, 3
    nmo = o + v
    rng = np.random.default_rng(11)
    mus = []
    for _ in range(3):
        m = rng.standard_normal((nmo, nmo))
        mus.append(0.5 * (m + m.T))
    mol = {"nocc": o, "nvirt": v,
           "mu_oo": np.array([m[:o, :o] for m in mus]),
           "mu_vv": np.array([m[o:, o:] for m in mus]),
           "mu_0ov": np.array([math.sqrt(2.0) * m[:o, o:] for m in mus])}
    d = np.array([0.36, -0.48, 0.8])
    h = sum(d[x] * mus[x] for x in range(3))
    ground = 0
    for i in range(o):
        ground |= (1 << (2 * i)) | (1 << (2 * i + 1))
    csfs = [{ground: 1.0}]
    for i in range(o):
        for a in range(v):
            e = np.zeros((nmo, nmo))
            e[o + a, i] = 1.0
            st = _apply_one_body({ground: 1.0}, e)
            csfs.append({det: c / math.sqrt(2.0) for det, c in st.items()})
    n = len(csfs)
    Mb = np.array([[_dot(csfs[x], _apply_one_body(csfs[y], h)) for y in range(n)] for x in range(n)])
    Mo = orc.build_M(*orc.dipole_along(mol, d))
    assert np.allclose(Mo, Mb - Mb[0, 0] * np.eye(n), atol=1e-13)


def test_M_two_level_and_sparsity():
    mu_oo = np.array([[0.3]])
    mu_vv = np.array([[-0.2]])
    m0 = np.array([[1.1]])
    M = orc.build_M(mu_oo, mu_vv, m0)
    assert np.array_equal(M, np.array([[0.0, 1.1], [1.1, -0.5]]))
    mol = small_mol(3, 4, 2, seed=9)
    moo, mvv, m0 = orc.dipole_along(mol, (0.0, 0.6, 0.8))
    M = orc.build_M(moo, mvv, m0)
    assert np.array_equal(M, M.T)
    for i, a, j, b in itertools.product(range(3), range(4), range(3), range(4)):
        if i != j and a != b:
            assert M[orc.csf_index(i, a, 4), orc.csf_index(j, b, 4)] == 0.0
    rows = [0, 2, 5, 11]
    assert np.array_equal(orc.M_rows(moo, mvv, m0, rows), M[rows])


# ---------------------------------------------------------------------------
# Pulses
# ---------------------------------------------------------------------------

def test_pulse_shapes():
    tl = orc.Pulse(kind=orc.GAUSS_TL, E0=2.0, omega=0.7, t0=30.0, fwhm=12.0)
    env = lambda t: math.exp(-((t - tl.t0) / (tl.fwhm / orc.FWHM_TO_SIGMA)) ** 2 / 2)
    assert abs(env(tl.t0 + tl.fwhm / 2) - 0.5) < 1e-5     # FWHM definition
    # carrier phase is measured from t0: zero field at the peak
    assert orc.field(tl, tl.t0) == 0.0
    t = tl.t0 + 0.3
    assert abs(orc.field(tl, t) - 2.0 * env(t) * math.sin(0.7 * 0.3)) < 1e-15
    # chirp: instantaneous frequency d/dt phase = omega + beta (t - t0)
    ch = orc.Pulse(kind=orc.CHIRP, E0=1.0, omega=0.5, t0=0.0, fwhm=1e9, beta=0.01)
    tau, h = 20.0, 1e-4
    assert abs(orc.field(ch, tau) - math.sin((0.5 + 0.005 * tau) * tau)) < 1e-12
    # the phase (omega + beta tau / 2) tau has derivative omega + beta tau
    ph = lambda x: (ch.omega + 0.5 * ch.beta * x) * x
    assert abs((ph(tau + h) - ph(tau - h)) / (2 * h) - (0.5 + 0.01 * tau)) < 1e-8
    cw = orc.Pulse(kind=orc.CW, E0=0.1, omega=0.3)
    assert abs(orc.field(cw, 2.0) - 0.1 * math.sin(0.6)) < 1e-16
    s2 = orc.Pulse(kind=orc.SIN2, E0=1.0, omega=0.4, duration=100.0)
    assert orc.field(s2, -1.0) == 0.0 and orc.field(s2, 100.5) == 0.0
    assert abs(orc.field(s2, 50.0) - math.sin(20.0)) < 1e-15
    assert orc.field(orc.Pulse(kind=orc.KICK, E0=1.0), 3.0) == 0.0


# ---------------------------------------------------------------------------
# RK4 propagation against the eigendecomposition
# ---------------------------------------------------------------------------

def _field_free(mol, c_x, nsteps, dt, seed=2):
    A = orc.build_A(mol, c_x)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    c0 = synth.random_state(A.shape[0], 1, seed=seed)[0]
    tr = orc.propagate(A, M, orc.Pulse(kind=orc.CW, E0=0.0), c0, dt, nsteps)
    lam, V = np.linalg.eigh(A)
    b = V.T @ c0
    return A, M, c0, tr, lam, V, b


@pytest.mark.parametrize("shape", [(3, 5, 7), (8, 24, 96)])
def test_rk4_field_free_equals_eigenbasis_polynomial(shape):
    mol = synth.molecule(*shape, seed=0)
    dt, n = 0.05, 200
    A, M, c0, tr, lam, V, b = _field_free(mol, 0.2, n, dt)
    ref = V @ (rk4_R(-1j * lam * dt) ** n * b)
    assert np.max(np.abs(tr.c - ref)) < 1e-12
    # with the exact propagator the difference is bounded by the per-step
    # amplification error of RK4 (componentwise in the eigenbasis)
    exact = V @ (np.exp(-1j * lam * dt * n) * b)
    bound = n * np.max(np.abs(rk4_R(-1j * lam * dt) - np.exp(-1j * lam * dt)))
    assert np.linalg.norm(tr.c - exact) <= bound * np.linalg.norm(c0) + 1e-13
    # norm after every step follows |R|^(2n)
    g = np.abs(rk4_R(-1j * lam * dt)) ** 2
    pred = np.array([np.sum(g ** k * np.abs(b) ** 2) for k in range(n + 1)])
    assert np.max(np.abs(tr.norm - pred)) < 1e-13


def test_rk4_is_fourth_order_with_time_dependent_field():
    mol = small_mol(2, 3, 4, seed=4)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (1, 0, 0)))
    p = orc.Pulse(kind=orc.GAUSS_TL, E0=0.05, omega=0.9, t0=4.0, fwhm=3.0)
    T = 8.0
    run = lambda dt: orc.propagate(A, M, p, None, dt, int(round(T / dt))).c
    ref = run(0.2 / 64)
    errs = [np.linalg.norm(run(dt) - ref) for dt in (0.2, 0.1, 0.05)]
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(abs(s - 4.0) < 0.1 for s in slopes), slopes


# ---------------------------------------------------------------------------
# Symplectic split-operator integrator
# ---------------------------------------------------------------------------

def leapfrog_power(x, n):
    """n steps of Stormer-Verlet on one harmonic mode q' = w p, p' = -w q
    with x = w dt, as the 2x2 map (q, p) -> T^n (q, p).  Textbook facts used:
    T has unit determinant and trace 2 - x^2, so its eigenvalues are
    exp(+-i theta) with cos(theta) = 1 - x^2/2, and for such a matrix
    T^n = sin(n theta)/sin(theta) T - sin((n-1) theta)/sin(theta) I
    (Chebyshev recursion).  T itself is the product of the three shears
    p -= (x/2) q, q += x p, p -= (x/2) q."""
    x = np.asarray(x, dtype=np.float64)
    kick = lambda a: np.array([[np.ones_like(a), np.zeros_like(a)], [-a / 2, np.ones_like(a)]])
    drift = lambda a: np.array([[np.ones_like(a), a], [np.zeros_like(a), np.ones_like(a)]])
    T = np.einsum("ij...,jk...,kl...->il...", kick(x), drift(x), kick(x))
    th = np.arccos(1 - x ** 2 / 2)
    I = np.array([[np.ones_like(x), np.zeros_like(x)], [np.zeros_like(x), np.ones_like(x)]])
    small = np.abs(th) < 1e-12          # x = 0 (the ground row): sin(k th)/sin(th) -> k
    st = np.where(small, 1.0, np.sin(th))
    un = np.where(small, n, np.sin(n * th) / st)
    un1 = np.where(small, n - 1, np.sin((n - 1) * th) / st)
    return un * T - un1 * I


@pytest.mark.parametrize("shape", [(2, 3, 4), (3, 5, 7)])
def test_sso_field_free_equals_per_mode_leapfrog(shape):
    """Field-free SSO in the eigenbasis of A is Stormer-Verlet on each mode."""
    mol = synth.molecule(*shape, seed=1)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    lam, V = np.linalg.eigh(A)
    c0 = synth.random_state(A.shape[0], 1, seed=2)[0]
    dt, n = 0.05, 300
    tr = orc.propagate_sso(A, M, orc.Pulse(kind=orc.CW, E0=0.0, omega=1.0), c0, dt, n)
    bq, bp = V.T @ c0.real, V.T @ c0.imag
    Tn = leapfrog_power(lam * dt, n)
    q = Tn[0, 0] * bq + Tn[0, 1] * bp
    p = Tn[1, 0] * bq + Tn[1, 1] * bp
    ref = V @ q + 1j * (V @ p)
    assert np.max(np.abs(tr.c - ref)) < 1e-12


def test_sso_is_time_reversible():
    mol = small_mol(3, 4, 5, seed=6)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (1, 0, 0)))
    p0 = orc.Pulse(kind=orc.CW, E0=0.0, omega=1.0)
    c0 = synth.random_state(A.shape[0], 1, seed=3)[0]
    c = c0.copy()
    for k in range(100):
        c = orc.sso_step(A, M, p0, k * 0.05, 0.05, c)
    for k in range(100):
        c = orc.sso_step(A, M, p0, (100 - k) * 0.05, -0.05, c)
    assert np.max(np.abs(c - c0)) < 1e-12


def test_sso_mean_norm_error_is_second_order_as_in_paper():
    """Sec. 3.4: start from a stationary state in the real part, run a fixed
    50 au, and the norm error averaged over the run falls with slope 2 in
    dt.  For one mode of frequency w the leapfrog norm is
    1 - (w dt / 2)^2 sin^2(n theta), so the mean error is (w dt)^2 / 8 to
    leading order."""
    mol = small_mol(3, 4, 6, seed=9)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (0, 1, 0)))
    lam, V = np.linalg.eigh(A)
    k = int(np.argsort(lam)[1])          # first excited state (lam[0] is the ground row)
    c0 = V[:, k].astype(np.complex128)
    p0 = orc.Pulse(kind=orc.CW, E0=0.0, omega=1.0)
    errs = []
    dts = [0.2, 0.1, 0.05, 0.025]
    for dt in dts:
        tr = orc.propagate_sso(A, M, p0, c0, dt, int(round(50.0 / dt)))
        errs.append(np.mean(np.abs(tr.norm - 1.0)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(dts) - 1)]
    assert all(abs(s - 2.0) < 0.1 for s in slopes), slopes
    w = lam[k]
    assert abs(errs[-1] / ((w * dts[-1]) ** 2 / 8) - 1.0) < 0.05
    # RK4 on the same problem loses norm monotonically instead
    tr4 = orc.propagate(A, M, p0, c0, 0.2, 250)
    assert np.all(np.diff(tr4.norm) <= 1e-15)


def test_sso_is_second_order_with_time_dependent_field():
    """The field enters each sub-step at the middle of the interval it
    advances; a first-order placement would show slope 1 here."""
    mol = small_mol(2, 3, 4, seed=4)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (1, 0, 0)))
    p = orc.Pulse(kind=orc.GAUSS_TL, E0=0.05, omega=0.9, t0=4.0, fwhm=3.0)
    T = 8.0
    ref = orc.propagate(A, M, p, None, 0.2 / 64, int(round(T / (0.2 / 64)))).c
    errs = [np.linalg.norm(orc.propagate_sso(A, M, p, None, dt, int(round(T / dt))).c - ref)
            for dt in (0.1, 0.05, 0.025)]
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(abs(s - 2.0) < 0.1 for s in slopes), slopes


# ---------------------------------------------------------------------------
# Stationary states and populations
# ---------------------------------------------------------------------------

def test_populations_over_all_states_sum_to_the_norm():
    """Completeness: the TI states plus |0> are an orthonormal basis, so the
    populations of all of them add up to |c|^2 at every step (a driven
    trajectory, so the state is not stationary)."""
    mol = small_mol(2, 3, 4, seed=5)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (0, 1, 0)))
    n = A.shape[0]
    w, X = orc.ti_states(A, n - 1)
    e0 = np.zeros(n)
    e0[0] = 1.0
    allX = np.vstack([e0, X])
    p = orc.Pulse(kind=orc.GAUSS_TL, E0=0.08, omega=0.8, t0=2.0, fwhm=2.0)
    c = np.zeros(n, dtype=np.complex128)
    c[0] = 1.0
    for s in range(60):
        c = orc.rk4_step(A, M, p, s * 0.05, 0.05, c)
        assert abs(np.sum(orc.populations(allX, c)) - np.vdot(c, c).real) < 1e-13
    # and the states really are eigenvectors of A
    assert np.max(np.abs(A @ X.T - X.T * w)) < 1e-12


def test_field_free_rk4_populations_follow_the_stability_polynomial():
    mol = small_mol(3, 4, 5, seed=2)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    w, X = orc.ti_states(A, 5)
    c0 = synth.random_state(A.shape[0], 1, seed=8)[0]
    dt, n = 0.05, 120
    tr = orc.propagate(A, M, orc.Pulse(kind=orc.CW, E0=0.0, omega=1.0), c0, dt, n)
    b = X @ c0
    pred = np.abs(rk4_R(-1j * w * dt)) ** (2 * n) * np.abs(b) ** 2
    assert np.max(np.abs(orc.populations(X, tr.c) - pred)) < 1e-13


def test_resonant_two_level_population_is_rabi_flopping():
    """Two levels (nocc = nvirt = 1), resonant CW drive E0 sin(w0 t) with
    coupling m: in the rotating-wave approximation the upper population is
    sin^2(m E0 t / 2) (a textbook result); the neglected counter-rotating
    terms are of relative size m E0 / w0."""
    w0, m, E0 = 0.5, 1.0, 0.004
    mol = zero_mol(1, 1)
    mol["eps_virt"][:] = w0
    mol["mu_0ov"][2, 0, 0] = m
    A = orc.build_A(mol, 0.0)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    w, X = orc.ti_states(A, 1)
    assert abs(w[0] - w0) < 1e-15
    p = orc.Pulse(kind=orc.CW, E0=E0, omega=w0)
    T = 2 * math.pi / (m * E0)
    dt = 0.05
    nsteps = int(round(T / dt))
    c = np.array([1.0, 0.0], dtype=np.complex128)
    worst = 0.0
    for s in range(nsteps):
        c = orc.rk4_step(A, M, p, s * dt, dt, c)
        if (s + 1) % 200 == 0:
            t = (s + 1) * dt
            worst = max(worst, abs(orc.populations(X, c)[0] - math.sin(m * E0 * t / 2) ** 2))
    assert worst < 3 * m * E0 / w0


# ---------------------------------------------------------------------------
# Autocorrelation spectrum (the paper's mode)
# ---------------------------------------------------------------------------

def _direct_acf_spectrum(R, dt, npad, nfreq):
    """The same spectrum by a direct sum over the mirrored, windowed record
    at the padded-grid frequencies (no FFT): written from the definition."""
    R = np.atleast_2d(R)
    n = R.shape[1]
    M = 2 * n - 1
    w = 2 * np.pi * np.arange(nfreq) / ((M + npad) * dt)
    S = np.zeros(nfreq)
    for r in R:
        for k in range(nfreq):
            F = 0.0
            for m in range(M):
                j = m - (n - 1)
                val = r[j] if j >= 0 else np.conj(r[-j])
                win = 0.5 - 0.5 * math.cos(2 * math.pi * m / (M - 1))
                F += win * val * np.exp(1j * w[k] * j * dt) * dt
            S[k] += w[k] * F.real
    return S / R.shape[0]


def test_autocorrelation_of_a_kicked_run_is_its_eigen_expansion():
    """Field free after the kick: with b = V^T c(eps), RK4 gives
    R(t_n) = sum_i |b_i|^2 R4(-i lambda_i dt)^n exactly."""
    mol = small_mol(3, 4, 5, seed=12)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    tr = orc.propagate(A, M, orc.Pulse(kind=orc.KICK, E0=0.05), None, 0.05, 80, keep_every=1)
    R = orc.autocorrelation(tr.c_history[0], tr.c_history)
    lam, V = np.linalg.eigh(A)
    b = V.T @ tr.c_history[0]
    ref = np.array([np.sum(np.abs(b) ** 2 * rk4_R(-1j * lam * 0.05) ** n) for n in range(81)])
    assert np.max(np.abs(R - ref)) < 1e-13


def test_autocorr_spectrum_fft_equals_direct_sum():
    rng = np.random.default_rng(4)
    R = rng.standard_normal((2, 40)) + 1j * rng.standard_normal((2, 40))
    R[:, 0] = 1.0
    got = orc.spectrum_autocorr(R, 0.1, 25, 30, normalize=False)
    ref = _direct_acf_spectrum(R, 0.1, 25, 30)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_autocorr_spectrum_peaks_at_state_energies_with_weights():
    """R(t) = sum_i |b_i|^2 exp(-i E_i t) for a state b expanded in
    eigenstates (exact for a stationary H): peaks at w = E_i on the grid,
    heights proportional to E_i |b_i|^2 (the w prefactor of Eq.
    (21)), the Hann window's peak value being the same for
    every line; the |0> line at w = 0 is removed by the w factor."""
    dt, n, npad = 0.1, 3001, 50000
    grid = orc.autocorr_grid(n, dt, npad, 4000)
    E = np.array([grid[700], grid[1500]])
    wts = np.array([0.3, 0.1])
    t = dt * np.arange(n)
    R = 0.6 + (wts[:, None] * np.exp(-1j * E[:, None] * t)).sum(axis=0)
    S = orc.spectrum_autocorr(R, dt, npad, 4000, normalize=False)
    peaks = [int(np.argmax(S[600:800])) + 600, int(np.argmax(S[1400:1600])) + 1400]
    assert peaks == [700, 1500]
    ratio = S[1500] / S[700]
    assert abs(ratio / ((E[1] * wts[1]) / (E[0] * wts[0])) - 1.0) < 1e-3
    assert abs(S[0]) < 1e-12
    Sn = orc.spectrum_autocorr(R, dt, npad, 4000)
    assert abs(np.max(Sn) - 1.0) < 1e-15


# ---------------------------------------------------------------------------
# Kick
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kappa", [1e-3, 0.3])
def test_kick_equals_matrix_exponential(kappa):
    mol = small_mol(3, 4, 5, seed=8)
    M = orc.build_M(*orc.dipole_along(mol, (0.6, 0.0, 0.8)))
    w, U = np.linalg.eigh(M)
    e0 = np.zeros(M.shape[0])
    e0[0] = 1.0
    ref = U @ (np.exp(1j * kappa * w) * (U.T @ e0))
    got = orc.kick(M, kappa, e0)
    assert np.max(np.abs(got - ref)) < 1e-14
    assert abs(np.vdot(got, got).real - 1.0) < 1e-14


# ---------------------------------------------------------------------------
# Two-level Rabi oscillation against the paper's table
# ---------------------------------------------------------------------------

def test_two_level_rabi_periods_match_paper_table():
    gold = np.loadtxt(os.path.join(GOLDEN, "rabi_periods.txt"))
    omega0 = 11.78 / HARTREE_EV
    tdm = 1.5624
    E0 = math.sqrt(1e12 / AU_INTENSITY_W_CM2)
    mol = zero_mol(1, 1, 1)
    mol["eps_virt"][0] = omega0
    mol["mu_0ov"][2, 0, 0] = tdm
    A = orc.build_A(mol, 0.0)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    p = orc.Pulse(kind=orc.CW, E0=E0, omega=omega0)
    dt = 0.05
    T_exact = 2 * math.pi / (tdm * E0)
    nsteps = int(5.3 * T_exact / dt)
    c = np.array([1.0 + 0j, 0.0])
    pg = np.empty(nsteps + 1)
    pg[0] = 1.0
    for s in range(nsteps):
        c = orc.rk4_step(A, M, p, s * dt, dt, c)
        pg[s + 1] = abs(c[0]) ** 2
    t = dt * np.arange(nsteps + 1)
    # The inversion 2 P_ground - 1 is cos(Omega t) plus small fast wiggles from
    # the counter-rotating term; a least-squares fit of the slow cosine over
    # five cycles gives the Rabi frequency.
    from scipy.optimize import curve_fit
    model = lambda tt, amp, om, ph, off: amp * np.cos(om * tt + ph) + off
    (amp, om, ph, off), _ = curve_fit(model, t, 2 * pg - 1,
                                      p0=(1.0, 2 * math.pi / T_exact, 0.0, 0.0))
    T_fit = 2 * math.pi / abs(om)
    periods_fs = np.arange(1, 6) * T_fit * AU_TIME_FS
    assert np.max(np.abs(periods_fs - gold[:, 2])) < 0.05
    assert np.max(np.abs(periods_fs - gold[:, 1])) < 0.1     # the paper's RT-TDA column
    assert pg.min() < 0.01                                    # full inversion


# ---------------------------------------------------------------------------
# Spectrum
# ---------------------------------------------------------------------------

def _damped_cos_integral(beta, gamma, T):
    z = 1j * beta - gamma
    return np.real((np.exp(z * T) - 1.0) / z)


def test_spectrum_matches_closed_form_integral():
    dt, n, w0, gamma = 0.01, 40001, 0.8, 0.02
    t = dt * np.arange(n)
    trace = 3.0 + np.sin(w0 * t)            # constant offset is removed
    om = np.linspace(0.5, 1.1, 61)
    S = orc.spectrum(trace, dt, 1.0, gamma, om)
    T = t[-1]
    ref = om * 0.5 * (_damped_cos_integral(om - w0, gamma, T)
                      - _damped_cos_integral(om + w0, gamma, T))
    assert np.max(np.abs(S - ref)) < 1e-4 * np.max(np.abs(ref))
    # average over several traces is the mean of the single spectra
    S2 = orc.spectrum(np.stack([trace, 2 * trace]), dt, 1.0, gamma, om)
    assert np.allclose(S2, 1.5 * S, rtol=1e-13, atol=0)


def test_frequency_resolution_matches_paper():
    """Sec. 3.1 gives 0.057 eV for a 3000 au record, i.e. 2 pi / T.  On the
    oracle's spectrum of such a record (undamped), two equal lines 2 pi / T
    apart are resolved: a single line's spectrum vanishes pi / T from its
    centre, so at their midpoint both vanish; the two maxima sit about that
    far apart (each pushed out by the other's side lobe).  Lines a quarter
    of that apart merge into one peak."""
    T, dt, res_ev = np.loadtxt(os.path.join(GOLDEN, "energy_resolution.txt"))
    res = 2 * math.pi / T
    assert abs(res * HARTREE_EV - res_ev) < 5e-4
    t = dt * np.arange(int(round(T / dt)) + 1)
    w1 = 0.5

    def lines(sep):
        trace = np.sin(w1 * t) + np.sin((w1 + sep) * t)
        om = np.linspace(w1 - 1.5 * res, w1 + sep + 1.5 * res, 601)
        S = orc.spectrum(trace, dt, 1.0, 0.0, om)
        peaks = [k for k in range(1, len(om) - 1) if S[k] > S[k - 1] and S[k] >= S[k + 1] and S[k] > 0.5 * S.max()]
        return om, S, peaks

    om, S, peaks = lines(res)
    assert len(peaks) == 2
    mid = np.argmin(np.abs(om - (w1 + 0.5 * res)))
    assert abs(S[mid]) < 0.05 * S.max()
    assert abs(om[peaks[1]] - om[peaks[0]] - res) < 0.2 * res
    _, _, peaks = lines(0.25 * res)
    assert len(peaks) == 1


def test_kicked_dipole_is_linear_response_and_peaks_at_eigenvalues():
    """mu(t)/kappa equals -2 sum_k (v_k . m)^2 Im R_k^n (first order in kappa,
    RK4 amplification R_k), and the spectrum peaks at the singles-block
    eigenvalues carrying dipole strength."""
    mol = small_mol(2, 3, 4, seed=21)
    c_x, kappa, dt, n = 0.2, 1e-5, 0.05, 16000
    A = orc.build_A(mol, c_x)
    M = orc.build_M(*orc.dipole_along(mol, (0, 0, 1)))
    tr = orc.propagate(A, M, orc.Pulse(kind=orc.KICK, E0=kappa), None, dt, n)
    lam, V = np.linalg.eigh(A[1:, 1:])
    wgt = (V.T @ M[0, 1:]) ** 2
    R = rk4_R(-1j * lam * dt)
    steps = np.arange(n + 1)
    lin = -2.0 * np.sum(wgt[None, :] * np.imag(R[None, :] ** steps[:, None]), axis=1)
    got = (tr.dipole - tr.dipole[0]) / kappa
    assert np.max(np.abs(got - lin)) < 1e-3 * np.max(np.abs(lin))
    gamma = 0.01
    T = n * dt
    bright = [k for k in range(len(lam)) if wgt[k] > 0.05 * wgt.max()]
    assert bright

    def closed_form(om):
        # continuous-time linear response of the same eigenpairs
        out = np.zeros_like(om)
        for k in range(len(lam)):
            out += wgt[k] * (_damped_cos_integral(om - lam[k], gamma, T)
                             - _damped_cos_integral(om + lam[k], gamma, T))
        return om * out

    def refined_peak(om, S):
        j = int(np.argmax(S))
        assert 0 < j < len(om) - 1
        y0, y1, y2 = S[j - 1], S[j], S[j + 1]
        return om[j] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * (om[1] - om[0])

    for k in bright:
        om = np.linspace(lam[k] - 0.003, lam[k] + 0.003, 601)
        S = orc.spectrum(tr.dipole, dt, kappa, gamma, om)
        ref = closed_form(om)
        assert np.max(np.abs(S - ref)) < 2e-3 * np.max(np.abs(ref))
        p_got, p_ref = refined_peak(om, S), refined_peak(om, ref)
        assert abs(p_got - p_ref) < 1e-5, (k, p_got, p_ref)
        # the peak sits at the eigenvalue within a tenth of the line width
        # (tails of the neighbouring lines and the w prefactor pull it)
        assert abs(p_ref - lam[k]) < 0.1 * gamma


def _trapezoid_geometric(beta, gamma, dt, npts):
    """sum_n w_n exp((i beta - gamma) t_n), trapezoid weights, in closed form."""
    q = np.exp((1j * beta - gamma) * dt)
    full = (1.0 - q ** npts) / (1.0 - q)
    return full - 0.5 * (1.0 + q ** (npts - 1))


@pytest.mark.parametrize("gamma", [0.0, 0.003])
def test_spectrum_sum_equals_geometric_series(gamma):
    """The discrete damped transform of a sampled sinusoid has an exact
    geometric-series value; this pins the trapezoid end weights and the
    sign of the exponent."""
    dt, npts, w0, kappa = 0.05, 3001, 0.9, 2e-3
    t = dt * np.arange(npts)
    trace = -1.5 + kappa * np.sin(w0 * t)
    om = np.linspace(0.6, 1.2, 37)
    S = orc.spectrum(trace, dt, kappa, gamma, om)
    G = lambda b: _trapezoid_geometric(b, gamma, dt, npts)
    ref = om * np.imag((G(om + w0) - G(om - w0)) / 2j) * dt
    assert np.max(np.abs(S - ref)) < 1e-10 * np.max(np.abs(ref))


def test_field_sign_matches_linear_response_convolution():
    """H = A - E(t) M (Eq. (16)) fixes the sign of the first-order dipole
    response: delta mu(t) = int_0^t chi(t - t') E(t') dt' with
    chi(tau) = 2 sum_n (v_n . m)^2 sin(lambda_n tau) from the eigenpairs."""
    mol = small_mol(2, 3, 4, seed=13)
    A = orc.build_A(mol, 0.2)
    M = orc.build_M(*orc.dipole_along(mol, (0, 1, 0)))
    p = orc.Pulse(kind=orc.GAUSS_TL, E0=1e-6, omega=1.1, t0=15.0, fwhm=8.0)
    dt, n = 0.01, 4000
    tr = orc.propagate(A, M, p, None, dt, n)
    lam, V = np.linalg.eigh(A[1:, 1:])
    wgt = (V.T @ M[0, 1:]) ** 2
    t = dt * np.arange(n + 1)
    E = np.array([orc.field(p, x) for x in t])
    chi = lambda tau: 2.0 * np.sum(wgt[None, :] * np.sin(np.outer(tau, lam)), axis=1)
    ref = np.zeros(n + 1)
    for k in range(1, n + 1, 50):
        tt = t[: k + 1]
        ref[k] = np.trapezoid(chi(t[k] - tt) * E[: k + 1], tt)
    got = tr.dipole - tr.dipole[0]
    sel = np.arange(1, n + 1, 50)
    scale = np.max(np.abs(ref[sel]))
    assert scale > 0
    assert np.max(np.abs(got[sel] - ref[sel])) < 1e-3 * scale
