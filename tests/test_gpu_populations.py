"""TI-TDA eigenstates (Davidson on the library's sigma) and population /
overlap recording (Eq. (22)) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import oracle_pulse, unit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PULSES3 = [
    dict(kind=2, E0=0.06, omega=0.9, t0=2.0, fwhm=1.7, direction=(1, 0, 0)),
    dict(kind=4, E0=0.05, omega=1.1, duration=4.0, direction=(0, 1, 1)),
    dict(kind=0, E0=2e-3, direction=(0, 0, 1)),
]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


@pytest.mark.parametrize("shape,k", [((5, 12, 17), 6), ((3, 40, 30), 9)])
def test_eigenstates_fp64_match_dense_diagonalisation(rb, shape, k):
    mol = synth.molecule(*shape, seed=21)
    prop = rb.Propagator(mol, 0.2, "fp64")
    prop.set_field(PULSES3)
    w, X, iters = prop.eigenstates(k, tol=1e-9, max_iter=300)
    A = orc.build_A(mol, 0.2)
    w_ref, X_ref = orc.ti_states(A, k)
    assert np.max(np.abs(w - w_ref)) < 1e-10, (w, w_ref)
    assert np.all(X[:, 0] == 0.0)
    # unit vectors parallel to the reference states (up to sign; the spectra
    # of these molecules have no degenerate levels among the lowest k)
    dots = np.abs(np.sum(X * X_ref, axis=1))
    assert np.max(np.abs(dots - 1.0)) < 1e-9
    assert np.max(np.abs(A @ X.T - X.T * w)) < 1e-8
    prop.close()


def test_eigenstates_bf16x2_close_to_fp64(rb):
    mol = synth.molecule(16, 96, 64, seed=3)
    prop = rb.Propagator(mol, 0.2, "bf16x2")
    prop.set_field(PULSES3)
    w, X, iters = prop.eigenstates(8, tol=1e-5, max_iter=300)
    w_ref, X_ref = orc.ti_states(orc.build_A(mol, 0.2), 8)
    assert np.max(np.abs(w - w_ref)) < 1e-5 * np.max(np.abs(w_ref)), (w - w_ref)
    assert np.min(np.abs(np.sum(X * X_ref, axis=1))) > 1 - 1e-4
    prop.close()


def _oracle_overlaps(mol, c_x, pulses, dt, nsteps, P, integrator):
    A = orc.build_A(mol, c_x)
    out = []
    for p in pulses:
        M = orc.build_M(*orc.dipole_along(mol, unit(p.get("direction", (0, 0, 1)))))
        op = oracle_pulse(p)
        c = np.zeros(A.shape[0], dtype=np.complex128)
        c[0] = 1.0
        if op.kind == orc.KICK:
            c = orc.kick(M, op.E0, c)
        rows = [orc.overlaps(P, c)]
        for s in range(nsteps):
            step = orc.rk4_step if integrator == "rk4" else orc.sso_step
            c = step(A, M, op, s * dt, dt, c)
            rows.append(orc.overlaps(P, c))
        out.append(np.array(rows))
    return np.array(out)


@pytest.mark.parametrize("integrator", ["rk4", "sso"])
def test_recorded_overlaps_match_oracle_fp64(rb, integrator):
    mol = synth.molecule(4, 9, 11, seed=6)
    A = orc.build_A(mol, 0.3)
    w, X = orc.ti_states(A, 5)
    e0 = np.zeros((1, A.shape[0]))
    e0[0, 0] = 1.0
    P = np.vstack([e0, X])
    prop = rb.Propagator(mol, 0.3, "fp64", integrator=integrator)
    prop.set_field(PULSES3)
    prop.set_projectors(P)
    nsteps = 120
    _, _, nrm = prop.propagate(0.05, nsteps)
    got = prop.overlaps(nsteps)
    ref = _oracle_overlaps(mol, 0.3, PULSES3, 0.05, nsteps, P, integrator)
    assert got.shape == ref.shape == (3, nsteps + 1, 6)
    assert np.max(np.abs(got - ref)) < 1e-12
    # a second call records its own steps (from the state it resumes)
    prop.resume(0.05, 10)
    assert prop.overlaps(10).shape == (3, 11, 6)
    prop.close()


def test_populations_of_a_complete_basis_sum_to_the_norm(rb):
    mol = synth.molecule(2, 3, 4, seed=7)
    A = orc.build_A(mol, 0.2)
    n = A.shape[0]
    w, X = orc.ti_states(A, n - 1)
    e0 = np.zeros((1, n))
    e0[0, 0] = 1.0
    prop = rb.Propagator(mol, 0.2, "bf16x2")
    prop.set_field(PULSES3)
    prop.set_projectors(np.vstack([e0, X]))
    _, _, nrm = prop.propagate(0.05, 200)
    pops = np.abs(prop.overlaps(200)) ** 2
    assert np.max(np.abs(pops.sum(axis=2) - nrm)) < 1e-12
    prop.close()


def test_overlap_errors(rb):
    mol = synth.molecule(2, 3, 4, seed=1)
    prop = rb.Propagator(mol, 0.2, "fp64")
    prop.set_field([dict(kind=0, E0=1e-3)])
    with pytest.raises(rb.RTTDAError) as e:
        prop.nproj = 1
        prop.overlaps(5)
    assert e.value.status == rb.E_STATE
    prop.set_projectors(np.eye(1, 7))
    prop.propagate(0.05, 5)
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_get_overlaps(prop.h, 1, 4, 1)
    assert e.value.status == rb.E_ARG
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_eigenstates(prop.h, 0, 7)
    assert e.value.status == rb.E_ARG
    prop.close()


@pytest.mark.parametrize("integrator", ["rk4", "sso"])
def test_autocorrelation_matches_oracle_fp64(rb, integrator):
    """R(t) = X(eps)^dagger X(eps + t) of kicked x/y/z runs (eps right after
    the kick) against the oracle's trajectories."""
    mol = synth.molecule(4, 9, 11, seed=6)
    pulses = [dict(kind=0, E0=0.02, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    prop = rb.Propagator(mol, 0.3, "fp64", integrator=integrator)
    prop.set_field(pulses)
    rb.rttda_set_autocorrelation(prop.h, True)
    nsteps = 150
    prop.propagate(0.05, nsteps)
    got = prop.autocorrelation(nsteps)
    A = orc.build_A(mol, 0.3)
    for t, p in enumerate(pulses):
        M = orc.build_M(*orc.dipole_along(mol, unit(p["direction"])))
        c = orc.kick(M, p["E0"], np.eye(1, A.shape[0])[0])
        hist = [c]
        for s in range(nsteps):
            step = orc.rk4_step if integrator == "rk4" else orc.sso_step
            c = step(A, M, oracle_pulse(p), s * 0.05, 0.05, c)
            hist.append(c)
        ref = orc.autocorrelation(hist[0], hist)
        assert np.max(np.abs(got[t] - ref)) < 1e-12, t
    # resume continues against the same X(eps)
    prop.resume(0.05, 20)
    assert prop.autocorrelation(20).shape == (3, 21)
    prop.close()


def test_autocorrelation_spectrum_matches_oracle_fft_and_finds_the_states(rb):
    """The paper's spectrum mode (mirror, Hann, 50000 zeros of padding, w Re F,
    x/y/z average, peak normalisation) from GPU records, against the
    oracle's FFT of the same records; its strongest line sits on a TI-TDA
    excitation energy from rttda_eigenstates, within the grid spacing."""
    mol = synth.molecule(4, 12, 16, seed=9)
    # kappa 0.05: the excited-state weights (~kappa^2) stand well above the
    # Hann sidelobes of the |0> line at w = 0 over this 200 au record
    pulses = [dict(kind=0, E0=0.05, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    prop = rb.Propagator(mol, 0.2, "bf16x2")
    prop.set_field(pulses)
    rb.rttda_set_autocorrelation(prop.h, True)
    nsteps, dt = 4000, 0.05
    prop.propagate(dt, nsteps)
    R = prop.autocorrelation(nsteps)
    om, S = rb.rttda_spectrum_autocorr(R, dt, npad=50000, nfreq=3000)
    S_ref = orc.spectrum_autocorr(R, dt, 50000, 3000)
    assert np.allclose(om, orc.autocorr_grid(nsteps + 1, dt, 50000, 3000), rtol=1e-14, atol=0)
    assert np.max(np.abs(S - S_ref)) < 1e-9
    w, _, _ = prop.eigenstates(4 * 12, tol=1e-4)     # every excited state
    # the |0> component of X(eps) puts a line at w = 0 whose Hann main lobe
    # (width ~ 2 pi / (nsteps dt)) the w factor does not remove: look above
    # it; each of the strongest local maxima sits on an excitation energy
    lo = int(np.searchsorted(om, 0.2))
    peaks = [j for j in range(lo + 1, len(S) - 1) if S[j] >= S[j - 1] and S[j] >= S[j + 1]]
    peaks = sorted(peaks, key=lambda j: -S[j])[:2]
    resolution = 2 * np.pi / (nsteps * dt)     # lines closer than this merge
    for j in peaks:
        assert np.min(np.abs(w - om[j])) <= 0.5 * resolution, (om[j], S[j])
    prop.close()
