"""TI-TDA eigenstates (Davidson on the library's sigma) and population /
overlap recording (Eq. populations) against the FP64 oracle."""
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
