"""Degenerate and boundary cases of the CUDA path against the oracle:
zero steps, a single auxiliary function, a single occupied or virtual
orbital, the smallest batch in every precision, empty fields, and resume
of zero steps."""
import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import oracle_runs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRECS = ["fp64", "fp32", "bf16", "bf16x3", "bf16x2"]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("integrator", ["rk4", "sso"])
@pytest.mark.parametrize("kappa", [0.01, 0.3])
def test_zero_steps_returns_the_kicked_state(rb, prec, integrator, kappa):
    """The kicked state: the Taylor series of exp(i kappa M_d) accumulated in
    FP64, its first-order term from FP64 field products in every precision.
    In the precisions whose field products are FP32 the terms of order >= 2
    take FP32 products, so the state is exact to FP64 rounding plus FP32
    rounding of those terms: n eps_32 (x^2 / 2) e^x for x = kappa ||M_d||_2
    and inner length n <= o + v + 1."""
    mol = synth.molecule(3, 8, 5, seed=2)
    pulses = [dict(kind=0, E0=kappa, direction=(0, 1, 0))]
    prop = rb.Propagator(mol, 0.2, prec, integrator=integrator)
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 0)
    ref = oracle_runs(mol, 0.2, pulses, 0.05, 0)[0]
    assert dip.shape == (1, 1) and nrm.shape == (1, 1)
    x = kappa * np.linalg.norm(orc.build_M(*orc.dipole_along(mol, (0, 1, 0))), 2)
    ktol = 1e-12 if prec == "fp64" else 1e-12 + (3 + 8 + 1) * 2.0 ** -24 * x * x / 2 * np.exp(x)
    assert np.max(np.abs(c[0] - ref.c)) < ktol
    assert abs(nrm[0, 0] - ref.norm[0]) < 2 * ktol
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert abs(dip[0, 0] - ref.dipole[0]) < tol * max(1.0, abs(ref.dipole[0]))
    # resuming zero steps changes nothing
    c2, d2, _ = prop.resume(0.05, 0)
    assert np.array_equal(c2, c)
    prop.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 40, 3), (40, 1, 3), (6, 10, 1)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x2", 1e-2)])
def test_degenerate_shapes_propagate_like_the_oracle(rb, shape, prec, tol):
    mol = synth.molecule(*shape, seed=5)
    pulses = [dict(kind=4, E0=0.05, omega=0.8, duration=3.0, direction=(1, 0, 1)),
              dict(kind=0, E0=0.02, direction=(0, 0, 1))]
    prop = rb.Propagator(mol, 0.3, prec)
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 60)
    refs = oracle_runs(mol, 0.3, pulses, 0.05, 60)
    for t, ref in enumerate(refs):
        if prec == "fp64":
            assert np.max(np.abs(c[t] - ref.c)) < tol, t
        else:
            d = ref.dipole - ref.dipole[0]
            rel = np.max(np.abs(dip[t] - ref.dipole)) / max(np.max(np.abs(d)), 1e-30)
            assert rel < tol, (t, rel)
        assert np.max(np.abs(nrm[t] - ref.norm)) < 1e-6, t
    prop.close()


def test_zero_field_pulses_leave_the_ground_state_stationary(rb):
    """E0 = 0 for every pulse kind: |0> is an eigenvector of A with
    eigenvalue 0, so the state, the dipole and the norm do not change."""
    mol = synth.molecule(4, 9, 6, seed=1)
    pulses = [dict(kind=k, E0=0.0, omega=0.7, t0=1.0, fwhm=1.0, beta=0.1, duration=2.0) for k in range(5)]
    prop = rb.Propagator(mol, 0.2, "bf16x2")
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 40)
    e0 = np.zeros(prop.n)
    e0[0] = 1.0
    assert np.max(np.abs(c - e0)) == 0.0
    assert np.all(dip == 0.0) and np.all(nrm == 1.0)
    prop.close()


def test_many_trajectories_of_a_tiny_molecule(rb):
    """64 trajectories (128 real columns) of a 2-occupied, 3-virtual molecule:
    the column-batched kernels at their widest for a tiny row count."""
    mol = synth.molecule(2, 3, 4, seed=3)
    rng = np.random.default_rng(0)
    pulses = [dict(kind=int(k % 5), E0=0.01 + 0.04 * rng.random(), omega=0.5 + rng.random(), t0=1.0,
                   fwhm=1.5, beta=0.2, duration=3.0, direction=tuple(rng.standard_normal(3)))
              for k in range(64)]
    prop = rb.Propagator(mol, 0.2, "fp64")
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 50)
    refs = oracle_runs(mol, 0.2, pulses, 0.05, 50)
    for t, ref in enumerate(refs):
        assert np.max(np.abs(c[t] - ref.c)) < 1e-12, t
    prop.close()
