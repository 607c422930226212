"""GPU parity of the symplectic split-operator integrator (Sec. 2.2) against
the FP64 oracle's split-operator steps, through the C ABI."""
import numpy as np
import pytest

from paper_2601_16949_b300 import synth
from tests._util import oracle_runs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PULSES4 = [
    dict(kind=1, E0=0.03, omega=0.7, direction=(0, 0, 1)),
    dict(kind=2, E0=0.05, omega=0.9, t0=2.0, fwhm=1.7, direction=(1, 0, 0)),
    dict(kind=3, E0=0.04, omega=0.6, t0=1.5, fwhm=2.5, beta=0.3, direction=(0, 1, 1)),
    dict(kind=4, E0=0.05, omega=1.1, duration=4.0, direction=(1, 1, 0)),
]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def test_sso_config1_fp64_2000_steps_within_1e10(rb):
    """o=8, v=24, P=96, z kick kappa=1e-3, c_x=0.2, dt=0.05, 2000 split-operator
    steps: amplitudes, dipole and norm against the oracle."""
    mol = synth.molecule(8, 24, 96, seed=0)
    pulses = [dict(kind=0, E0=1e-3, direction=(0, 0, 1))]
    prop = rb.Propagator(mol, 0.2, "fp64", integrator="sso")
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 2000)
    ref = oracle_runs(mol, 0.2, pulses, 0.05, 2000, integrator="sso")[0]
    assert np.max(np.abs(c[0] - ref.c)) <= 1e-10
    assert np.max(np.abs(dip[0] - ref.dipole)) <= 1e-10 * max(1.0, np.max(np.abs(ref.dipole)))
    assert np.max(np.abs(nrm[0] - ref.norm)) <= 1e-12
    prop.close()


def test_sso_fp64_driven_batch_matches_oracle(rb):
    mol = synth.molecule(4, 9, 11, seed=2)
    prop = rb.Propagator(mol, 0.3, "fp64", integrator="sso")
    prop.set_field(PULSES4)
    c0 = synth.random_state(prop.n, len(PULSES4), seed=4)
    c, dip, nrm = prop.propagate(0.05, 150, c0=c0)
    refs = oracle_runs(mol, 0.3, PULSES4, 0.05, 150, c0=c0, integrator="sso")
    for t, ref in enumerate(refs):
        assert np.max(np.abs(c[t] - ref.c)) < 1e-12, t
        assert np.max(np.abs(dip[t] - ref.dipole)) < 1e-11, t
        assert np.max(np.abs(nrm[t] - ref.norm)) < 1e-13, t
    prop.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x2"])
def test_sso_resume_is_bitwise(rb, prec):
    mol = synth.molecule(6, 64, 20, seed=8)
    pulses = [PULSES4[1], PULSES4[3]]
    a = rb.Propagator(mol, 0.2, prec, integrator="sso")
    a.set_field(pulses)
    c_full, d_full, n_full = a.propagate(0.05, 80)
    a.propagate(0.05, 40)
    state, t = a.get_state()
    b = rb.Propagator(mol, 0.2, prec, integrator="sso")
    b.set_field(pulses)
    b.set_state(state, t)
    c_res, d_res, n_res = b.resume(0.05, 40)
    assert np.array_equal(c_res, c_full)
    assert np.array_equal(d_res[:, -1], d_full[:, -1])
    assert np.array_equal(n_res[:, -1], n_full[:, -1])
    a.close()
    b.close()


# about 10x the measured relative dipole error after 400 steps (7e-9, 3e-7,
# 7e-10 with the FP64-accurate observable)
@pytest.mark.parametrize("prec,dip_tol", [("bf16x3", 1e-7), ("bf16x2", 3e-6), ("fp32", 1e-8)])
def test_sso_reduced_precision_against_oracle(rb, prec, dip_tol):
    mol = synth.molecule(8, 64, 48, seed=5)
    pulses = [dict(kind=0, E0=1e-3, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    prop = rb.Propagator(mol, 0.2, prec, integrator="sso")
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 400)
    refs = oracle_runs(mol, 0.2, pulses, 0.05, 400, integrator="sso")
    for t, ref in enumerate(refs):
        d = ref.dipole - ref.dipole[0]
        rel = np.max(np.abs(dip[t] - ref.dipole)) / np.max(np.abs(d))
        assert rel < dip_tol, (prec, t, rel)
        assert np.max(np.abs(nrm[t] - ref.norm)) < 1e-9, (prec, t)
    prop.close()


def test_sso_norm_stays_bounded_where_rk4_decays(rb):
    """Long field-free run from a random state: the split operator's norm
    error oscillates without a trend, RK4's decreases monotonically."""
    mol = synth.molecule(5, 40, 30, seed=3)
    c0 = synth.random_state(1 + 5 * 40, 1, seed=6)
    out = {}
    for integ in ("sso", "rk4"):
        prop = rb.Propagator(mol, 0.2, "fp64", integrator=integ)
        prop.set_field([dict(kind=1, E0=0.0, omega=1.0)])
        _, _, nrm = prop.propagate(0.2, 3000, c0=c0)
        out[integ] = nrm[0]
        prop.close()
    sso, rk4 = out["sso"], out["rk4"]
    assert np.all(np.diff(rk4) <= 1e-15) and rk4[-1] < rk4[0] - 1e-9
    first, last = np.abs(sso[:1000] - 1.0).max(), np.abs(sso[-1000:] - 1.0).max()
    assert last < 1.5 * first + 1e-14


def test_unknown_integrator_is_rejected(rb):
    mol = synth.molecule(2, 3, 4, seed=1)
    prop = rb.Propagator(mol, 0.2, "fp64")
    with pytest.raises(rb.RTTDAError) as e:
        rb.rttda_set_integrator(prop.h, 7)
    assert e.value.status == rb.E_ARG
    prop.close()
