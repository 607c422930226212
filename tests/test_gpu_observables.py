"""The recorded observables are the FP64-accurate expectation values of the
state the GPU holds, in every precision.

The dipole trace records mu_d(t_n) = Re c_n^dagger M_d c_n (Sec. 2.2, the
expectation of the dipole operator of Eqs. (12)-(16) along the pulse's
polarisation) and the norm |c_n|^2.  In the reduced-precision modes the
sigma builds are BF16 or FP32, but the field product that feeds the
observable is taken in double-float arithmetic from the FP64 dipole blocks,
and the reduction is FP64.  So whatever the precision, the recorded value
must agree with the oracle's dense FP64 expectation of the GPU's own state
(returned by the same call) to about the FP64 rounding of the sum, far
below the sigma build's own error.  This pins the observable separately
from the propagation's accuracy.
"""
import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import unit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# a CW pulse (no kick: the given state is the state at t = 0)
MIXED = [dict(kind=1, E0=0.02, omega=0.6, direction=d) for d in ((0, 0, 1), (1, 0, 0), (1, 2, -1))]
ONE_DIR = [dict(kind=1, E0=0.01 * (k + 1), omega=0.5 + 0.1 * k, direction=(0, 1, 1)) for k in range(5)]
# relative to sum |c_i| |M_ij| |c_j|: FP64 rounding of the sum is ~1e-16
# per term; the double-float product keeps ~44 bits
REL_TOL = 2e-13


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def _expectation(M, c):
    return float(np.real(np.vdot(c, M @ c))), float(np.abs(c) @ (np.abs(M) @ np.abs(c)))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x2", "bf16x3", "fp64", "fp64oz"])
@pytest.mark.parametrize("shape,pulses", [((5, 37, 23), MIXED), ((8, 64, 40), ONE_DIR), ((3, 9, 11), ONE_DIR[:1])])
def test_recorded_dipole_is_the_fp64_expectation_of_the_held_state(rb, prec, shape, pulses):
    mol = synth.molecule(*shape, seed=7)
    prop = rb.Propagator(mol, 0.2, prec)
    prop.set_field(pulses)
    n, T = prop.n, len(pulses)
    c0 = synth.random_state(n, T, seed=11)
    Ms = [orc.build_M(*orc.dipole_along(mol, unit(p["direction"]))) for p in pulses]
    # t = 0: the given state itself
    _, dip0, nrm0 = prop.propagate(0.05, 0, c0=c0)
    # after 9 steps: the state the call returns
    c9, dip9, nrm9 = prop.propagate(0.05, 9, c0=c0)
    prop.close()
    assert np.allclose(dip9[:, 0], dip0[:, 0], rtol=0, atol=0)
    for t in range(T):
        for c, mu, nr in ((c0[t], dip0[t, 0], nrm0[t, 0]), (c9[t], dip9[t, -1], nrm9[t, -1])):
            ref, scale = _expectation(Ms[t], c)
            assert abs(mu - ref) <= REL_TOL * scale, (prec, t, mu, ref, scale)
            assert abs(nr - float(np.vdot(c, c).real)) <= 1e-14 * nr, (prec, t)
