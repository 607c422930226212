"""FP64_OZ: the exchange on tensor-core Ozaki digits against the FP64 oracle
(sigma, propagation, several Z chunks, several exactness blocks per P) and
against the FP64 CUDA-core path at the full linear-absorption size."""
import os

import numpy as np
import pytest

from oracle import rttda_oracle as orc
from paper_2601_16949_b300 import synth
from tests._util import oracle_runs, oracle_sigma, to_ri, unit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PULSES = [
    dict(kind=1, E0=0.03, omega=0.7, direction=(0, 0, 1)),
    dict(kind=4, E0=0.05, omega=1.1, duration=4.0, direction=(1, 1, 0)),
]


@pytest.fixture(scope="module")
def rb():
    from paper_2601_16949_b300 import binding
    return binding


def _sigma_gpu(rb, prop, c, t):
    cd = torch.tensor(to_ri(c), dtype=torch.float64, device="cuda")
    sd = torch.zeros_like(cd)
    rb.rttda_sigma(prop.h, cd.data_ptr(), t, sd.data_ptr(), 0)
    torch.cuda.synchronize()
    s = sd.cpu().numpy()
    return s[..., 0] + 1j * s[..., 1]


# (nocc, nvirt, naux): tiny, ragged (nvirt not a multiple of 64, nocc not a
# multiple of 8), several 128-row tiles, and nvirt > 512 (two exactness blocks
# per P along b)
SHAPES = [(1, 1, 1), (3, 5, 7), (5, 37, 19), (17, 70, 33), (9, 130, 21), (4, 600, 5)]


@pytest.mark.parametrize("shape", SHAPES)
def test_sigma_fp64oz_matches_oracle(rb, shape):
    mol = synth.molecule(*shape, seed=4)
    c_x = 0.2
    prop = rb.Propagator(mol, c_x, "fp64oz")
    prop.set_field(PULSES)
    assert rb.rttda_plan(prop.h)["main_kernel"] == 3
    c = synth.random_state(prop.n, len(PULSES), seed=7)
    for t in (0.0, 1.3):
        got = _sigma_gpu(rb, prop, c, t)
        ref = oracle_sigma(mol, c_x, PULSES, c, t)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) < 2e-12 * max(scale, 1.0), (shape, t, np.max(np.abs(got - ref)) / scale)
    prop.close()


@pytest.mark.parametrize("zchunk", ["1", "4"])
def test_sigma_fp64oz_over_several_z_chunks(rb, zchunk):
    """Z built and contracted a few P at a time (FP64 partials accumulated
    across chunks, B_vv digits and exponents offset per chunk)."""
    mol = synth.molecule(6, 90, 11, seed=3)
    os.environ["RTTDA_ZCHUNK"] = zchunk
    try:
        prop = rb.Propagator(mol, 0.3, "fp64oz")
        prop.set_field(PULSES)
    finally:
        del os.environ["RTTDA_ZCHUNK"]
    assert rb.rttda_plan(prop.h)["z_chunk"] == int(zchunk)
    c = synth.random_state(prop.n, len(PULSES), seed=2)
    got = _sigma_gpu(rb, prop, c, 0.6)
    ref = oracle_sigma(mol, 0.3, PULSES, c, 0.6)
    assert np.max(np.abs(got - ref)) < 2e-12 * np.max(np.abs(ref))
    prop.close()


def test_fp64oz_propagation_matches_oracle(rb):
    mol = synth.molecule(6, 40, 24, seed=9)
    pulses = [dict(kind=2, E0=0.05, omega=0.9, t0=2.0, fwhm=1.7, direction=(1, 0, 0)),
              dict(kind=0, E0=1e-3, direction=(0, 0, 1))]
    prop = rb.Propagator(mol, 0.2, "fp64oz")
    prop.set_field(pulses)
    c, dip, nrm = prop.propagate(0.05, 200)
    refs = oracle_runs(mol, 0.2, pulses, 0.05, 200)
    for t, ref in enumerate(refs):
        assert np.max(np.abs(c[t] - ref.c)) < 1e-11, t
        assert np.max(np.abs(dip[t] - ref.dipole)) < 1e-11 * max(1.0, np.max(np.abs(ref.dipole))), t
        assert np.max(np.abs(nrm[t] - ref.norm)) < 1e-12, t
    prop.close()


def test_fp64oz_equals_fp64_at_full_size(rb):
    """Linear-absorption molecule (o=64, v=448, P=1536): one sigma of a
    random batch of three trajectories in FP64_OZ against the FP64
    CUDA-core path (all rows) and against the oracle's element-wise rows."""
    mol = synth.molecule(64, 448, 1536, seed=0)
    pulses = [dict(kind=1, E0=0.01, omega=0.5, direction=d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    n = 1 + 64 * 448
    c = synth.random_state(n, 3, seed=11)
    t = 0.9
    got = {}
    for prec in ("fp64oz", "fp64"):
        prop = rb.Propagator(mol, 0.2, prec)
        prop.set_field(pulses)
        got[prec] = _sigma_gpu(rb, prop, c, t)
        prop.close()
    scale = np.max(np.abs(got["fp64"]), axis=1)
    err = np.max(np.abs(got["fp64oz"] - got["fp64"]), axis=1) / scale
    assert np.all(err < 1e-12), err
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, 1, n - 1], rng.choice(np.arange(2, n - 1), 13, replace=False)])
    Arows = orc.A_rows(mol, 0.2, rows)
    for k, p in enumerate(pulses):
        Mrows = orc.M_rows(*orc.dipole_along(mol, unit(p["direction"])), rows)
        E = orc.field(orc.Pulse(kind=1, E0=0.01, omega=0.5), t)
        ref = Arows @ c[k] - E * (Mrows @ c[k])
        rs = np.abs(Arows) @ np.abs(c[k]) + abs(E) * (np.abs(Mrows) @ np.abs(c[k]))
        assert np.max(np.abs(got["fp64oz"][k, rows] - ref) / rs) < 1e-12, k


def test_fp64oz_rejects_nocc_above_512(rb):
    mol = synth.molecule(513, 1, 1, seed=1)
    with pytest.raises(rb.RTTDAError) as e:
        rb.Propagator(mol, 0.2, "fp64oz")
    assert e.value.status == rb.E_ARG


def test_fp64oz_split_operator_and_resume(rb):
    """The split-operator stepper on the digit path: driven batch from a
    given state against the oracle's split operator, and a bitwise resume."""
    mol = synth.molecule(4, 9, 11, seed=2)
    pulses = [dict(kind=1, E0=0.03, omega=0.7, direction=(0, 0, 1)),
              dict(kind=3, E0=0.04, omega=0.6, t0=1.5, fwhm=2.5, beta=0.3, direction=(0, 1, 1))]
    c0 = synth.random_state(1 + 4 * 9, len(pulses), seed=4)
    a = rb.Propagator(mol, 0.3, "fp64oz", integrator="sso")
    a.set_field(pulses)
    c, dip, nrm = a.propagate(0.05, 150, c0=c0)
    refs = oracle_runs(mol, 0.3, pulses, 0.05, 150, c0=c0, integrator="sso")
    for t, ref in enumerate(refs):
        assert np.max(np.abs(c[t] - ref.c)) < 1e-11, t
        assert np.max(np.abs(nrm[t] - ref.norm)) < 1e-12, t
    a.propagate(0.05, 80, c0=c0)
    c_full = a.resume(0.05, 40)[0]
    b = rb.Propagator(mol, 0.3, "fp64oz", integrator="sso")
    b.set_field(pulses)
    b.propagate(0.05, 80, c0=c0)
    state, t_now = b.get_state()
    b.set_state(state, t_now)
    assert np.array_equal(b.resume(0.05, 40)[0], c_full)
    a.close()
    b.close()


def test_fp64oz_eigenstates_match_dense_diagonalisation(rb):
    """Davidson on the digit path's sigma finds the dense eigenpairs."""
    mol = synth.molecule(5, 12, 17, seed=21)
    prop = rb.Propagator(mol, 0.2, "fp64oz")
    prop.set_field([dict(kind=0, E0=1e-3, direction=(0, 0, 1))])
    w, X, iters = prop.eigenstates(6, tol=1e-9, max_iter=300)
    w_ref, X_ref = orc.ti_states(orc.build_A(mol, 0.2), 6)
    assert np.max(np.abs(w - w_ref)) < 1e-10, (w, w_ref)
    assert np.max(np.abs(np.abs(np.sum(X * X_ref, axis=1)) - 1.0)) < 1e-9
    prop.close()


def _extreme_digit_value(sign):
    """A value in (-1, 1) whose six centred base-128 digits are all at the
    largest magnitude the split produces for a block maximum of 1:
    +-(127, 63, 63, 63, 63, 63)."""
    F = 127 * 128 ** 5 + 63 * sum(128 ** k for k in range(5))
    return sign * F / 2.0 ** 42


@pytest.mark.parametrize("pattern", ["equal", "alternating"])
def test_fp64oz_group_sums_at_their_bound_stay_exact(rb, pattern):
    """Exactness of the tensor-core group sums at their worst case.  With
    nocc = 1, nvirt = 512 (one exactness block of 512 b per P), B_oo = 1 and
    every amplitude and B_vv entry at +-(127, 63, 63, 63, 63, 63), the
    digit-pair sums of the main contraction reach (g + 3) 2^12 x 512 per
    group: 2^23.96 for g = 5, 2^23 for the leading groups.  A rounded partial
    sum in a leading group would show as a relative error near 1e-7; the
    dropped pairs (s + t >= 6) allow about 2^-44."""
    o, v, P = 1, 512, 1
    x = _extreme_digit_value(1.0)
    sgn = np.ones(v) if pattern == "equal" else np.where(np.arange(v) % 2 == 0, 1.0, -1.0)
    mol = dict(nocc=o, nvirt=v, naux=P,
               eps_occ=np.zeros(o), eps_virt=np.zeros(v),
               B_ov=np.zeros((P, o, v)), B_oo=np.ones((P, o, o)),
               B_vv=np.full((P, v, v), x), mu_oo=np.zeros((3, o, o)),
               mu_vv=np.zeros((3, v, v)), mu_0ov=np.zeros((3, o, v)))
    c = np.zeros((1, 1 + v), dtype=complex)
    c[0, 1:] = x * sgn
    pulses = [dict(kind=1, E0=0.0, omega=0.5, direction=(0, 0, 1))]
    prop = rb.Propagator(mol, 1.0, "fp64oz")
    prop.set_field(pulses)
    got = _sigma_gpu(rb, prop, c, 0.0)
    prop.close()
    ref = oracle_sigma(mol, 1.0, pulses, c, 0.0)
    exact = -x * x * np.sum(sgn)   # every row a: -c_x sum_b x_b B_ab
    scale = x * x * v
    assert np.max(np.abs(ref[0, 1:] - exact)) <= 1e-14 * scale   # the oracle, up to FP64 summation
    assert abs(got[0, 0]) == 0.0
    err = np.max(np.abs(got[0, 1:] - exact)) / scale
    assert err <= 1e-12, err
